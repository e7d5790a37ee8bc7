"""The model's variants on the CUDA path against the FP64 oracle, flip for flip:
the edge forms and the ising array of the geometry figure, the parallel-only
switching criterion of the pinwheel section, local and spatial external fields
and encoded protocols (Sec. "External field", Sec. "Simulation framework"),
annealing by a per-step thermal deviation and the spin-spin correlation (Sec.
"Domain size in square ASI").

Tolerances as for the main path: flip sequences, flips per step, hashes, final
spins and correlation counts bit-exact; fields within 1e-12 of max|h| (FS_FP64).
"""
import math

import numpy as np
import pytest

from paper_2002_11401_b300 import inputs as I

from .helpers import first_divergence

pytestmark = pytest.mark.gpu

FP64, FP32 = 0, 1


@pytest.fixture(scope="module")
def B():
    from paper_2002_11401_b300 import build
    build.build()
    from paper_2002_11401_b300 import binding
    return binding


def _pair(B, O, kind, nx, ny, *, alpha=1e-3, cutoff=3.0, hk=0.2, kdis=0.05, seed=5,
          sigma=0.0, astroid=(1.0, 1.0, 3.0, 3.0), criterion=0, precision=FP64):
    b, c, beta, gamma = astroid
    sim = B.Sim.geometry(kind, nx, ny)
    sim.set_params(B.make_params(alpha=alpha, hk=hk, k_disorder=kdis, b=b, c=c, beta=beta,
                                 gamma=gamma, cutoff=cutoff, sigma_th=sigma, seed=seed,
                                 precision=precision, criterion=criterion))
    x, y, th = O.geometry(kind, nx, ny)
    S = O.Sim(x, y, th, O.draw_hk(len(x), hk, kdis, seed), alpha=alpha, b=b, c=c, beta=beta,
              gamma=gamma, sigma_th=sigma, cutoff_abs=cutoff, seed=seed, criterion=criterion)
    return sim, S


def _same(got, ref):
    d = first_divergence(ref["log_step"], ref["log_spin"], got["log_step"], got["log_spin"])
    assert d is None, (d, ref["ties"])
    assert got["n_flips"] == ref["n_flips"] and got["hash"] == ref["hash"]
    np.testing.assert_array_equal(got["flips_per_step"], ref["flips_per_step"])


# ---------------------------------------------------------------------------
# Geometries and the switching criterion
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("kind,n,cutoff", [(3, 14, 3.0), (4, 12, 5.0), (5, 12, 5.0),
                                           (6, 16, 4.0)])
def test_geometry_variants_sequences(B, oracle, kind, n, cutoff, prec):
    sim, S = _pair(B, oracle, kind, n, n, cutoff=cutoff, seed=kind, precision=prec,
                   alpha=2e-3 if kind == 6 else 1e-3)
    hx, hy = I.loop_protocol(160, 30.0 if kind in (4, 5) else 10.0, -0.3, 0.3)
    ref = S.run(np.ones(S.n, dtype=np.int8), hx, hy)
    got = sim.run_protocol(hx, hy)
    assert ref["n_flips"] >= S.n
    _same(got, ref)
    np.testing.assert_array_equal(sim.spins(), ref["spins"])


@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("angle", [0.0, 30.0])
def test_parallel_criterion_pinwheel_reversal(B, oracle, angle, prec):
    """The paper's pinwheel reversal (its astroid parameters and coupling) under the
    parallel-only criterion: every flip as the oracle's; it differs from the
    reversal under Eq. 5."""
    kw = dict(alpha=0.00033, hk=0.098, kdis=0.05, cutoff=10.0, seed=1,
              astroid=(0.28, 1.0, 4.8, 3.0))
    sim, S = _pair(B, oracle, I.PINWHEEL, 16, 16, criterion=1, precision=prec, **kw)
    K = 300
    h = -0.2 + 0.4 * np.arange(K) / (K - 1)
    a = math.radians(angle)
    hx, hy = h * math.cos(a), h * math.sin(a)
    ref = S.run(np.ones(S.n, dtype=np.int8), hx, hy)
    got = sim.run_protocol(hx, hy)
    _same(got, ref)
    _, S5 = _pair(B, oracle, I.PINWHEEL, 16, 16, criterion=0, **kw)
    assert S5.run(np.ones(S.n, dtype=np.int8), hx, hy)["hash"] != ref["hash"]
    # the LHS it ranks by
    sim.set_spins(I.random_spins(sim.n, 3))
    sim.set_field(float(hx[200]), float(hy[200]), step=0)
    hp, hq = sim.fields()
    if prec == FP64:
        np.testing.assert_allclose(sim.lhs(), np.abs(hp) / sim.hk(), rtol=4e-16)


# ---------------------------------------------------------------------------
# Local and spatial external fields, encoders
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("resweep", [True, False])
def test_local_field_series_matches_oracle(B, oracle, prec, resweep):
    """A kagome array with thermal noise under a rotating global field plus a local
    field: a spatial gradient along x that changes with time."""
    sim, S = _pair(B, oracle, I.KAGOME, 10, 10, alpha=8e-4, cutoff=4.0, kdis=0.08, seed=2,
                   sigma=0.004, precision=prec)
    K = 90
    hx, hy = I.rotation_protocol(K, 4.0, 0.09)
    x, _, _ = sim.geometry_arrays()
    g = (x - x.mean()) / (x.max() - x.min())
    lhx = 0.04 * np.outer(np.sin(np.arange(K) / 9.0), g)
    lhy = 0.03 * np.outer(np.cos(np.arange(K) / 7.0), g ** 2)
    sim.set_field_local(lhx, lhy)
    ref = S.run(np.ones(S.n, dtype=np.int8), hx, hy, lhx=lhx, lhy=lhy)
    got = sim.run_protocol(hx, hy, resweep=resweep)
    assert ref["n_flips"] > 100
    _same(got, ref)
    # the fields at one step, with the local part
    s = I.random_spins(sim.n, 8)
    sim.set_spins(s)
    sim.set_field(float(hx[40]), float(hy[40]), step=40)
    hp, hq = sim.fields()
    op, oq = S.fields(s, float(hx[40]), float(hy[40]), step=40, lx=lhx[40], ly=lhy[40])
    scale = max(np.abs(op).max(), np.abs(oq).max())
    tol = 1e-12 if prec == FP64 else 1e-5
    assert max(np.abs(hp - op).max(), np.abs(hq - oq).max()) <= tol * scale
    # without the series the same protocol is a different one
    sim.set_field_local(np.zeros((0, 0)), np.zeros((0, 0)))
    sim.set_spins(np.ones(sim.n, dtype=np.int8))
    assert sim.run_protocol(hx, hy)["hash"] != ref["hash"]


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_spatial_field_matches_oracle(B, oracle, prec):
    sim, S = _pair(B, oracle, I.PINWHEEL, 14, 14, cutoff=5.0, seed=4, precision=prec)
    K, gw, gh = 120, 4, 3
    h = np.linspace(-0.3, 0.3, K)
    w = np.linspace(0.6, 1.4, gw * gh).reshape(gh, gw)
    gx = h[:, None, None] * w[None] * math.cos(math.radians(25.0))
    gy = h[:, None, None] * w[None, ::-1, ::-1] * math.sin(math.radians(25.0))
    x0, y0, dx, dy = 0.5, -0.2, 3.7, 4.9
    sim.set_field_spatial(gx, gy, x0, y0, dx, dy)
    xs, ys, _ = oracle.geometry(I.PINWHEEL, 14, 14)
    lx, ly = oracle.sample_grid(xs, ys, gw, gh, x0, y0, dx, dy, gx, gy)
    zero = np.zeros(K)
    ref = S.run(np.ones(S.n, dtype=np.int8), zero, zero, lhx=lx, lhy=ly)
    got = sim.run_protocol(zero, zero)
    assert ref["n_flips"] > S.n
    _same(got, ref)


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_encoded_protocol_matches_oracle(B, oracle, prec):
    """Inputs through the sawtooth and sinusoid encoders drive a square array."""
    sim, S = _pair(B, oracle, I.SQUARE, 12, 12, seed=9, precision=prec)
    u = np.array([0.2, 0.9, 0.5, 1.0])
    ax, ay = B.encode(B.FS_ENCODE_SAWTOOTH, u, 30, 0.15, 0.35, 40.0)
    bx, by = B.encode(B.FS_ENCODE_SINUSOID, u[::-1], 24, 0.1, 0.3, 220.0)
    hx, hy = np.concatenate([ax, bx]), np.concatenate([ay, by])
    ox = np.concatenate([oracle.encode(1, u, 30, 0.15, 0.35, 40.0)[0],
                         oracle.encode(0, u[::-1], 24, 0.1, 0.3, 220.0)[0]])
    ref = S.run(np.ones(S.n, dtype=np.int8), hx, hy)
    got = sim.run_protocol(hx, hy)
    np.testing.assert_allclose(hx, ox, rtol=2e-16, atol=1e-17)
    assert ref["n_flips"] > S.n
    _same(got, ref)


def test_series_shorter_than_the_protocol_is_rejected(B):
    sim = B.Sim.geometry(I.SQUARE, 4, 4)
    sim.set_params(B.make_params(alpha=1e-3, sigma_th=0.01))
    sim.set_field_local(np.zeros((5, sim.n)), np.zeros((5, sim.n)))
    with pytest.raises(B.FsError) as e:
        sim.run_protocol(np.zeros(6), np.zeros(6))
    assert e.value.code == B.FS_ERR_INVALID
    sim.run_protocol(np.zeros(3), np.zeros(3), step0=2)  # steps 2..4: inside
    sim.set_sigma_series([0.01, 0.0])
    with pytest.raises(B.FsError):
        sim.run_protocol(np.zeros(3), np.zeros(3))
    cold = B.Sim.geometry(I.SQUARE, 4, 4)
    cold.set_params(B.make_params(alpha=1e-3))
    with pytest.raises(B.FsError) as e:
        cold.set_sigma_series([0.01])
    assert e.value.code == B.FS_ERR_STATE


def test_batch_members_with_local_fields(B, oracle):
    hx, hy = I.ramp_protocol(60, 45.0, 0.3)
    K = len(hx)
    sims, refs = [], []
    for q, n in enumerate((5, 9, 7)):
        sim, S = _pair(B, oracle, I.SQUARE, n, n, seed=30 + q, precision=FP32)
        lhx = 0.02 * np.outer(np.ones(K), np.linspace(-1, 1, sim.n)) * (q + 1)
        sim.set_field_local(lhx, np.zeros_like(lhx))
        sims.append(sim)
        refs.append(S.run(np.ones(S.n, dtype=np.int8), hx, hy, lhx=lhx, lhy=np.zeros_like(lhx)))
    # the persistent schedule takes no local fields; the default falls back to per step
    with pytest.raises(B.FsError) as e:
        B.batch_run_protocol(sims, hx, hy, schedule=B.FS_BATCH_PERSISTENT)
    assert e.value.code == B.FS_ERR_INVALID
    out = B.batch_run_protocol(sims, hx, hy)
    for q, ref in enumerate(refs):
        assert int(out["hash"][q]) == ref["hash"] and int(out["n_flips"][q]) == ref["n_flips"]


# ---------------------------------------------------------------------------
# Annealing and the spin-spin correlation
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", [FP64, FP32])
def test_annealing_and_correlation_match_oracle(B, oracle, prec):
    """The domain-size study's protocol on a 24 x 24 square array (its astroid
    b = 0.4, c = 1, beta = gamma = 3, h_k 0.186, k_disorder 0.05): an exponentially
    decreasing thermal field at zero external field, every flip as the oracle's, and
    the correlation of the annealed state bin for bin."""
    kw = dict(alpha=0.0025, hk=0.186, kdis=0.05, cutoff=4.0, seed=7, sigma=0.2,
              astroid=(0.4, 1.0, 3.0, 3.0))
    sim, S = _pair(B, oracle, I.SQUARE, 24, 24, precision=prec, **kw)
    K = 140
    sig = 0.2 * 0.95 ** np.arange(K)
    sim.set_sigma_series(sig)
    zero = np.zeros(K)
    ref = S.run(np.ones(S.n, dtype=np.int8), zero, zero, sigma=sig)
    got = sim.run_protocol(zero, zero)
    assert ref["n_flips"] > S.n
    _same(got, ref)
    final = sim.spins()
    np.testing.assert_array_equal(final, ref["spins"])
    cnt, sm = sim.correlation(10.0, 0.5, 20)
    x, y, th = oracle.geometry(I.SQUARE, 24, 24)
    ocnt, osm = oracle.correlation(x, y, th, final, 10.0, 0.5, 20)
    np.testing.assert_array_equal(cnt, ocnt)
    np.testing.assert_array_equal(sm, osm)
    c = np.abs(sm[1]) / cnt[1]
    assert c > 0.5  # the annealed state is ordered at short range


@pytest.mark.parametrize("kind,n,rmax,w,nb", [(I.KAGOME, 12, 6.0, 0.25, 24),
                                               (I.PINWHEEL, 15, 9.5, 0.5, 19),
                                               (6, 30, 12.0, 0.1, 121),
                                               (3, 20, 3.0, 1.0, 3)])
def test_correlation_matches_oracle(B, oracle, kind, n, rmax, w, nb):
    sim = B.Sim.geometry(kind, n, n)
    sim.set_params(B.make_params(alpha=1e-3))
    for seed in (1, 2):
        s = I.random_spins(sim.n, seed)
        sim.set_spins(s)
        cnt, sm = sim.correlation(rmax, w, nb)
        x, y, th = oracle.geometry(kind, n, n)
        ocnt, osm = oracle.correlation(x, y, th, s, rmax, w, nb)
        np.testing.assert_array_equal(cnt, ocnt)
        np.testing.assert_array_equal(sm, osm)
        assert cnt.sum() > 0
