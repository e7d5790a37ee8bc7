"""The multi-flip relax (FS_RELAX_MULTI, FS_RELAX_MULTI_CTA) against the FP64
oracle, flip for flip.

A round flips several of the islands with the largest LHS at once, as long as
each is the island the single-flip relax of Sec. "Dynamics" takes next (its exact
value beats everything outside the round, it lies more than twice the cutoff from
the round's earlier islands, and no earlier flip's neighbour overtakes it). The
flip sequence, the flips per field step, the hash and the final spins must equal
the oracle's: the same cases as the single-flip path's parity tests, forced into
the multi-flip mode, plus ties that overflow a round's candidate set.
"""
import math

import numpy as np
import pytest

from paper_2002_11401_b300 import inputs as I

from .helpers import first_divergence, lib_sim, oracle_sim, small

pytestmark = pytest.mark.gpu

FP64, FP32 = 0, 1


@pytest.fixture(scope="module")
def B():
    from paper_2002_11401_b300 import build
    build.build()
    from paper_2002_11401_b300 import binding
    return binding


def _multi(B, w, prec, mode=None, **over):
    sim = lib_sim(w, precision=prec, **over)
    sim.set_relax_mode(B.FS_RELAX_MULTI if mode is None else mode)
    return sim


def _compare(B, oracle, w, hx, hy, precs=(FP64, FP32), resweeps=(True,), **over):
    S = oracle_sim(oracle, w, **over)
    ref = S.run(np.ones(S.n, dtype=np.int8), hx, hy)
    assert ref["status"] == 0
    # the rounds on a cluster of CTAs, and on one CTA (the build that runs where a
    # cluster does not fit)
    for mode in (B.FS_RELAX_MULTI, B.FS_RELAX_MULTI_CTA):
        for prec in precs:
            for rs in resweeps:
                _check_one(B, w, hx, hy, ref, prec, rs, mode, **over)
    return ref


def _check_one(B, w, hx, hy, ref, prec, rs, mode, **over):
    sim = _multi(B, w, prec, mode, **over)
    got = sim.run_protocol(hx, hy, resweep=rs)
    d = first_divergence(ref["log_step"], ref["log_spin"], got["log_step"], got["log_spin"])
    assert d is None, (mode, prec, rs, d, ref["ties"])
    assert (got["n_flips"], got["hash"]) == (ref["n_flips"], ref["hash"])
    np.testing.assert_array_equal(got["flips_per_step"], ref["flips_per_step"])
    np.testing.assert_array_equal(sim.spins(), ref["spins"])
    sim.close()


def test_square16_sequence(B, oracle):
    w = I.WORKLOADS["square16"]
    hx, hy = I.protocol_of(w["protocol"])
    ref = _compare(B, oracle, w, hx, hy, resweeps=(True, False))
    assert ref["n_flips"] == 1088


@pytest.mark.parametrize("case", range(8))
def test_small_systems_sequences(B, oracle, case):
    rng = np.random.default_rng(2000 + case)
    kind = [I.SQUARE, I.PINWHEEL, I.KAGOME][case % 3]
    astroids = [(1, 1, 3, 3), (0.28, 1, 4.8, 3), (0.42, 1, 1.7, 3.4), (0.38, 1, 1.5, 3.2)]
    b, c, beta, gamma = astroids[case % 4]
    n = int(rng.integers(8, 20))
    sigma = 0.004 if case % 2 else 0.0
    w = small(kind, n, b=b, c=c, beta=beta, gamma=gamma, sigma_th=sigma, seed=case,
              alpha=[1e-3, 3e-3, 1e-2][case % 3], k_disorder=[0.05, 0.1, 0.02][case % 3])
    hmax = 0.35 if b >= 1 else 0.2
    proto = [I.ramp_protocol(50, float(rng.uniform(0, 360)), hmax),
             I.rotation_protocol(50, 7.0, hmax * 0.6),
             I.loop_protocol(50, float(rng.uniform(0, 360)), -hmax, hmax)][case % 3]
    _compare(B, oracle, w, *proto, resweeps=(True, False))


def test_pinwheel_mid_size(B, oracle):
    w = small(I.PINWHEEL, 60, seed=1)
    hx, hy = I.loop_protocol(120, 30.0, -0.25, 0.25)
    _compare(B, oracle, w, hx, hy)


def test_kagome_thermal_mid_size(B, oracle):
    w = small(I.KAGOME, 70, sigma_th=0.005, k_disorder=0.08, seed=2)
    hx, hy = I.rotation_protocol(100, 3.0, 0.11)
    ref = _compare(B, oracle, w, hx, hy)
    assert ref["n_flips"] > 10_000


@pytest.mark.parametrize("angle", [0.0, 30.0])
def test_pinwheel_reversal_with_the_papers_parameters(B, oracle, angle):
    w = small(I.PINWHEEL, 24, alpha=0.00033, hk=0.098, k_disorder=0.05, cutoff=10.0, b=0.28,
              c=1.0, beta=4.8, gamma=3.0, seed=1)
    K = 300
    h = -0.06 + 0.12 * np.arange(K) / (K - 1)
    a = math.radians(angle)
    _compare(B, oracle, w, h * math.cos(a), h * math.sin(a))


@pytest.mark.parametrize("n", [70, 400, 1500])
def test_exact_ties(B, n):
    # identical islands out of each other's reach: every pick ties with all the
    # others, lowest index first; 1500 of them overflow a round's candidate set
    x = np.arange(n, dtype=np.float64) * 10.0
    for prec in (FP64, FP32):
        sim = B.Sim.custom(x, np.zeros(n), np.zeros(n))
        sim.set_params(B.make_params(alpha=0.0, cutoff=1.0, precision=prec))
        sim.set_relax_mode(B.FS_RELAX_MULTI)
        sim.set_hk(np.full(n, 0.2))
        got = sim.run_protocol(np.array([-0.3, 0.3]), np.zeros(2), log_cap=2 * n)
        assert got["status"] == 0
        assert got["log_spin"].tolist() == list(range(n)) * 2


def test_flip_guard(B):
    w = small(I.SQUARE, 6, max_flips_per_step=5)
    sim = _multi(B, w, FP64)
    got = sim.run_protocol(np.array([-0.4]), np.array([-0.4]))
    assert got["status"] == B.FS_ERR_NOT_CONVERGED
    assert got["n_flips"] == 5


def test_resume_relax_and_short_log(B, oracle):
    w = small(I.KAGOME, 16, sigma_th=0.01)
    hx, hy = I.rotation_protocol(60, 6.0, 0.12)
    S = oracle_sim(oracle, w)
    ref = S.run(np.ones(S.n, dtype=np.int8), hx, hy)
    for prec in (FP64, FP32):
        a = _multi(B, w, prec)
        r1 = a.run_protocol(hx[:25], hy[:25], log_cap=7)
        b = _multi(B, w, prec)
        b.set_spins(a.spins())
        r2 = b.run_protocol(hx[25:], hy[25:], step0=25, hash_in=r1["hash"])
        assert r2["hash"] == ref["hash"]
        np.testing.assert_array_equal(r1["log_spin"], ref["log_spin"][:7])
        c = _multi(B, w, prec)
        c.set_field(float(hx[0]), float(hy[0]), step=0)
        nf, log = c.relax(log_cap=100)
        assert nf == ref["flips_per_step"][0]
        np.testing.assert_array_equal(log[:100], ref["log_spin"][:min(nf, 100)])


def test_with_local_field_and_annealing(B, oracle):
    w = small(I.SQUARE, 30, alpha=0.0025, hk=0.186, cutoff=4.0, seed=7, b=0.4, sigma_th=0.2)
    K = 80
    sig = 0.2 * 0.93 ** np.arange(K)
    x, _, _ = oracle.geometry(I.SQUARE, 30, 30)
    lhx = 0.01 * np.outer(np.ones(K), np.sin(x / 5.0))
    zero = np.zeros(K)
    S = oracle_sim(oracle, w)
    ref = S.run(np.ones(S.n, dtype=np.int8), zero, zero, lhx=lhx, lhy=np.zeros_like(lhx),
                sigma=sig)
    for prec in (FP64, FP32):
        sim = _multi(B, w, prec)
        sim.set_sigma_series(sig)
        sim.set_field_local(lhx, np.zeros_like(lhx))
        got = sim.run_protocol(zero, zero)
        assert (got["n_flips"], got["hash"]) == (ref["n_flips"], ref["hash"])
