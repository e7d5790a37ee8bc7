"""The FP32 error model under stress (Sec. "Switching", Eq. 5 and 6).

Both precision paths rest on the FP32 bounds: FS_FP32_RECHECK takes a pick from
them when they separate the winner from every other island, and FS_FP64 uses
them as a prefilter that decides which islands get an FP64 evaluation at all.
A bound that is too narrow shows up as a flip order that differs from the FP64
oracle's. These systems are built to sit where the bounds are tightest:

- strong fields on small coercive fields, so that the astroid terms are large
  (LHS 5 to 50) and the FP32 exponent's rounding, |p - (float)p| |ln x|, is a
  sizeable part of the error;
- coercive fields a few parts in 1e8 apart, so that many pairs of FP64 LHS values
  lie 0 to 3 FP32 ulps apart, and exact FP64 ties among them;
- islands within a few parts in 1e8 of the threshold LHS = 1;
- the paper's four astroid parameter sets (Stoner-Wohlfarth and the fitted ones of
  Sec. "Switching" and the pinwheel and switching-order sections).

The islands are 10 lattice spacings apart with a cutoff of 1, so none interact
and the oracle's flip order is the order of the exact values; every flip is
compared with the oracle's, on both paths.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FP64, FP32 = 0, 1
U = 2.0**-24
ASTROIDS = [(1.0, 1.0, 3.0, 3.0), (0.28, 1.0, 4.8, 3.0), (0.42, 1.0, 1.7, 3.4),
            (0.38, 1.0, 1.5, 3.2)]


@pytest.fixture(scope="module")
def B():
    from paper_2002_11401_b300 import build
    build.build()
    from paper_2002_11401_b300 import binding
    return binding


def _near_tie_system(seed, n=240, hk0=1e-3):
    """Positions, angles and coercive fields of non-interacting islands in six angle
    classes, h_k = hk0 (1 + k 3e-8) with k in 0..11 (ties included)."""
    rng = np.random.default_rng(seed)
    x = np.arange(n, dtype=np.float64) * 10.0
    y = np.zeros(n)
    classes = np.array([0.0, 0.3, 0.7, 1.1, 1.6, 2.5])
    th = classes[np.arange(n) % len(classes)]
    k = rng.integers(0, 12, size=n)
    hk = hk0 * (1.0 + k * 3e-8)
    return x, y, th, hk


def _strong_protocol():
    """Alternating field directions, magnitudes from 4 to 80 h_k: every step flips
    every flippable island, in order of its LHS (about 3 to 30 for the
    Stoner-Wohlfarth astroid, more for the others)."""
    mags = np.array([0.004, 0.01, 0.03, 0.08, 0.08, 0.05, 0.02])
    phi = math.radians(200.0) + math.pi * np.arange(len(mags))
    return mags * np.cos(phi), mags * np.sin(phi)


def _run_both(B, oracle, x, y, th, hk, astroid, sigma, hx, hy, seed):
    b, c, beta, gamma = astroid
    S = oracle.Sim(x, y, th, hk, alpha=1e-3, b=b, c=c, beta=beta, gamma=gamma,
                   sigma_th=sigma, cutoff_abs=1.0, seed=seed)
    ref = S.run(np.ones(len(x), dtype=np.int8), hx, hy)
    assert ref["status"] == 0
    for prec in (FP64, FP32):
        sim = B.Sim.custom(x, y, th)
        sim.set_params(B.make_params(alpha=1e-3, b=b, c=c, beta=beta, gamma=gamma,
                                     cutoff=1.0, sigma_th=sigma, seed=seed, precision=prec))
        sim.set_hk(hk)
        got = sim.run_protocol(hx, hy, log_cap=max(ref["n_flips"], 1))
        assert got["status"] == 0
        assert got["n_flips"] == ref["n_flips"], prec
        np.testing.assert_array_equal(got["log_step"], ref["log_step"])
        np.testing.assert_array_equal(got["log_spin"], ref["log_spin"])
        assert got["hash"] == ref["hash"]
        np.testing.assert_array_equal(sim.spins(), ref["spins"])
        sim.close()
    return ref


@pytest.mark.parametrize("sigma", [0.0, 1e-9])
@pytest.mark.parametrize("astroid", ASTROIDS)
def test_near_ties_at_large_lhs_match_oracle(B, oracle, astroid, sigma):
    x, y, th, hk = _near_tie_system(seed=17)
    hx, hy = _strong_protocol()
    ref = _run_both(B, oracle, x, y, th, hk, astroid, sigma, hx, hy, seed=5)
    # the large-LHS regime is reached: check the oracle's values on one step
    S = oracle.Sim(x, y, th, hk, alpha=1e-3, b=astroid[0], c=astroid[1], beta=astroid[2],
                   gamma=astroid[3], cutoff_abs=1.0)
    hp, hq = S.fields(np.ones(len(x), dtype=np.int8), hx[3], hy[3])
    lhs = np.array([oracle.astroid_lhs(hp[i], hq[i], hk[i], *astroid) for i in range(len(x))])
    assert lhs.max() > 20.0
    assert ref["n_flips"] >= len(x)
    # many pairs of values lie within three FP32 ulps of each other, some tie exactly
    v = np.sort(lhs)
    gap = np.diff(v) / v[1:]
    assert int(((gap > 0) & (gap <= 3 * 2.0**-23)).sum()) >= 20
    assert int((gap == 0).sum()) >= 20


@pytest.mark.parametrize("astroid", ASTROIDS)
def test_threshold_within_a_few_ulps_matches_oracle(B, oracle, astroid):
    """Islands along x, a field along -x: LHS = (|h| / (b h_k))^(2/gamma) with
    h_k = |h| / b (1 + k 1e-8), k in -6..6 without 0, i.e. within a few FP32 ulps
    of one on either side; only those below it flip, largest first."""
    b, c, beta, gamma = astroid
    n = 96
    rng = np.random.default_rng(3)
    x = np.arange(n, dtype=np.float64) * 10.0
    y = np.zeros(n)
    th = np.zeros(n)
    k = rng.integers(1, 7, size=n) * rng.choice([-1, 1], size=n)
    h = 0.1
    hk = h / b * (1.0 + k * 1e-8)
    hx = np.array([-h])
    hy = np.array([0.0])
    ref = _run_both(B, oracle, x, y, th, hk, astroid, 0.0, hx, hy, seed=1)
    assert ref["n_flips"] == int((k < 0).sum())


@pytest.mark.parametrize("astroid", ASTROIDS)
def test_bounds_bracket_fp64_at_large_lhs(B, astroid):
    """[lo, hi] of the FP32 evaluation contains the FS_FP64 LHS on interacting
    arrays with small coercive fields (LHS up to ~50) and thermal noise."""
    from paper_2002_11401_b300 import inputs as I
    from .helpers import lib_sim, small
    b, c, beta, gamma = astroid
    w = small(I.KAGOME, 10, b=b, c=c, beta=beta, gamma=gamma, sigma_th=0.002, alpha=4e-3)
    s32 = lib_sim(w, precision=FP32)
    s64 = lib_sim(w, precision=FP64)
    rng = np.random.default_rng(11)
    hk = s64.hk() * rng.choice([1.0, 0.1, 0.02, 0.005], size=s64.n)
    s32.set_hk(hk)
    s64.set_hk(hk)
    top = 0.0
    for trial in range(10):
        s = I.random_spins(s32.n, 40 + trial)
        ang = rng.uniform(0, 2 * math.pi)
        mag = [0.05, 0.2, 0.4][trial % 3]
        for sim in (s32, s64):
            sim.set_spins(s)
            sim.set_field(mag * math.cos(ang), mag * math.sin(ang), step=trial)
        _, lo, hi = s32.lhs(bounds=True)
        l64 = s64.lhs()
        assert (lo <= l64).all() and (l64 <= hi).all(), trial
        top = max(top, float(l64.max()))
    assert top > 20.0
