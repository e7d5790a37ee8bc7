"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, a value printed in the paper, a brute-force enumeration, an invariant,
or an independent third-party implementation. A plausible slip in the oracle
(a dropped term, a wrong sign, swapped exponents, a wrong index) fails one.
"""
import math

import numpy as np
import pytest

from paper_2002_11401_b300 import inputs as I

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


# ---------------------------------------------------------------------------
# Eq. (3): the point-dipole field
# ---------------------------------------------------------------------------

def test_dipole_head_to_tail(oracle):
    # r parallel to m: h = 2 alpha / d^3 along m (Sec. "Magnetic dipole-dipole interactions").
    for d in (0.5, 1.0, 1.7, 3.0):
        hx, hy = oracle.dipole_field(d, 0.0, 1.0, 0.0, 1e-3)
        assert hx == pytest.approx(2e-3 / d**3, rel=1e-15)
        assert hy == 0.0


def test_dipole_side_by_side(oracle):
    # r perpendicular to m: h = -alpha / d^3 along m.
    for d in (0.5, 1.0, 2.5):
        hx, hy = oracle.dipole_field(0.0, d, 1.0, 0.0, 1e-3)
        assert hx == pytest.approx(-1e-3 / d**3, rel=1e-15)
        assert abs(hy) < 1e-30


def test_dipole_polar_closed_form(oracle):
    # Textbook polar form: radial 2 cos(psi - rho) / d^3, azimuthal -sin(psi - rho) / d^3,
    # for a moment at angle psi seen from direction rho at distance d.
    rng = np.random.default_rng(7)
    for _ in range(200):
        d = rng.uniform(0.3, 6.0)
        rho = rng.uniform(-math.pi, math.pi)
        psi = rng.uniform(-math.pi, math.pi)
        alpha = rng.uniform(1e-4, 1e-2)
        hr = 2.0 * math.cos(psi - rho) * alpha / d**3
        hphi = -math.sin(psi - rho) * alpha / d**3
        ex = hr * math.cos(rho) - hphi * math.sin(rho)
        ey = hr * math.sin(rho) + hphi * math.cos(rho)
        hx, hy = oracle.dipole_field(d * math.cos(rho), d * math.sin(rho), math.cos(psi),
                                     math.sin(psi), alpha)
        scale = alpha / d**3
        assert abs(hx - ex) <= 1e-13 * scale
        assert abs(hy - ey) <= 1e-13 * scale


def test_two_island_system_field(oracle):
    # Superposition in a two-island system: the total field equals the closed-form
    # pair field of the other island plus the external field, projected on the frame.
    x = np.array([0.0, 1.3])
    y = np.array([0.0, 0.4])
    th = np.array([0.3, 1.9])
    hk = np.array([0.2, 0.2])
    S = oracle.Sim(x, y, th, hk, alpha=2e-3, cutoff_abs=5.0)
    s = np.array([1, -1], dtype=np.int8)
    hp, hq = S.fields(s, 0.01, -0.02)
    for i, j in ((0, 1), (1, 0)):
        rx, ry = x[i] - x[j], y[i] - y[j]
        d = math.hypot(rx, ry)
        rho = math.atan2(ry, rx)
        psi = th[j] + (math.pi if s[j] < 0 else 0.0)
        hr = 2.0 * math.cos(psi - rho) * 2e-3 / d**3
        hphi = -math.sin(psi - rho) * 2e-3 / d**3
        ex = hr * math.cos(rho) - hphi * math.sin(rho) + 0.01
        ey = hr * math.sin(rho) + hphi * math.cos(rho) - 0.02
        par = ex * math.cos(th[i]) + ey * math.sin(th[i])
        perp = -ex * math.sin(th[i]) + ey * math.cos(th[i])
        assert hp[i] == pytest.approx(par, abs=1e-15)
        assert hq[i] == pytest.approx(perp, abs=1e-15)


# ---------------------------------------------------------------------------
# Eq. (4)-(6): switching astroid
# ---------------------------------------------------------------------------

def _threshold(oracle, phi, hk, b, c, beta, gamma):
    """Field magnitude at which Eq. (5) reaches 1 for a field at angle phi from the
    easy axis (bisection on the oracle's left-hand side)."""
    ux = 0.0 if phi == math.pi / 2 else math.cos(phi)
    uy = math.sin(phi)
    lo, hi = 0.0, 10.0 * hk
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        L = oracle.astroid_lhs(mid * ux, mid * uy, hk, b, c, beta, gamma)
        if L > 1.0:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def test_sw_astroid_reduction(oracle):
    # b = c = 1, beta = gamma = 3 gives the Stoner-Wohlfarth astroid, Eq. (4): the
    # switching field is h_k along the easy axis and h_k / 2 at 45 degrees.
    hk = 0.2
    assert _threshold(oracle, 0.0, hk, 1, 1, 3, 3) == pytest.approx(hk, rel=1e-12)
    assert _threshold(oracle, math.pi / 4, hk, 1, 1, 3, 3) == pytest.approx(hk / 2, rel=1e-12)


def test_sw_astroid_closed_form_curve(oracle):
    # h_sw(phi) = h_k / (|cos phi|^(2/3) + |sin phi|^(2/3))^(3/2), every degree.
    hk = 0.2
    for deg in range(0, 90):
        phi = math.radians(deg)
        expect = hk / (abs(math.cos(phi)) ** (2 / 3) + abs(math.sin(phi)) ** (2 / 3)) ** 1.5
        assert _threshold(oracle, phi, hk, 1, 1, 3, 3) == pytest.approx(expect, rel=1e-11)


def test_generalised_astroid_axes(oracle):
    # Eq. (5): b scales the easy-axis threshold, c the hard-axis one.
    hk, b, c = 0.098, 0.28, 1.0
    assert _threshold(oracle, 0.0, hk, b, c, 4.8, 3.0) == pytest.approx(b * hk, rel=1e-12)
    assert _threshold(oracle, math.pi / 2, hk, 0.4, 0.7, 4.8, 3.0) == pytest.approx(0.7 * hk,
                                                                                  rel=1e-12)


def test_generalised_astroid_exponents_as_printed(oracle):
    # Eq. (5) puts 2/gamma on the parallel term and 2/beta on the perpendicular one.
    # b = 0.5, c = 1, beta = 2, gamma = 4, h_par = h_perp = 0.1, h_k = 0.2:
    # (0.1/0.1)^(1/2) + (0.1/0.2)^1 = 1.5 (swapped exponents would give 1 + 0.5^0.5).
    L = oracle.astroid_lhs(0.1, 0.1, 0.2, 0.5, 1.0, 2.0, 4.0)
    assert L == pytest.approx(1.5, rel=1e-15)
    # and the sign of each component does not matter (fractional powers of |h|)
    assert oracle.astroid_lhs(-0.1, -0.1, 0.2, 0.5, 1.0, 2.0, 4.0) == L


def test_astroid_lhs_against_high_precision(oracle):
    # Eq. (5) on random fields, coercive fields and the paper's four astroids, against
    # a 60-digit evaluation (mpmath, an independent implementation of the powers):
    # the oracle's FP64 value is within a few ulps of the exact one.
    import mpmath
    mpmath.mp.dps = 60
    rng = np.random.default_rng(7)
    shapes = [(1.0, 1.0, 3.0, 3.0), (0.28, 1.0, 4.8, 3.0), (0.42, 1.0, 1.7, 3.4),
              (0.38, 1.0, 1.5, 3.2)]
    for b, c, beta, gamma in shapes:
        for _ in range(200):
            hp, hq = rng.normal(0.0, 0.15, 2)
            hk = float(rng.uniform(0.05, 0.3))
            got = oracle.astroid_lhs(hp, hq, hk, b, c, beta, gamma)
            B_, C_, K_ = mpmath.mpf(b), mpmath.mpf(c), mpmath.mpf(hk)
            exact = (abs(mpmath.mpf(hp)) / (B_ * K_)) ** (2 / mpmath.mpf(gamma)) + \
                (abs(mpmath.mpf(hq)) / (C_ * K_)) ** (2 / mpmath.mpf(beta))
            assert abs(got - float(exact)) <= 8 * np.spacing(float(exact)), (b, hp, hq, hk)


def test_antialignment_condition(oracle):
    # Eq. (6): a field outside the astroid switches only when h . m_i < 0.
    assert oracle.flippable(+1, -0.3, 2.0)
    assert not oracle.flippable(+1, +0.3, 2.0)
    assert oracle.flippable(-1, +0.3, 2.0)
    assert not oracle.flippable(-1, -0.3, 2.0)
    # a purely perpendicular field never switches (h_par = 0), however strong
    assert not oracle.flippable(+1, 0.0, 100.0)
    # strictly greater than one
    assert not oracle.flippable(+1, -0.3, 1.0)


# ---------------------------------------------------------------------------
# Geometry (Sec. "Geometries")
# ---------------------------------------------------------------------------

def test_kagome_count_printed_in_paper(oracle):
    # 29 x 29 hexagons hold 2638 islands (Sec. "Dirac strings in kagome ASI").
    x, _, _ = oracle.geometry(I.KAGOME, 29, 29)
    assert len(x) == 2638


@pytest.mark.parametrize("n,m", [(1, 1), (2, 3), (5, 4), (10, 10), (7, 12)])
def test_kagome_count_formula(oracle, n, m):
    x, y, t = oracle.geometry(I.KAGOME, n, m)
    assert len(x) == 3 * n * m + 2 * n + 2 * m - 1
    deg = np.round(np.degrees(t)).astype(int)
    assert set(deg.tolist()) <= {0, 60, 120}
    # no two islands share a position
    assert len(set(zip(np.round(x, 9), np.round(y, 9)))) == len(x)


@pytest.mark.parametrize("n", [1, 2, 3, 16, 25])
def test_square_and_pinwheel_counts(oracle, n):
    xs, ys, ts = oracle.geometry(I.SQUARE, n, n)
    xp, yp, tp = oracle.geometry(I.PINWHEEL, n, n)
    assert len(xs) == 2 * n * (n + 1)
    np.testing.assert_array_equal(xs, xp)
    np.testing.assert_array_equal(ys, yp)
    # pinwheel: every square island turned 45 degrees about its centre
    np.testing.assert_allclose(np.degrees(tp) - np.degrees(ts), 45.0, atol=1e-12)
    assert set(np.round(np.degrees(ts)).astype(int).tolist()) <= {0, 90}


def test_canonical_order(oracle):
    for kind in (I.SQUARE, I.KAGOME):
        x, y, _ = oracle.geometry(kind, 9, 7)
        key = list(zip(y.tolist(), x.tolist()))
        assert key == sorted(key)


def test_square_closed_edges_cell_has_four_islands(oracle):
    # Closed edges: each of the n x n cells is bounded by four islands.
    n = 6
    x, y, t = oracle.geometry(I.SQUARE, n, n)
    pos = set(zip((2 * x).round().astype(int).tolist(), (2 * y).round().astype(int).tolist()))
    for cx in range(n):
        for cy in range(n):
            X, Y = 2 * cx + 1, 2 * cy + 1  # cell centre in half spacings
            for dx, dy in ((0, -1), (0, 1), (-1, 0), (1, 0)):
                assert (X + dx, Y + dy) in pos


# ---------------------------------------------------------------------------
# Neighbourhoods
# ---------------------------------------------------------------------------

def test_eight_spin_neighbourhood(oracle):
    # Sec. "Performance": square ASI with the standard 8-spin neighbourhood, i.e. a
    # cutoff of one lattice spacing that includes the islands exactly at distance 1.
    x, y, _ = oracle.geometry(I.SQUARE, 12, 12)
    rp, _ = oracle.neighbors(x, y, 1.0)
    deg = np.diff(rp)
    assert deg.max() == 8
    interior = (x > 2) & (x < 10) & (y > 2) & (y < 10)
    assert (deg[interior] == 8).all()


@pytest.mark.parametrize("kind,n,rc", [(I.SQUARE, 10, 3.0), (I.PINWHEEL, 12, 5.0),
                                       (I.KAGOME, 8, 4.0), (I.SQUARE, 7, 1.0)])
def test_cell_grid_equals_brute_force(oracle, kind, n, rc):
    x, y, _ = oracle.geometry(kind, n, n)
    rp1, c1 = oracle.neighbors(x, y, rc)
    rp2, c2 = oracle.neighbors(x, y, rc, brute=True)
    np.testing.assert_array_equal(rp1, rp2)
    np.testing.assert_array_equal(c1, c2)
    # symmetric neighbour relation, no self pairs, rows ascending
    pairs = set()
    for i in range(len(x)):
        row = c1[rp1[i]:rp1[i + 1]]
        assert (np.diff(row) > 0).all()
        assert i not in row
        pairs.update((i, int(j)) for j in row)
    assert all((j, i) in pairs for (i, j) in pairs)


def test_bulk_degrees_of_the_workloads(oracle):
    # Interior degrees, counted by brute force on smaller arrays of the same kind.
    for kind, n, rc, expect in ((I.SQUARE, 16, 3.0, 60), (I.PINWHEEL, 24, 5.0, 160),
                                (I.KAGOME, 20, 4.0, 62)):
        x, y, _ = oracle.geometry(kind, n, n)
        rp, _ = oracle.neighbors(x, y, rc, brute=True)
        assert np.diff(rp).max() == expect


# ---------------------------------------------------------------------------
# Philox4x32-10 and Box-Muller
# ---------------------------------------------------------------------------

_TRITON_PHILOX = r"""
import json, sys
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def kern(out_ptr, c0_ptr, c1_ptr, c2_ptr, c3_ptr, seed, N: tl.constexpr):
    o = tl.arange(0, N)
    a, b, c, d = tl.philox(seed, tl.load(c0_ptr + o), tl.load(c1_ptr + o),
                           tl.load(c2_ptr + o), tl.load(c3_ptr + o))
    tl.store(out_ptr + o * 4 + 0, a)
    tl.store(out_ptr + o * 4 + 1, b)
    tl.store(out_ptr + o * 4 + 2, c)
    tl.store(out_ptr + o * 4 + 3, d)

req = json.loads(sys.stdin.read())
ctrs = np.asarray(req["ctrs"], dtype=np.uint64).astype(np.uint32)
n = len(ctrs)
cols = [torch.from_numpy(ctrs[:, q].view(np.int32).copy()) for q in range(4)]
res = {}
for seed in req["seeds"]:
    out = torch.zeros(4 * n, dtype=torch.int32)
    kern[(1,)](out, *cols, seed, N=n)
    res[str(seed)] = out.numpy().view(np.uint32).reshape(n, 4).tolist()
print(json.dumps(res))
"""


def _triton_philox(ctrs, seeds):
    """Philox4x32-10 from Triton's own implementation, run by its CPU interpreter
    in a fresh process (the interpreter must be chosen before Triton loads)."""
    import json
    import os
    import subprocess
    import sys
    env = dict(os.environ, TRITON_INTERPRET="1")
    req = json.dumps({"ctrs": np.asarray(ctrs).tolist(), "seeds": list(seeds)})
    out = subprocess.run([sys.executable, "-c", _TRITON_PHILOX], input=req, env=env,
                         capture_output=True, text=True, timeout=600, check=True)
    res = json.loads(out.stdout.strip().splitlines()[-1])
    return {int(k): np.asarray(v, dtype=np.uint32) for k, v in res.items()}


def test_philox_against_independent_implementation(oracle):
    pytest.importorskip("triton")
    rng = np.random.default_rng(3)
    ctrs = rng.integers(0, 2**32, size=(16, 4), dtype=np.uint64).astype(np.uint32)
    ctrs[0] = 0
    seeds = (0, 1, 2**32 + 5, 0xDEADBEEFCAFEF00D)
    refs = _triton_philox(ctrs, seeds)
    for seed in seeds:
        ref = refs[seed]
        key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
        for q in range(len(ctrs)):
            np.testing.assert_array_equal(oracle.philox4x32_10(ctrs[q], key), ref[q])


def test_box_muller_normals(oracle):
    from scipy import stats
    tp, tq = oracle.thermal(200_000, 1.0, 11, 0, 3)
    for z in (tp, tq):
        assert abs(z.mean()) < 0.01
        assert abs(z.std() - 1.0) < 0.01
        assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(tp, tq)[0, 1]) < 0.01
    # the draw is a function of (seed, step, island): another step is another sample
    tp2, _ = oracle.thermal(1000, 1.0, 11, 0, 4)
    assert not np.allclose(tp[:1000], tp2)


def test_coercive_field_disorder(oracle):
    # Sec. "Imperfections and disorder": h_k^(i) ~ N(h_k, k_disorder h_k), positive.
    hk = oracle.draw_hk(200_000, 0.2, 0.05, 0)
    assert hk.min() > 0
    assert hk.mean() == pytest.approx(0.2, rel=2e-3)
    assert hk.std() == pytest.approx(0.01, rel=1e-2)
    # a huge spread forces redraws, which still yield positive fields
    wide = oracle.draw_hk(20_000, 0.2, 1.5, 9)
    assert wide.min() > 0


# ---------------------------------------------------------------------------
# Dynamics (Sec. "Dynamics")
# ---------------------------------------------------------------------------

def _brute_tables(x, y, th, hk, alpha, rc, b, c, beta, gamma, hex_, hey):
    """For every spin state of a tiny array: the next flip under the paper's rule
    (largest Eq. (5) left-hand side among islands satisfying Eq. (5) > 1 and Eq. (6),
    lowest index on ties), or -1. Fields from all pairs within the cutoff."""
    n = len(x)
    mx, my = np.cos(th), np.sin(th)
    rx = x[:, None] - x[None, :]
    ry = y[:, None] - y[None, :]
    r2 = rx * rx + ry * ry
    near = (r2 <= rc * rc * (1 + 1e-9)) & ~np.eye(n, dtype=bool)
    r = np.sqrt(np.where(near, r2, 1.0))
    states = ((np.arange(2**n)[:, None] >> np.arange(n)[None, :]) & 1) * 2 - 1  # [S, n]
    nxt = np.full(2**n, -1)
    for S in range(2**n):
        s = states[S]
        mjx, mjy = s * mx, s * my
        mr = mjx[None, :] * rx + mjy[None, :] * ry
        hx = alpha * np.where(near, 3 * rx * mr / r**5 - mjx[None, :] / r**3, 0).sum(1) + hex_
        hy = alpha * np.where(near, 3 * ry * mr / r**5 - mjy[None, :] / r**3, 0).sum(1) + hey
        hp = hx * mx + hy * my
        hq = -hx * my + hy * mx
        L = (np.abs(hp) / (b * hk)) ** (2 / gamma) + (np.abs(hq) / (c * hk)) ** (2 / beta)
        ok = (s * hp < 0) & (L > 1)
        if ok.any():
            cand = np.where(ok, L, -np.inf)
            nxt[S] = int(np.argmax(cand))  # argmax returns the lowest index on ties
    return nxt


def _pinwheel_reversal(oracle, angle_deg, cells=20, K=400, hmax=0.06):
    # The paper's pinwheel reversal parameters (Sec. "Superferromagnetism in pinwheel
    # ASI"): b = 0.28, c = 1, beta = 4.8, gamma = 3, alpha = 0.00033, h_k = 0.098,
    # k_disorder = 0.05, neighbour distance 10; a linear loop -hmax -> +hmax at the
    # given angle from +x. Returns, per field step, the fraction of each sublattice
    # (islands at 45 and at 135 degrees) reversed since the first step's saturation.
    x, y, th = oracle.geometry(I.PINWHEEL, cells, cells)
    hk = oracle.draw_hk(len(x), 0.098, 0.05, 1)
    S = oracle.Sim(x, y, th, hk, alpha=0.00033, b=0.28, c=1.0, beta=4.8, gamma=3.0,
                   cutoff_abs=10.0)
    h = -hmax + 2 * hmax * np.arange(K) / (K - 1)
    a = math.radians(angle_deg)
    r = S.run(np.ones(len(x), dtype=np.int8), h * math.cos(a), h * math.sin(a))
    sub_a = np.isclose(np.degrees(th) % 180.0, 45.0)
    s = np.ones(len(x), dtype=np.int8)
    ls, lk = r["log_step"], r["log_spin"]
    j, s0, rows = 0, None, []
    for t in range(K):
        while j < len(ls) and ls[j] == t:
            s[lk[j]] *= -1
            j += 1
        if t == 0:
            s0 = s.copy()
        rows.append(((s[sub_a] != s0[sub_a]).mean(), (s[~sub_a] != s0[~sub_a]).mean()))
    return np.array(rows)


def test_pinwheel_reversal_angle_controls_avalanche_or_two_steps(oracle):
    # The paper's key pinwheel result: a field equally aligned to both sublattices
    # (theta = 0) reverses them in a single avalanche; one more aligned to one
    # sublattice (theta = 30 degrees) reverses it completely before the other starts.
    both = _pinwheel_reversal(oracle, 0.0)
    assert both[-1].min() > 0.99
    tot = both.mean(axis=1)  # (equal sublattice sizes)
    t10, t90 = int(np.argmax(tot >= 0.1)), int(np.argmax(tot >= 0.9))
    assert t90 - t10 <= 3, (t10, t90)
    assert np.abs(both[:, 0] - both[:, 1]).max() < 0.3
    two = _pinwheel_reversal(oracle, 30.0)
    assert two[-1].min() > 0.99
    assert ((two[:, 0] >= 0.99) & (two[:, 1] <= 0.01)).sum() >= 5  # A done, B not begun
    assert not ((two[:, 1] >= 0.5) & (two[:, 0] <= 0.5)).any()     # never the other way


def test_relax_matches_brute_force_state_table(oracle):
    # 2 x 2 closed square: 12 islands, all 4096 states enumerated.
    x, y, th = oracle.geometry(I.SQUARE, 2, 2)
    assert len(x) == 12
    rng = np.random.default_rng(5)
    for trial in range(3):
        hk = 0.2 * (1 + 0.05 * rng.standard_normal(12))
        alpha = [0.02, 0.05, 0.01][trial]
        K = 24
        hx, hy = I.ramp_protocol(K, [45.0, 30.0, 10.0][trial], 0.3)
        S = oracle.Sim(x, y, th, hk, alpha=alpha, cutoff_abs=3.0)
        s0 = np.ones(12, dtype=np.int8)
        res = S.run(s0, hx, hy)
        assert res["status"] == 0
        state = s0.copy()
        q = 0
        for t in range(K):
            table = _brute_tables(x, y, th, hk, alpha, 3.0, 1, 1, 3, 3, hx[t], hy[t])
            while True:
                idx = int((((state + 1) // 2).astype(np.int64) << np.arange(12)).sum())
                k = table[idx]
                if k < 0:
                    break
                assert q < res["n_flips"]
                assert res["log_step"][q] == t and res["log_spin"][q] == k
                state[k] = -state[k]
                q += 1
        assert q == res["n_flips"]
        np.testing.assert_array_equal(state, res["spins"])


def test_energy_strictly_decreases_every_flip(oracle):
    # P_ij = P_ji makes E = -1/2 sum s_i h_dip,par,i - sum s_i (h_ext + h_th) . mhat_i a
    # Lyapunov function: a flip allowed by Eq. (6) changes E by 2 s_k h_par,k < 0.
    x, y, th = oracle.geometry(I.SQUARE, 5, 5)
    n = len(x)
    hk = oracle.draw_hk(n, 0.2, 0.05, 3)
    S = oracle.Sim(x, y, th, hk, alpha=0.01, cutoff_abs=3.0, sigma_th=0.003, seed=4)
    hx, hy = I.ramp_protocol(60, 40.0, 0.3)
    s0 = np.ones(n, dtype=np.int8)
    res = S.run(s0, hx, hy)
    assert res["n_flips"] > n
    mx, my = np.cos(th), np.sin(th)

    def energy(s, t):
        hdx, hdy = S.dip_fields(s)
        tp, _ = oracle.thermal(n, 0.003, 4, 0, t)
        edip = -0.5 * float((s * (hdx * mx + hdy * my)).sum())
        eext = -float((s * (hx[t] * mx + hy[t] * my + tp)).sum())
        return edip + eext

    state = s0.astype(np.int64)
    q = 0
    for t in range(len(hx)):
        e_prev = energy(state, t)
        while q < res["n_flips"] and res["log_step"][q] == t:
            state[res["log_spin"][q]] *= -1
            e = energy(state, t)
            assert e < e_prev
            e_prev = e
            q += 1


def test_noninteracting_limit_closed_form(oracle):
    # alpha = 0: island i switches when |h_ext| exceeds h_k^(i) h_sw(phi_i) while
    # anti-aligned, h_sw from the Stoner-Wohlfarth closed form; within one field
    # step the order is by |h| / h_sw descending (monotone in Eq. (5)).
    x, y, th = oracle.geometry(I.KAGOME, 6, 6)
    n = len(x)
    hk = oracle.draw_hk(n, 0.2, 0.05, 8)
    S = oracle.Sim(x, y, th, hk, alpha=0.0, cutoff_abs=4.0)
    hx, hy = I.rotation_protocol(90, 4.0, 0.15)
    s0 = np.ones(n, dtype=np.int8)
    res = S.run(s0, hx, hy)
    mx, my = np.cos(th), np.sin(th)
    state = s0.astype(np.int64)
    q = 0
    for t in range(len(hx)):
        hpar = hx[t] * mx + hy[t] * my
        hperp = -hx[t] * my + hy[t] * mx
        mag = math.hypot(hx[t], hy[t])
        phi = np.arctan2(np.abs(hperp), np.abs(hpar))
        hsw = hk / (np.abs(np.cos(phi)) ** (2 / 3) + np.abs(np.sin(phi)) ** (2 / 3)) ** 1.5
        ratio = mag / hsw
        cand = np.where((state * hpar < 0) & (ratio > 1))[0]
        order = sorted(cand.tolist(), key=lambda i: (-ratio[i], i))
        got = res["log_spin"][res["log_step"] == t].tolist()
        assert got == order
        state[order] *= -1
        q += len(order)
    assert q == res["n_flips"]


def test_definition_mode_equals_incremental(oracle):
    # Recomputing every field after every flip (the paper's literal loop) and updating
    # only the flipped island's neighbours give the same sequence on square16.
    w = I.WORKLOADS["square16"]
    x, y, th = oracle.geometry(w["kind"], w["nx"], w["ny"])
    hk = oracle.draw_hk(len(x), w["hk"], w["k_disorder"], w["seed"])
    S = oracle.Sim(x, y, th, hk, alpha=w["alpha"], cutoff_abs=w["cutoff"])
    hx, hy = I.protocol_of(w["protocol"])
    s0 = np.ones(len(x), dtype=np.int8)
    a = S.run(s0, hx, hy)
    b = S.run(s0, hx, hy, mode=oracle.MODE_DEFINITION)
    assert a["n_flips"] == b["n_flips"] == 2 * len(x)
    np.testing.assert_array_equal(a["log_spin"], b["log_spin"])
    np.testing.assert_array_equal(a["log_step"], b["log_step"])
    assert a["hash"] == b["hash"] == oracle.hash_flips(a["log_step"], a["log_spin"])
    assert a["ties"].sum() == 0


def test_tree_argmax_equals_linear_scan(oracle):
    x, y, th = oracle.geometry(I.PINWHEEL, 48, 48)
    n = len(x)
    assert n > 4096
    hk = oracle.draw_hk(n, 0.2, 0.05, 1)
    S = oracle.Sim(x, y, th, hk, alpha=1e-3, cutoff_abs=5.0)
    hx, hy = I.loop_protocol(120, 30.0, -0.25, 0.25)
    s0 = np.ones(n, dtype=np.int8)
    a = S.run(s0, hx, hy)
    b = S.run(s0, hx, hy, mode=oracle.MODE_LINEAR)
    assert a["n_flips"] == b["n_flips"] > n
    np.testing.assert_array_equal(a["log_spin"], b["log_spin"])
    assert a["hash"] == b["hash"]


def test_ties_go_to_lowest_index(oracle):
    # Identical, non-interacting islands see identical fields: every pick is a tie
    # and the paper's "deterministic, arbitrary" rule is read as lowest index first.
    x = np.arange(6, dtype=np.float64) * 10.0
    y = np.zeros(6)
    th = np.zeros(6)
    hk = np.full(6, 0.2)
    S = oracle.Sim(x, y, th, hk, alpha=0.0, cutoff_abs=1.0)
    res = S.run(np.ones(6, dtype=np.int8), np.array([-0.3]), np.array([0.0]))
    assert res["log_spin"].tolist() == [0, 1, 2, 3, 4, 5]
    assert res["ties"][0] == 5


def test_flip_guard(oracle):
    x, y, th = oracle.geometry(I.SQUARE, 4, 4)
    hk = oracle.draw_hk(len(x), 0.2, 0.05, 0)
    S = oracle.Sim(x, y, th, hk, alpha=1e-3, cutoff_abs=3.0)
    res = S.run(np.ones(len(x), dtype=np.int8), np.array([-0.3]), np.array([-0.3]),
                max_flips_per_step=3)
    assert res["status"] == oracle.ERR_NOT_CONVERGED
    assert res["n_flips"] == 3


def test_resume_is_exact(oracle):
    # State = (spins, step index, seed): a protocol split at step t and resumed
    # gives the same sequence and hash (thermal draws are keyed by step).
    x, y, th = oracle.geometry(I.KAGOME, 6, 6)
    n = len(x)
    hk = oracle.draw_hk(n, 0.2, 0.05, 2)
    S = oracle.Sim(x, y, th, hk, alpha=8e-4, cutoff_abs=4.0, sigma_th=0.01, seed=2)
    hx, hy = I.rotation_protocol(80, 4.5, 0.12)
    s0 = np.ones(n, dtype=np.int8)
    full = S.run(s0, hx, hy)
    a = S.run(s0, hx[:37], hy[:37])
    b = S.run(a["spins"], hx[37:], hy[37:], step0=37, hash_in=a["hash"])
    assert b["hash"] == full["hash"]
    np.testing.assert_array_equal(b["spins"], full["spins"])
    assert a["n_flips"] + b["n_flips"] == full["n_flips"]


def test_golden_square16_reproduces(oracle):
    # the stored square16 values were written by tests/golden/make_golden.py from the
    # oracle; recomputing them must give the same sequence
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "square16.json")))
    w = I.WORKLOADS["square16"]
    x, y, th = oracle.geometry(w["kind"], w["nx"], w["ny"])
    hk = oracle.draw_hk(len(x), w["hk"], w["k_disorder"], w["seed"])
    S = oracle.Sim(x, y, th, hk, alpha=w["alpha"], cutoff_abs=w["cutoff"])
    hx, hy = I.protocol_of(w["protocol"])
    r = S.run(np.ones(len(x), dtype=np.int8), hx, hy)
    assert f"{r['hash']:#018x}" == g["seq_hash"]
    assert r["log_spin"].tolist() == g["log_spin"]
    assert r["flips_per_step"].tolist() == g["flips_per_step"]
