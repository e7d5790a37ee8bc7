"""Pins of the oracle's variants of the model: the edge forms and the ising array
of the geometry figure, the parallel-only switching criterion of the pinwheel
section, local and spatial external fields and the input encoders (Sec.
"External field", Sec. "Simulation framework"), thermal protocols and the
spin-spin correlation (Sec. "Domain size in square ASI").

Each test checks the oracle against something other than itself: a count
printed in the paper, a closed form, an identity between two ways of stating the
same input, or an independent formula.
"""
import math

import numpy as np
import pytest

from paper_2002_11401_b300 import inputs as I


def _sites(O, kind, n, m=None):
    x, y, t = O.geometry(kind, n, n if m is None else m)
    return {(round(2 * a), round(2 * b)): round(math.degrees(c)) for a, b, c in zip(x, y, t)}


# ---------------------------------------------------------------------------
# Geometry variants (Fig. "geometries")
# ---------------------------------------------------------------------------

def test_pinwheel_diamond_count_printed_in_paper(oracle):
    # Sec. "Performance": the 25 x 25 pinwheel array of the pinwheel section has 1250 magnets.
    x, _, t = oracle.geometry(oracle.PINWHEEL_DIAMOND, 25, 25)
    assert len(x) == 1250
    assert sorted(set(np.round(np.degrees(t)).astype(int))) == [45, 135]


@pytest.mark.parametrize("n,m", [(1, 1), (2, 5), (7, 3), (16, 16)])
def test_variant_counts(oracle, n, m):
    def count(kind):
        return len(oracle.geometry(kind, n, m)[0]) if n * m > 0 else 0
    assert count(oracle.PINWHEEL_DIAMOND) == 2 * n * m
    assert count(oracle.ISING) == n * m
    if (n, m) != (1, 1):  # a 1 x 1 open square has no island left
        assert count(oracle.SQUARE_OPEN) == 2 * n * m - n - m
        assert count(oracle.PINWHEEL_LUCKY_KNOT) == 2 * n * m - n - m


def test_open_edges_are_the_closed_square_without_its_boundary(oracle):
    n, m = 6, 4
    closed = _sites(oracle, oracle.SQUARE, n, m)
    opened = _sites(oracle, oracle.SQUARE_OPEN, n, m)
    # half-spacing coordinates: horizontal islands at even Y, vertical ones at even X
    boundary = {k for k in closed if (k[1] % 2 == 0 and k[1] in (0, 2 * m)) or
                (k[0] % 2 == 0 and k[0] in (0, 2 * n))}
    assert set(opened) == set(closed) - boundary
    assert all(opened[k] == closed[k] for k in opened)
    lucky = _sites(oracle, oracle.PINWHEEL_LUCKY_KNOT, n, m)
    assert set(lucky) == set(opened) and all(lucky[k] == opened[k] + 45 for k in lucky)


def test_diamond_is_the_unit_cell_tiling_turned_45_degrees(oracle):
    n, m = 5, 7
    closed = _sites(oracle, oracle.SQUARE, n, m)
    diamond = _sites(oracle, oracle.PINWHEEL_DIAMOND, n, m)
    # closed square less its top row of horizontal and right column of vertical islands
    top_right = {k for k in closed if (k[1] % 2 == 0 and k[1] == 2 * m) or
                 (k[0] % 2 == 0 and k[0] == 2 * n)}
    assert set(diamond) == set(closed) - top_right
    assert all(diamond[k] == closed[k] + 45 for k in diamond)


def test_ising_is_one_aligned_sublattice(oracle):
    x, y, t = oracle.geometry(oracle.ISING, 4, 3)
    assert (t == 0.0).all()
    assert sorted(zip(y.tolist(), x.tolist())) == [(float(b), float(a)) for b in range(3)
                                                  for a in range(4)]


def test_open_square_eight_spin_neighbourhood(oracle):
    # Sec. "Performance": square ASI with open edges and the standard 8-spin
    # neighbourhood; bulk islands see 8 neighbours at a cutoff of one spacing.
    x, y, _ = oracle.geometry(oracle.SQUARE_OPEN, 12, 12)
    rp, _ = oracle.neighbors(x, y, 1.0)
    deg = np.diff(rp)
    assert deg.max() == 8
    bulk = (x > 2) & (x < 10) & (y > 2) & (y < 10)
    assert (deg[bulk] == 8).all()


# ---------------------------------------------------------------------------
# The parallel-only criterion (pinwheel section)
# ---------------------------------------------------------------------------

def test_parallel_criterion_threshold_closed_form(oracle):
    # One island along x, a field at angle phi: the parallel-only criterion switches
    # when |h| |cos phi| > h_k, i.e. at |h| = h_k / |cos phi|, whatever the
    # perpendicular part; Eq. 5 (Stoner-Wohlfarth) at 45 degrees already at h_k / 2.
    hk = 0.2
    for phi_deg in (0.0, 30.0, 45.0, 60.0, 80.0):
        phi = math.radians(180.0 + phi_deg)  # opposing the +1 island
        h = np.linspace(0.0, 2.0, 2001)
        hx, hy = h * math.cos(phi), h * math.sin(phi)
        S = oracle.Sim([0.0], [0.0], [0.0], [hk], alpha=1e-3, cutoff_abs=1.0,
                       criterion=oracle.PARALLEL)
        r = S.run(np.ones(1, dtype=np.int8), hx, hy)
        assert r["n_flips"] == 1
        t = int(r["log_step"][0])
        thr = hk / math.cos(math.radians(phi_deg))
        assert h[t] * math.cos(math.radians(phi_deg)) > hk >= h[t - 1] * math.cos(math.radians(phi_deg))
        assert abs(h[t] - thr) <= 1e-3 + 1e-12  # one grid step
        hp, hq = S.fields(np.ones(1, dtype=np.int8), hx[t], hy[t])
        assert S.lhs(hp, hq)[0] == oracle.parallel_lhs(hp[0], hk) == abs(hp[0]) / hk
    # the two criteria differ: at 45 degrees Eq. 5 switches at half the field
    h45 = 0.15  # between h_k / 2 and sqrt(2) h_k
    a = math.radians(225.0)
    for crit, expect in ((oracle.ASTROID, 1), (oracle.PARALLEL, 0)):
        S = oracle.Sim([0.0], [0.0], [0.0], [hk], alpha=1e-3, cutoff_abs=1.0, criterion=crit)
        r = S.run(np.ones(1, dtype=np.int8), [h45 * math.cos(a)], [h45 * math.sin(a)])
        assert r["n_flips"] == expect


# ---------------------------------------------------------------------------
# Local and spatial external fields (Sec. "External field")
# ---------------------------------------------------------------------------

def _kagome_system(O, sigma=0.004):
    w = dict(kind=I.KAGOME, nx=8, ny=8, alpha=3e-3, cutoff=4.0, hk=0.2, k_disorder=0.08, seed=3,
             b=1.0, c=1.0, beta=3.0, gamma=3.0, sigma_th=sigma)
    x, y, th = O.geometry(w["kind"], w["nx"], w["ny"])
    hk = O.draw_hk(len(x), w["hk"], w["k_disorder"], w["seed"])
    return x, y, th, hk, w


def test_uniform_local_field_equals_the_global_field(oracle):
    x, y, th, hk, w = _kagome_system(oracle)
    hx, hy = I.rotation_protocol(60, 6.0, 0.12)
    n, K = len(x), len(hx)
    S = oracle.Sim(x, y, th, hk, alpha=w["alpha"], sigma_th=w["sigma_th"], cutoff_abs=4.0, seed=3)
    ref = S.run(np.ones(n, dtype=np.int8), hx, hy)
    loc = S.run(np.ones(n, dtype=np.int8), np.zeros(K), np.zeros(K),
                lhx=np.repeat(hx[:, None], n, axis=1), lhy=np.repeat(hy[:, None], n, axis=1))
    assert ref["n_flips"] > 100
    assert loc["hash"] == ref["hash"] and loc["n_flips"] == ref["n_flips"]


def test_uniform_spatial_field_equals_the_global_field(oracle):
    x, y, th, hk, w = _kagome_system(oracle)
    hx, hy = I.rotation_protocol(60, 6.0, 0.12)
    n, K = len(x), len(hx)
    gw, gh = 3, 2
    gx = np.repeat(hx[:, None, None], gh, axis=1).repeat(gw, axis=2)
    gy = np.repeat(hy[:, None, None], gh, axis=1).repeat(gw, axis=2)
    lx, ly = oracle.sample_grid(x, y, gw, gh, 0.0, 0.0, 5.0, 7.0, gx, gy)
    S = oracle.Sim(x, y, th, hk, alpha=w["alpha"], sigma_th=w["sigma_th"], cutoff_abs=4.0, seed=3)
    ref = S.run(np.ones(n, dtype=np.int8), hx, hy)
    sp = S.run(np.ones(n, dtype=np.int8), np.zeros(K), np.zeros(K), lhx=lx, lhy=ly)
    assert sp["hash"] == ref["hash"] and sp["n_flips"] == ref["n_flips"]


def test_spatial_sampling_takes_the_cell_of_each_centre(oracle):
    # cells of 2 x 1 from (1, -1): x in [1, 3) -> 0, [3, 5) -> 1, ...; outside -> clamped
    x = np.array([1.0, 2.99, 3.0, 4.5, -7.0, 100.0, 2.0])
    y = np.array([-1.0, 0.5, -0.5, 1.0, 0.2, 3.2, 25.0])
    gw, gh = 4, 3
    cell = np.arange(gw * gh, dtype=np.float64).reshape(1, gh, gw)
    lx, ly = oracle.sample_grid(x, y, gw, gh, 1.0, -1.0, 2.0, 1.0, cell, -cell)
    want = [0 + 0, 0 + 4, 1 + 0, 1 + 8, 0 + 4, 3 + 8, 0 + 8]
    assert lx[0].tolist() == [float(v) for v in want]
    assert ly[0].tolist() == [-float(v) for v in want]


def test_local_field_gradient_orders_noninteracting_switches(oracle):
    # Islands out of each other's reach, equal h_k, all along x; island i feels
    # f_i times a ramp opposing it: it switches at the first step where f_i |h| > h_k
    # (Eq. 5 at 0 degrees), and within a step the larger f_i first.
    n = 40
    rng = np.random.default_rng(2)
    f = rng.permutation(np.linspace(0.5, 1.5, n))
    x = np.arange(n) * 10.0
    S = oracle.Sim(x, np.zeros(n), np.zeros(n), np.full(n, 0.2), alpha=1e-3, cutoff_abs=1.0)
    h = np.linspace(0.0, 0.45, 90)
    lhx = -np.outer(h, f)
    r = S.run(np.ones(n, dtype=np.int8), np.zeros(len(h)), np.zeros(len(h)), lhx=lhx,
              lhy=np.zeros_like(lhx))
    assert r["n_flips"] == n
    expect_step = np.array([int(np.argmax(h * fi > 0.2)) for fi in f])
    order = sorted(range(n), key=lambda i: (expect_step[i], -f[i]))
    assert r["log_spin"].tolist() == order
    assert r["log_step"].tolist() == [int(expect_step[i]) for i in order]


# ---------------------------------------------------------------------------
# Thermal protocols (Sec. "Domain size in square ASI": annealing)
# ---------------------------------------------------------------------------

def test_constant_sigma_series_equals_sigma_th(oracle):
    x, y, th, hk, w = _kagome_system(oracle, sigma=0.006)
    hx, hy = I.rotation_protocol(40, 9.0, 0.11)
    n, K = len(x), len(hx)
    S = oracle.Sim(x, y, th, hk, alpha=w["alpha"], sigma_th=0.006, cutoff_abs=4.0, seed=3)
    ref = S.run(np.ones(n, dtype=np.int8), hx, hy)
    ser = S.run(np.ones(n, dtype=np.int8), hx, hy, sigma=np.full(K, 0.006))
    assert ser["hash"] == ref["hash"] and ser["n_flips"] == ref["n_flips"] > 50


def test_zero_sigma_series_equals_no_thermal_field(oracle):
    x, y, th, hk, w = _kagome_system(oracle)
    hx, hy = I.rotation_protocol(40, 9.0, 0.11)
    n, K = len(x), len(hx)
    cold = oracle.Sim(x, y, th, hk, alpha=w["alpha"], sigma_th=0.0, cutoff_abs=4.0, seed=3)
    ref = cold.run(np.ones(n, dtype=np.int8), hx, hy)
    S = oracle.Sim(x, y, th, hk, alpha=w["alpha"], sigma_th=0.01, cutoff_abs=4.0, seed=3)
    ser = S.run(np.ones(n, dtype=np.int8), hx, hy, sigma=np.zeros(K))
    assert ser["hash"] == ref["hash"] and ser["n_flips"] == ref["n_flips"]
    hot = S.run(np.ones(n, dtype=np.int8), hx, hy)
    assert hot["hash"] != ref["hash"]


def test_annealing_orders_the_square_array(oracle):
    # Sec. "Domain size in square ASI" (its astroid b = 0.4, c = 1, beta = gamma = 3,
    # h_k 0.186, k_disorder 0.05): an exponentially decreasing thermal field at zero
    # external field takes a polarised square array to a state of lower dipolar
    # energy, ordered at short range: the nearest pairs are strongly correlated and
    # the correlation falls off with separation.
    n = 20
    x, y, th = oracle.geometry(oracle.SQUARE, n, n)
    hk = oracle.draw_hk(len(x), 0.186, 0.05, 7)
    S = oracle.Sim(x, y, th, hk, alpha=0.0025, b=0.4, c=1.0, beta=3.0, gamma=3.0,
                   sigma_th=0.2, cutoff_abs=4.0, seed=7)
    K = 120
    sig = 0.2 * 0.95 ** np.arange(K)
    s0 = np.ones(len(x), dtype=np.int8)
    r = S.run(s0, np.zeros(K), np.zeros(K), sigma=sig)
    assert r["status"] == 0

    def energy(s):
        hdx, hdy = S.dip_fields(s)
        return -0.5 * float(np.sum(s * (hdx * np.cos(th) + hdy * np.sin(th))))

    assert energy(r["spins"]) < energy(s0)
    cnt, sm = oracle.correlation(x, y, th, r["spins"], 8.0, 0.5, 16)
    c = np.where(cnt > 0, np.abs(sm) / np.maximum(cnt, 1), np.nan)
    near = c[1]  # separation 0.5 .. 1: the vertex pairs
    assert near > 0.5
    assert np.nanmean(c[12:16]) < near


# ---------------------------------------------------------------------------
# Spin-spin correlation
# ---------------------------------------------------------------------------

def test_correlation_of_the_aligned_ising_array_closed_form(oracle):
    # All spins +1 along x on an n x n grid. Pair at offset (dx, dy): the energy is
    # minimal (+1) when 3 (mhat.rhat)^2 - 1 > 0. Separation 1: n(n-1) head-to-tail
    # pairs (+1) and n(n-1) side-by-side (-1); sqrt 2: 2(n-1)^2 pairs, 3/2 - 1 > 0;
    # 2: like 1; sqrt 5: 2(n-1)(n-2) at (2, +-1) (+1) and as many at (1, +-2) (-1).
    n = 9
    x, y, th = oracle.geometry(oracle.ISING, n, n)
    cnt, sm = oracle.correlation(x, y, th, np.ones(n * n, dtype=np.int8), 2.3, 0.1, 24)
    assert (cnt[10], sm[10]) == (2 * n * (n - 1), 0)
    assert (cnt[14], sm[14]) == (2 * (n - 1) ** 2, 2 * (n - 1) ** 2)
    assert (cnt[20], sm[20]) == (2 * n * (n - 2), 0)
    assert (cnt[22], sm[22]) == (4 * (n - 1) * (n - 2), 0)
    assert cnt.sum() == cnt[10] + cnt[14] + cnt[20] + cnt[22]


def test_correlation_sign_is_that_of_the_pair_energy(oracle):
    # The same correlation from the point-dipole field of Eq. 3: the energy of the
    # pair, -m_i . h_j(r_i), is below zero exactly when the correlation is +1.
    x, y, th = oracle.geometry(oracle.KAGOME, 4, 3)
    s = I.random_spins(len(x), 5)
    rmax, wd, nb = 3.1, 0.25, 13
    cnt, sm = oracle.correlation(x, y, th, s, rmax, wd, nb)
    ec, es = np.zeros(nb, dtype=np.int64), np.zeros(nb, dtype=np.int64)
    for i in range(len(x)):
        for j in range(i + 1, len(x)):
            rx, ry = x[i] - x[j], y[i] - y[j]
            r = math.hypot(rx, ry)
            if r * r > rmax * rmax * (1 + 1e-9):
                continue
            b = int(math.floor(r / wd + 1e-7))
            if b >= nb:
                continue
            hx, hy = oracle.dipole_field(rx, ry, s[j] * math.cos(th[j]), s[j] * math.sin(th[j]),
                                         1.0)
            e = -(s[i] * math.cos(th[i]) * hx + s[i] * math.sin(th[i]) * hy)
            v = -e * r**3 * s[i] * s[j]
            if abs(v) <= 1e-9:
                continue
            ec[b] += 1
            es[b] += 1 if e < 0 else -1
    np.testing.assert_array_equal(cnt, ec)
    np.testing.assert_array_equal(sm, es)


def test_correlation_is_invariant_under_a_global_flip(oracle):
    x, y, th = oracle.geometry(oracle.PINWHEEL, 6, 6)
    s = I.random_spins(len(x), 9)
    a = oracle.correlation(x, y, th, s, 4.0, 0.5, 8)
    b = oracle.correlation(x, y, th, -s, 4.0, 0.5, 8)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


# ---------------------------------------------------------------------------
# Input encoders (Sec. "Simulation framework")
# ---------------------------------------------------------------------------

def test_sinusoid_encoder_closed_form(oracle):
    u = np.array([0.0, 0.5, 1.0])
    hx, hy = oracle.encode(oracle.SINUSOID, u, 8, 0.1, 0.3, 0.0)
    assert len(hx) == 24 and (hy == 0.0).all()
    for k, A in enumerate((0.1, 0.2, 0.3)):
        per = hx[8 * k:8 * k + 8]
        assert per[2] == A and per[6] == -A and per[0] == 0.0  # quarter periods
        assert abs(per[1] - A * math.sqrt(0.5)) <= 1e-16
    hx, hy = oracle.encode(oracle.SINUSOID, [1.0], 4, 0.0, 0.2, 90.0)
    assert abs(hy[1] - 0.2) <= 1e-16 and abs(hx[1]) <= 1e-16


def test_sawtooth_encoder_closed_form(oracle):
    hx, hy = oracle.encode(oracle.SAWTOOTH, [0.25, 1.0], 5, 0.0, 0.4, 30.0)
    c, s = math.cos(math.radians(30.0)), math.sin(math.radians(30.0))
    for k, A in enumerate((0.1, 0.4)):
        h = hx[5 * k:5 * k + 5] / c
        np.testing.assert_allclose(h, A * np.array([-1.0, -0.5, 0.0, 0.5, 1.0]), rtol=0,
                                   atol=1e-16)
        np.testing.assert_allclose(hy[5 * k:5 * k + 5], h * s, rtol=1e-15, atol=1e-17)


def test_rotation_encoder_closed_form(oracle):
    hx, hy = oracle.encode(oracle.ROTATION, [0.5], 12, 0.1, 0.3, 15.0)
    np.testing.assert_allclose(np.hypot(hx, hy), 0.2, rtol=1e-15)
    ang = np.degrees(np.arctan2(hy, hx)) % 360.0
    np.testing.assert_allclose(ang, (15.0 + 30.0 * np.arange(12)) % 360.0, atol=1e-12)


def test_single_island_switching_times_under_a_sawtooth(oracle):
    # One island along x (s = +1), h_k = 0.2, the Stoner-Wohlfarth astroid, a
    # sawtooth along 30 degrees rising from -A to +A: the island switches to -1 at the
    # first value (|h| = A > h_sw) and back at the first j with
    # A (2 j / (T - 1) - 1) > h_sw(30 deg) = h_k / (cos^(2/3) + sin^(2/3))^(3/2).
    hk, A, T = 0.2, 0.3, 101
    hx, hy = oracle.encode(oracle.SAWTOOTH, [1.0], T, 0.0, A, 30.0)
    S = oracle.Sim([0.0], [0.0], [0.0], [hk], alpha=1e-3, cutoff_abs=1.0)
    r = S.run(np.ones(1, dtype=np.int8), hx, hy)
    c, s = math.cos(math.radians(30.0)), math.sin(math.radians(30.0))
    hsw = hk / (c ** (2 / 3) + s ** (2 / 3)) ** 1.5
    j_back = next(j for j in range(T) if A * (2 * j / (T - 1) - 1) > hsw)
    assert r["log_step"].tolist() == [0, j_back]
