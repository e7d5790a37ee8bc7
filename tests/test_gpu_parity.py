"""CUDA path against the FP64 oracle, element by element, on seeded inputs.

Tolerances: flip sequences (step, island) and spin states bit-exact; coercive
fields bit-exact (both sides draw them with Philox4x32-10 + Box-Muller in host
double precision); fields within 1e-12 of max|h| (FS_FP64) or 1e-5 of max|h|
(FS_FP32_RECHECK, the FP32 evaluation itself).
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


def _pair_field_frame(O, xi, yi, ti, xj, yj, tj, alpha):
    hx, hy = O.dipole_field(xi - xj, yi - yj, math.cos(tj), math.sin(tj), alpha)
    c, s = math.cos(ti), math.sin(ti)
    return hx * c + hy * s, -hx * s + hy * c


# ---------------------------------------------------------------------------
# Inputs and tensors
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind,n", [(I.SQUARE, 16), (I.PINWHEEL, 10), (I.KAGOME, 8)])
def test_hk_and_neighbour_tensor(B, oracle, kind, n):
    w = small(kind, n)
    sim = lib_sim(w)
    S = oracle_sim(oracle, w)
    np.testing.assert_array_equal(sim.hk(), S.hk)  # bit-exact draws
    rp, col, P, Q = sim.csr()
    orp, ocol = S.neighbors()
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(col, ocol)
    x, y, t = S.x, S.y, S.theta
    scale = 0.0
    errs = []
    for i in range(S.n):
        for e in range(rp[i], rp[i + 1]):
            j = col[e]
            ep, eq = _pair_field_frame(oracle, x[i], y[i], t[i], x[j], y[j], t[j], w["alpha"])
            errs.append(max(abs(P[e] - ep), abs(Q[e] - eq)))
            scale = max(scale, abs(ep), abs(eq))
    assert max(errs) <= 1e-14 * scale
    # P_ij = P_ji exactly (symmetric tensor, symmetric neighbourhood)
    pos = {(i, int(col[e])): e for i in range(S.n) for e in range(rp[i], rp[i + 1])}
    for (i, j), e in pos.items():
        assert P[e] == P[pos[(j, i)]]


# ---------------------------------------------------------------------------
# Fields (Eq. 2, 3) and the astroid (Eq. 5)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec,tol", [(FP64, 1e-12), (FP32, 1e-5)])
@pytest.mark.parametrize("kind,n,sigma", [(I.SQUARE, 12, 0.0), (I.PINWHEEL, 9, 0.0),
                                          (I.KAGOME, 9, 0.005)])
def test_fields_match_oracle(B, oracle, prec, tol, kind, n, sigma):
    w = small(kind, n, sigma_th=sigma, alpha=3e-3)
    sim = lib_sim(w, precision=prec)
    S = oracle_sim(oracle, w)
    worst = 0.0
    for trial in range(4):
        s = I.random_spins(S.n, 100 + trial)
        hx, hy = 0.05 * math.cos(trial), -0.07 * math.sin(trial + 1)
        sim.set_spins(s)
        sim.set_field(hx, hy, step=trial * 7)
        hp, hq = sim.fields()
        op, oq = S.fields(s, hx, hy, step=trial * 7)
        hmax = max(np.abs(op).max(), np.abs(oq).max())
        err = max(np.abs(hp - op).max(), np.abs(hq - oq).max()) / hmax
        worst = max(worst, err)
        assert err <= tol, (trial, err)
        lhs = sim.lhs()
        olhs = np.array([oracle.astroid_lhs(op[i], oq[i], S.hk[i], 1, 1, 3, 3)
                         for i in range(S.n)])
        assert np.abs(lhs - olhs).max() <= (1e-11 if prec == FP64 else 1e-4) * olhs.max()


@pytest.mark.parametrize("kind,n", [(I.PINWHEEL, 9), (I.KAGOME, 9)])
def test_fp64_astroid_within_a_few_ulps(B, oracle, kind, n):
    """Eq. 5 on the FS_FP64 path, taken on the library's own fields so that only the
    astroid is compared: the oracle's libm pow against the kernels' x^(2/3), within
    4e-15 relative (a dropped second-order term of its refinement would be ~3e-14)."""
    w = small(kind, n, alpha=3e-3)
    sim = lib_sim(w, precision=FP64)
    S = oracle_sim(oracle, w)
    checked = 0
    for trial in range(6):
        s = I.random_spins(S.n, 300 + trial)
        hx, hy = 0.3 * math.cos(trial), 0.25 * math.sin(2 * trial + 1)
        sim.set_spins(s)
        sim.set_field(hx, hy, step=trial)
        hp, hq = sim.fields()
        lhs = sim.lhs()
        for i in range(S.n):
            o = oracle.astroid_lhs(hp[i], hq[i], S.hk[i], 1, 1, 3, 3)
            if o > 0.0:
                assert abs(lhs[i] - o) <= 4e-15 * o, (trial, i, lhs[i], o)
                checked += 1
    assert checked > 100


# ---------------------------------------------------------------------------
# Flip sequences (Sec. "Dynamics")
# ---------------------------------------------------------------------------

def _compare_runs(oracle, w, hx, hy, precs=(FP64, FP32), resweeps=(True,), **over):
    S = oracle_sim(oracle, w, **over)
    ref = S.run(np.ones(S.n, dtype=np.int8), hx, hy)
    assert ref["status"] == 0
    out = []
    for prec in precs:
        for rs in resweeps:
            sim = lib_sim(w, precision=prec, **over)
            got = sim.run_protocol(hx, hy, resweep=rs)
            d = first_divergence(ref["log_step"], ref["log_spin"], got["log_step"],
                                 got["log_spin"])
            assert d is None, (prec, rs, d, ref["ties"])
            assert got["n_flips"] == ref["n_flips"]
            assert got["hash"] == ref["hash"]
            np.testing.assert_array_equal(got["flips_per_step"], ref["flips_per_step"])
            np.testing.assert_array_equal(sim.spins(), ref["spins"])
            out.append(got)
    return ref, out


@pytest.mark.parametrize("angle", [0.0, 30.0])
def test_pinwheel_reversal_with_the_papers_parameters(B, oracle, angle):
    """The paper's pinwheel reversal (asymmetric astroid b = 0.28, beta = 4.8,
    alpha = 0.00033, h_k = 0.098, neighbour distance 10; a loop -0.06 -> +0.06 T):
    every flip as the oracle's, both paths (the oracle's own pin checks the
    avalanche at 0 degrees and the two steps at 30)."""
    w = small(I.PINWHEEL, 20, alpha=0.00033, hk=0.098, k_disorder=0.05, cutoff=10.0, b=0.28,
              c=1.0, beta=4.8, gamma=3.0, seed=1)
    K = 400
    h = -0.06 + 0.12 * np.arange(K) / (K - 1)
    a = math.radians(angle)
    ref, _ = _compare_runs(oracle, w, h * math.cos(a), h * math.sin(a))
    # the first step saturates one sublattice (420 islands); then all 840 reverse
    assert ref["n_flips"] == 420 + 840


def test_square16_sequence(B, oracle):
    w = I.WORKLOADS["square16"]
    hx, hy = I.protocol_of(w["protocol"])
    ref, _ = _compare_runs(oracle, w, hx, hy, resweeps=(True, False))
    assert ref["n_flips"] == 2 * 544


@pytest.mark.parametrize("case", range(8))
def test_small_systems_sequences(B, oracle, case):
    rng = np.random.default_rng(1000 + case)
    kind = [I.SQUARE, I.PINWHEEL, I.KAGOME][case % 3]
    astroids = [(1, 1, 3, 3), (0.28, 1, 4.8, 3), (0.42, 1, 1.7, 3.4), (0.38, 1, 1.5, 3.2)]
    b, c, beta, gamma = astroids[case % 4]
    n = int(rng.integers(5, 14))
    sigma = 0.004 if case % 2 else 0.0
    w = small(kind, n, b=b, c=c, beta=beta, gamma=gamma, sigma_th=sigma, seed=case,
              alpha=[1e-3, 3e-3, 1e-2][case % 3], k_disorder=[0.05, 0.1, 0.02][case % 3])
    hmax = 0.35 if b >= 1 else 0.2
    proto = [I.ramp_protocol(60, float(rng.uniform(0, 360)), hmax),
             I.rotation_protocol(60, 6.0, hmax * 0.6),
             I.loop_protocol(60, float(rng.uniform(0, 360)), -hmax, hmax)][case % 3]
    _compare_runs(oracle, w, *proto, resweeps=(True, False))


def test_pinwheel_mid_size(B, oracle):
    w = small(I.PINWHEEL, 48, seed=1)
    hx, hy = I.loop_protocol(150, 30.0, -0.25, 0.25)
    ref, _ = _compare_runs(oracle, w, hx, hy)
    assert ref["n_flips"] > w["nx"] * w["nx"]


def test_kagome_thermal_mid_size(B, oracle):
    w = small(I.KAGOME, 40, sigma_th=0.005, k_disorder=0.08, seed=2)
    hx, hy = I.rotation_protocol(120, 3.0, 0.11)
    _compare_runs(oracle, w, hx, hy)


# ---------------------------------------------------------------------------
# Edge cases
# ---------------------------------------------------------------------------

def test_single_island(B, oracle):
    sim = B.Sim.custom([0.0], [0.0], [0.3])
    sim.set_params(B.make_params(alpha=1e-3, cutoff=2.0))
    hx = np.array([0.0, -0.1, -0.3, 0.3])
    hy = np.zeros(4)
    got = sim.run_protocol(hx, hy)
    S = oracle.Sim([0.0], [0.0], [0.3], sim.hk(), alpha=1e-3, cutoff_abs=2.0)
    ref = S.run(np.ones(1, dtype=np.int8), hx, hy)
    assert got["hash"] == ref["hash"] and got["n_flips"] == ref["n_flips"] == 2


def test_exact_ties_lowest_index(B, oracle):
    # identical non-interacting islands with equal h_k: every pick is an exact tie
    n = 70
    x = np.arange(n, dtype=np.float64) * 10.0
    for prec in (FP64, FP32):
        sim = B.Sim.custom(x, np.zeros(n), np.zeros(n))
        sim.set_params(B.make_params(alpha=0.0, cutoff=1.0, precision=prec))
        sim.set_hk(np.full(n, 0.2))
        got = sim.run_protocol(np.array([-0.3, 0.3]), np.zeros(2))
        assert got["log_spin"].tolist() == list(range(n)) * 2


def test_exact_ties_beyond_the_candidate_cap(B):
    # 400 identical non-interacting islands: every pick is an exact tie among more
    # islands than one warp's exact comparison holds (256), so the block-wide scan
    # settles them; the order is still the lowest index first
    n = 400
    x = np.arange(n, dtype=np.float64) * 10.0
    for prec in (FP64, FP32):
        sim = B.Sim.custom(x, np.zeros(n), np.zeros(n))
        sim.set_params(B.make_params(alpha=0.0, cutoff=1.0, precision=prec))
        sim.set_hk(np.full(n, 0.2))
        got = sim.run_protocol(np.array([-0.3, 0.3]), np.zeros(2), log_cap=2 * n)
        assert got["status"] == 0
        assert got["log_spin"].tolist() == list(range(n)) * 2
        assert sim.profile()["fallbacks"] > 0


def test_custom_geometry_matches_oracle(B, oracle):
    rng = np.random.default_rng(9)
    n = 300
    x = rng.uniform(0, 12, n)
    y = rng.uniform(0, 12, n)
    t = rng.uniform(0, math.pi, n)
    hx, hy = I.rotation_protocol(50, 7.0, 0.12)
    for prec in (FP64, FP32):
        sim = B.Sim.custom(x, y, t)
        sim.set_params(B.make_params(alpha=2e-3, cutoff=2.5, k_disorder=0.1, seed=3,
                                     precision=prec))
        # (300 islands: every column offset fits 16 bits, which the FP32 path reads)
        assert sim.info().col_offsets16 == (1 if prec == FP32 else 0)
        S = oracle.Sim(x, y, t, sim.hk(), alpha=2e-3, cutoff_abs=2.5)
        ref = S.run(np.ones(n, dtype=np.int8), hx, hy)
        got = sim.run_protocol(hx, hy)
        assert got["hash"] == ref["hash"], first_divergence(
            ref["log_step"], ref["log_spin"], got["log_step"], got["log_spin"])


def test_custom_geometry_far_indices_matches_oracle(B, oracle):
    # Islands in random order: neighbours lie up to the whole array apart in index,
    # so the FP32 sweeps cannot use 16-bit column offsets and read the 32-bit
    # columns (arrays of at most 32,768 islands, and lattices in their canonical
    # order, always fit 16 bits); above 32,768 islands the multi-flip relax runs.
    rng = np.random.default_rng(21)
    n = 50_000
    side = math.sqrt(n)
    x = rng.uniform(0, side, n)
    y = rng.uniform(0, side, n)
    t = rng.uniform(0, math.pi, n)
    hx, hy = I.rotation_protocol(10, 9.0, 0.11)
    for prec in (FP32, FP64):
        sim = B.Sim.custom(x, y, t)
        sim.set_params(B.make_params(alpha=2e-3, cutoff=2.0, k_disorder=0.1, seed=5,
                                     precision=prec))
        assert sim.info().col_offsets16 == 0
        if prec == FP32:
            rp, col, _, _ = sim.csr()
            rows = np.repeat(np.arange(n), np.diff(rp))
            assert np.abs(col.astype(np.int64) - rows).max() > 32767
            S = oracle.Sim(x, y, t, sim.hk(), alpha=2e-3, cutoff_abs=2.0)
            ref = S.run(np.ones(n, dtype=np.int8), hx, hy)
        got = sim.run_protocol(hx, hy)
        assert sum(ref["flips_per_step"]) > 1000
        assert got["hash"] == ref["hash"], first_divergence(
            ref["log_step"], ref["log_spin"], got["log_step"], got["log_spin"])


def test_flip_guard_reports_not_converged(B):
    w = small(I.SQUARE, 6, max_flips_per_step=5)
    sim = lib_sim(w)
    got = sim.run_protocol(np.array([-0.4]), np.array([-0.4]))
    assert got["status"] == B.FS_ERR_NOT_CONVERGED
    assert got["n_flips"] == 5


def test_empty_protocol_and_relax(B, oracle):
    w = small(I.SQUARE, 5)
    sim = lib_sim(w)
    got = sim.run_protocol(np.zeros(0), np.zeros(0))
    assert got["n_flips"] == 0 and got["hash"] == B.hash_init()
    sim.set_field(-0.25, -0.25, step=3)
    nf, log = sim.relax(log_cap=10_000)
    S = oracle_sim(oracle, w)
    ref = S.run(np.ones(S.n, dtype=np.int8), np.array([-0.25]), np.array([-0.25]), step0=3)
    assert nf == ref["n_flips"]
    np.testing.assert_array_equal(log, ref["log_spin"])


def test_resume_split_protocol(B, oracle):
    w = small(I.KAGOME, 10, sigma_th=0.01)
    hx, hy = I.rotation_protocol(80, 4.5, 0.12)
    for prec in (FP64, FP32):
        sim = lib_sim(w, precision=prec)
        full = sim.run_protocol(hx, hy)
        sim2 = lib_sim(w, precision=prec)
        a = sim2.run_protocol(hx[:37], hy[:37])
        spins = sim2.spins()
        sim3 = lib_sim(w, precision=prec)
        sim3.set_spins(spins)
        b = sim3.run_protocol(hx[37:], hy[37:], step0=37, hash_in=a["hash"])
        assert b["hash"] == full["hash"]
        np.testing.assert_array_equal(sim3.spins(), sim.spins())


def test_log_shorter_than_flips(B):
    w = small(I.SQUARE, 8)
    sim = lib_sim(w)
    hx, hy = I.protocol_of(("ramp", (40, 45.0, 0.3)))
    full = sim.run_protocol(hx, hy)
    sim2 = lib_sim(w)
    part = sim2.run_protocol(hx, hy, log_cap=10)
    assert part["hash"] == full["hash"] and part["n_flips"] == full["n_flips"]
    np.testing.assert_array_equal(part["log_spin"], full["log_spin"][:10])


# ---------------------------------------------------------------------------
# Batches
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("schedule", [1, 2, 3])  # FS_BATCH_PERSISTENT, _PER_STEP, _TWO_CHAINS
def test_batch_equals_solo_and_oracle(B, oracle, prec, schedule):
    rng = np.random.default_rng(4)
    sides = rng.integers(3, 15, size=12)
    hx, hy = I.ramp_protocol(50, 45.0, 0.3)
    members = []
    for q, s in enumerate(sides):
        w = small(I.SQUARE, int(s), seed=1000 + q)
        members.append((w, lib_sim(w, precision=prec)))
    out = B.batch_run_protocol([m for _, m in members], hx, hy, with_counts=True,
                               schedule=schedule)
    for q, (w, _) in enumerate(members):
        S = oracle_sim(oracle, w)
        ref = S.run(np.ones(S.n, dtype=np.int8), hx, hy)
        assert int(out["hash"][q]) == ref["hash"]
        assert out["n_flips"][q] == ref["n_flips"]
        np.testing.assert_array_equal(out["flips_per_step"][q], ref["flips_per_step"])
        solo = lib_sim(w, precision=prec).run_protocol(hx, hy)
        assert solo["hash"] == ref["hash"]


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_persistent_batch_mixed_members_match_oracle(B, oracle, prec):
    """The persistent schedule on members of every geometry and of very different
    sizes (a one-node tree of 24 islands up to ~20,000 islands, whose sweep spans many
    claimed chunks), with and without thermal noise, more members than one CTA each
    can hold at once: every member's flips per step, flip count and hash equal the
    oracle's, and the final spins equal a per-step batch run's."""
    rng = np.random.default_rng(9)
    hx, hy = I.ramp_protocol(40, 30.0, 0.3)
    ws = []
    kinds = [I.SQUARE, I.PINWHEEL, I.KAGOME]
    for q in range(20):
        kind = kinds[q % 3]
        n = int(rng.integers(3, 30))
        ws.append(small(kind, n, seed=2000 + q, sigma_th=0.004 if q % 4 == 1 else 0.0))
    ws.append(small(I.SQUARE, 3, seed=2100))    # 24 islands: a one-node tree
    ws.append(small(I.KAGOME, 80, seed=2101))   # 19,519 islands
    sims = [lib_sim(w, precision=prec) for w in ws]
    out = B.batch_run_protocol(sims, hx, hy, with_counts=True, schedule=1)
    assert (out["status"] == 0).all()
    spins = [s.spins() for s in sims]
    sims2 = [lib_sim(w, precision=prec) for w in ws]
    B.batch_run_protocol(sims2, hx, hy, schedule=2)
    for q, w in enumerate(ws):
        S = oracle_sim(oracle, w)
        ref = S.run(np.ones(S.n, dtype=np.int8), hx, hy)
        assert int(out["hash"][q]) == ref["hash"], q
        assert out["n_flips"][q] == ref["n_flips"], q
        np.testing.assert_array_equal(out["flips_per_step"][q], ref["flips_per_step"])
        np.testing.assert_array_equal(spins[q], sims2[q].spins())


def test_batch_schedule_arguments(B):
    """An unknown schedule is refused; an empty protocol runs on every schedule and
    flips nothing."""
    sims = [lib_sim(small(I.SQUARE, n, seed=2300 + n), precision=FP32) for n in (4, 6)]
    hx, hy = I.ramp_protocol(10, 45.0, 0.3)
    with pytest.raises(B.FsError) as e:
        B.batch_run_protocol(sims, hx, hy, schedule=7)
    assert e.value.code == B.FS_ERR_INVALID
    for sched in (B.FS_BATCH_AUTO, B.FS_BATCH_PERSISTENT, B.FS_BATCH_PER_STEP,
                  B.FS_BATCH_TWO_CHAINS):
        out = B.batch_run_protocol(sims, hx[:0], hy[:0], schedule=sched)
        assert (out["n_flips"] == 0).all() and (out["status"] == 0).all()


def test_persistent_batch_twice_in_a_row(B, oracle):
    """Two persistent protocols in a row on the same members (the second continues
    from the first's final state, with a new step offset): both equal solo runs."""
    hx, hy = I.ramp_protocol(30, 45.0, 0.3)
    ws = [small(I.SQUARE, n, seed=2200 + n) for n in (4, 9, 17, 33)]
    sims = [lib_sim(w, precision=FP32) for w in ws]
    solo = [lib_sim(w, precision=FP32) for w in ws]
    for rep in range(2):
        out = B.batch_run_protocol(sims, hx, hy, schedule=1)
        for q, s in enumerate(solo):
            r = s.run_protocol(hx, hy)
            assert int(out["n_flips"][q]) == r["n_flips"]
        for q in range(len(ws)):
            np.testing.assert_array_equal(sims[q].spins(), solo[q].spins())


# ---------------------------------------------------------------------------
# Serving: each result is the same alone and in the mix
# ---------------------------------------------------------------------------

def _served_params(B, r, prec):
    return B.make_params(alpha=r["alpha"], hk=r["hk"], k_disorder=r["k_disorder"],
                         cutoff=r["cutoff"], sigma_th=r["sigma_th"], seed=r["seed"],
                         precision=prec)


def test_server_results_equal_solo_runs_and_oracle(B, oracle):
    """30 requests of mixed geometry, size (200..6000 islands), precision and thermal
    noise, submitted in three waves so that later ones arrive while earlier ones run
    and a small slot count makes them wait for slots to free up: every served
    result (sequence hash, flip count, final spins) equals the oracle's run of the
    same request and a solo library run of it."""
    import time
    reqs = I.serving_stream(n_requests=30, n_lo=200, n_hi=6000, steps_lo=20, steps_hi=80,
                            seed=21)
    for q, r in enumerate(reqs):
        r["sigma_th"] = 0.004 if q % 3 == 2 else 0.0
    srv = B.Server(hbm_budget=2 << 30, max_active=6)
    entries = []
    seen = {}  # results polled early (a result is handed out once)
    overlapped = 0
    for wave in range(3):
        for q in range(10 * wave, 10 * wave + 10):
            r = reqs[q]
            hx, hy = I.protocol_of(r["protocol"])
            prec = FP32 if q % 2 else FP64
            n = B.Sim.geometry(r["kind"], r["nx"], r["ny"]).n
            buf = np.zeros(n, dtype=np.int8)
            t = srv.submit(r["kind"], r["nx"], r["ny"], _served_params(B, r, prec), hx, hy,
                           spins_out=buf)
            entries.append((t, r, prec, hx, hy, buf))
        if wave < 2:
            # a short pause (the wave's requests are admitted and start), then the
            # requests still in flight when the next wave arrives
            time.sleep(0.002)
            for e in entries:
                if e[0] not in seen:
                    res = srv.poll(e[0])
                    if res is None:
                        overlapped += 1
                    else:
                        seen[e[0]] = res
    srv.drain()
    assert overlapped > 0
    for t, r, prec, hx, hy, buf in entries:
        res = seen[t] if t in seen else srv.poll(t)
        assert res is not None and res["status"] == 0
        w = small(r["kind"], r["nx"], alpha=r["alpha"], cutoff=r["cutoff"], seed=r["seed"],
                  sigma_th=r["sigma_th"])
        ref = oracle_sim(oracle, w).run(np.ones(res["n"], dtype=np.int8), hx, hy)
        assert ref["status"] == 0
        assert (res["hash"], res["n_flips"]) == (ref["hash"], ref["n_flips"]), (t, prec)
        np.testing.assert_array_equal(buf, ref["spins"])
        solo_sim = lib_sim(w, precision=prec)
        solo = solo_sim.run_protocol(hx, hy)
        assert (solo["hash"], solo["n_flips"]) == (res["hash"], res["n_flips"])
        np.testing.assert_array_equal(buf, solo_sim.spins())
        solo_sim.close()
    srv.close()


@pytest.mark.parametrize("kind,astroid,sigma", [(I.SQUARE, (1, 1, 3, 3), 0.0),
                                                (I.PINWHEEL, (0.28, 1, 4.8, 3), 0.0),
                                                (I.KAGOME, (0.42, 1, 1.7, 3.4), 0.006),
                                                (I.SQUARE, (0.38, 1, 1.5, 3.2), 0.01)])
def test_fp32_bounds_bracket_fp64(B, kind, astroid, sigma):
    # the FP32 evaluation's [lo, hi] must contain the FS_FP64 value of the LHS
    b, c, beta, gamma = astroid
    w = small(kind, 12, b=b, c=c, beta=beta, gamma=gamma, sigma_th=sigma, alpha=4e-3)
    s32 = lib_sim(w, precision=FP32)
    s64 = lib_sim(w, precision=FP64)
    rng = np.random.default_rng(5)
    worst = 0.0
    for trial in range(12):
        s = I.random_spins(s32.n, trial)
        ang = rng.uniform(0, 2 * math.pi)
        mag = [0.0, 0.05, 0.2, 0.4][trial % 4]
        for sim in (s32, s64):
            sim.set_spins(s)
            sim.set_field(mag * math.cos(ang), mag * math.sin(ang), step=trial)
        l32, lo, hi = s32.lhs(bounds=True)
        l64 = s64.lhs()
        assert (lo <= l64).all() and (l64 <= hi).all(), trial
        near = l64 > 0.5  # the band matters only near the switching threshold
        if near.any():
            worst = max(worst, float(np.max(hi[near] - lo[near])))
    assert worst < 2e-3


def test_fp32_thermal_draw_within_bound(B):
    # alpha = 0 and no external field: the total field is the thermal draw alone,
    # FP32 Box-Muller in one simulation, FP64 in the other. The FP32 path's error
    # model takes |th32 - th64| <= 12 u (|th_par| + |th_perp|), u = 2^-24, derived
    # from the documented ulp bounds of logf, log1pf, sqrtf and sincospif.
    w = small(I.KAGOME, 60, sigma_th=1.0, alpha=0.0)
    s32 = lib_sim(w, precision=FP32)
    s64 = lib_sim(w, precision=FP64)
    worst = 0.0
    for step in range(0, 40, 3):
        for sim in (s32, s64):
            sim.set_field(0.0, 0.0, step=step)
        p32, q32 = s32.fields()
        p64, q64 = s64.fields()
        r = np.abs(p64) + np.abs(q64)
        err = np.maximum(np.abs(p32 - p64), np.abs(q32 - q64)) / r
        worst = max(worst, float(err.max()))
    assert worst <= 12 * 2.0**-24, worst


# ---------------------------------------------------------------------------
# Caller-owned workspace (fs_workspace_bytes, fs_bind_workspace)
# ---------------------------------------------------------------------------

def _params_of(B, w, prec):
    return B.make_params(alpha=w["alpha"], hk=w["hk"], k_disorder=w["k_disorder"], b=w["b"],
                         c=w["c"], beta=w["beta"], gamma=w["gamma"], cutoff=w["cutoff"],
                         sigma_th=w["sigma_th"], seed=w["seed"], precision=prec)


@pytest.mark.parametrize("kind,n,sigma,prec", [(I.SQUARE, 16, 0.0, FP64),
                                               (I.PINWHEEL, 12, 0.0, FP32),
                                               (I.KAGOME, 10, 0.004, FP32),
                                               (I.KAGOME, 10, 0.004, FP64)])
def test_bound_workspace_of_the_stated_size_runs_identically(B, kind, n, sigma, prec):
    """A simulation built inside a torch-owned buffer of exactly fs_workspace_bytes
    bytes gives the same flips as one on the library's pool; one 256 bytes short
    fails with FS_ERR_OOM and can be bound again."""
    import torch
    w = small(kind, n, sigma_th=sigma)
    p = _params_of(B, w, prec)
    hx, hy = I.ramp_protocol(120, 30.0, 0.3)
    ref = lib_sim(w, precision=prec)
    r0 = ref.run_protocol(hx, hy)
    s0 = ref.spins()
    state_bytes = ref.info().device_bytes
    ref.close()

    sim = B.Sim.geometry(kind, n, n)
    need = sim.workspace_bytes(p)
    assert need > state_bytes > 0
    short = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    sim.bind_workspace(short.data_ptr(), short.numel())
    with pytest.raises(B.FsError) as e:
        sim.set_params(p)
    assert e.value.code == B.FS_ERR_OOM
    buf = torch.empty(need, dtype=torch.uint8, device="cuda")
    sim.bind_workspace(buf.data_ptr(), buf.numel(), torch.cuda.current_stream().cuda_stream)
    sim.set_params(p)
    assert sim.info().device_bytes == state_bytes
    r1 = sim.run_protocol(hx, hy)
    assert (r1["n_flips"], r1["hash"]) == (r0["n_flips"], r0["hash"])
    np.testing.assert_array_equal(r1["log_spin"], r0["log_spin"])
    np.testing.assert_array_equal(sim.spins(), s0)
    # bound state is the caller's: binding again needs new parameters first
    with pytest.raises(B.FsError) as e:
        sim.bind_workspace(0, 0)
    assert e.value.code == B.FS_ERR_STATE
    sim.close()
    del buf, short


def test_workspace_must_be_device_memory(B):
    host = np.zeros(1 << 16, dtype=np.uint8)
    addr = (host.ctypes.data + 255) & ~255
    sim = B.Sim.geometry(I.SQUARE, 4, 4)
    with pytest.raises(B.FsError) as e:
        sim.bind_workspace(addr, 1 << 15)
    assert e.value.code == B.FS_ERR_INVALID
    sim.close()
