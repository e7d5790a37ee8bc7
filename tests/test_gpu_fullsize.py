"""The CUDA path at the workloads' full sizes, in the launch configuration the
benchmark uses, against values the oracle wrote (tests/golden/, by
tests/golden/make_golden.py) and against the oracle's fields sampled at the
device's final state. Flip sequences bit-exact; fields within 1e-12 (FS_FP64)
or 1e-5 (FS_FP32_RECHECK) of max|h|."""
import json
import math
import os

import numpy as np
import pytest

from paper_2002_11401_b300 import inputs as I

from .helpers import lib_sim, oracle_sim

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def gold(name):
    with open(os.path.join(GOLD, name + ".json")) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def B():
    from paper_2002_11401_b300 import build
    build.build()
    from paper_2002_11401_b300 import binding
    return binding


def _check_against(g, got):
    assert got["n_flips"] == g["n_flips"]
    assert f"{got['hash']:#018x}" == g["seq_hash"]
    assert got["flips_per_step"].tolist() == g["flips_per_step"]
    if "log_spin" in g:
        m = len(g["log_spin"])
        assert got["log_spin"][:m].tolist() == g["log_spin"]
        assert got["log_step"][:m].tolist() == g["log_step"]


@pytest.mark.parametrize("prec", [0, 1])
def test_pinwheel300_prefix_matches_oracle(B, prec):
    g = gold("pinwheel300_prefix40")
    w = I.WORKLOADS["pinwheel300"]
    hx, hy = I.protocol_of(w["protocol"])
    sim = lib_sim(w, precision=prec)
    sim.autotune()
    got = sim.run_protocol(hx[:40], hy[:40])
    _check_against(g, got)


@pytest.mark.parametrize("prec", [0, 1])
def test_kagome1000_prefix_matches_oracle(B, prec):
    g = gold("kagome1000_prefix3")
    w = I.WORKLOADS["kagome1000"]
    hx, hy = I.protocol_of(w["protocol"])
    sim = lib_sim(w, precision=prec)
    got = sim.run_protocol(hx[:3], hy[:3])
    _check_against(g, got)


def test_pinwheel300_full_protocol_invariants_and_fields(B, oracle):
    # the whole 1000-step protocol on both paths, with and without the resweep:
    # the oracle's sequence (flips per step and hash); the final state is saturated
    # along +0.25 T at 30 degrees; the fields at the final state agree with the
    # oracle's recomputation from positions
    w = I.WORKLOADS["pinwheel300"]
    hx, hy = I.protocol_of(w["protocol"])
    runs = {}
    for prec in (0, 1):
        for rs in (True, False):
            sim = lib_sim(w, precision=prec)
            r = sim.run_protocol(hx, hy, resweep=rs, log_cap=0)
            assert r["status"] == 0
            runs[(prec, rs)] = (r, sim)
    hashes = {k: v[0]["hash"] for k, v in runs.items()}
    assert len(set(hashes.values())) == 1, hashes
    # the whole protocol as the oracle ran it (tests/golden/make_golden.py --full)
    g = gold("pinwheel300_full")
    for (r, _) in runs.values():
        _check_against(g, r)
    r, sim = runs[(0, True)]
    assert r["n_flips"] == 270900
    s = sim.spins()
    x, y, th = sim.geometry_arrays()
    align = np.cos(th - math.radians(30.0))
    assert (s == np.where(align > 0, 1, -1)).all()
    S = oracle_sim(oracle, w)
    op, oq = S.fields(s, hx[-1], hy[-1], step=len(hx) - 1)
    hp, hq = sim.fields()
    scale = max(np.abs(op).max(), np.abs(oq).max())
    assert max(np.abs(hp - op).max(), np.abs(hq - oq).max()) <= 1e-12 * scale
    r32, sim32 = runs[(1, True)]
    p32, q32 = sim32.fields()
    assert max(np.abs(p32 - op).max(), np.abs(q32 - oq).max()) <= 1e-5 * scale


@pytest.mark.parametrize("prec,mode", [(0, 0), (1, 0), (1, 1)])
def test_kagome1000_full_protocol_matches_oracle(B, prec, mode):
    # the whole 720-step rotation with thermal noise (3.0M islands, 3,146,771 flips):
    # flips per step and the sequence hash as the oracle ran it; the default relax
    # (multi-flip rounds at this size) and the single-flip chain
    g = gold("kagome1000_full")
    w = I.WORKLOADS["kagome1000"]
    hx, hy = I.protocol_of(w["protocol"])
    sim = lib_sim(w, precision=prec)
    sim.set_relax_mode(mode)
    got = sim.run_protocol(hx, hy, log_cap=0)
    assert got["status"] == 0
    _check_against(g, got)


@pytest.mark.parametrize("prec", [0, 1])
def test_pinwheel300_full_protocol_multi_flip(B, prec):
    g = gold("pinwheel300_full")
    w = I.WORKLOADS["pinwheel300"]
    hx, hy = I.protocol_of(w["protocol"])
    sim = lib_sim(w, precision=prec)
    sim.set_relax_mode(B.FS_RELAX_MULTI)
    got = sim.run_protocol(hx, hy, log_cap=0)
    assert got["status"] == 0
    _check_against(g, got)


def test_kagome1000_fields_at_full_size(B, oracle):
    # a random state of the 3.0M-island array with its thermal draw: every field
    w = I.WORKLOADS["kagome1000"]
    s = I.random_spins(3003999, 77)
    S = oracle_sim(oracle, w)
    op, oq = S.fields(s, 0.06, -0.03, step=123)
    scale = max(np.abs(op).max(), np.abs(oq).max())
    for prec, tol in ((0, 1e-12), (1, 1e-5)):
        sim = lib_sim(w, precision=prec)
        sim.set_spins(s)
        sim.set_field(0.06, -0.03, step=123)
        hp, hq = sim.fields()
        assert max(np.abs(hp - op).max(), np.abs(hq - oq).max()) <= tol * scale


@pytest.mark.parametrize("schedule", [0, 1, 2])  # FS_BATCH_AUTO (two chains), _PERSISTENT, _PER_STEP
def test_ensemble512_members_match_oracle(B, schedule):
    members, proto = I.ensemble_workload()
    hx, hy = I.protocol_of(proto)
    sims = [lib_sim(m, precision=1) for m in members]
    out = B.batch_run_protocol(sims, hx, hy, with_counts=True, schedule=schedule)
    assert (out["status"] == 0).all()
    for q in (0, 37, 211, 500):
        g = gold(f"ensemble512_member{q}")
        assert int(out["n_flips"][q]) == g["n_flips"]
        assert f"{int(out['hash'][q]):#018x}" == g["seq_hash"]
        assert out["flips_per_step"][q].tolist() == g["flips_per_step"]
    # every member of a square array under this ramp flips each island twice
    ns = np.array([s.n for s in sims])
    assert (out["n_flips"] == 2 * ns).all()
