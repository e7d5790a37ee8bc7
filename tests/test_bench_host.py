"""Host-side logic of bench.py (no GPU): the algorithmic and layout byte counts, the
composition of the oracle's whole-protocol rate from its per-sweep and per-flip
costs, and the traffic figures that follow only the kernel sources they were
profiled from."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_bytes_by_hand():
    # per sweep: 12 nnz + 30 n (FP32), 20 nnz + 42 n (FP64)
    assert bench.sweep_alg_bytes(10, 40, True) == 480 + 300
    assert bench.sweep_alg_bytes(10, 40, False) == 800 + 420
    # per flip: 42 B (FP32) or 70 B (FP64) per neighbour
    assert bench.flip_alg_bytes(62.0, True) == 62 * 42
    assert bench.flip_alg_bytes(62.0, False) == 62 * 70


def test_layout_sweep_bytes_by_hand():
    # 10 islands, 40 pairs: FP32 resweep = 12*40 + 8*11 + 59*10
    assert bench.sweep_bytes(10, 40, True, True, False) == 480 + 88 + 590
    # the FP32 path's 16-bit column offsets: 10 B per pair
    assert bench.sweep_bytes(10, 40, True, True, False, True) == 400 + 88 + 590
    # FP64 resweep adds the 64-bit sums (75 B per island) and 20 B per pair
    assert bench.sweep_bytes(10, 40, False, True, False) == 800 + 88 + 750
    # without the resweep only per-island bytes remain (FP32 reads its 32-bit sums)
    assert bench.sweep_bytes(10, 40, True, False, False) == 67 * 10
    # thermal noise writes the step's FP32 draw
    assert bench.sweep_bytes(10, 40, True, True, True) == 480 + 88 + 670


def test_composed_rate():
    # 720 sweeps of 0.5 s and 1e6 flips of 10 us: 1e6 / (360 + 10) flips/s
    assert abs(bench.composed_rate(0.5, 1e-5, 720, 10**6) - 1e6 / 370.0) < 1e-9


def test_traffic_follows_the_profiled_sources(monkeypatch):
    import hashlib
    entry = dict(bench.TRAFFIC["k_sweep"], bytes_per_unit=10.0)
    m = hashlib.sha256()
    for name in entry["sources"]:
        with open(os.path.join(ROOT, "paper_2002_11401_b300", "csrc", name), "rb") as f:
            m.update(f.read())
    monkeypatch.setitem(bench.TRAFFIC, "k_sweep", dict(entry, sha256_16="0" * 16))
    assert bench.traffic_of("k_sweep", 5) is None  # sources differ from the profiled ones
    monkeypatch.setitem(bench.TRAFFIC, "k_sweep", dict(entry, sha256_16=m.hexdigest()[:16]))
    assert bench.traffic_of("k_sweep", 5) == 50.0
    monkeypatch.setitem(bench.TRAFFIC, "k_sweep", dict(entry, bytes_per_unit=None))
    assert bench.traffic_of("k_sweep", 5) is None  # no capture of these sources yet
