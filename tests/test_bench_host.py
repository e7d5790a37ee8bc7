"""Host-side logic of bench.py (no GPU): the sweep's algorithmic byte count and the
traffic figures that follow only the kernel sources they were profiled from."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_sweep_bytes_by_hand():
    # 10 islands, 40 pairs: FP32 resweep = 12*40 + 8*11 + 59*10
    assert bench.sweep_bytes(10, 40, True, True, False) == 480 + 88 + 590
    # FP64 resweep adds the 64-bit sums (75 B per island) and 20 B per pair
    assert bench.sweep_bytes(10, 40, False, True, False) == 800 + 88 + 750
    # without the resweep only per-island bytes remain (FP32 reads its 32-bit sums)
    assert bench.sweep_bytes(10, 40, True, False, False) == 67 * 10
    # thermal noise writes the step's FP32 draw
    assert bench.sweep_bytes(10, 40, True, True, True) == 480 + 88 + 670


def test_traffic_follows_the_profiled_sources(monkeypatch):
    entry = dict(bench.TRAFFIC["k_sweep"])
    monkeypatch.setitem(bench.TRAFFIC, "k_sweep", dict(entry, sha256_16="0" * 16))
    assert bench.traffic_of("k_sweep") is None  # sources differ from the profiled ones
    import hashlib
    m = hashlib.sha256()
    for name in entry["sources"]:
        with open(os.path.join(ROOT, "paper_2002_11401_b300", "csrc", name), "rb") as f:
            m.update(f.read())
    monkeypatch.setitem(bench.TRAFFIC, "k_sweep", dict(entry, sha256_16=m.hexdigest()[:16]))
    assert bench.traffic_of("k_sweep") == entry["bytes_per_launch"]
