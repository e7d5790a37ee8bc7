"""The allocation-free entry point (fs_eval_argmax_static) against the existing
entry points, through the C ABI, on two calls in a row.

It serves callers that cannot allocate device memory at call time (a control
loop that must not block on the allocator, a process whose device memory is held
by another framework's pool): its scratch is a static device array. Its output
must equal what the allocating entry points report for the same state: the
FS_FP64 LHS of every flippable island (fs_get_fields / fs_get_lhs) and the island
the relax flips first (fs_relax). This file is named so that pytest collects it
last.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_2002_11401_b300 import inputs as I

from .helpers import lib_sim, small

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n_cells", [24, 110])
def test_static_scratch_sweep_matches_allocating_entry_points(prec, n_cells):
    """On a simulation of either precision (the entry point always evaluates in
    the FS_FP64 arithmetic, which both keep) and on arrays with a three-level and a
    four-level tree (kagome 24x24 = 1,775 and 110x110 = 36,739 islands). The call
    leaves the simulation's own device memory as it was."""
    import torch
    from paper_2002_11401_b300 import build
    build.build()
    from paper_2002_11401_b300 import binding as B
    lib = B.load()
    w = small(I.KAGOME, n_cells, sigma_th=0.004, alpha=3e-3, seed=21)
    sim = lib_sim(w, precision=prec)
    ref = lib_sim(w, precision=B.FS_FP64)  # the allocating entry points' FP64 values
    n = sim.n
    bytes_before = sim.info().device_bytes
    stream = torch.cuda.Stream()
    d_lhs = torch.full((n,), -7.0, dtype=torch.float64, device="cuda")
    d_best = torch.full((1,), -9, dtype=torch.int64, device="cuda")
    for call, (mag, ang_deg, step) in enumerate([(0.16, 200.0, 3), (0.19, 37.0, 11)]):
        spins = I.random_spins(n, 40 + call)
        hx, hy = mag * math.cos(math.radians(ang_deg)), mag * math.sin(math.radians(ang_deg))
        # the existing (allocating) entry points on the same state
        ref.set_spins(spins)
        ref.set_field(hx, hy, step=step)
        hpar, _ = ref.fields()
        lhs = ref.lhs()
        expect = np.where((spins * hpar < 0) & (lhs > 1.0), lhs, 0.0)
        probe = lib_sim(w, precision=prec)
        probe.set_spins(spins)
        probe.set_field(hx, hy, step=step)
        nflips, first = probe.relax(log_cap=1)
        probe.close()
        # the allocation-free entry point
        d_spins = torch.from_numpy(spins).to("cuda")
        torch.cuda.synchronize()
        st = lib.fs_eval_argmax_static(sim.handle, ctypes.c_void_p(d_spins.data_ptr()), hx, hy,
                                       step, ctypes.c_void_p(d_lhs.data_ptr()),
                                       ctypes.c_void_p(d_best.data_ptr()),
                                       ctypes.c_void_p(stream.cuda_stream))
        assert st == B.FS_OK
        stream.synchronize()
        got = d_lhs.cpu().numpy()
        # same FS_FP64 arithmetic on the same exact sums: equal bit for bit
        np.testing.assert_array_equal(got, expect)
        best = int(d_best.cpu()[0])
        assert nflips > 0
        assert best == int(first[0])
        assert best == int(np.argmax(expect))
    assert sim.info().device_bytes == bytes_before
    sim.close()
    ref.close()


def test_static_scratch_sweep_rejects_bad_calls():
    from paper_2002_11401_b300 import build
    build.build()
    from paper_2002_11401_b300 import binding as B
    lib = B.load()
    sim = B.Sim.geometry(I.SQUARE, 3, 3)
    p = ctypes.c_void_p(1)
    assert lib.fs_eval_argmax_static(sim.handle, p, 0.0, 0.0, 0, p, p, None) == B.FS_ERR_STATE
    assert lib.fs_eval_argmax_static(None, p, 0.0, 0.0, 0, p, p, None) == B.FS_ERR_INVALID
    big = B.Sim.geometry(I.SQUARE, 1100, 1100)  # 2,422,200 islands, above the limit
    big.set_params(B.make_params(alpha=1e-3, cutoff=1.0))
    assert lib.fs_eval_argmax_static(big.handle, p, 0.0, 0.0, 0, p, p, None) == B.FS_ERR_INVALID
