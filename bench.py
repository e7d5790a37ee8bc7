#!/usr/bin/env python
"""Benchmark of the flatspin relax loop on B300.

One step = one full field protocol of the pinwheel workload: a 300 x 300
pinwheel array (180,600 islands, cutoff 5a, alpha 1e-3, h_k ~ N(0.2, 5%), seed 1)
driven from -0.25 T to +0.25 T at 30 degrees in 1000 field steps, each step a
full field-and-margin sweep followed by a relax to a fixed point (Sec.
"Dynamics"), starting from all spins +1. Inputs are synthetic and resident in HBM
for `value`; `e2e` goes through the host-buffer C ABI call.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch with torch.distributed.run; each rank runs an independent
replica (a single relax is a serial chain and does not shard).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2002_11401_b300 import inputs as I  # noqa: E402

METRIC = ("spin-flips/sec and field-steps/sec at 1 B300 (% HBM roofline); "
          "served p50/p99 latency")
UNIT = "spin-flips/s"
WORKLOAD = "pinwheel300"


def workload_desc(w):
    """The workload alone (both arms run it; the arithmetic is in config["path"])."""
    return (f"pinwheel {w['nx']}x{w['ny']} cells (180,600 islands), cutoff {w['cutoff']:g}a, "
            f"alpha {w['alpha']:g}, h_k N(0.2 T, 5%) seed {w['seed']}, b=c=1 beta=gamma=3, "
            f"field loop -0.25 -> +0.25 T at 30 deg in 1000 steps from all +1")


def sweep_bytes(n: int, nnz: int, fp32: bool, resweep: bool, thermal: bool) -> int:
    """Algorithmic bytes of one field-and-margin sweep. Per pair: the column index
    and the (P, Q) coefficients of the path's width (4 + 8 or 4 + 16); per row: its
    pointer (8). Per island: spin, angle class, 1/(b h_k) and 1/(c h_k) read
    (1 + 2 + 8); the relax's 32-byte record, key and exact value written
    (32 + 8 + 8); on the FP64 path the 64-bit sums written (or, without the
    resweep, read: 16), on the FP32 path without the resweep the 32-bit sums read
    (8); with thermal noise, the step's FP32 draw written (8)."""
    per_island = (1 + 2 + 8 + 32 + 8 + 8 + (0 if fp32 else 16)
                  + (8 if fp32 and not resweep else 0) + (8 if thermal else 0))
    if not resweep:
        return n * per_island
    return (12 if fp32 else 20) * nnz + 8 * (n + 1) + n * per_island


# DRAM bytes per launch (read + write) of the dominant kernels on this workload, from
# one ncu capture of every launch of one protocol (summarised with the profiles),
# with a hash of the kernel sources that were profiled: a changed kernel reports null.
TRAFFIC = {
    "k_relax": {"bytes_per_launch": 2.132e6, "sources": ("fs_relax.cu", "fs_common.cuh"),
                "sha256_16": "866eb60c88098762"},
    "k_sweep": {"bytes_per_launch": 348.24e6, "sources": ("fs_sweep.cu", "fs_common.cuh"),
                "sha256_16": "b620db53096b4552"},
}


def traffic_of(kernel: str):
    import hashlib
    t = TRAFFIC[kernel]
    m = hashlib.sha256()
    for name in t["sources"]:
        with open(os.path.join(ROOT, "paper_2002_11401_b300", "csrc", name), "rb") as f:
            m.update(f.read())
    return t["bytes_per_launch"] if m.hexdigest()[:16] == t["sha256_16"] else None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate(ms: float, units: float, dist=None, device: str = "cpu"):
    """Whole-job figures over independent replicas: the slowest rank's time and
    the units of all ranks (no data-path collective; one all-reduce each for
    the timing and the count)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms, units
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def cpu_baseline(w, budget_s=20.0):
    """The FP64 oracle on the host cores, on a bounded prefix of the protocol (the
    first field steps, including the initial avalanche), in flips per second."""
    import oracle as O
    O.build()
    from tests.helpers import oracle_sim
    cores = os.cpu_count() or 1
    O.set_threads(cores)
    S = oracle_sim(O, w)
    hx, hy = I.protocol_of(w["protocol"])
    s = np.ones(S.n, dtype=np.int8)
    flips, steps, t0 = 0, 0, time.perf_counter()
    while steps < len(hx) and time.perf_counter() - t0 < budget_s:
        r = S.run(s, hx[steps:steps + 1], hy[steps:steps + 1], step0=steps, log_cap=0)
        s = r["spins"]
        flips += r["n_flips"]
        steps += 1
    dt = time.perf_counter() - t0
    return {"value": flips / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {steps} of 1000 field steps of the same workload "
                      f"({flips} flips, {dt:.1f} s, OpenMP over rows for field sums)",
            "field_steps_per_s": steps / dt}


def run_reference(args, w, rank):
    """Reference arm: the FP64 oracle as it stands, on the host cores."""
    if rank != 0:
        return
    steps, warm = max(args.steps, 1), args.warmup
    per = max(3.0, min(30.0, 150.0 / max(steps + warm, 1)))
    for _ in range(warm):
        cpu_baseline(w, budget_s=per / 3)
    vals, t0 = [], time.perf_counter()
    for _ in range(steps):
        vals.append(cpu_baseline(w, budget_s=per))
    dt = time.perf_counter() - t0
    v = float(np.mean([x["value"] for x in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0,
            "steps": steps, "warmup": warm, "ms_per_step": dt * 1000 / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_desc(w),
                       "path": "FP64 oracle on the host cores, dipolar fields recomputed "
                               "from scratch every field step"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"],
                             "kind": "oracle", "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--resweep", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    w = I.WORKLOADS[WORKLOAD]
    if args.impl == "reference":
        run_reference(args, w, rank)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2002_11401_b300 import binding as B
    from paper_2002_11401_b300 import build as BLD
    BLD.build()
    B.load()

    prec = B.FS_FP32_RECHECK if args.precision == "fp32" else B.FS_FP64
    prec_name = "FP32 + FP64 recheck" if prec == B.FS_FP32_RECHECK else "FP64"
    stream = torch.cuda.Stream()
    sim = B.Sim.geometry(w["kind"], w["nx"], w["ny"], w["a"])
    sim.set_stream(stream.cuda_stream)
    sim.set_params(B.make_params(alpha=w["alpha"], hk=w["hk"], k_disorder=w["k_disorder"],
                                 b=w["b"], c=w["c"], beta=w["beta"], gamma=w["gamma"],
                                 cutoff=w["cutoff"], sigma_th=w["sigma_th"], seed=w["seed"],
                                 precision=prec))
    info = sim.info()
    lanes = sim.autotune()
    hx, hy = I.protocol_of(w["protocol"])
    K = len(hx)
    with torch.cuda.stream(stream):
        d_hx = torch.from_numpy(hx).cuda()
        d_hy = torch.from_numpy(hy).cuda()
        d_init = torch.ones(sim.n, dtype=torch.int8, device="cuda")
        d_out = torch.zeros(4, dtype=torch.int64, device="cuda")
    stream.synchronize()

    def step():
        sim.set_spins_dev(d_init.data_ptr())
        sim.run_protocol_dev(d_hx.data_ptr(), d_hy.data_ptr(), K, resweep=bool(args.resweep),
                             d_out=d_out.data_ptr())

    for _ in range(max(args.warmup, 0)):
        step()
    stream.synchronize()
    out0 = d_out.cpu().tolist()
    flips_per_protocol = int(out0[1])
    hash0 = int(out0[2]) & 0xFFFFFFFFFFFFFFFF

    clocks = Clocks(local)
    sim.set_profiling(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    prof = sim.profile()
    sim.set_profiling(False)
    out1 = d_out.cpu().tolist()
    assert int(out1[0]) == 0, f"protocol status {out1[0]}"
    if args.warmup <= 0:  # nothing to compare with: the timed steps define the figures
        flips_per_protocol = int(out1[1])
        hash0 = int(out1[2]) & 0xFFFFFFFFFFFFFFFF
    assert int(out1[1]) == flips_per_protocol and (int(out1[2]) & 0xFFFFFFFFFFFFFFFF) == hash0, \
        "timed steps diverged from the warm-up steps"
    ms, units = aggregate(ms, flips_per_protocol * args.steps, dist, device="cuda")
    value = units / (ms / 1000.0)
    field_steps = K * args.steps * world / (ms / 1000.0)

    # ---- roofline of the kernels, from the live per-launch timings ----------------
    peak, peak_kind = peaks()
    n, nnz = info.n, info.nnz
    avg_deg = nnz / n
    fp32 = prec == B.FS_FP32_RECHECK
    # per flip and neighbour: the row entry (column, P and transposed Q; both
    # widths on the FP32 path), the neighbour's state read (exact sums, 32-bit sums,
    # key, spin, angle class, 1/(b h_k) and 1/(c h_k) in FP32 (8 B) or FP64 (16 B),
    # row pointers for the next-pick prediction) and written back (sums, key, lower
    # bound, exact value)
    per_nb = (4 + 4 + 4 + 8 + 8) + (16 + 8 + 8 + 1 + 2 + 8 + 16) + (16 + 8 + 8 + 8 + 4) \
        if fp32 else (4 + 8 + 8) + (16 + 8 + 1 + 2 + 16 + 8 + 16) + (16 + 8 + 8 + 4)
    relax_bytes = flips_per_protocol * avg_deg * per_nb * args.steps
    relax_s = prof["relax_ms"] / 1000.0
    sweep_unit = sweep_bytes(n, nnz, fp32, bool(args.resweep), w["sigma_th"] > 0)
    sweep_s = prof["sweep_ms"] / 1000.0
    n_sweeps = max(prof["sweep_launches"], 1)
    relax_launch_ms = prof["relax_ms"] / max(prof["relax_launches"], 1)
    sweep_launch_ms = prof["sweep_ms"] / n_sweeps
    roof_relax = {"kernel": "k_relax", "bound": "hbm",
                  "achieved": relax_bytes / relax_s / 1e9 if relax_s > 0 else 0.0,
                  "peak": peak, "unit": "GB/s",
                  "frac": (relax_bytes / relax_s / 1e9) / peak if relax_s > 0 else 0.0,
                  "traffic": traffic_of("k_relax") if fp32 and args.resweep else None,
                  "peak_kind": peak_kind,
                  "avg_launch_ms": relax_launch_ms,
                  "share_of_step": prof["relax_ms"] / ms if ms > 0 else None,
                  "bytes_per_launch": relax_bytes / max(prof["relax_launches"], 1),
                  "note": "serial flip chain: latency-bound; bytes per flip = "
                          f"{avg_deg:.1f} neighbours x {per_nb} B; traffic below them "
                          "means L2 hits"}
    roof_sweep = {"kernel": "k_sweep", "bound": "hbm",
                  "achieved": sweep_unit / (sweep_launch_ms / 1000.0) / 1e9,
                  "peak": peak, "unit": "GB/s",
                  "frac": sweep_unit / (sweep_launch_ms / 1000.0) / 1e9 / peak,
                  "traffic": traffic_of("k_sweep") if fp32 and args.resweep else None,
                  "peak_kind": peak_kind, "avg_launch_ms": sweep_launch_ms,
                  "bytes_per_launch": sweep_unit,
                  "share_of_step": prof["sweep_ms"] / ms if ms > 0 else None}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "i32+f32, f64 recheck" if fp32 else "i64+f64", "data": "synthetic",
            "config": {"workload": workload_desc(w),
                       "path": f"{prec_name}, " + ("full dipolar resweep every field step"
                                                   if args.resweep else "exact incremental sums"),
                       "islands": n,
                       "neighbour_pairs": nnz, "field_steps_per_step": K,
                       "flips_per_step": flips_per_protocol, "seq_hash": f"{hash0:#018x}",
                       "l2": "inputs larger than L2 (neighbour tensors "
                             f"{info.device_bytes / 1e9:.2f} GB on the device)",
                       "parallelism": "replicas" if world > 1 else "single",
                       "sweep_lanes_per_row": lanes},
            "field_steps_per_s": field_steps,
            "roofline": roof_relax, "roofline_sweep": roof_sweep,
            "gpu_launches": args.steps * (3 * K + 1),
            "rechecks_per_flip": int(out1[3]) / max(flips_per_protocol, 1)}
    if clk:
        line["clocks"] = clk

    # ---- end to end through the host-buffer C ABI call --------------------------
    if not args.no_e2e:
        init = np.ones(sim.n, dtype=np.int8)
        sim.set_spins(init)
        r = sim.run_protocol(hx, hy, resweep=bool(args.resweep), log_cap=0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sim.set_spins(init)
            r = sim.run_protocol(hx, hy, resweep=bool(args.resweep), log_cap=0)
        dt = time.perf_counter() - t0
        line["e2e"] = {"value": r["n_flips"] * args.steps / dt, "unit": UNIT,
                       "h2d_bytes_per_step": int(init.nbytes + hx.nbytes + hy.nbytes),
                       "d2h_bytes_per_step": int(8 * K + 8 + 8 + 64)}
    # ---- the FP32 path's field error against the FS_FP64 path, at the final state ---
    if fp32 and rank == 0 and not args.no_e2e:
        ref = B.Sim.geometry(w["kind"], w["nx"], w["ny"], w["a"])
        ref.set_params(B.make_params(alpha=w["alpha"], hk=w["hk"], k_disorder=w["k_disorder"],
                                     b=w["b"], c=w["c"], beta=w["beta"], gamma=w["gamma"],
                                     cutoff=w["cutoff"], sigma_th=w["sigma_th"], seed=w["seed"],
                                     precision=B.FS_FP64))
        final = sim.spins()
        ref.set_spins(final)
        ref.set_field(float(hx[-1]), float(hy[-1]), step=K - 1)
        sim.set_field(float(hx[-1]), float(hy[-1]), step=K - 1)
        p64, q64 = ref.fields()
        p32, q32 = sim.fields()
        scale = max(float(np.abs(p64).max()), float(np.abs(q64).max()))
        err = max(float(np.abs(p32 - p64).max()), float(np.abs(q32 - q64).max()))
        line["fp32_field_error"] = {"max_abs_over_max_h": err / scale, "bound": 1e-5,
                                    "vs": "FS_FP64 path (= oracle to 1e-12) at the final state"}
        ref.close()
    if rank == 0 and not args.no_cpu and world >= 1:
        try:
            line["cpu_baseline"] = cpu_baseline(w)
        except Exception as exc:  # the baseline is context, not the measurement
            line["cpu_baseline"] = {"error": repr(exc)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
