#!/usr/bin/env python
"""Benchmark of the flatspin relax loop on B300.

Headline workload: the kagome array of 1000 x 1000 hexagons (3,003,999 islands,
cutoff 4a, alpha 8e-4, h_k ~ N(0.2 T, 8%) seed 2, thermal field sigma 0.005 T
keyed by (seed, step, island)) under a 0.09 T field rotating in 720 steps of 0.5
degrees, from the polarised state, on the FP32 + FP64-recheck path. Each field
step is a full field-and-margin sweep followed by a relax to a fixed point (Sec.
"Dynamics"). One bench step is one tenth of the rotation, 72 consecutive field
steps, continuing from the previous step's state; every tenth step starts the
rotation again from the polarised state, so ten consecutive bench steps run the
whole protocol (3,146,771 flips), and every flip count per field step is
checked against the oracle's stored values. Inputs are synthetic and resident in
HBM for `value`; `e2e` goes through the host-buffer C ABI call.

Beside the headline, the line carries timed figures of the other
workloads: the square 16x16 ramp, the pinwheel 300x300 loop on both paths, the
kagome rotation on the FP64 path, the 512-member batched ensemble against the
same members run one at a time on the FP64 path, and a short Poisson stream
through the continuous-batching server (p50/p99 latency and throughput).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--extras all|none]
For N > 1 launch with torch.distributed.run; each rank runs an independent
replica (a single relax is a serial chain and does not shard).
"""
from __future__ import annotations

import argparse
import json
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
HEADLINE = "kagome1000"
CHUNK = 72          # field steps per bench step
CHUNKS = 10         # bench steps per whole rotation
GOLDEN = os.path.join(ROOT, "tests", "golden")


def workload_desc(w):
    """The workload alone (both arms run it; the arithmetic is in config["path"])."""
    return (f"kagome {w['nx']}x{w['ny']} hexagons (3,003,999 islands), cutoff "
            f"{w['cutoff']:g}a, alpha {w['alpha']:g}, h_k N(0.2 T, 8%) seed {w['seed']}, "
            f"b=c=1 beta=gamma=3, thermal sigma {w['sigma_th']:g} T, 0.09 T field rotating "
            f"in 720 steps of 0.5 deg from the polarised state")


def golden(name):
    with open(os.path.join(GOLDEN, f"{name}.json")) as f:
        return json.load(f)


# ---------------------------------------------------------------------------
# Byte counts
# ---------------------------------------------------------------------------

def sweep_alg_bytes(n: int, nnz: int, fp32: bool) -> int:
    """Algorithmic bytes of one field-and-margin sweep: per pair the column index
    and the (P, Q) coefficients (4 + 2w), per island its row pointer (8), spin and
    angle class (1 + 1), h_k (w), and the written fields (2w) and key (8); w = 4
    on the FP32 path, 8 on the FP64 path: 12 nnz + 30 n, or 20 nnz + 42 n."""
    return (12 * nnz + 30 * n) if fp32 else (20 * nnz + 42 * n)


def flip_alg_bytes(degree: float, fp32: bool) -> float:
    """Algorithmic bytes of one flip: per neighbour the column index and the
    coefficients (4 + 2w), the neighbour's fields read and written (4w), its h_k
    (w), its spin and angle class (2) and its key (8): 42 B (FP32) or 70 B (FP64)
    per neighbour."""
    return degree * (42.0 if fp32 else 70.0)


def sweep_bytes(n: int, nnz: int, fp32: bool, resweep: bool, thermal: bool,
                col16: bool = False) -> int:
    """Bytes of one sweep as this implementation lays its arrays out. Per pair: the
    column index and the (P, Q) coefficients of the path's width (4 + 8 or 4 + 16;
    with col16, the FP32 path's 16-bit column offsets: 2 + 8);
    per row: its pointer (8). Per island: spin, angle class, 1/(b h_k) and
    1/(c h_k) read (1 + 2 + 8); the relax's 32-byte record, key and exact value
    written (32 + 8 + 8); on the FP64 path the 64-bit sums written (or, without the
    resweep, read: 16), on the FP32 path without the resweep the 32-bit sums read
    (8); with thermal noise, the step's FP32 draw written (8)."""
    per_island = (1 + 2 + 8 + 32 + 8 + 8 + (0 if fp32 else 16)
                  + (8 if fp32 and not resweep else 0) + (8 if thermal else 0))
    if not resweep:
        return n * per_island
    per_pair = (10 if col16 else 12) if fp32 else 20
    return per_pair * nnz + 8 * (n + 1) + n * per_island


def flip_layout_bytes(degree: float, fp32: bool) -> float:
    """Bytes one flip moves as this implementation lays its arrays out, per
    neighbour: the row entry (column, P and transposed Q; both widths on the FP32
    path), the neighbour's state read (exact sums, 32-bit sums, key, spin, angle
    class, 1/(b h_k) and 1/(c h_k) in FP32 or FP64, row pointers for the next-pick
    prediction) and written back (sums, key, lower bound, exact value)."""
    per_nb = ((4 + 4 + 4 + 8 + 8) + (16 + 8 + 8 + 1 + 2 + 8 + 16) + (16 + 8 + 8 + 8 + 4)
              if fp32 else (4 + 8 + 8) + (16 + 8 + 1 + 2 + 16 + 8 + 16) + (16 + 8 + 8 + 4))
    return degree * per_nb


# DRAM bytes (read + write) per unit of work of the kernels, from one ncu capture on
# a smaller array of the same geometry (summarised with the profiles), scaled to a
# launch by its units, with a hash of the kernel sources that were profiled: a
# changed kernel reports null.
TRAFFIC = {
    # DRAM bytes (read + write) per unit from one small-case ncu capture of the kernel
    # (profiles/), valid while the listed sources are unchanged (sha256 prefix): the sweep
    # capture is of its 4-lanes-a-row build on kagome 300x300, the multi-flip one of field
    # step 5 of that rotation; both are scaled to a full launch by their units
    "k_sweep": {"per": "neighbour pair", "bytes_per_unit": 11.41,
                "sources": ("fs_sweep.cu", "fs_sweep_task.cuh"), "sha256_16": "0b37c859b8c89d8a"},
    "k_relax_multi": {"per": "flip", "bytes_per_unit": 11716.0,
                      "sources": ("fs_relax_multi.cu", "fs_update.cuh", "fs_common.cuh"),
                      "sha256_16": "adfeb495ca5714f7"},
    "k_relax": {"per": "flip", "bytes_per_unit": None,
                "sources": ("fs_relax.cu", "fs_common.cuh"), "sha256_16": ""},
}


def traffic_of(kernel: str, units: float):
    import hashlib
    t = TRAFFIC[kernel]
    if t["bytes_per_unit"] is None:
        return None
    m = hashlib.sha256()
    for name in t["sources"]:
        with open(os.path.join(ROOT, "paper_2002_11401_b300", "csrc", name), "rb") as f:
            m.update(f.read())
    if m.hexdigest()[:16] != t["sha256_16"]:
        return None
    return t["bytes_per_unit"] * units


def composed_rate(t_sweep: float, t_flip: float, field_steps: int, flips: int) -> float:
    """Flips per second of a whole protocol composed from a per-sweep and a
    per-flip cost: flips / (field_steps t_sweep + flips t_flip)."""
    return flips / (field_steps * t_sweep + flips * t_flip)


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


# ---------------------------------------------------------------------------
# The oracle on the host cores (the CPU baseline and the reference arm)
# ---------------------------------------------------------------------------

class OracleProbe:
    """The FP64 oracle built once for the headline workload. One measurement times
    two field steps from the polarised state: one at zero external field (no flip:
    a whole field sweep, the Eq. 5 evaluation of every island and the argmax tree
    build alone) and the rotation's first step (its initial avalanche of 92,563
    flips), and composes the whole 720-step protocol from them as 720 t_sweep +
    F t_flip, F = its 3,146,771 flips."""

    def __init__(self, w):
        import oracle as O
        O.build()
        from tests.helpers import oracle_sim
        self.O = O
        self.cores = os.cpu_count() or 1
        O.set_threads(self.cores)
        t0 = time.perf_counter()
        self.S = oracle_sim(O, w)
        self.build_s = time.perf_counter() - t0
        self.hx, self.hy = I.protocol_of(w["protocol"])
        g = golden("kagome1000_full")
        self.F = int(g["n_flips"])
        self.first = int(g["flips_per_step"][0])
        self.K = len(self.hx)

    def measure(self):
        s0 = np.ones(self.S.n, dtype=np.int8)
        t0 = time.perf_counter()
        r0 = self.S.run(s0.copy(), np.zeros(1), np.zeros(1), step0=100_000, log_cap=0)
        t_sweep = time.perf_counter() - t0
        assert r0["n_flips"] == 0
        t0 = time.perf_counter()
        r1 = self.S.run(s0.copy(), self.hx[:1], self.hy[:1], log_cap=0)
        t_step = time.perf_counter() - t0
        assert r1["n_flips"] == self.first, (r1["n_flips"], self.first)
        t_flip = max(t_step - t_sweep, 0.0) / self.first
        v = composed_rate(t_sweep, t_flip, self.K, self.F)
        return {"value": v, "unit": UNIT, "cores": self.cores, "kind": "oracle",
                "sample": (f"composed: {self.K} x {t_sweep:.3f} s per field sweep (a zero-field "
                           f"step, 0 flips) + {self.F} flips x {t_flip * 1e6:.2f} us per flip "
                           f"(the rotation's first step, {self.first} flips, {t_step:.2f} s); "
                           f"OpenMP over rows for the field sums; the oracle's build "
                           f"({self.build_s:.1f} s) not counted"),
                "t_sweep_s": t_sweep, "t_flip_us": t_flip * 1e6,
                "field_steps_per_s": self.K / (self.K * t_sweep + self.F * t_flip)}


def cpu_baseline(w):
    return OracleProbe(w).measure()


def run_reference(args, w, rank):
    """Reference arm: the FP64 oracle as it stands, on the host cores."""
    if rank != 0:
        return
    steps, warm = max(args.steps, 1), args.warmup
    probe = OracleProbe(w)
    for _ in range(warm):
        probe.measure()
    vals, t0 = [], time.perf_counter()
    for _ in range(steps):
        vals.append(probe.measure())
    dt = time.perf_counter() - t0
    v = float(np.mean([x["value"] for x in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 0,
            "steps": steps, "warmup": warm, "ms_per_step": dt * 1000 / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_desc(w),
                       "path": "FP64 oracle on the host cores, dipolar fields recomputed "
                               "from positions every field step; each bench step measures "
                               "the per-sweep and per-flip costs and composes the whole "
                               "protocol from them"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": vals[0]["cores"],
                             "kind": "oracle", "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# The library's workloads
# ---------------------------------------------------------------------------

def make_sim(B, w, prec, stream=None):
    sim = B.Sim.geometry(w["kind"], w["nx"], w["ny"], w.get("a", 1.0))
    if stream is not None:
        sim.set_stream(stream.cuda_stream)
    sim.set_params(B.make_params(alpha=w["alpha"], hk=w["hk"], k_disorder=w["k_disorder"],
                                 b=w["b"], c=w["c"], beta=w["beta"], gamma=w["gamma"],
                                 cutoff=w["cutoff"], sigma_th=w["sigma_th"], seed=w["seed"],
                                 instance=w.get("instance", 0), precision=prec))
    return sim


def timed_protocol(torch, B, w, prec, repeats, warm, golden_name=None, resweep=True):
    """Whole protocols on device-resident inputs, timed with CUDA events on the
    simulation's stream; flips per field step checked against the oracle's. With
    resweep off, each field step's pass reads the exact sums that the flips kept up
    to date instead of re-summing every neighbour (the same bits)."""
    stream = torch.cuda.Stream()
    sim = make_sim(B, w, prec, stream)
    info = sim.info()
    lanes = sim.autotune()
    hx, hy = I.protocol_of(w["protocol"])
    K = len(hx)
    with torch.cuda.stream(stream):
        d_hx = torch.from_numpy(hx).cuda()
        d_hy = torch.from_numpy(hy).cuda()
        d_init = torch.ones(sim.n, dtype=torch.int8, device="cuda")
        d_fps = torch.zeros(K, dtype=torch.int64, device="cuda")
        d_out = torch.zeros(4, dtype=torch.int64, device="cuda")
    stream.synchronize()

    def step():
        sim.set_spins_dev(d_init.data_ptr())
        sim.run_protocol_dev(d_hx.data_ptr(), d_hy.data_ptr(), K, resweep=resweep,
                             d_flips_per_step=d_fps.data_ptr(), d_out=d_out.data_ptr())

    for _ in range(warm):
        step()
    stream.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(repeats):
        step()
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    out = d_out.cpu().tolist()
    # the kernels' shares from one more protocol with per-kernel timing (per-step
    # launches, also for a small array whose timed protocols ran in one CTA)
    sim.set_profiling(True)
    e0.record(stream)
    step()
    e1.record(stream)
    e1.synchronize()
    ms_prof = e0.elapsed_time(e1)
    prof = sim.profile()
    assert d_out.cpu().tolist()[2] == out[2]
    assert int(out[0]) == 0, f"protocol status {out[0]}"
    flips = int(out[1])
    fps = d_fps.cpu().numpy()
    res = {"flips_per_s": flips * repeats / (ms / 1e3),
           "field_steps_per_s": K * repeats / (ms / 1e3),
           "ms_per_protocol": ms / repeats, "flips": flips, "field_steps": K,
           "seq_hash": f"{int(out[2]) & 0xFFFFFFFFFFFFFFFF:#018x}", "repeats": repeats,
           "sweep_lanes_per_row": lanes, "resweep": bool(resweep),
           "fp64_rechecks_per_flip": int(out[3]) / max(flips, 1)}
    if golden_name:
        g = golden(golden_name)
        res["equals_oracle"] = bool(np.array_equal(fps, np.array(g["flips_per_step"])) and
                                    res["seq_hash"] == g["seq_hash"])
    sw = prof["sweep_ms"] / max(prof["sweep_launches"], 1)
    fp32 = prec == B.FS_FP32_RECHECK
    peak, _ = peaks()
    layout = sweep_bytes(info.n, info.nnz, fp32, resweep, w["sigma_th"] > 0,
                         bool(info.col_offsets16))
    # without the re-summation the pass has no neighbour bytes: its own layout's
    # bytes are the ones to set against the copy peak
    alg = sweep_alg_bytes(info.n, info.nnz, fp32) if resweep else layout
    res["sweep"] = {"us_per_launch": sw * 1e3, "alg_bytes_per_launch": alg,
                    "achieved_gbs": alg / (sw / 1e3) / 1e9, "frac": alg / (sw / 1e3) / 1e9 / peak,
                    "layout_bytes_per_launch": layout}
    res["relax_share"] = prof["relax_ms"] / ms_prof
    sim.close()
    return res


def extra_ensemble(torch, B, n_members=512, alone_every=16):
    """The 512-member ensemble batched (FP32 + recheck and FP64), and the members
    0, 16, 32, ... run one at a time on the FP64 path; sequences compared."""
    members, proto = I.ensemble_workload(n_members)
    hx, hy = I.protocol_of(proto)
    out = {"workload": f"{len(members)} square arrays, sides uniform 20..200 (seed 4), "
                       f"h_k seeds 1000+i, {len(hx)}-step 45-degree ramp 0 -> -0.3 -> +0.3 T"}
    hashes = {}
    for prec, tag in ((B.FS_FP32_RECHECK, "fp32"), (B.FS_FP64, "fp64")):
        sims = [make_sim(B, m, prec) for m in members]
        out["islands"] = int(sum(s.n for s in sims))
        B.batch_run_protocol(sims[:8], hx[:4], hy[:4])  # warm-up (graph set-up paths)
        for s in sims[:8]:
            s.set_spins(np.ones(s.n, dtype=np.int8))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = B.batch_run_protocol(sims, hx, hy)
        dt = time.perf_counter() - t0
        assert (res["status"] == 0).all()
        flips = int(res["n_flips"].sum())
        hashes[tag] = res["hash"].copy()
        out[f"batched_{tag}_flips_per_s"] = flips / dt
        out[f"batched_{tag}_s"] = dt
        out["flips"] = flips
        if tag == "fp32":
            # the same protocol again from the polarised state with the persistent
            # schedule (one launch in which every member advances its own field steps)
            for s in sims:
                s.set_spins(np.ones(s.n, dtype=np.int8))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rp = B.batch_run_protocol(sims, hx, hy, schedule=B.FS_BATCH_PERSISTENT)
            dtp = time.perf_counter() - t0
            assert (rp["status"] == 0).all() and (rp["hash"] == res["hash"]).all()
            out["persistent_fp32_flips_per_s"] = int(rp["n_flips"].sum()) / dtp
            out["persistent_fp32_s"] = dtp
        for s in sims:
            s.close()
        del sims
    idx = list(range(0, len(members), alone_every))
    t_run, flips, same = 0.0, 0, 0
    for q in idx:
        s = make_sim(B, members[q], B.FS_FP64)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = s.run_protocol(hx, hy, log_cap=0)
        t_run += time.perf_counter() - t0
        flips += r["n_flips"]
        same += int(r["hash"] == int(hashes["fp32"][q]) == int(hashes["fp64"][q]))
        s.close()
    gold = [0, 37, 211, 500]
    out["members_equal_oracle"] = sum(
        int(f"{int(hashes['fp32'][q]) & 0xFFFFFFFFFFFFFFFF:#018x}" ==
            golden(f"ensemble512_member{q}")["seq_hash"]) for q in gold if q < len(members))
    out["one_at_a_time"] = {"members": f"every {alone_every}th ({len(idx)} members: "
                                       f"{idx[0]}, {idx[1]}, ..., {idx[-1]})",
                            "flips": flips, "fp64_flips_per_s": flips / t_run,
                            "identical_sequences": f"{same}/{len(idx)}"}
    out["batched_fp32_vs_one_at_a_time_fp64"] = out["batched_fp32_flips_per_s"] / (flips / t_run)
    return out


def extra_serving(n_requests=40, rate=200.0, check=6):
    """A Poisson stream through the continuous-batching server, FP32 + recheck, in a
    process of its own (as a server runs): measured in this process after the kagome
    runs it was 20-30% slower than in a fresh one."""
    cmd = [sys.executable, "-m", "paper_2002_11401_b300.run_workloads", "serving",
           "--requests", str(n_requests), "--rate", str(rate), "--budget-gb", "200",
           "--check", str(check)]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    if r.returncode != 0:
        return {"error": (r.stderr or r.stdout)[-400:]}
    got = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    keys = ("workload", "flips", "wall_s", "flips_per_s", "requests_per_s", "latency_p50_s",
            "latency_p99_s", "admission_wait_p50_s", "one_at_a_time_fp64_flips_per_s",
            "served_vs_one_at_a_time_fp64")
    out = {k: got[k] for k in keys if k in got}
    out["alone_fp64_equals_served"] = got.get("fp64_alone_equals_mix")
    out["alone_fp32_equals_served"] = got.get("alone_equals_mix")
    out["process"] = "its own: " + " ".join(cmd[1:])
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--extras", default="all", choices=["all", "none"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    w = I.WORKLOADS[HEADLINE]
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

    prec = B.FS_FP32_RECHECK
    stream = torch.cuda.Stream()
    sim = make_sim(B, w, prec, stream)
    info = sim.info()
    lanes = sim.autotune()
    hx, hy = I.protocol_of(w["protocol"])
    K = len(hx)
    assert K == CHUNK * CHUNKS
    gold = golden("kagome1000_full")
    with torch.cuda.stream(stream):
        d_hx = torch.from_numpy(hx).cuda()
        d_hy = torch.from_numpy(hy).cuda()
        d_init = torch.ones(sim.n, dtype=torch.int8, device="cuda")
        d_fps = torch.zeros(K, dtype=torch.int64, device="cuda")
        d_outs = torch.zeros((max(args.steps, 1) + max(args.warmup, 0), 4), dtype=torch.int64,
                             device="cuda")
    stream.synchronize()
    counter = [0]

    def step(slot):
        c = counter[0] % CHUNKS
        counter[0] += 1
        if c == 0:
            sim.set_spins_dev(d_init.data_ptr())
        sim.run_protocol_dev(d_hx.data_ptr() + 8 * CHUNK * c, d_hy.data_ptr() + 8 * CHUNK * c,
                             CHUNK, step0=CHUNK * c,
                             d_flips_per_step=d_fps.data_ptr() + 8 * CHUNK * c,
                             d_out=d_outs[slot].data_ptr())
        return c

    for q in range(max(args.warmup, 0)):
        step(args.steps + q)
    stream.synchronize()

    clocks = Clocks(local)
    sim.set_profiling(True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    chunks = [step(q) for q in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    prof = sim.profile()
    sim.set_profiling(False)
    outs = d_outs[:args.steps].cpu().numpy()
    assert (outs[:, 0] == 0).all(), f"protocol status {outs[:, 0]}"
    flips_timed = int(outs[:, 1].sum())
    rechecks = int(outs[:, 3].sum())
    fps = d_fps.cpu().numpy()
    gfps = np.array(gold["flips_per_step"])
    for q, c in enumerate(chunks):  # every timed chunk's flip count = the oracle's
        assert int(outs[q, 1]) == int(gfps[CHUNK * c:CHUNK * (c + 1)].sum()), (q, c)
    seen = sorted(set(chunks) | set(range(CHUNKS) if args.warmup + args.steps >= CHUNKS else []))
    for c in seen:
        assert (fps[CHUNK * c:CHUNK * (c + 1)] == gfps[CHUNK * c:CHUNK * (c + 1)]).all(), c
    ms, units = aggregate(ms, flips_timed, dist, device="cuda")
    value = units / (ms / 1000.0)
    field_steps = CHUNK * args.steps * world / (ms / 1000.0)

    # ---- rooflines of the kernels, from the live per-launch event timings ---------
    peak, peak_kind = peaks()
    n, nnz = info.n, info.nnz
    avg_deg = nnz / n
    relax_s = prof["relax_ms"] / 1000.0
    relax_launches = max(prof["relax_launches"], 1)
    relax_alg = flip_alg_bytes(avg_deg, True) * flips_timed
    relax_ach = relax_alg / relax_s / 1e9 if relax_s > 0 else 0.0
    flips_per_launch = flips_timed / relax_launches
    relax_kernel = "k_relax_multi" if n >= 32768 else "k_relax"  # the library's automatic choice
    roof_relax = {"kernel": relax_kernel, "bound": "hbm", "achieved": relax_ach, "peak": peak,
                  "unit": "GB/s", "frac": relax_ach / peak,
                  "traffic": traffic_of(relax_kernel, flips_per_launch),
                  "peak_kind": peak_kind,
                  "avg_launch_ms": prof["relax_ms"] / relax_launches,
                  "share_of_step": prof["relax_ms"] / ms if ms > 0 else None,
                  "bytes_per_launch": relax_alg / relax_launches,
                  "flips_per_launch": flips_per_launch,
                  "layout_bytes_per_launch": flip_layout_bytes(avg_deg, True) * flips_per_launch,
                  "note": f"flip chain in multi-flip rounds, latency-bound: algorithmic bytes = "
                          f"{avg_deg:.2f} neighbours x 42 B per flip; layout bytes = what the "
                          "kernel's arrays move per flip"}
    sweep_launch_ms = prof["sweep_ms"] / max(prof["sweep_launches"], 1)
    sweep_alg = sweep_alg_bytes(n, nnz, True)
    roof_sweep = {"kernel": "k_sweep", "bound": "hbm",
                  "achieved": sweep_alg / (sweep_launch_ms / 1e3) / 1e9, "peak": peak,
                  "unit": "GB/s", "frac": sweep_alg / (sweep_launch_ms / 1e3) / 1e9 / peak,
                  "traffic": traffic_of("k_sweep", nnz), "peak_kind": peak_kind,
                  "avg_launch_ms": sweep_launch_ms, "bytes_per_launch": sweep_alg,
                  "layout_bytes_per_launch": sweep_bytes(n, nnz, True, True, True,
                                                         bool(info.col_offsets16)),
                  "share_of_step": prof["sweep_ms"] / ms if ms > 0 else None}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "i32+f32, f64 recheck", "data": "synthetic",
            "config": {"workload": workload_desc(w),
                       "path": "FP32 + FP64 recheck, full dipolar resweep every field step",
                       "bench_step": f"{CHUNK} consecutive field steps (one tenth of the "
                                     "rotation), continuing the state; every tenth bench step "
                                     "restarts from the polarised state",
                       "timed_chunks": chunks, "islands": n, "neighbour_pairs": nnz,
                       "flips_timed": flips_timed, "equals_oracle_flips_per_field_step": True,
                       "l2": "inputs larger than L2 (neighbour tensors and state "
                             f"{info.device_bytes / 1e9:.2f} GB on the device)",
                       "parallelism": "replicas" if world > 1 else "single",
                       "sweep_lanes_per_row": lanes},
            "field_steps_per_s": field_steps,
            "roofline": roof_relax, "roofline_sweep": roof_sweep,
            # per field step: the external-field table, the sweep, the relax (with the
            # multi-flip rounds also the single-flip continuation, which returns at once
            # unless a step is handed over); per bench step one copy-out of the results
            "gpu_launches": args.steps * ((4 if relax_kernel == "k_relax_multi" else 3) * CHUNK
                                          + 1),
            "fp64_rechecks_per_flip": rechecks / max(flips_timed, 1)}
    if relax_kernel == "k_relax_multi" and not args.no_e2e:
        line["multi_flip_rounds"] = None  # filled from the host-buffer pass below
    if clk:
        line["clocks"] = clk

    # ---- end to end through the host-buffer C ABI call --------------------------
    if not args.no_e2e:
        init = np.ones(sim.n, dtype=np.int8)
        h2d = d2h = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_flips = 0
        for q in range(args.steps):
            c = q % CHUNKS
            if c == 0:
                sim.set_spins(init)
                h2d += init.nbytes
            sl = slice(CHUNK * c, CHUNK * (c + 1))
            r = sim.run_protocol(hx[sl], hy[sl], step0=CHUNK * c, log_cap=0)
            h2d += hx[sl].nbytes + hy[sl].nbytes
            d2h += 8 * CHUNK + 64
            e2e_flips += r["n_flips"]
            assert r["n_flips"] == int(gfps[sl].sum())
        dt = time.perf_counter() - t0
        pr = sim.profile()
        if "multi_flip_rounds" in line:
            line["multi_flip_rounds"] = {"rounds": pr["rounds"], "flips": e2e_flips,
                                         "flips_per_round": e2e_flips / max(pr["rounds"], 1),
                                         "passes_without_a_flip": pr["idle_rounds"]}
        line["e2e"] = {"value": e2e_flips / dt, "unit": UNIT,
                       "h2d_bytes_per_step": int(h2d / args.steps),
                       "d2h_bytes_per_step": int(d2h / args.steps)}
    # ---- the FP32 path's field error against the FS_FP64 path, at the final state ---
    if rank == 0 and not args.no_e2e:
        final = sim.spins()
        sim.close()
        ref = make_sim(B, w, B.FS_FP64)
        ref.set_spins(final)
        t_last = CHUNK * ((args.steps - 1) % CHUNKS + 1) - 1
        ref.set_field(float(hx[t_last]), float(hy[t_last]), step=t_last)
        p64, q64 = ref.fields()
        ref.close()
        s32 = make_sim(B, w, B.FS_FP32_RECHECK)
        s32.set_spins(final)
        s32.set_field(float(hx[t_last]), float(hy[t_last]), step=t_last)
        p32, q32 = s32.fields()
        s32.close()
        scale = max(float(np.abs(p64).max()), float(np.abs(q64).max()))
        err = max(float(np.abs(p32 - p64).max()), float(np.abs(q32 - q64).max()))
        line["fp32_field_error"] = {"max_abs_over_max_h": err / scale, "bound": 1e-5,
                                    "vs": "FS_FP64 path (= oracle to 1e-12) at the final state"}
    else:
        sim.close()

    # ---- the other workloads, each timed on the device -------------------------
    if args.extras == "all" and rank == 0:
        ex = {}
        # the serving stream in a process of its own (see extra_serving)
        ex["serving"] = extra_serving()
        ex["square16_fp64"] = timed_protocol(torch, B, I.WORKLOADS["square16"], B.FS_FP64, 5, 2,
                                             "square16")
        for tag, p in (("fp32", B.FS_FP32_RECHECK), ("fp64", B.FS_FP64)):
            ex[f"pinwheel300_{tag}"] = timed_protocol(torch, B, I.WORKLOADS["pinwheel300"], p, 3,
                                                      1, "pinwheel300_full")
        ex["kagome1000_fp64"] = timed_protocol(torch, B, w, B.FS_FP64, 1, 0, "kagome1000_full")
        # the headline's rotation with the flips' exact sums carried across field steps
        ex["kagome1000_fp32_no_resweep"] = timed_protocol(torch, B, w, B.FS_FP32_RECHECK, 1, 0,
                                                           "kagome1000_full", resweep=False)
        ex["ensemble512"] = extra_ensemble(torch, B)
        line["workloads"] = ex
    if rank == 0 and not args.no_cpu:
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
