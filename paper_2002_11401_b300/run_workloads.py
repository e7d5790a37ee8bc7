"""Runner for the library's workloads (the single-GPU counterpart of flatspin's
runner, Sec. "Simulation framework"): builds each workload from `inputs.py`,
runs it through the C ABI and prints one JSON line of measurements.

  python -m paper_2002_11401_b300.run_workloads square16|pinwheel300|kagome1000 \
      [--precision fp32|fp64] [--steps K] [--resweep 0|1] [--cells N]
      [--relax auto|single|multi|multi_cta]
  python -m paper_2002_11401_b300.run_workloads ensemble512 [--members M] [--steps K]
      [--schedule per_step|persistent|auto]
  python -m paper_2002_11401_b300.run_workloads serving [--requests R] [--rate HZ]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

from . import binding as B
from . import inputs as I


def _peak():
    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    try:
        with open(os.path.join(here, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def make_sim(w, precision):
    sim = B.Sim.geometry(w["kind"], w["nx"], w["ny"], w.get("a", 1.0))
    sim.set_params(B.make_params(alpha=w["alpha"], hk=w["hk"], k_disorder=w["k_disorder"],
                                 b=w["b"], c=w["c"], beta=w["beta"], gamma=w["gamma"],
                                 cutoff=w["cutoff"], sigma_th=w["sigma_th"], seed=w["seed"],
                                 precision=precision))
    return sim


def sweep_bytes(info, fp32: bool, resweep: bool, thermal: bool) -> int:
    """Bytes one field-and-margin sweep moves as the arrays are laid out. Per pair:
    the column index and the (P, Q) coefficients of the path's width (4 + 8 or
    4 + 16; 2 + 8 where the FP32 path reads 16-bit column offsets); per row: its
    pointer (8). Per island: spin, angle class, 1/(b h_k) and 1/(c h_k) read
    (1 + 2 + 8); the relax's 32-byte record, key and exact value written
    (32 + 8 + 8); on the FP64 path the 64-bit sums written (or, without the
    resweep, read: 16), on the FP32 path without the resweep the 32-bit sums read
    (8); with thermal noise, the step's FP32 draw written (8)."""
    n, nnz = info.n, info.nnz
    per_island = (1 + 2 + 8 + 32 + 8 + 8 + (0 if fp32 else 16)
                  + (8 if fp32 and not resweep else 0) + (8 if thermal else 0))
    if not resweep:
        return n * per_island
    per_pair = (10 if info.col_offsets16 else 12) if fp32 else 20
    return per_pair * nnz + 8 * (n + 1) + n * per_island


def run_single(name, precision, steps, resweep, cells=0, relax="auto"):
    w = dict(I.WORKLOADS[name])
    if cells:
        w["nx"] = w["ny"] = cells
    fp32 = precision == B.FS_FP32_RECHECK
    t0 = time.perf_counter()
    sim = make_sim(w, precision)
    sim.set_relax_mode({"auto": B.FS_RELAX_AUTO, "single": B.FS_RELAX_SINGLE,
                        "multi": B.FS_RELAX_MULTI, "multi_cta": B.FS_RELAX_MULTI_CTA}[relax])
    build_s = time.perf_counter() - t0
    lanes = sim.autotune()
    hx, hy = I.protocol_of(w["protocol"])
    if steps:
        hx, hy = hx[:steps], hy[:steps]
    sim.set_spins(np.ones(sim.n, dtype=np.int8))
    sim.set_profiling(True)
    t0 = time.perf_counter()
    r = sim.run_protocol(hx, hy, resweep=resweep, log_cap=0)
    dt = time.perf_counter() - t0
    prof = sim.profile()
    info = sim.info()
    peak, kind = _peak()
    sw_ms = prof["sweep_ms"] / max(prof["sweep_launches"], 1)
    sb = sweep_bytes(info, fp32, resweep, w["sigma_th"] > 0)
    return {"workload": name, "precision": "fp32+fp64-recheck" if fp32 else "fp64",
            "islands": info.n, "neighbour_pairs": info.nnz, "field_steps": len(hx),
            "resweep": bool(resweep), "build_s": build_s, "lanes_per_row": lanes,
            "protocol_s": dt, "flips": r["n_flips"], "flips_per_s": r["n_flips"] / dt,
            "field_steps_per_s": len(hx) / dt, "seq_hash": f"{r['hash']:#018x}",
            "status": r["status"], "sweep_us_per_launch": sw_ms * 1e3,
            "sweep_gbs": sb / (sw_ms / 1e3) / 1e9 if sw_ms > 0 else None,
            "sweep_frac_of_peak": sb / (sw_ms / 1e3) / 1e9 / peak if sw_ms > 0 else None,
            "peak_gbs": peak, "peak_kind": kind,
            "relax_share": prof["relax_ms"] / (dt * 1e3), "rechecks": prof["rechecks"],
            "multi_rounds": prof["rounds"], "multi_idle_rounds": prof["idle_rounds"],
            "multi_round_flips": prof["round_flips"], "multi_handoffs": prof["handoffs"],
            "relax_us_per_launch": prof["relax_ms"] * 1e3 / max(prof["relax_launches"], 1),
            "device_bytes": info.device_bytes,
            "flips_per_step_head": r["flips_per_step"][:16].tolist()}


def step_barrier(fps, slots=2 * 148):
    """What the batch's per-step barrier costs, with a member's relax time taken as its
    flips in the step: fps [members, K]. With the barrier every step lasts as long as
    its largest member's relax, or the step's flips spread over the resident relax CTAs
    (`slots`), whichever is longer; without it (each member advancing on its own) the
    protocol lasts as long as the longest member chain, or all flips over the slots."""
    fps = np.asarray(fps, dtype=np.float64)
    per_step = np.maximum(fps.max(axis=0), fps.sum(axis=0) / slots)
    with_barrier = float(per_step.sum())
    without = float(max(fps.sum(axis=1).max(), fps.sum() / slots))
    return {"flip_steps_with_barrier": with_barrier, "flip_steps_without": without,
            "bound_on_gain": with_barrier / without if without > 0 else None,
            "largest_member_is_the_slowest_in_steps": int(
                (fps.argmax(axis=0) == fps.sum(axis=1).argmax()).sum()),
            "steps": int(fps.shape[1]), "slots": slots}


def run_ensemble(members, sample, steps=0, schedule="per_step"):
    mem, proto = I.ensemble_workload()
    mem = mem[:members]
    hx, hy = I.protocol_of(proto)
    if steps:
        hx, hy = hx[:steps], hy[:steps]
    sched = {"auto": B.FS_BATCH_AUTO, "persistent": B.FS_BATCH_PERSISTENT,
             "per_step": B.FS_BATCH_PER_STEP, "two_chains": B.FS_BATCH_TWO_CHAINS}[schedule]
    out = {"workload": f"ensemble of {len(mem)} square arrays (sides 20..200), "
                       f"{len(hx)}-step 45-degree ramp", "schedule": schedule}
    hashes = {}
    for prec, tag in ((B.FS_FP32_RECHECK, "fp32"), (B.FS_FP64, "fp64")):
        sims = [make_sim(m, prec) for m in mem]
        out["islands"] = int(sum(s.n for s in sims))
        t0 = time.perf_counter()
        res = B.batch_run_protocol(sims, hx, hy, with_counts=tag == "fp32", schedule=sched)
        dt = time.perf_counter() - t0
        flips = int(res["n_flips"].sum())
        hashes[tag] = res["hash"].copy()
        if tag == "fp32":
            out["step_barrier"] = step_barrier(res["flips_per_step"])
        out[f"batched_{tag}_s"] = dt
        out[f"batched_{tag}_flips_per_s"] = flips / dt
        out["flips"] = flips
        for s in sims:
            s.close()
    assert (hashes["fp32"] == hashes["fp64"]).all()
    # one simulation at a time, FP64, on an evenly spaced sample (build not timed)
    idx = np.linspace(0, len(mem) - 1, sample).astype(int)
    t_run, flips = 0.0, 0
    for q in idx:
        s = make_sim(mem[q], B.FS_FP64)
        t0 = time.perf_counter()
        r = s.run_protocol(hx, hy, log_cap=0)
        t_run += time.perf_counter() - t0
        flips += r["n_flips"]
        assert r["hash"] == int(hashes["fp64"][q])
        s.close()
    out["one_at_a_time_fp64_flips_per_s"] = flips / t_run
    out["one_at_a_time_sample"] = len(idx)
    out["speedup_batched_fp32_vs_one_at_a_time_fp64"] = \
        out["batched_fp32_flips_per_s"] / out["one_at_a_time_fp64_flips_per_s"]
    return out


def run_serving(n_requests, rate, budget_gb, check):
    reqs = I.serving_stream(n_requests=n_requests, rate_hz=rate)
    srv = B.Server(hbm_budget=int(budget_gb * (1 << 30)), max_active=256)
    tickets = []
    t_start = srv.now()
    for r in reqs:
        hx, hy = I.protocol_of(r["protocol"])
        prec = B.FS_FP32_RECHECK
        p = B.make_params(alpha=r["alpha"], hk=r["hk"], k_disorder=r["k_disorder"],
                          cutoff=r["cutoff"], seed=r["seed"], precision=prec)
        while srv.now() - t_start < r["arrival"]:
            time.sleep(min(0.002, max(0.0, r["arrival"] - (srv.now() - t_start))))
        tickets.append((srv.submit(r["kind"], r["nx"], r["ny"], p, hx, hy), r, hx, hy))
    srv.drain()
    t_end = srv.now()
    lat, wait, run, flips, islands, results = [], [], [], 0, 0, []
    for t, r, hx, hy in tickets:
        res = srv.poll(t)
        assert res is not None and res["status"] == 0, res
        lat.append(res["t_done"] - res["t_submit"])
        wait.append(res["t_admit"] - res["t_submit"])
        run.append(res["t_done"] - res["t_admit"])
        flips += res["n_flips"]
        islands += res["n"]
        results.append((res, r, hx, hy))
    srv.close()
    out = {"workload": f"Poisson stream of {n_requests} requests at {rate:g}/s, mixed "
                       "square/pinwheel/kagome, 1e3..2e6 islands, 50..500 ramp steps",
           "requests": n_requests, "islands": islands, "flips": flips,
           "wall_s": t_end - t_start, "flips_per_s": flips / (t_end - t_start),
           "requests_per_s": n_requests / (t_end - t_start),
           "latency_p50_s": float(np.percentile(lat, 50)),
           "latency_p99_s": float(np.percentile(lat, 99)),
           "latency_max_s": float(np.max(lat)),
           "admission_wait_p50_s": float(np.percentile(wait, 50)),
           "admission_wait_p99_s": float(np.percentile(wait, 99)),
           "build_and_run_p50_s": float(np.percentile(run, 50)),
           "build_and_run_p99_s": float(np.percentile(run, 99)),
           "largest_request_islands": int(max(res["n"] for res, _, _, _ in results)),
           "hbm_budget_gb": budget_gb}
    # the same requests alone (a sample): identical results; and the plain
    # one-simulation-at-a-time FP64 path on them (build not timed), for comparison
    same, same64, t64, f64 = 0, 0, 0.0, 0
    for res, r, hx, hy in results[:check]:
        w = dict(r)
        w.pop("protocol")
        s = make_sim(w, B.FS_FP32_RECHECK)
        alone = s.run_protocol(hx, hy, log_cap=0)
        same += int(alone["hash"] == res["hash"] and alone["n_flips"] == res["n_flips"])
        s.close()
        s = make_sim(w, B.FS_FP64)
        t0 = time.perf_counter()
        r64 = s.run_protocol(hx, hy, log_cap=0)
        t64 += time.perf_counter() - t0
        f64 += r64["n_flips"]
        same64 += int(r64["hash"] == res["hash"] and r64["n_flips"] == res["n_flips"])
        s.close()
    n_chk = min(check, len(results))
    out["alone_equals_mix"] = f"{same}/{n_chk}"
    out["fp64_alone_equals_mix"] = f"{same64}/{n_chk}"
    out["one_at_a_time_fp64_flips_per_s"] = f64 / t64 if t64 > 0 else None
    out["served_vs_one_at_a_time_fp64"] = out["flips_per_s"] / (f64 / t64) if f64 else None
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("workload")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--steps", type=int, default=0)
    ap.add_argument("--cells", type=int, default=0, help="override the array side (cells)")
    ap.add_argument("--resweep", type=int, default=1)
    ap.add_argument("--relax", default="auto", choices=["auto", "single", "multi", "multi_cta"])
    ap.add_argument("--members", type=int, default=512)
    ap.add_argument("--schedule", default="per_step", choices=["auto", "persistent", "per_step", "two_chains"])
    ap.add_argument("--sample", type=int, default=12)
    ap.add_argument("--requests", type=int, default=1000)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--budget-gb", type=float, default=240.0)
    ap.add_argument("--check", type=int, default=20)
    a = ap.parse_args(argv)
    from . import build
    build.build()
    B.load()
    prec = B.FS_FP32_RECHECK if a.precision == "fp32" else B.FS_FP64
    if a.workload in I.WORKLOADS:
        out = run_single(a.workload, prec, a.steps, bool(a.resweep), a.cells, a.relax)
        out["relax"] = a.relax
    elif a.workload == "ensemble512":
        out = run_ensemble(a.members, a.sample, a.steps, a.schedule)
    elif a.workload == "serving":
        out = run_serving(a.requests, a.rate, a.budget_gb, a.check)
    else:
        raise SystemExit(f"unknown workload {a.workload}")
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    sys.exit(main())
