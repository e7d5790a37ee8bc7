"""Writes the stored expected values under tests/golden/ from the FP64 oracle
alone (no library code): the square16 protocol in full, and prefixes of the
pinwheel, kagome and ensemble workloads at their full sizes. With --full, the
whole pinwheel 300x300 and kagome 1000x1000 protocols instead (flip counts per
step and the sequence hash; minutes to tens of minutes on a few cores).

    python tests/golden/make_golden.py [--threads N] [--full pinwheel300,kagome1000]
"""
import argparse
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2002_11401_b300 import inputs as I  # noqa: E402

# protocol prefixes (field steps) kept for the large workloads
PREFIX = {"pinwheel300": 40, "kagome1000": 3}
ENSEMBLE_MEMBERS = (0, 37, 211, 500)


def oracle_sim(w):
    x, y, th = O.geometry(w["kind"], w["nx"], w["ny"], w.get("a", 1.0))
    hk = O.draw_hk(len(x), w["hk"], w["k_disorder"], w["seed"], w.get("instance", 0))
    return O.Sim(x, y, th, hk, alpha=w["alpha"], b=w["b"], c=w["c"], beta=w["beta"],
                 gamma=w["gamma"], sigma_th=w["sigma_th"], cutoff_abs=w["cutoff"] * w.get("a", 1.0),
                 seed=w["seed"], instance=w.get("instance", 0))


def record(name, w, hx, hy, keep_log):
    S = oracle_sim(w)
    r = S.run(np.ones(S.n, dtype=np.int8), hx, hy)
    assert r["status"] == 0
    out = {"workload": name, "islands": S.n, "neighbour_pairs": S.nnz, "field_steps": len(hx),
           "n_flips": r["n_flips"], "seq_hash": f"{r['hash']:#018x}",
           "flips_per_step": r["flips_per_step"].tolist(),
           "near_ties": r["ties"].tolist(),
           "spins_plus": int((r["spins"] > 0).sum())}
    if keep_log:
        out["log_step"] = r["log_step"][:keep_log].tolist()
        out["log_spin"] = r["log_spin"][:keep_log].tolist()
    with open(os.path.join(HERE, f"{name}.json"), "w") as f:
        json.dump(out, f)
    print(name, S.n, r["n_flips"], out["seq_hash"], flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--full", default="", help="comma-separated workloads to record in full")
    a = ap.parse_args()
    O.build()
    O.set_threads(a.threads)
    if a.full:
        for name in a.full.split(","):
            w = I.WORKLOADS[name]
            hx, hy = I.protocol_of(w["protocol"])
            record(f"{name}_full", w, hx, hy, keep_log=0)
        return
    w = I.WORKLOADS["square16"]
    hx, hy = I.protocol_of(w["protocol"])
    record("square16", w, hx, hy, keep_log=10_000)
    for name, k in PREFIX.items():
        w = I.WORKLOADS[name]
        hx, hy = I.protocol_of(w["protocol"])
        record(f"{name}_prefix{k}", w, hx[:k], hy[:k], keep_log=5000)
    members, proto = I.ensemble_workload()
    hx, hy = I.protocol_of(proto)
    for q in ENSEMBLE_MEMBERS:
        record(f"ensemble512_member{q}", members[q], hx, hy, keep_log=0)


if __name__ == "__main__":
    main()
