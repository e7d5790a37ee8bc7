"""Shared test helpers: build the same seeded system on the CUDA library and on
the oracle, each from its own code (the oracle generates its own geometry and
coercive fields; only the workload description is shared)."""
import numpy as np

from paper_2002_11401_b300 import inputs as I


def lib_sim(w, precision=0, **over):
    from paper_2002_11401_b300 import binding as B
    p = dict(w)
    p.update(over)
    sim = B.Sim.geometry(p["kind"], p["nx"], p["ny"], p.get("a", 1.0))
    sim.set_params(B.make_params(alpha=p["alpha"], hk=p["hk"], k_disorder=p["k_disorder"],
                                 b=p["b"], c=p["c"], beta=p["beta"], gamma=p["gamma"],
                                 cutoff=p["cutoff"], sigma_th=p["sigma_th"], seed=p["seed"],
                                 instance=p.get("instance", 0), precision=precision,
                                 max_flips_per_step=p.get("max_flips_per_step", 0)))
    return sim


def oracle_sim(O, w, **over):
    p = dict(w)
    p.update(over)
    x, y, th = O.geometry(p["kind"], p["nx"], p["ny"], p.get("a", 1.0))
    hk = O.draw_hk(len(x), p["hk"], p["k_disorder"], p["seed"], p.get("instance", 0))
    return O.Sim(x, y, th, hk, alpha=p["alpha"], b=p["b"], c=p["c"], beta=p["beta"],
                 gamma=p["gamma"], sigma_th=p["sigma_th"], cutoff_abs=p["cutoff"] * p.get("a", 1.0),
                 seed=p["seed"], instance=p.get("instance", 0))


def small(kind, n, **kw):
    base = dict(kind=kind, nx=n, ny=n, a=1.0, alpha=1e-3, cutoff=3.0, hk=0.2, k_disorder=0.05,
                seed=11, b=1.0, c=1.0, beta=3.0, gamma=3.0, sigma_th=0.0)
    if kind == I.PINWHEEL:
        base["cutoff"] = 5.0
    if kind == I.KAGOME:
        base.update(alpha=8e-4, cutoff=4.0)
    base.update(kw)
    return base


def first_divergence(a_steps, a_spins, b_steps, b_spins):
    m = min(len(a_spins), len(b_spins))
    d = np.nonzero((a_spins[:m] != b_spins[:m]) | (a_steps[:m] != b_steps[:m]))[0]
    if len(d):
        return int(d[0])
    return None if len(a_spins) == len(b_spins) else m
