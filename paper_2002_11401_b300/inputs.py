"""Seeded synthetic inputs shared by the library's tests, the oracle's tests and
the benchmark: workload definitions, external-field protocols and random spin
states. This module holds none of the model's arithmetic (no fields, no
astroid, no relax); it only describes what is fed in.

Workloads are synthetic lattices shaped like the paper's experiments (square,
pinwheel and kagome arrays with normally distributed coercive fields, Sec.
"Imperfections and disorder"; field ramps, loops and rotations, Sec. "External
field"). No dataset is involved.
"""
from __future__ import annotations

import math

import numpy as np

SQUARE, PINWHEEL, KAGOME = 0, 1, 2
KIND_NAMES = {SQUARE: "square", PINWHEEL: "pinwheel", KAGOME: "kagome"}

# Per-geometry defaults used by the mixed serving stream: (alpha, cutoff).
KIND_DEFAULTS = {SQUARE: (1e-3, 3.0), PINWHEEL: (1e-3, 5.0), KAGOME: (8e-4, 4.0)}


def deg2rad(d: float) -> float:
    return d * math.pi / 180.0


def ramp_protocol(K: int, angle_deg: float, hmax: float):
    """0 -> -hmax -> +hmax along one direction, K values uniform in path length
    (u_t = 3 hmax t / (K-1); h = -u for u <= hmax, else u - 2 hmax)."""
    t = np.arange(K, dtype=np.float64)
    u = (3.0 * hmax) * t / max(K - 1, 1)
    h = np.where(u <= hmax, -u, u - 2.0 * hmax)
    a = deg2rad(angle_deg)
    return h * math.cos(a), h * math.sin(a)


def loop_protocol(K: int, angle_deg: float, h0: float, h1: float):
    """Linear sweep h0 -> h1 in K values along one direction."""
    t = np.arange(K, dtype=np.float64)
    h = h0 + (h1 - h0) * t / max(K - 1, 1)
    a = deg2rad(angle_deg)
    return h * math.cos(a), h * math.sin(a)


def rotation_protocol(K: int, step_deg: float, magnitude: float, start_deg: float = 0.0):
    """Field of fixed magnitude rotating counter-clockwise by step_deg per value."""
    phi = np.array([deg2rad(start_deg + step_deg * t) for t in range(K)], dtype=np.float64)
    return magnitude * np.cos(phi), magnitude * np.sin(phi)


def square_cells_for(n_magnets: float) -> int:
    """Side n of the n x n closed square (or pinwheel) array closest to n_magnets
    islands (2 n (n + 1) islands)."""
    return max(1, int(round((-1.0 + math.sqrt(1.0 + 2.0 * n_magnets)) / 2.0)))


def kagome_cells_for(n_magnets: float) -> int:
    """Side n of the n x n kagome array closest to n_magnets islands."""
    # 3 n^2 + 4 n - 1 islands
    return max(1, int(round((-4.0 + math.sqrt(16.0 + 12.0 * (n_magnets + 1.0))) / 6.0)))


# The five workloads. `protocol` is (name, args) for the helpers above.
WORKLOADS = {
    # Square ASI 16x16, FP64, 400-step 45-degree ramp 0 -> -0.3 -> +0.3 T.
    "square16": dict(kind=SQUARE, nx=16, ny=16, a=1.0, alpha=1e-3, cutoff=3.0, hk=0.2,
                     k_disorder=0.05, seed=0, b=1.0, c=1.0, beta=3.0, gamma=3.0,
                     sigma_th=0.0, protocol=("ramp", (400, 45.0, 0.3))),
    # Pinwheel 300x300 (180,600 islands), loop at 30 degrees, -0.25 -> +0.25 T in 1000 steps.
    "pinwheel300": dict(kind=PINWHEEL, nx=300, ny=300, a=1.0, alpha=1e-3, cutoff=5.0, hk=0.2,
                        k_disorder=0.05, seed=1, b=1.0, c=1.0, beta=3.0, gamma=3.0,
                        sigma_th=0.0, protocol=("loop", (1000, 30.0, -0.25, 0.25))),
    # Kagome 1000x1000 (3,003,999 islands), thermal sigma 0.005 T, rotating 0.09 T field.
    "kagome1000": dict(kind=KAGOME, nx=1000, ny=1000, a=1.0, alpha=8e-4, cutoff=4.0, hk=0.2,
                       k_disorder=0.08, seed=2, b=1.0, c=1.0, beta=3.0, gamma=3.0,
                       sigma_th=0.005, protocol=("rotation", (720, 0.5, 0.09))),
}


def protocol_of(spec) -> tuple[np.ndarray, np.ndarray]:
    name, args = spec
    if name == "ramp":
        return ramp_protocol(*args)
    if name == "loop":
        return loop_protocol(*args)
    if name == "rotation":
        return rotation_protocol(*args)
    raise ValueError(name)


def ensemble_workload(n_instances: int = 512, lo: int = 20, hi: int = 200, steps: int = 200,
                      seed: int = 4):
    """Batched ensemble: square arrays with sides drawn uniformly from lo..hi
    cells, coercive-field seeds 1000 + i, one shared 45-degree ramp."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(lo, hi + 1, size=n_instances)
    members = [dict(kind=SQUARE, nx=int(s), ny=int(s), a=1.0, alpha=1e-3, cutoff=3.0, hk=0.2,
                    k_disorder=0.05, seed=1000 + i, b=1.0, c=1.0, beta=3.0, gamma=3.0,
                    sigma_th=0.0) for i, s in enumerate(sides)]
    return members, ("ramp", (steps, 45.0, 0.3))


def serving_stream(n_requests: int = 1000, rate_hz: float = 200.0, n_lo: float = 1e3,
                   n_hi: float = 2e6, steps_lo: int = 50, steps_hi: int = 500, seed: int = 5):
    """Poisson stream of simulation requests mixing the three geometries, island
    counts log-uniform in [n_lo, n_hi], random field angle, ramp of 50..500 steps."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=n_requests)
    arrival = np.cumsum(gaps) - gaps[0]
    reqs = []
    for r in range(n_requests):
        kind = int(rng.integers(0, 3))
        target = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        side = kagome_cells_for(target) if kind == KAGOME else square_cells_for(target)
        alpha, cutoff = KIND_DEFAULTS[kind]
        angle = float(rng.uniform(0.0, 360.0))
        steps = int(rng.integers(steps_lo, steps_hi + 1))
        reqs.append(dict(arrival=float(arrival[r]), kind=kind, nx=side, ny=side, a=1.0,
                         alpha=alpha, cutoff=cutoff, hk=0.2, k_disorder=0.05, seed=50_000 + r,
                         b=1.0, c=1.0, beta=3.0, gamma=3.0, sigma_th=0.0,
                         protocol=("ramp", (steps, angle, 0.3))))
    return reqs


def random_spins(n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.where(rng.random(n) < 0.5, -1, 1).astype(np.int8)
