"""Plain FP64 CPU oracle of the flatspin relax loop (arXiv 2002.11401).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are its only users. The library never imports it
and it imports nothing from the library.

The arithmetic lives in ``flatspin_oracle.c`` (plain C, double precision,
single-threaded per row, optionally OpenMP over independent rows); this module
compiles it with gcc on first use and wraps it with ctypes. Each wrapper names
the part of the paper its C function writes out.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flatspin_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

SQUARE, PINWHEEL, KAGOME = 0, 1, 2
SQUARE_OPEN, PINWHEEL_DIAMOND, PINWHEEL_LUCKY_KNOT, ISING = 3, 4, 5, 6
ASTROID, PARALLEL = 0, 1  # switching criteria
SINUSOID, SAWTOOTH, ROTATION = 0, 1, 2  # input encoders
MODE_INCREMENTAL, MODE_DEFINITION, MODE_LINEAR = 0, 1, 2
OK, ERR_NOT_CONVERGED = 0, 4


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2, no fast-math,
    no floating-point contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        i64, u64, u32, i32, dbl = C.c_int64, C.c_uint64, C.c_uint32, C.c_int32, C.c_double
        P = C.c_void_p
        lib.or_set_threads.argtypes = [C.c_int]
        lib.or_get_threads.restype = C.c_int
        lib.or_philox4x32_10.argtypes = [P, P, P]
        lib.or_box_muller.argtypes = [P, P, P]
        lib.or_draw_hk.argtypes = [i64, dbl, dbl, u64, u32, P]
        lib.or_thermal.argtypes = [i64, dbl, u64, u32, u32, P, P]
        lib.or_geometry_capacity.argtypes = [C.c_int, i32, i32]
        lib.or_geometry_capacity.restype = i64
        lib.or_geometry.argtypes = [C.c_int, i32, i32, dbl, P, P, P]
        lib.or_geometry.restype = i64
        lib.or_dipole_field.argtypes = [dbl, dbl, dbl, dbl, dbl, P, P]
        lib.or_astroid_lhs.argtypes = [dbl, dbl, dbl, dbl, dbl, dbl, dbl]
        lib.or_astroid_lhs.restype = dbl
        lib.or_flippable.argtypes = [C.c_int, dbl, dbl]
        lib.or_flippable.restype = C.c_int
        lib.or_neighbors.argtypes = [i64, P, P, dbl, C.c_int, P, P, i64]
        lib.or_neighbors.restype = i64
        lib.or_sim_create.argtypes = [i64, P, P, P, P, dbl, dbl, dbl, dbl, dbl, dbl, dbl, u64,
                                      u32, C.c_int]
        lib.or_sim_create.restype = P
        lib.or_sim_destroy.argtypes = [P]
        lib.or_sim_n.argtypes = [P]
        lib.or_sim_n.restype = i64
        lib.or_sim_nnz.argtypes = [P]
        lib.or_sim_nnz.restype = i64
        lib.or_sim_neighbors.argtypes = [P, P, P]
        lib.or_sim_dip_fields.argtypes = [P, P, P, P]
        lib.or_sim_fields.argtypes = [P, P, dbl, dbl, u32, P, P]
        lib.or_sim_run.argtypes = [P, P, P, P, i64, u32, P, P, i64, P, P, P, i64, C.c_int, P]
        lib.or_sim_run.restype = C.c_int
        lib.or_sim_set_criterion.argtypes = [P, C.c_int]
        lib.or_parallel_lhs.argtypes = [dbl, dbl]
        lib.or_parallel_lhs.restype = dbl
        lib.or_sim_lhs.argtypes = [P, i64, dbl, dbl]
        lib.or_sim_lhs.restype = dbl
        lib.or_sim_fields_ext.argtypes = [P, P, dbl, dbl, P, P, dbl, u32, P, P]
        lib.or_sim_run_ext.argtypes = [P, P, P, P, P, P, P, i64, u32, P, P, i64, P, P, P, i64,
                                       C.c_int, P]
        lib.or_sim_run_ext.restype = C.c_int
        lib.or_sample_grid.argtypes = [i64, P, P, i64, i32, i32, dbl, dbl, dbl, dbl, P, P, P, P]
        lib.or_encode.argtypes = [C.c_int, i64, P, i32, dbl, dbl, dbl, P, P]
        lib.or_encode.restype = i64
        lib.or_correlation.argtypes = [i64, P, P, P, P, dbl, dbl, i32, P, P]
        lib.or_hash_init.restype = u64
        lib.or_hash_flip.argtypes = [u64, u32, u32]
        lib.or_hash_flip.restype = u64
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def set_threads(n: int) -> None:
    """Threads used for the per-row loops (full field recomputation)."""
    _load().or_set_threads(int(n))


def get_threads() -> int:
    return int(_load().or_get_threads())


# --- Philox4x32-10 + Box-Muller (Salmon et al. SC'11; Sec. "Thermal field",
# --- Sec. "Imperfections and disorder") ---------------------------------------

def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def box_muller(words) -> tuple[float, float]:
    w = np.ascontiguousarray(words, dtype=np.uint32)
    z0, z1 = C.c_double(), C.c_double()
    _load().or_box_muller(_ptr(w), C.byref(z0), C.byref(z1))
    return z0.value, z1.value


def draw_hk(n: int, hk: float, k_disorder: float, seed: int, instance: int = 0) -> np.ndarray:
    """h_k^(i) ~ N(h_k, k_disorder h_k), redrawn while non-positive."""
    out = np.empty(n, dtype=np.float64)
    _load().or_draw_hk(n, hk, k_disorder, seed, instance, _ptr(out))
    return out


def thermal(n: int, sigma: float, seed: int, instance: int, step: int):
    """(th_par, th_perp) of every island for one field step."""
    tp = np.empty(n, dtype=np.float64)
    tq = np.empty(n, dtype=np.float64)
    _load().or_thermal(n, sigma, seed, instance, step, _ptr(tp), _ptr(tq))
    return tp, tq


# --- Geometry (Sec. "Geometries") ----------------------------------------------

def geometry(kind: int, nx: int, ny: int, a: float = 1.0):
    """Island centres and angles (radians) in canonical order (ascending y, then x)."""
    lib = _load()
    cap = lib.or_geometry_capacity(kind, nx, ny)
    if cap <= 0:
        raise ValueError("bad geometry")
    x = np.empty(cap, dtype=np.float64)
    y = np.empty(cap, dtype=np.float64)
    t = np.empty(cap, dtype=np.float64)
    n = lib.or_geometry(kind, nx, ny, a, _ptr(x), _ptr(y), _ptr(t))
    if n <= 0:
        raise ValueError("bad geometry")
    return x[:n].copy(), y[:n].copy(), t[:n].copy()


# --- Eq. (3), (5), (6) ------------------------------------------------------------

def dipole_field(rx, ry, mx, my, alpha) -> tuple[float, float]:
    """Field of a dipole with moment (mx, my) at offset r = r_i - r_j (Eq. 3, one term)."""
    hx, hy = C.c_double(), C.c_double()
    _load().or_dipole_field(rx, ry, mx, my, alpha, C.byref(hx), C.byref(hy))
    return hx.value, hy.value


def astroid_lhs(hpar, hperp, hk, b, c, beta, gamma) -> float:
    """Left-hand side of Eq. (5)."""
    return float(_load().or_astroid_lhs(hpar, hperp, hk, b, c, beta, gamma))


def parallel_lhs(hpar, hk) -> float:
    """The parallel-only criterion's LHS, |h_par| / h_k (pinwheel section)."""
    return float(_load().or_parallel_lhs(hpar, hk))


def sample_grid(x, y, gw, gh, x0, y0, dx, dy, gx, gy):
    """A spatial field h_ext(r) on a gw x gh grid (K steps of gh x gw vectors, arrays
    of shape (K, gh, gw)) sampled at the island centres: (K, n) arrays per component."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    gx = np.ascontiguousarray(gx, dtype=np.float64)
    gy = np.ascontiguousarray(gy, dtype=np.float64)
    K = gx.shape[0]
    n = len(x)
    ox = np.empty((K, n))
    oy = np.empty((K, n))
    _load().or_sample_grid(n, _ptr(x), _ptr(y), K, gw, gh, x0, y0, dx, dy, _ptr(gx), _ptr(gy),
                           _ptr(ox), _ptr(oy))
    return ox, oy


def encode(kind: int, inputs, period: int, h_lo: float, h_hi: float, angle_deg: float):
    """Input encoder (Sec. "Simulation framework"): one period of a sinusoid, sawtooth
    or rotation per input value, amplitude h_lo + (h_hi - h_lo) u."""
    u = np.ascontiguousarray(inputs, dtype=np.float64)
    m = len(u)
    hx = np.empty(max(m * period, 1))
    hy = np.empty(max(m * period, 1))
    k = _load().or_encode(kind, m, _ptr(u), period, h_lo, h_hi, angle_deg, _ptr(hx), _ptr(hy))
    if k < 0:
        raise ValueError("bad encoder arguments")
    return hx[:k].copy(), hy[:k].copy()


def correlation(x, y, theta, s, rmax: float, width: float, nbins: int):
    """Spin-spin correlation against separation (Sec. "Domain size in square ASI"):
    per bin the number of pairs and the sum of their correlations."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    t = np.ascontiguousarray(theta, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.int8)
    cnt = np.zeros(nbins, dtype=np.int64)
    sm = np.zeros(nbins, dtype=np.int64)
    _load().or_correlation(len(x), _ptr(x), _ptr(y), _ptr(t), _ptr(s), rmax, width, nbins,
                           _ptr(cnt), _ptr(sm))
    return cnt, sm


def flippable(s: int, hpar: float, lhs: float) -> bool:
    """Eq. (5) > 1 and Eq. (6)."""
    return bool(_load().or_flippable(int(s), hpar, lhs))


def neighbors(x, y, cutoff_abs: float, brute: bool = False):
    """CSR of all pairs within the (inclusive) cutoff, rows ascending."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    lib = _load()
    n = len(x)
    nnz = lib.or_neighbors(n, _ptr(x), _ptr(y), cutoff_abs, int(brute), None, None, 0)
    if nnz < 0:
        raise ValueError("neighbour search failed")
    rp = np.empty(n + 1, dtype=np.int64)
    col = np.empty(max(nnz, 1), dtype=np.int32)
    lib.or_neighbors(n, _ptr(x), _ptr(y), cutoff_abs, int(brute), _ptr(rp), _ptr(col), nnz)
    return rp, col[:nnz]


def hash_init() -> int:
    return int(_load().or_hash_init())


def hash_flips(steps, spins, h: int | None = None) -> int:
    """FNV-1a 64 over (step, spin) records, the flip-sequence hash."""
    lib = _load()
    h = hash_init() if h is None else h
    for t, k in zip(np.asarray(steps).tolist(), np.asarray(spins).tolist()):
        h = lib.or_hash_flip(h, t, k)
    return int(h)


class Sim:
    """One simulated array: positions, angles, per-island h_k and the model's
    parameters (alpha, astroid b, c, beta, gamma, sigma_th, cutoff, seed)."""

    def __init__(self, x, y, theta, hk, *, alpha, b=1.0, c=1.0, beta=3.0, gamma=3.0,
                 sigma_th=0.0, cutoff_abs, seed=0, instance=0, brute_neighbors=False,
                 criterion=ASTROID):
        self._lib = _load()
        self.x = np.ascontiguousarray(x, dtype=np.float64)
        self.y = np.ascontiguousarray(y, dtype=np.float64)
        self.theta = np.ascontiguousarray(theta, dtype=np.float64)
        self.hk = np.ascontiguousarray(hk, dtype=np.float64)
        self.n = len(self.x)
        self.params = dict(alpha=alpha, b=b, c=c, beta=beta, gamma=gamma, sigma_th=sigma_th,
                           cutoff_abs=cutoff_abs, seed=seed, instance=instance)
        self._h = self._lib.or_sim_create(self.n, _ptr(self.x), _ptr(self.y), _ptr(self.theta),
                                          _ptr(self.hk), alpha, b, c, beta, gamma, sigma_th,
                                          cutoff_abs, seed, instance, int(brute_neighbors))
        if not self._h:
            raise MemoryError("oracle: could not create the system")
        self.criterion = criterion
        self._lib.or_sim_set_criterion(self._h, int(criterion))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.or_sim_destroy(h)
            self._h = None

    @property
    def nnz(self) -> int:
        return int(self._lib.or_sim_nnz(self._h))

    def neighbors(self):
        rp = np.empty(self.n + 1, dtype=np.int64)
        col = np.empty(max(self.nnz, 1), dtype=np.int32)
        self._lib.or_sim_neighbors(self._h, _ptr(rp), _ptr(col))
        return rp, col[:self.nnz]

    def dip_fields(self, s):
        """Eq. (3) for every island, lab frame, from positions."""
        s = np.ascontiguousarray(s, dtype=np.int8)
        hx = np.empty(self.n)
        hy = np.empty(self.n)
        self._lib.or_sim_dip_fields(self._h, _ptr(s), _ptr(hx), _ptr(hy))
        return hx, hy

    def fields(self, s, hex_=0.0, hey=0.0, step=0, lx=None, ly=None, sigma=None):
        """Eq. (2) in each island's frame: (h_par, h_perp); lx, ly: the per-island
        external field (lab frame, added to the global one); sigma: the thermal
        standard deviation of this step (default sigma_th)."""
        s = np.ascontiguousarray(s, dtype=np.int8)
        hp = np.empty(self.n)
        hq = np.empty(self.n)
        lx = None if lx is None else np.ascontiguousarray(lx, dtype=np.float64)
        ly = None if ly is None else np.ascontiguousarray(ly, dtype=np.float64)
        sig = self.params["sigma_th"] if sigma is None else sigma
        self._lib.or_sim_fields_ext(self._h, _ptr(s), hex_, hey,
                                    _ptr(lx) if lx is not None else None,
                                    _ptr(ly) if ly is not None else None, sig, step, _ptr(hp),
                                    _ptr(hq))
        return hp, hq

    def lhs(self, hp, hq):
        """The LHS the switching rule ranks by (Eq. 5, or the parallel-only
        criterion), per island, for fields in the islands' frames."""
        return np.array([self._lib.or_sim_lhs(self._h, i, float(hp[i]), float(hq[i]))
                         for i in range(self.n)])

    def run(self, s, hx, hy, *, step0=0, log_cap=None, mode=MODE_INCREMENTAL,
            max_flips_per_step=0, hash_in=None, lhx=None, lhy=None, sigma=None):
        """Field steps t = 0..K-1, each a relax to a fixed point (Sec. "Dynamics").
        lhx, lhy: (K, n) per-island external fields added to the global (hx[t],
        hy[t]); sigma: K per-step thermal standard deviations.

        Returns a dict with the final spins, the flip log (step, spin), flips per
        step, the sequence hash, the status and the near-tie counters."""
        s = np.array(s, dtype=np.int8, copy=True)
        hx = np.ascontiguousarray(hx, dtype=np.float64)
        hy = np.ascontiguousarray(hy, dtype=np.float64)
        K = len(hx)
        if log_cap is None:
            log_cap = 4 * self.n * max(K, 1)
            log_cap = min(log_cap, 50_000_000)
        ls = np.zeros(max(log_cap, 1), dtype=np.uint32)
        lk = np.zeros(max(log_cap, 1), dtype=np.uint32)
        fps = np.zeros(max(K, 1), dtype=np.int64)
        h = C.c_uint64(hash_init() if hash_in is None else hash_in)
        nf = C.c_int64(0)
        ties = np.zeros(3, dtype=np.int64)
        lx = None if lhx is None else np.ascontiguousarray(lhx, dtype=np.float64)
        ly = None if lhy is None else np.ascontiguousarray(lhy, dtype=np.float64)
        sg = None if sigma is None else np.ascontiguousarray(sigma, dtype=np.float64)
        if lx is not None:
            assert lx.size == K * self.n and ly is not None and ly.size == K * self.n
        if sg is not None:
            assert sg.size == K
        st = self._lib.or_sim_run_ext(self._h, _ptr(s), _ptr(hx), _ptr(hy),
                                      _ptr(lx) if lx is not None else None,
                                      _ptr(ly) if ly is not None else None,
                                      _ptr(sg) if sg is not None else None, K, step0, _ptr(ls),
                                      _ptr(lk), log_cap, _ptr(fps), C.byref(h), C.byref(nf),
                                      max_flips_per_step, mode, _ptr(ties))
        m = min(nf.value, log_cap)
        return dict(status=st, spins=s, log_step=ls[:m].copy(), log_spin=lk[:m].copy(),
                    flips_per_step=fps[:K].copy(), hash=int(h.value), n_flips=int(nf.value),
                    ties=ties)
