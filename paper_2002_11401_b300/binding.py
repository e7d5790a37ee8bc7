"""Thin ctypes binding of the C ABI in ``include/flatspin_b300.h``.

Only argument marshalling lives here: every step of the model runs in the CUDA
library. Loading fails loudly when the library is missing; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libflatspin_b300.so")

FS_OK, FS_ERR_INVALID, FS_ERR_OOM, FS_ERR_CUDA = 0, 1, 2, 3
FS_ERR_NOT_CONVERGED, FS_ERR_TIMEOUT, FS_ERR_BOUNDS, FS_ERR_STATE = 4, 5, 6, 8
FS_SQUARE, FS_PINWHEEL, FS_KAGOME = 0, 1, 2
FS_SQUARE_OPEN, FS_PINWHEEL_DIAMOND, FS_PINWHEEL_LUCKY_KNOT, FS_ISING = 3, 4, 5, 6
FS_FP64, FS_FP32_RECHECK = 0, 1
FS_CRITERION_ASTROID, FS_CRITERION_PARALLEL = 0, 1
FS_ENCODE_SINUSOID, FS_ENCODE_SAWTOOTH, FS_ENCODE_ROTATION = 0, 1, 2
FS_RELAX_AUTO, FS_RELAX_SINGLE, FS_RELAX_MULTI, FS_RELAX_MULTI_CTA = 0, 1, 2, 3
FS_BATCH_AUTO, FS_BATCH_PERSISTENT, FS_BATCH_PER_STEP, FS_BATCH_TWO_CHAINS = 0, 1, 2, 3

EXPORTS = (
    "fs_last_error", "fs_hash_init", "fs_create_geometry", "fs_create_custom", "fs_destroy",
    "fs_set_stream", "fs_set_params", "fs_set_hk", "fs_set_spins", "fs_set_field", "fs_relax",
    "fs_run_protocol", "fs_run_protocol_dev", "fs_get_spins", "fs_get_fields", "fs_get_lhs",
    "fs_get_hk", "fs_get_geometry", "fs_get_info", "fs_get_csr", "fs_batch_run_protocol",
    "fs_server_create", "fs_server_submit", "fs_server_poll", "fs_server_drain",
    "fs_server_now", "fs_server_destroy", "fs_server_last_error", "fs_set_spins_dev",
    "fs_set_profiling", "fs_get_profile", "fs_eval_argmax_static", "fs_autotune",
    "fs_workspace_bytes", "fs_bind_workspace", "fs_set_field_local", "fs_set_field_spatial",
    "fs_set_sigma_series", "fs_encode", "fs_correlation", "fs_set_relax_mode",
    "fs_batch_run_protocol_ex",
)


class FsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[fs status {code}] {msg}")
        self.code = code


class fs_params(C.Structure):
    _fields_ = [("alpha", C.c_double), ("hk", C.c_double), ("k_disorder", C.c_double),
                ("b", C.c_double), ("c", C.c_double), ("beta", C.c_double),
                ("gamma", C.c_double), ("cutoff", C.c_double), ("sigma_th", C.c_double),
                ("seed", C.c_uint64), ("instance", C.c_uint32), ("precision", C.c_int32),
                ("max_flips_per_step", C.c_int64), ("criterion", C.c_int32),
                ("reserved", C.c_int32)]


class fs_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("nnz_padded", C.c_int64),
                ("max_degree", C.c_int32), ("e64", C.c_int32), ("e32", C.c_int32),
                ("device_bytes", C.c_int64), ("band_rel", C.c_double), ("band_abs", C.c_double),
                ("col_offsets16", C.c_int32), ("reserved_info", C.c_int32)]


class fs_profile(C.Structure):
    _fields_ = [("sweep_ms", C.c_double), ("relax_ms", C.c_double),
                ("sweep_launches", C.c_int64), ("relax_launches", C.c_int64),
                ("rechecks", C.c_int64), ("fallbacks", C.c_int64), ("rounds", C.c_int64),
                ("idle_rounds", C.c_int64), ("round_flips", C.c_int64), ("handoffs", C.c_int64)]


class fs_request(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32), ("a", C.c_double),
                ("params", fs_params), ("K", C.c_int64), ("hx", C.c_void_p),
                ("hy", C.c_void_p), ("spins_out", C.c_void_p)]


class fs_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("done", C.c_int32), ("n", C.c_int64),
                ("n_flips", C.c_int64), ("seq_hash", C.c_uint64), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double)]


_lock = threading.Lock()
_lib = None


def load():
    """Loads the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library missing: {LIB_PATH}; run "
                              "`python -m paper_2002_11401_b300.build` (no CPU fallback)")
        lib = C.CDLL(LIB_PATH)
        P, i32, i64, u32, u64, dbl = (C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_uint64,
                                      C.c_double)
        sig = {
            "fs_last_error": ([P], C.c_char_p),
            "fs_hash_init": ([], u64),
            "fs_create_geometry": ([i32, i32, i32, dbl, P], i32),
            "fs_create_custom": ([i64, P, P, P, dbl, P], i32),
            "fs_destroy": ([P], None),
            "fs_set_stream": ([P, P], i32),
            "fs_set_params": ([P, P], i32),
            "fs_set_hk": ([P, P, i64], i32),
            "fs_set_spins": ([P, P, i64], i32),
            "fs_set_field": ([P, dbl, dbl, u32], i32),
            "fs_relax": ([P, P, i64, P], i32),
            "fs_run_protocol": ([P, P, P, i64, u32, i32, P, P, i64, P, P, P], i32),
            "fs_run_protocol_dev": ([P, P, P, i64, u32, i32, P, P, i64, P, P], i32),
            "fs_get_spins": ([P, P, i64], i32),
            "fs_get_fields": ([P, P, P, i64], i32),
            "fs_get_lhs": ([P, P, P, P, i64], i32),
            "fs_get_hk": ([P, P, i64], i32),
            "fs_get_geometry": ([P, P, P, P, i64], i32),
            "fs_get_info": ([P, P], i32),
            "fs_get_csr": ([P, P, P, P, P], i32),
            "fs_batch_run_protocol": ([P, i32, P, P, i64, i32, P, P, P, P], i32),
            "fs_batch_run_protocol_ex": ([P, i32, P, P, i64, i32, i32, P, P, P, P], i32),
            "fs_server_create": ([C.c_size_t, i32, P], i32),
            "fs_server_submit": ([P, P, P], i32),
            "fs_server_poll": ([P, u64, P], i32),
            "fs_server_drain": ([P], i32),
            "fs_server_now": ([P], dbl),
            "fs_server_destroy": ([P], None),
            "fs_server_last_error": ([P], C.c_char_p),
            "fs_set_spins_dev": ([P, P, i64], i32),
            "fs_set_profiling": ([P, i32], i32),
            "fs_get_profile": ([P, P], i32),
            "fs_eval_argmax_static": ([P, P, dbl, dbl, u32, P, P, P], i32),
            "fs_autotune": ([P, P], i32),
            "fs_workspace_bytes": ([P, P, P], i32),
            "fs_bind_workspace": ([P, P, C.c_size_t, P], i32),
            "fs_set_field_local": ([P, P, P, i64, i64], i32),
            "fs_set_field_spatial": ([P, P, P, i64, i32, i32, dbl, dbl, dbl, dbl], i32),
            "fs_set_sigma_series": ([P, P, i64], i32),
            "fs_encode": ([i32, P, i64, i32, dbl, dbl, dbl, P, P], i32),
            "fs_correlation": ([P, dbl, dbl, i32, P, P], i32),
            "fs_set_relax_mode": ([P, i32], i32),
        }
        for name, (args, res) in sig.items():
            if not hasattr(lib, name):
                continue
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def hash_init() -> int:
    return int(load().fs_hash_init())


def make_params(alpha, hk=0.2, k_disorder=0.05, b=1.0, c=1.0, beta=3.0, gamma=3.0, cutoff=3.0,
                sigma_th=0.0, seed=0, instance=0, precision=FS_FP64,
                max_flips_per_step=0, criterion=0) -> fs_params:
    return fs_params(alpha, hk, k_disorder, b, c, beta, gamma, cutoff, sigma_th, seed, instance,
                     precision, max_flips_per_step, criterion, 0)


class Sim:
    """One simulation (an ``fs_sim``)."""

    def __init__(self, handle):
        self._lib = load()
        self._h = handle
        self.n = 0
        self.n = self.info().n

    @classmethod
    def geometry(cls, kind: int, nx: int, ny: int, a: float = 1.0) -> "Sim":
        lib = load()
        h = C.c_void_p()
        st = lib.fs_create_geometry(kind, nx, ny, a, C.byref(h))
        if st != FS_OK:
            raise FsError(st, lib.fs_last_error(None).decode())
        return cls(h)

    @classmethod
    def custom(cls, x, y, theta, a: float = 1.0) -> "Sim":
        lib = load()
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        t = np.ascontiguousarray(theta, dtype=np.float64)
        h = C.c_void_p()
        st = lib.fs_create_custom(len(x), _p(x), _p(y), _p(t), a, C.byref(h))
        if st != FS_OK:
            raise FsError(st, lib.fs_last_error(None).decode())
        return cls(h)

    def _check(self, st: int):
        if st != FS_OK:
            raise FsError(st, self._lib.fs_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fs_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    @property
    def handle(self):
        return self._h

    def set_stream(self, stream_ptr: int):
        self._check(self._lib.fs_set_stream(self._h, C.c_void_p(stream_ptr)))

    def set_params(self, params: fs_params):
        self._check(self._lib.fs_set_params(self._h, C.byref(params)))

    def workspace_bytes(self, params: fs_params) -> int:
        """Device bytes set_params(params) would allocate (state + build temporaries)."""
        out = C.c_size_t(0)
        self._check(self._lib.fs_workspace_bytes(self._h, C.byref(params), C.byref(out)))
        return out.value

    def bind_workspace(self, dev_ptr: int, nbytes: int, stream_ptr: int = 0):
        """Carves the state from a caller-owned device buffer (0: the library's pool)."""
        self._check(self._lib.fs_bind_workspace(self._h, C.c_void_p(dev_ptr or None),
                                                 C.c_size_t(nbytes),
                                                 C.c_void_p(stream_ptr or None)))

    def set_hk(self, hk):
        hk = np.ascontiguousarray(hk, dtype=np.float64)
        self._check(self._lib.fs_set_hk(self._h, _p(hk), len(hk)))

    def set_spins(self, s):
        s = np.ascontiguousarray(s, dtype=np.int8)
        self._check(self._lib.fs_set_spins(self._h, _p(s), len(s)))

    def set_spins_dev(self, d_ptr: int):
        self._check(self._lib.fs_set_spins_dev(self._h, C.c_void_p(d_ptr), self.n))

    def set_profiling(self, on: bool):
        self._check(self._lib.fs_set_profiling(self._h, int(bool(on))))

    def autotune(self) -> int:
        lanes = C.c_int32(0)
        self._check(self._lib.fs_autotune(self._h, C.byref(lanes)))
        return int(lanes.value)

    def profile(self) -> dict:
        out = fs_profile()
        self._check(self._lib.fs_get_profile(self._h, C.byref(out)))
        return {k: getattr(out, k) for k, _ in fs_profile._fields_}

    def set_field(self, hx: float, hy: float, step: int = 0):
        self._check(self._lib.fs_set_field(self._h, hx, hy, step))

    def relax(self, log_cap: int = 0):
        log = np.zeros(max(log_cap, 1), dtype=np.uint32)
        nf = C.c_int64(0)
        self._check(self._lib.fs_relax(self._h, _p(log) if log_cap else None, log_cap,
                                       C.byref(nf)))
        return nf.value, log[:min(nf.value, log_cap)].copy()

    def run_protocol(self, hx, hy, *, step0: int = 0, resweep: bool = True,
                     log_cap: int | None = None, hash_in: int | None = None):
        hx = np.ascontiguousarray(hx, dtype=np.float64)
        hy = np.ascontiguousarray(hy, dtype=np.float64)
        K = len(hx)
        if log_cap is None:
            log_cap = min(4 * self.n * max(K, 1), 50_000_000)
        ls = np.zeros(max(log_cap, 1), dtype=np.uint32)
        lk = np.zeros(max(log_cap, 1), dtype=np.uint32)
        fps = np.zeros(max(K, 1), dtype=np.int64)
        h = C.c_uint64(hash_init() if hash_in is None else hash_in)
        nf = C.c_int64(0)
        st = self._lib.fs_run_protocol(self._h, _p(hx), _p(hy), K, step0, int(bool(resweep)),
                                       _p(ls) if log_cap else None,
                                       _p(lk) if log_cap else None, log_cap, _p(fps),
                                       C.byref(h), C.byref(nf))
        m = min(nf.value, log_cap)
        res = dict(status=st, log_step=ls[:m].copy(), log_spin=lk[:m].copy(),
                   flips_per_step=fps[:K].copy(), hash=int(h.value), n_flips=int(nf.value))
        if st not in (FS_OK, FS_ERR_NOT_CONVERGED):
            self._check(st)
        return res

    def run_protocol_dev(self, d_hx: int, d_hy: int, K: int, *, step0: int = 0,
                         resweep: bool = True, d_log_step: int = 0, d_log_spin: int = 0,
                         log_cap: int = 0, d_flips_per_step: int = 0, d_out: int):
        """Device-pointer form (torch ``data_ptr()`` values); queued, not waited on."""
        self._check(self._lib.fs_run_protocol_dev(
            self._h, C.c_void_p(d_hx), C.c_void_p(d_hy), K, step0, int(bool(resweep)),
            C.c_void_p(d_log_step or None), C.c_void_p(d_log_spin or None), log_cap,
            C.c_void_p(d_flips_per_step or None), C.c_void_p(d_out)))

    def spins(self) -> np.ndarray:
        out = np.empty(self.n, dtype=np.int8)
        self._check(self._lib.fs_get_spins(self._h, _p(out), self.n))
        return out

    def fields(self):
        hp = np.empty(self.n)
        hq = np.empty(self.n)
        self._check(self._lib.fs_get_fields(self._h, _p(hp), _p(hq), self.n))
        return hp, hq

    def lhs(self, bounds: bool = False):
        out = np.empty(self.n)
        lo = np.empty(self.n) if bounds else None
        hi = np.empty(self.n) if bounds else None
        self._check(self._lib.fs_get_lhs(self._h, _p(out), _p(lo), _p(hi), self.n))
        return (out, lo, hi) if bounds else out

    def hk(self):
        out = np.empty(self.n)
        self._check(self._lib.fs_get_hk(self._h, _p(out), self.n))
        return out

    def geometry_arrays(self):
        x, y, t = np.empty(self.n), np.empty(self.n), np.empty(self.n)
        self._check(self._lib.fs_get_geometry(self._h, _p(x), _p(y), _p(t), self.n))
        return x, y, t

    def info(self) -> fs_info:
        out = fs_info()
        self._check(self._lib.fs_get_info(self._h, C.byref(out)))
        return out

    def set_relax_mode(self, mode: int):
        """FS_RELAX_AUTO, FS_RELAX_SINGLE, FS_RELAX_MULTI or FS_RELAX_MULTI_CTA."""
        self._check(self._lib.fs_set_relax_mode(self._h, mode))

    def set_field_local(self, hx, hy):
        """Local external field series: (K, n) arrays per component (K = 0 clears)."""
        hx = np.ascontiguousarray(hx, dtype=np.float64)
        hy = np.ascontiguousarray(hy, dtype=np.float64)
        K = hx.shape[0] if hx.ndim == 2 else 0
        self._check(self._lib.fs_set_field_local(self._h, _p(hx) if K else None,
                                                 _p(hy) if K else None, K, self.n))

    def set_field_spatial(self, gx, gy, x0, y0, dx, dy):
        """Spatial external field series: (K, gh, gw) arrays per component."""
        gx = np.ascontiguousarray(gx, dtype=np.float64)
        gy = np.ascontiguousarray(gy, dtype=np.float64)
        K, gh, gw = gx.shape
        self._check(self._lib.fs_set_field_spatial(self._h, _p(gx), _p(gy), K, gw, gh, x0, y0,
                                                   dx, dy))

    def set_sigma_series(self, sigma):
        """Thermal standard deviation per field step (empty clears)."""
        sg = np.ascontiguousarray(sigma, dtype=np.float64)
        self._check(self._lib.fs_set_sigma_series(self._h, _p(sg) if len(sg) else None, len(sg)))

    def correlation(self, rmax: float, width: float, nbins: int):
        """Spin-spin correlation against separation: (pairs, sums) per bin."""
        cnt = np.zeros(nbins, dtype=np.int64)
        sm = np.zeros(nbins, dtype=np.int64)
        self._check(self._lib.fs_correlation(self._h, rmax, width, nbins, _p(cnt), _p(sm)))
        return cnt, sm

    def csr(self):
        inf = self.info()
        rp = np.empty(self.n + 1, dtype=np.int64)
        col = np.empty(max(inf.nnz, 1), dtype=np.int32)
        P = np.empty(max(inf.nnz, 1))
        Q = np.empty(max(inf.nnz, 1))
        self._check(self._lib.fs_get_csr(self._h, _p(rp), _p(col), _p(P), _p(Q)))
        return rp, col[:inf.nnz], P[:inf.nnz], Q[:inf.nnz]


def encode(kind: int, inputs, period: int, h_lo: float, h_hi: float, angle_deg: float):
    """Input encoder (``fs_encode``): one period of a sinusoid, sawtooth or rotation
    per input value; returns the (hx, hy) field series."""
    lib = load()
    u = np.ascontiguousarray(inputs, dtype=np.float64)
    m = len(u)
    hx = np.empty(max(m * period, 1))
    hy = np.empty(max(m * period, 1))
    st = lib.fs_encode(kind, _p(u), m, period, h_lo, h_hi, angle_deg, _p(hx), _p(hy))
    if st != FS_OK:
        raise FsError(st, "bad encoder arguments")
    return hx[:m * period].copy(), hy[:m * period].copy()


def batch_run_protocol(sims, hx, hy, *, resweep: bool = True, with_counts: bool = False,
                       schedule: int = FS_BATCH_AUTO):
    """Runs every simulation of `sims` through one protocol together (schedule:
    FS_BATCH_AUTO, FS_BATCH_PERSISTENT, FS_BATCH_PER_STEP or FS_BATCH_TWO_CHAINS)."""
    lib = load()
    n = len(sims)
    handles = (C.c_void_p * n)(*[s.handle for s in sims])
    hx = np.ascontiguousarray(hx, dtype=np.float64)
    hy = np.ascontiguousarray(hy, dtype=np.float64)
    K = len(hx)
    nf = np.zeros(n, dtype=np.int64)
    hs = np.full(n, hash_init(), dtype=np.uint64)
    stv = np.zeros(n, dtype=np.int32)
    fps = np.zeros(n * K, dtype=np.int64) if with_counts else None
    st = lib.fs_batch_run_protocol_ex(handles, n, _p(hx), _p(hy), K, int(bool(resweep)),
                                      int(schedule), _p(nf), _p(hs), _p(stv), _p(fps))
    if st != FS_OK:
        raise FsError(st, lib.fs_last_error(sims[0].handle).decode())
    out = dict(n_flips=nf, hash=hs, status=stv)
    if with_counts:
        out["flips_per_step"] = fps.reshape(n, K)
    return out


class Server:
    """Continuous-batching server (``fs_server``)."""

    def __init__(self, hbm_budget: int, max_active: int = 256):
        self._lib = load()
        h = C.c_void_p()
        st = self._lib.fs_server_create(hbm_budget, max_active, C.byref(h))
        if st != FS_OK:
            raise FsError(st, self._lib.fs_last_error(None).decode())
        self._h = h
        self._keep = {}

    def submit(self, kind, nx, ny, params: fs_params, hx, hy, a=1.0, spins_out=None) -> int:
        hx = np.ascontiguousarray(hx, dtype=np.float64)
        hy = np.ascontiguousarray(hy, dtype=np.float64)
        req = fs_request(kind, nx, ny, a, params, len(hx), hx.ctypes.data, hy.ctypes.data,
                         spins_out.ctypes.data if spins_out is not None else None)
        t = C.c_uint64(0)
        st = self._lib.fs_server_submit(self._h, C.byref(req), C.byref(t))
        if st != FS_OK:
            raise FsError(st, self._lib.fs_server_last_error(self._h).decode())
        if spins_out is not None:
            self._keep[t.value] = spins_out
        return int(t.value)

    def poll(self, ticket: int):
        r = fs_result()
        st = self._lib.fs_server_poll(self._h, ticket, C.byref(r))
        if st == FS_ERR_STATE:
            return None
        if st != FS_OK:
            raise FsError(st, self._lib.fs_server_last_error(self._h).decode())
        self._keep.pop(ticket, None)
        return dict(status=r.status, n=r.n, n_flips=r.n_flips, hash=int(r.seq_hash),
                    t_submit=r.t_submit, t_admit=r.t_admit, t_done=r.t_done)

    def drain(self):
        st = self._lib.fs_server_drain(self._h)
        if st != FS_OK:
            raise FsError(st, self._lib.fs_server_last_error(self._h).decode())

    def now(self) -> float:
        return float(self._lib.fs_server_now(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fs_server_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()
