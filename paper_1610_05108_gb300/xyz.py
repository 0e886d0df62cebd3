"""Thin ctypes binding of libxyz (include/xyz.h).

Argument marshalling only: every step of the search runs in the library's
CUDA kernels.  There is no CPU fallback; if ``libxyz.so`` is missing or the
GPU is unavailable the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libxyz.so")

XYZ_OK, XYZ_EINVAL, XYZ_ENOMEM, XYZ_ECUDA, XYZ_ETIMEDOUT, XYZ_ECANCELED, XYZ_EAGAIN = range(7)
XYZ_MAX_M = 64

_i64, _i32, _u64, _dbl, _p = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p


class XyzError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"xyz error {code}: {msg}")
        self.code = code


class Pair(ctypes.Structure):
    _fields_ = [("j", ctypes.c_int32), ("k", ctypes.c_int32), ("agree", ctypes.c_int32),
                ("strength", ctypes.c_float)]


PAIR_DTYPE = np.dtype([("j", np.int32), ("k", np.int32), ("agree", np.int32), ("strength", np.float32)])


class Stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "runs", "chunks", "runs_per_chunk", "candidates", "buckets", "passing", "unique_pairs",
        "sort_passes", "key_bits", "gpu_launches")] + \
        [(name, ctypes.c_double) for name in (
            "ms_keys", "ms_sort", "ms_join", "ms_verify", "ms_dedup", "ms_total")] + \
        [(name, ctypes.c_int64) for name in (
            "launches_keys", "launches_sort", "launches_join", "launches_verify", "launches_dedup",
            "survivors", "filter_kept", "attempts", "bucket_members",
            "segment_grouped_runs")]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class Tiles(ctypes.Structure):
    _fields_ = [("filter_threads", ctypes.c_int32), ("verify_blocks_per_sm", ctypes.c_int32),
                ("group_runs", ctypes.c_int64)]


class Peaks(ctypes.Structure):
    _fields_ = [("alu_ops_per_s", ctypes.c_double), ("iadd_ops_per_s", ctypes.c_double),
                ("popc_ops_per_s", ctypes.c_double), ("sm_mhz", ctypes.c_double), ("sms", ctypes.c_int32)]


def probe_peaks() -> dict:
    """Measured instruction throughputs of the current device (xyz_probe_peaks)."""
    pk = Peaks()
    _check(load().xyz_probe_peaks(ctypes.byref(pk)))
    return {name: getattr(pk, name) for name, _ in Peaks._fields_}


class ServerStats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "completed", "canceled", "failed", "queued", "active", "device_bytes", "budget_bytes")] + \
        [(name, ctypes.c_double) for name in ("p50_ms", "p99_ms", "pairs_screened", "elapsed_ms")]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


# name -> (restype, argtypes); every symbol declared in include/xyz.h
SIGNATURES = {
    "xyz_create": (ctypes.c_int, [_p, _p, _i64, _i64, _p]),
    "xyz_create_dev": (ctypes.c_int, [_p, _p, _i64, _i64, _p, _p]),
    "xyz_create_sign": (ctypes.c_int, [_p, _i64, _i64, _u64, _p]),
    "xyz_create_unbiased": (ctypes.c_int, [_p, _p, _i64, _i64, _p]),
    "xyz_set_y": (ctypes.c_int, [_p, _p]),
    "xyz_set_y_dev": (ctypes.c_int, [_p, _p]),
    "xyz_set_y_real": (ctypes.c_int, [_p, _p]),
    "xyz_set_y_real_dev": (ctypes.c_int, [_p, _p]),
    "xyz_destroy": (None, [_p]),
    "xyz_last_error": (ctypes.c_char_p, []),
    "xyz_info": (ctypes.c_int, [_p, _p, _p, _p]),
    "xyz_search": (ctypes.c_int, [_p, _i32, _i32, _dbl, _u64, _p, _p]),
    "xyz_search_range": (ctypes.c_int, [_p, _i64, _i64, _i32, _dbl, _u64, _p, _p]),
    "xyz_search_batch": (ctypes.c_int, [_p, _p, _i32, _i32, _i32, _dbl, _u64, _p, _p]),
    "xyz_search_batch_dev": (ctypes.c_int, [_p, _p, _i32, _i32, _i32, _dbl, _u64, _p, _p]),
    "xyz_brute_force": (ctypes.c_int, [_p, _dbl, _p, _p]),
    "xyz_search_abs": (ctypes.c_int, [_p, _i32, _i32, _dbl, _u64, _p, _p]),
    "xyz_search_many": (ctypes.c_int, [_p, _i32, _p, _p, _p, _p, _p, _p]),
    "xyz_autotune_M": (ctypes.c_int, [_p, _dbl, _dbl, _dbl, _i32, _i32, _u64, _i64, _p, _p, _p, _p]),
    "xyz_kkt_screen": (ctypes.c_int, [_p, _p, _dbl, _i32, _i32, _u64, _p, _p]),
    "xyz_free_pairs": (None, [_p]),
    "xyz_free": (None, [_p]),
    "xyz_get_stats": (ctypes.c_int, [_p, _p]),
    "xyz_set_timing": (ctypes.c_int, [_p, ctypes.c_int]),
    "xyz_set_chunk_entries": (ctypes.c_int, [_p, _i64]),
    "xyz_set_filter": (ctypes.c_int, [_p, ctypes.c_int]),
    "xyz_set_spill_flush": (ctypes.c_int, [_p, _i64]),
    "xyz_set_onchip_partitions": (ctypes.c_int, [_p, ctypes.c_int32]),
    "xyz_set_fused_filter": (ctypes.c_int, [_p, ctypes.c_int]),
    "xyz_run_keys": (ctypes.c_int, [_p, _i32, _u64, _i64, _p, _p]),
    "xyz_run_candidates": (ctypes.c_int, [_p, _i32, _u64, _i64, _p, _p]),
    "xyz_agree": (ctypes.c_int, [_p, _p, _p, _i64, _p]),
    "xyz_sample_agree": (ctypes.c_int, [_p, _i64, _u64, _p, _p, _p]),
    "xyz_amin": (_i64, [_i64, _dbl]),
    "xyz_eta": (_dbl, [_dbl, _i32, _i64]),
    "xyz_runs_for_recall": (_i64, [_dbl, _dbl]),
    "xyz_best_M": (ctypes.c_int, [_i64, _i64, _dbl, _p, _i64, _i32, _p, _p]),
    "xyz_M_for_gamma0": (_i32, [_i64, _dbl]),
    "xyz_run_candidates_noalloc": (ctypes.c_int, [_p, _i32, _u64, _i64, _p, _i64, _p]),
    "xyz_probe_peaks": (ctypes.c_int, [_p]),
    "xyz_set_tiles": (ctypes.c_int, [_p, _p]),
    "xyz_autotune_tiles": (ctypes.c_int, [_p, _i32, _dbl, _u64, _i64, _p, _p]),
    "xyz_server_create": (ctypes.c_int, [_i32, _i64, _i64, _p]),
    "xyz_server_add_dataset": (ctypes.c_int, [_p, _p, _p, _i64, _i64, _p]),
    "xyz_server_submit": (ctypes.c_int, [_p, _i32, _p, _i32, _i32, _dbl, _u64, _p]),
    "xyz_server_wait": (ctypes.c_int, [_p, _i64, _i64, _p, _p, _p]),
    "xyz_server_poll": (ctypes.c_int, [_p, _i64, _p, _p, _p]),
    "xyz_server_cancel": (ctypes.c_int, [_p, _i64]),
    "xyz_server_get_stats": (ctypes.c_int, [_p, _p]),
    "xyz_server_destroy": (None, [_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libxyz.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run paper_1610_05108_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int):
    if rc != XYZ_OK:
        raise XyzError(rc, load().xyz_last_error().decode())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _pairs_to_numpy(ptr: ctypes.c_void_p, count: int) -> np.ndarray:
    lib = load()
    if count == 0 or not ptr.value:
        if ptr.value:
            lib.xyz_free_pairs(ptr)
        return np.zeros(0, dtype=PAIR_DTYPE)
    buf = (ctypes.c_char * (count * PAIR_DTYPE.itemsize)).from_address(ptr.value)
    out = np.frombuffer(bytes(buf), dtype=PAIR_DTYPE).copy()
    lib.xyz_free_pairs(ptr)
    return out


# ------------------------------------------------------------- planner

def amin(n: int, kappa: float) -> int:
    return int(load().xyz_amin(n, float(kappa)))


def eta(gamma: float, M: int, L: int) -> float:
    return float(load().xyz_eta(float(gamma), int(M), int(L)))


def runs_for_recall(beta: float, eta_target: float) -> int:
    return int(load().xyz_runs_for_recall(float(beta), float(eta_target)))


def best_M(n: int, p: int, gamma: float, agree: np.ndarray, max_M: int = XYZ_MAX_M):
    agree = np.ascontiguousarray(agree, dtype=np.int32)
    M = ctypes.c_int32(0)
    cost = ctypes.c_double(0.0)
    _check(load().xyz_best_M(n, p, float(gamma), _ptr(agree), len(agree), max_M,
                             ctypes.byref(M), ctypes.byref(cost)))
    return int(M.value), float(cost.value)


def M_for_gamma0(p: int, gamma0: float) -> int:
    return int(load().xyz_M_for_gamma0(int(p), float(gamma0)))


# ------------------------------------------------------------- context

class Context:
    """A resident packed X (and Y) on the current CUDA device."""

    def __init__(self, handle: ctypes.c_void_p, n: int, p: int):
        self._h = handle
        self.n, self.p = n, p

    # construction ---------------------------------------------------
    @classmethod
    def from_host(cls, X: np.ndarray, Y: np.ndarray) -> "Context":
        X = np.asfortranarray(X, dtype=np.int8)
        Y = np.ascontiguousarray(Y, dtype=np.int8)
        n, p = X.shape
        if Y.shape != (n,):
            raise ValueError("Y must have shape (n,)")
        h = ctypes.c_void_p()
        _check(load().xyz_create(_ptr(X), _ptr(Y), n, p, ctypes.byref(h)))
        return cls(h, n, p)

    @classmethod
    def from_real_sign(cls, X: np.ndarray, coin_seed: int = 0) -> "Context":
        """Real X (n x p) through the sign transform of Section 3.2."""
        X = np.asfortranarray(X, dtype=np.float32)
        n, p = X.shape
        h = ctypes.c_void_p()
        _check(load().xyz_create_sign(_ptr(X), n, p, coin_seed & (2**64 - 1), ctypes.byref(h)))
        return cls(h, n, p)

    @classmethod
    def from_real_unbiased(cls, X: np.ndarray, Y: np.ndarray) -> "Context":
        """Real X (n x p) and real Y through the unbiased transform (Section 3.2)."""
        X = np.asfortranarray(X, dtype=np.float32)
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        n, p = X.shape
        if Y.shape != (n,):
            raise ValueError("Y must have shape (n,)")
        h = ctypes.c_void_p()
        _check(load().xyz_create_unbiased(_ptr(X), _ptr(Y), n, p, ctypes.byref(h)))
        return cls(h, n, p)

    @classmethod
    def from_device(cls, dX_ptr: int, dY_ptr: int, n: int, p: int, stream: int = 0) -> "Context":
        """X/Y given as device pointers (e.g. ``tensor.data_ptr()`` of int8
        CUDA tensors, X column-major) and a cudaStream_t handle."""
        h = ctypes.c_void_p()
        _check(load().xyz_create_dev(ctypes.c_void_p(dX_ptr), ctypes.c_void_p(dY_ptr), n, p,
                                     ctypes.c_void_p(stream or None), ctypes.byref(h)))
        return cls(h, n, p)

    def close(self):
        if self._h is not None and self._h.value:
            load().xyz_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("context is closed")
        return self._h

    # response --------------------------------------------------------
    def set_y(self, Y: np.ndarray):
        Y = np.ascontiguousarray(Y, dtype=np.int8)
        if Y.shape != (self.n,):
            raise ValueError("Y must have shape (n,)")
        _check(load().xyz_set_y(self.handle, _ptr(Y)))

    def set_y_dev(self, dY_ptr: int):
        _check(load().xyz_set_y_dev(self.handle, ctypes.c_void_p(dY_ptr)))

    def set_y_real(self, Y: np.ndarray):
        """Real-valued response (Section 3.1): weighted rows and strengths."""
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        if Y.shape != (self.n,):
            raise ValueError("Y must have shape (n,)")
        _check(load().xyz_set_y_real(self.handle, _ptr(Y)))

    def set_y_real_dev(self, dY_ptr: int):
        _check(load().xyz_set_y_real_dev(self.handle, ctypes.c_void_p(dY_ptr)))

    # search ----------------------------------------------------------
    def search(self, L: int, M: int, kappa: float, seed: int) -> np.ndarray:
        out = ctypes.c_void_p()
        cnt = ctypes.c_int64(0)
        _check(load().xyz_search(self.handle, int(L), int(M), float(kappa), seed & (2**64 - 1),
                                 ctypes.byref(out), ctypes.byref(cnt)))
        return _pairs_to_numpy(out, cnt.value)

    def search_range(self, l0: int, l1: int, M: int, kappa: float, seed: int) -> np.ndarray:
        out = ctypes.c_void_p()
        cnt = ctypes.c_int64(0)
        _check(load().xyz_search_range(self.handle, int(l0), int(l1), int(M), float(kappa),
                                       seed & (2**64 - 1), ctypes.byref(out), ctypes.byref(cnt)))
        return _pairs_to_numpy(out, cnt.value)

    def autotune_M(self, kappa: float, gamma: float, recall: float, M_lo: int, M_hi: int, seed: int = 1,
                   trial_runs: int = 2048):
        """(M, L, predicted ms, table) with the fastest measured search that
        reaches `recall` for a pair of strength gamma (interaction strength
        a/n, eq. def_gamma)."""
        Mb = ctypes.c_int32(0)
        Lb = ctypes.c_int64(0)
        ms = ctypes.c_double(0)
        table = np.zeros((M_hi - M_lo + 1, 3), dtype=np.float64)
        _check(load().xyz_autotune_M(self.handle, float(kappa), float(gamma), float(recall), int(M_lo),
                                     int(M_hi), seed & (2**64 - 1), int(trial_runs), ctypes.byref(Mb),
                                     ctypes.byref(Lb), ctypes.byref(ms), _ptr(table)))
        return Mb.value, Lb.value, ms.value, table

    def search_abs(self, L: int, M: int, kappa: float, seed: int) -> np.ndarray:
        """Pairs with |Y^T(X_j o X_k)| / n >= kappa (searches with +Y and -Y)."""
        out = ctypes.c_void_p()
        cnt = ctypes.c_int64(0)
        _check(load().xyz_search_abs(self.handle, int(L), int(M), float(kappa), seed & (2**64 - 1),
                                     ctypes.byref(out), ctypes.byref(cnt)))
        return _pairs_to_numpy(out, cnt.value)

    def kkt_screen(self, r: np.ndarray, lam: float, L: int, M: int, seed: int) -> np.ndarray:
        """Lasso KKT check: pairs with |r^T(X_j o X_k)| / n > lam."""
        r = np.ascontiguousarray(r, dtype=np.float64)
        if r.shape != (self.n,):
            raise ValueError("r must have shape (n,)")
        out = ctypes.c_void_p()
        cnt = ctypes.c_int64(0)
        _check(load().xyz_kkt_screen(self.handle, _ptr(r), float(lam), int(L), int(M), seed & (2**64 - 1),
                                     ctypes.byref(out), ctypes.byref(cnt)))
        return _pairs_to_numpy(out, cnt.value)

    def brute_force(self, kappa: float) -> np.ndarray:
        """Every pair j < k with strength >= kappa (exhaustive GPU screen)."""
        out = ctypes.c_void_p()
        cnt = ctypes.c_int64(0)
        _check(load().xyz_brute_force(self.handle, float(kappa), ctypes.byref(out), ctypes.byref(cnt)))
        return _pairs_to_numpy(out, cnt.value)

    def search_batch(self, Ys: np.ndarray, L: int, M: int, kappa: float, seed: int) -> list:
        """One search per row of Ys (B x n int8 +-1) on this X; list of B results."""
        Ys = np.ascontiguousarray(Ys, dtype=np.int8)
        if Ys.ndim != 2 or Ys.shape[1] != self.n:
            raise ValueError("Ys must have shape (B, n)")
        B = Ys.shape[0]
        out = ctypes.c_void_p()
        offs = np.zeros(B + 1, dtype=np.int64)
        _check(load().xyz_search_batch(self.handle, _ptr(Ys), B, int(L), int(M), float(kappa),
                                       seed & (2**64 - 1), ctypes.byref(out), _ptr(offs)))
        allp = _pairs_to_numpy(out, int(offs[-1]))
        return [allp[offs[b]:offs[b + 1]].copy() for b in range(B)]

    def stats(self) -> dict:
        st = Stats()
        _check(load().xyz_get_stats(self.handle, ctypes.byref(st)))
        return st.as_dict()

    def set_timing(self, on: bool):
        _check(load().xyz_set_timing(self.handle, 1 if on else 0))

    def set_chunk_entries(self, entries: int):
        _check(load().xyz_set_chunk_entries(self.handle, int(entries)))

    def set_filter(self, on):
        """True / 1: the survivor filter where it applies (default); False /
        0: group every column; 2: the class-split filter wherever it applies."""
        mode = int(on) if not isinstance(on, bool) else (1 if on else 0)
        _check(load().xyz_set_filter(self.handle, mode))

    def set_spill_flush(self, groups: int):
        _check(load().xyz_set_spill_flush(self.handle, int(groups)))

    def set_tiles(self, filter_threads: int = 0, verify_blocks_per_sm: int = 0, group_runs: int = 0):
        """Launch shapes of later searches (0 = the default rule); results never depend on them."""
        t = Tiles(filter_threads, verify_blocks_per_sm, group_runs)
        _check(load().xyz_set_tiles(self.handle, ctypes.byref(t)))

    def autotune_tiles(self, M: int, kappa: float, seed: int = 1, trial_runs: int = 4096):
        """Launch shapes picked by timing searches of trial_runs runs; set on the context.
        Returns (dict of the shapes, ms of the best trial)."""
        t = Tiles()
        ms = ctypes.c_double()
        _check(load().xyz_autotune_tiles(self.handle, M, kappa, seed & (2**64 - 1), trial_runs, ctypes.byref(t),
                                         ctypes.byref(ms)))
        return {name: getattr(t, name) for name, _ in Tiles._fields_}, ms.value

    def set_onchip_partitions(self, max_parts: int):
        _check(load().xyz_set_onchip_partitions(self.handle, int(max_parts)))

    def set_fused_filter(self, enable: bool):
        """Whether search_many may run this context's filter in a fused
        launch with the other searches of the call."""
        _check(load().xyz_set_fused_filter(self.handle, int(bool(enable))))

    def info(self) -> dict:
        n, p, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().xyz_info(self.handle, ctypes.byref(n), ctypes.byref(p), ctypes.byref(b)))
        return {"n": n.value, "p": p.value, "device_bytes": b.value}

    # parity hooks ----------------------------------------------------
    def run_keys(self, M: int, seed: int, run: int):
        kx = np.zeros(self.p, dtype=np.uint64)
        c = ctypes.c_uint64(0)
        _check(load().xyz_run_keys(self.handle, int(M), seed & (2**64 - 1), int(run), _ptr(kx),
                                   ctypes.byref(c)))
        return kx, int(c.value)

    def run_candidates(self, M: int, seed: int, run: int) -> np.ndarray:
        out = ctypes.c_void_p()
        cnt = ctypes.c_int64(0)
        lib = load()
        _check(lib.xyz_run_candidates(self.handle, int(M), seed & (2**64 - 1), int(run),
                                      ctypes.byref(out), ctypes.byref(cnt)))
        if cnt.value == 0:
            return np.zeros((0, 2), dtype=np.int32)
        buf = (ctypes.c_int32 * (2 * cnt.value)).from_address(out.value)
        arr = np.frombuffer(buf, dtype=np.int32).reshape(-1, 2).copy()
        lib.xyz_free(out)
        return arr

    def agree(self, j, k) -> np.ndarray:
        j = np.ascontiguousarray(j, dtype=np.int32)
        k = np.ascontiguousarray(k, dtype=np.int32)
        if j.shape != k.shape:
            raise ValueError("j and k must have the same shape")
        a = np.zeros(len(j), dtype=np.int32)
        _check(load().xyz_agree(self.handle, _ptr(j), _ptr(k), len(j), _ptr(a)))
        return a

    def sample_agree(self, count: int, seed: int):
        j = np.zeros(count, dtype=np.int32)
        k = np.zeros(count, dtype=np.int32)
        a = np.zeros(count, dtype=np.int32)
        _check(load().xyz_sample_agree(self.handle, int(count), seed & (2**64 - 1), _ptr(j), _ptr(k),
                                       _ptr(a)))
        return j, k, a


def create(X: np.ndarray, Y: np.ndarray) -> Context:
    return Context.from_host(X, Y)


def search_many(ctxs, L, M, kappa, seed) -> list:
    """One search per context (sequences of equal length), launched as one
    CUDA graph; list of per-search results."""
    k = len(ctxs)
    handles = (ctypes.c_void_p * k)(*[c.handle.value for c in ctxs])
    La = np.ascontiguousarray(L, dtype=np.int32)
    Ma = np.ascontiguousarray(M, dtype=np.int32)
    ka = np.ascontiguousarray(kappa, dtype=np.float64)
    sa = np.ascontiguousarray([int(v) & (2**64 - 1) for v in seed], dtype=np.uint64)
    offs = np.zeros(k + 1, dtype=np.int64)
    out = ctypes.c_void_p()
    _check(load().xyz_search_many(ctypes.cast(handles, ctypes.c_void_p), k, _ptr(La), _ptr(Ma), _ptr(ka),
                                  _ptr(sa), ctypes.byref(out), _ptr(offs)))
    allp = _pairs_to_numpy(out, int(offs[-1]))
    return [allp[offs[i]:offs[i + 1]].copy() for i in range(k)]


class Server:
    """Request loop over resident datasets (xyz_server_* in include/xyz.h).

    ``submit`` returns a request id; ``wait``/``poll`` return
    ``(pairs, latency_ms)``; a cancelled request raises XyzError with code
    XYZ_ECANCELED, an unfinished one XYZ_ETIMEDOUT (wait) or XYZ_EAGAIN (poll).
    """

    def __init__(self, workers: int = 2, hbm_budget_bytes: int = 120 << 30, slice_runs: int = 2048):
        h = ctypes.c_void_p()
        _check(load().xyz_server_create(int(workers), int(hbm_budget_bytes), int(slice_runs),
                                        ctypes.byref(h)))
        self._h = h
        self._n = {}

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("server is closed")
        return self._h

    def add_dataset(self, X: np.ndarray, Y: np.ndarray) -> int:
        X = np.asfortranarray(X, dtype=np.int8)
        Y = np.ascontiguousarray(Y, dtype=np.int8)
        n, p = X.shape
        if Y.shape != (n,):
            raise ValueError("Y must have shape (n,)")
        d = ctypes.c_int32(0)
        _check(load().xyz_server_add_dataset(self.handle, _ptr(X), _ptr(Y), n, p, ctypes.byref(d)))
        self._n[d.value] = n
        return d.value

    def submit(self, dataset: int, L: int, M: int, kappa: float, seed: int, Y: np.ndarray = None) -> int:
        yp = None
        if Y is not None:
            Y = np.ascontiguousarray(Y, dtype=np.int8)
            if Y.shape != (self._n[dataset],):
                raise ValueError("Y must have shape (n,)")
            yp = _ptr(Y)
        r = ctypes.c_int64(0)
        _check(load().xyz_server_submit(self.handle, int(dataset), yp, int(L), int(M), float(kappa),
                                        seed & (2**64 - 1), ctypes.byref(r)))
        return r.value

    def wait(self, request: int, timeout_ms: int = -1):
        out = ctypes.c_void_p()
        cnt = ctypes.c_int64(0)
        lat = ctypes.c_double(0)
        _check(load().xyz_server_wait(self.handle, int(request), int(timeout_ms), ctypes.byref(out),
                                      ctypes.byref(cnt), ctypes.byref(lat)))
        return _pairs_to_numpy(out, cnt.value), lat.value

    def poll(self, request: int):
        out = ctypes.c_void_p()
        cnt = ctypes.c_int64(0)
        lat = ctypes.c_double(0)
        _check(load().xyz_server_poll(self.handle, int(request), ctypes.byref(out), ctypes.byref(cnt),
                                      ctypes.byref(lat)))
        return _pairs_to_numpy(out, cnt.value), lat.value

    def cancel(self, request: int):
        _check(load().xyz_server_cancel(self.handle, int(request)))

    def stats(self) -> dict:
        st = ServerStats()
        _check(load().xyz_server_get_stats(self.handle, ctypes.byref(st)))
        return st.as_dict()

    def close(self):
        if self._h is not None and self._h.value:
            load().xyz_server_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
