"""Plain CPU oracle for the binary xyz search (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library never does.

The arithmetic lives in ``xyz_oracle.c`` (plain C, int8 loops, qsort); this
module only compiles it with gcc and marshals numpy arrays through ctypes.
Conventions: X is an (n, p) int8 array of +-1 values stored column-major
(``X[:, j]`` contiguous, i.e. ``np.asfortranarray``), Y an (n,) int8 array.

Each function cites the part of the paper it follows; the readings taken
where the paper is silent are listed at the top of ``xyz_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xyz_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle_xyz.so")
_lib = None

_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_u64 = ctypes.c_uint64
_dbl = ctypes.c_double
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle into a shared object next to its source."""
    if force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    ):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.run(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"],
            check=True,
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    sig = {
        "orc_splitmix64_at": (_u64, [_u64, _u64]),
        "orc_draw_rows": (None, [_u64, _i64, _i32, _i64, _p]),
        "orc_agree": (_i64, [_p, _p, _i64, _i64, _i64]),
        "orc_agree_pairs": (None, [_p, _p, _i64, _p, _p, _i64, _p]),
        "orc_amin": (_i64, [_i64, _dbl]),
        "orc_check_pm1": (ctypes.c_int, [_p, _i64]),
        "orc_brute_force": (_i64, [_p, _p, _i64, _i64, _dbl, _p, _i64]),
        "orc_keys": (None, [_p, _p, _i64, _i64, _p, _i32, _p, _p]),
        "orc_project_real": (None, [_p, _p, _i64, _i64, _p, _i32, _p, _p, _p]),
        "orc_equal_pairs": (_i64, [_p, _p, _i64, _p, _i64]),
        "orc_equal_pairs_real": (_i64, [_p, _p, _i64, _p, _i64]),
        "orc_candidates": (_i64, [_p, _p, _i64, _i64, _i32, _u64, _i64, _p, _i64]),
        "orc_xyz_range": (_i64, [_p, _p, _i64, _i64, _i64, _i64, _i32, _dbl, _u64, _p, _i64]),
        "orc_xyz": (_i64, [_p, _p, _i64, _i64, _i32, _i32, _dbl, _u64, _p, _i64]),
        "orc_quantize_y": (ctypes.c_int, [_p, _i64, _p, _p]),
        "orc_draw_rows_weighted": (None, [_p, _i64, _u64, _i64, _i32, _p]),
        "orc_weighted_agree": (_i64, [_p, _p, _p, _i64, _i64, _i64, _p]),
        "orc_xyz_weighted_range": (_i64, [_p, _p, _i64, _i64, _i64, _i64, _i32, _dbl, _u64, _p, _p,
                                          _i64]),
        "orc_brute_force_weighted": (_i64, [_p, _p, _i64, _i64, _dbl, _p, _p, _i64]),
        "orc_kkt_threshold": (_i64, [_p, _i64, _dbl]),
        "orc_kkt_brute": (_i64, [_p, _p, _i64, _i64, _dbl, _p, _p, _i64]),
        "orc_kkt_xyz": (_i64, [_p, _p, _i64, _i64, _i64, _i32, _dbl, _u64, _p, _p, _i64]),
        "orc_sign_transform": (ctypes.c_int, [_p, _i64, _i64, _u64, _p]),
        "orc_unbiased_scale": (None, [_p, _p, _i64, _i64, _p, _p]),
        "orc_unbiased_draw": (ctypes.c_int, [_p, _i64, _i64, _u64, _i64, _i32, _i32, _i64, _i64]),
        "orc_real_dot": (_dbl, [_p, _p, _i64, _i64, _i64]),
        "orc_xyz_unbiased_range": (_i64, [_p, _p, _i64, _i64, _i64, _i64, _i32, _dbl, _u64, _p, _p,
                                          _i64]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check_xy(X: np.ndarray, Y: np.ndarray):
    X = np.asfortranarray(X, dtype=np.int8)
    Y = np.ascontiguousarray(Y, dtype=np.int8)
    n, p = X.shape
    if Y.shape != (n,):
        raise ValueError("Y must have shape (n,)")
    lib = _load()
    if not lib.orc_check_pm1(_ptr(X), X.size) or not lib.orc_check_pm1(_ptr(Y), Y.size):
        raise ValueError("entries of X and Y must be -1 or +1")
    return X, Y, n, p


def splitmix64_at(seed: int, t: int) -> int:
    """Output number t of splitmix64 started at state ``seed`` (reading R2)."""
    return int(_load().orc_splitmix64_at(seed & (2**64 - 1), t))


def draw_rows(seed: int, run: int, M: int, n: int) -> np.ndarray:
    """Row indices i_1..i_M of one run, with replacement (eq. projR, R1)."""
    rows = np.zeros(max(M, 1), dtype=np.int64)
    _load().orc_draw_rows(seed & (2**64 - 1), run, M, n, _ptr(rows))
    return rows[:M]


def agree(X, Y, j: int, k: int) -> int:
    """a_jk = sum_i 1{Y_i = X_ij X_ik} (eq. def_gamma)."""
    X, Y, n, p = _check_xy(X, Y)
    return int(_load().orc_agree(_ptr(X), _ptr(Y), n, j, k))


def agree_pairs(X, Y, j, k) -> np.ndarray:
    """a_jk for each given pair (eq. def_gamma), one by one."""
    X, Y, n, p = _check_xy(X, Y)
    j = np.ascontiguousarray(j, dtype=np.int32)
    k = np.ascontiguousarray(k, dtype=np.int32)
    if j.shape != k.shape or (len(j) and (min(j.min(), k.min()) < 0 or max(j.max(), k.max()) >= p)):
        raise ValueError("bad pair indices")
    out = np.zeros(len(j), dtype=np.int32)
    _load().orc_agree_pairs(_ptr(X), _ptr(Y), n, _ptr(j), _ptr(k), len(j), _ptr(out))
    return out


def amin(n: int, kappa: float) -> int:
    """Least agreement count that passes (2a - n) >= kappa n (reading R5)."""
    return int(_load().orc_amin(n, float(kappa)))


def brute_force(X, Y, kappa: float) -> np.ndarray:
    """All pairs j < k with a_jk >= a_min, naive O(np^2) (eq. inter_search1).

    Returns an int32 array of shape (count, 3): columns j, k, a.
    """
    X, Y, n, p = _check_xy(X, Y)
    lib = _load()
    cnt = lib.orc_brute_force(_ptr(X), _ptr(Y), n, p, float(kappa), None, 0)
    out = np.zeros((max(cnt, 1), 3), dtype=np.int32)
    lib.orc_brute_force(_ptr(X), _ptr(Y), n, p, float(kappa), _ptr(out), cnt)
    return out[:cnt]


def keys(X, Y, rows: np.ndarray):
    """Integer keys (x, z) of the M sampled rows (the projection step of Algorithm 2, R3)."""
    X, Y, n, p = _check_xy(X, Y)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    x = np.zeros(p, dtype=np.uint64)
    z = np.zeros(p, dtype=np.uint64)
    _load().orc_keys(_ptr(X), _ptr(Y), n, p, _ptr(rows), len(rows), _ptr(x), _ptr(z))
    return x, z


def project_real(X, Y, rows: np.ndarray, D: np.ndarray):
    """The paper's projection x = X^T R, z = Z^T R with R from eq. projR."""
    X, Y, n, p = _check_xy(X, Y)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    D = np.ascontiguousarray(D, dtype=np.float64)
    x = np.zeros(p, dtype=np.float64)
    z = np.zeros(p, dtype=np.float64)
    _load().orc_project_real(_ptr(X), _ptr(Y), n, p, _ptr(rows), len(rows), _ptr(D), _ptr(x), _ptr(z))
    return x, z


def equal_pairs(x: np.ndarray, z: np.ndarray) -> np.ndarray:
    """Ordered pairs (j, k) with x_j = z_k, by the sort-and-walk of Figure 2."""
    lib = _load()
    if x.dtype == np.float64:
        fn = lib.orc_equal_pairs_real
        x = np.ascontiguousarray(x, dtype=np.float64)
        z = np.ascontiguousarray(z, dtype=np.float64)
    else:
        fn = lib.orc_equal_pairs
        x = np.ascontiguousarray(x, dtype=np.uint64)
        z = np.ascontiguousarray(z, dtype=np.uint64)
    p = len(x)
    cnt = fn(_ptr(x), _ptr(z), p, None, 0)
    out = np.zeros((max(cnt, 1), 2), dtype=np.int32)
    fn(_ptr(x), _ptr(z), p, _ptr(out), cnt)
    return out[:cnt]


def candidates(X, Y, M: int, seed: int, run: int) -> np.ndarray:
    """E_l of one run as sorted unordered pairs j < k (R4); shape (count, 2)."""
    X, Y, n, p = _check_xy(X, Y)
    lib = _load()
    args = (_ptr(X), _ptr(Y), n, p, M, seed & (2**64 - 1), run)
    cnt = lib.orc_candidates(*args, None, 0)
    out = np.zeros((max(cnt, 1), 2), dtype=np.int32)
    lib.orc_candidates(*args, _ptr(out), cnt)
    return out[:cnt]


def xyz_range(X, Y, l0: int, l1: int, M: int, kappa: float, seed: int) -> np.ndarray:
    """Algorithm 2 over runs [l0, l1): sorted (j, k, a) triples (R5, R6)."""
    X, Y, n, p = _check_xy(X, Y)
    lib = _load()
    args = (_ptr(X), _ptr(Y), n, p, l0, l1, M, float(kappa), seed & (2**64 - 1))
    cap = 4096
    while True:
        out = np.zeros((cap, 3), dtype=np.int32)
        cnt = lib.orc_xyz_range(*args, _ptr(out), cap)
        if cnt <= cap:
            return out[:cnt]
        cap = cnt


def xyz(X, Y, L: int, M: int, kappa: float, seed: int) -> np.ndarray:
    """Algorithm 2 (final xyz): union over L runs of verified candidates."""
    return xyz_range(X, Y, 0, L, M, kappa, seed)


# ------------------------------------------------------ continuous response
# Section 3.1 with readings R9-R11 of xyz_oracle.c.


def _check_x_real(X: np.ndarray, Y: np.ndarray):
    X = np.asfortranarray(X, dtype=np.int8)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    n, p = X.shape
    if Y.shape != (n,):
        raise ValueError("Y must have shape (n,)")
    if not _load().orc_check_pm1(_ptr(X), X.size):
        raise ValueError("entries of X must be -1 or +1")
    return X, Y, n, p


def quantize_y(Y) -> tuple:
    """Fixed-point weights q and signs of a real response (R9)."""
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    q = np.zeros(len(Y), dtype=np.int64)
    sgn = np.zeros(len(Y), dtype=np.int8)
    if _load().orc_quantize_y(_ptr(Y), len(Y), _ptr(q), _ptr(sgn)) != 0:
        raise ValueError("Y must be finite and not all zero")
    return q, sgn


def draw_rows_weighted(q, seed: int, run: int, M: int) -> np.ndarray:
    """Rows of one run drawn with probability q_i / sum q (R10)."""
    q = np.ascontiguousarray(q, dtype=np.int64)
    rows = np.zeros(max(M, 1), dtype=np.int64)
    _load().orc_draw_rows_weighted(_ptr(q), len(q), seed & (2**64 - 1), run, M, _ptr(rows))
    return rows[:M]


def weighted_agree(X, Y, j: int, k: int) -> tuple:
    """(count of sign-agreeing rows, their weight sum S_jk) under R9."""
    X, Y, n, p = _check_x_real(X, Y)
    q, sgn = quantize_y(Y)
    S = ctypes.c_int64(0)
    a = _load().orc_weighted_agree(_ptr(X), _ptr(sgn), _ptr(q), n, j, k, ctypes.byref(S))
    return int(a), int(S.value)


def _weighted_call(fn, X, Y, *args):
    X, Y, n, p = _check_x_real(X, Y)
    cap = 4096
    while True:
        out = np.zeros((cap, 3), dtype=np.int32)
        ws = np.zeros(cap, dtype=np.int64)
        cnt = fn(_ptr(X), _ptr(Y), n, p, *args, _ptr(out), _ptr(ws), cap)
        if cnt < 0:
            raise ValueError("Y must be finite and not all zero")
        if cnt <= cap:
            return out[:cnt], ws[:cnt]
        cap = cnt


def xyz_weighted_range(X, Y, l0: int, l1: int, M: int, kappa: float, seed: int) -> tuple:
    """Algorithm 2 with the continuous-Y modifications of Section 3.1 over
    runs [l0, l1): sorted (j, k, a) triples and their weight sums S."""
    return _weighted_call(_load().orc_xyz_weighted_range, X, Y, l0, l1, M, float(kappa),
                          seed & (2**64 - 1))


def xyz_weighted(X, Y, L: int, M: int, kappa: float, seed: int) -> tuple:
    return xyz_weighted_range(X, Y, 0, L, M, kappa, seed)


def brute_force_weighted(X, Y, kappa: float) -> tuple:
    """Every pair passing R11 by the naive loop over all pairs."""
    return _weighted_call(_load().orc_brute_force_weighted, X, Y, float(kappa))


# ------------------------------------------------- absolute value, KKT check
# Section 4 with reading R12 of xyz_oracle.c.


def xyz_abs(X, Y, L: int, M: int, kappa: float, seed: int) -> np.ndarray:
    """Pairs with |Y^T(X_j o X_k)| / n >= kappa: the binary search with Y and
    with -Y, united (Section 4 runs xyz on +-Y); (j, k, a) with a for +Y."""
    X, Y, n, p = _check_xy(X, Y)
    plus = xyz(X, Y, L, M, kappa, seed)
    minus = xyz(X, (-Y).astype(np.int8), L, M, kappa, seed)
    minus = minus.copy()
    minus[:, 2] = n - minus[:, 2]
    allp = {(int(j), int(k)): int(a) for j, k, a in minus}
    allp.update({(int(j), int(k)): int(a) for j, k, a in plus})
    return np.array([(j, k, allp[(j, k)]) for j, k in sorted(allp)], dtype=np.int32).reshape(-1, 3)


def kkt_threshold(r, lam: float) -> int:
    r = np.ascontiguousarray(r, dtype=np.float64)
    return int(_load().orc_kkt_threshold(_ptr(r), len(r), float(lam)))


def kkt_brute(X, r, lam: float) -> tuple:
    """KKT violators |r^T(X_j o X_k)| / n > lambda by the loop over all pairs
    (R12): (j, k, a) triples and the signed integers 2S - Q."""
    return _weighted_call(_load().orc_kkt_brute, X, r, float(lam))


def kkt_xyz(X, r, L: int, M: int, lam: float, seed: int) -> tuple:
    """The same check by the continuous-response search with +r and -r."""
    return _weighted_call(_load().orc_kkt_xyz, X, r, int(L), int(M), float(lam), seed & (2**64 - 1))


def sign_transform(X, coin_seed: int = 0) -> np.ndarray:
    """Section 3.2's sign transform of a real X (R14): column-major int8 +-1."""
    X = np.asfortranarray(X, dtype=np.float32)
    n, p = X.shape
    out = np.zeros((n, p), dtype=np.int8, order="F")
    if _load().orc_sign_transform(_ptr(X), n, p, coin_seed & (2**64 - 1), _ptr(out)) != 0:
        raise ValueError("entries of X must not be NaN")
    return out


def unbiased_scale(X, Y) -> tuple:
    """Row scaling of R15: X' = X / nu_i (float), Y' = Y nu_i^2."""
    X = np.asfortranarray(X, dtype=np.float32)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    n, p = X.shape
    Xs = np.zeros((n, p), dtype=np.float32, order="F")
    Ys = np.zeros(n, dtype=np.float64)
    _load().orc_unbiased_scale(_ptr(X), _ptr(Y), n, p, _ptr(Xs), _ptr(Ys))
    return Xs, Ys


def unbiased_draw(Xs, seed: int, run: int, M: int, m: int, i: int, j: int) -> int:
    Xs = np.asfortranarray(Xs, dtype=np.float32)
    n, p = Xs.shape
    return int(_load().orc_unbiased_draw(_ptr(Xs), n, p, seed & (2**64 - 1), run, M, m, i, j))


def xyz_unbiased_range(X, Y, l0: int, l1: int, M: int, kappa: float, seed: int) -> tuple:
    """The unbiased-transform search (R15) over runs [l0, l1): sorted pairs
    (count, 2) and their dot products sum_i Y'_i X'_ij X'_ik."""
    X = np.asfortranarray(X, dtype=np.float32)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    n, p = X.shape
    cap = 4096
    while True:
        out = np.zeros((cap, 2), dtype=np.int32)
        dots = np.zeros(cap, dtype=np.float64)
        cnt = _load().orc_xyz_unbiased_range(_ptr(X), _ptr(Y), n, p, l0, l1, M, float(kappa),
                                             seed & (2**64 - 1), _ptr(out), _ptr(dots), cap)
        if cnt < 0:
            raise ValueError("the scaled response must be finite and not all zero")
        if cnt <= cap:
            return out[:cnt], dots[:cnt]
        cap = cnt
