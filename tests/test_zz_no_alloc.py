"""The allocation-free entry point xyz_run_candidates_noalloc.

Some callers cannot allocate device memory when they want a result (their
HBM is owned by another allocator, or a cudaMalloc's device-wide
synchronisation is not acceptable in their loop).  For them the library
offers one entry point whose scratch is a fixed array inside the library.
These tests call it through the C ABI twice in a row and check each result
against the allocating entry point xyz_run_candidates and against the
oracle's E_l (integer results, so equality is exact): on a binary response,
and on a real-valued response after a thresholded search has run on the
context (the entry point must still return every candidate).  Contexts of
real X are refused, and so are sizes over its limits.  The file is named so
that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _rand(n, p, seed):
    rng = np.random.default_rng(seed)
    X = np.asfortranarray((rng.integers(0, 2, size=(n, p), dtype=np.int8) * 2 - 1).astype(np.int8))
    Y = (rng.integers(0, 2, size=n, dtype=np.int8) * 2 - 1).astype(np.int8)
    return X, Y


def _noalloc(lib, ctx, M, seed, run, cap):
    buf = np.zeros((cap, 2), dtype=np.int32)
    cnt = ctypes.c_int64(-1)
    rc = lib.xyz_run_candidates_noalloc(ctx.handle, M, seed, run,
                                        buf.ctypes.data_as(ctypes.c_void_p), cap, ctypes.byref(cnt))
    return rc, buf[: max(cnt.value, 0)].copy()


def test_noalloc_candidates_match_allocating_entry_point(orc):
    from paper_1610_05108_gb300 import build, xyz
    build.build()
    lib = xyz.load()
    X, Y = _rand(301, 3000, 21)          # ragged n and p
    M, seed, cap = 10, 0xC0FFEE, 32768
    with xyz.create(X, Y) as ctx:
        rc0, got0 = _noalloc(lib, ctx, M, seed, 0, cap)     # two calls in a row
        rc1, got1 = _noalloc(lib, ctx, M, seed, 1, cap)
        assert rc0 == xyz.XYZ_OK and rc1 == xyz.XYZ_OK, lib.xyz_last_error()
        want0 = ctx.run_candidates(M, seed, 0)
        want1 = ctx.run_candidates(M, seed, 1)
    assert len(want0) > 100 and len(want1) > 100
    assert np.array_equal(got0, want0)
    assert np.array_equal(got1, want1)
    assert np.array_equal(got0, orc.candidates(X, Y, M, seed, 0))
    assert np.array_equal(got1, orc.candidates(X, Y, M, seed, 1))


def test_noalloc_weighted_response_after_a_thresholded_search(orc):
    """A real-valued response, and a search with kappa = 0.5 run on the
    context first: the entry point still returns the whole E_l."""
    from paper_1610_05108_gb300 import xyz
    lib = xyz.load()
    X, _ = _rand(257, 2500, 24)
    rng = np.random.default_rng(25)
    Yr = rng.normal(size=257) + 0.3 * X[:, 3] * X[:, 7]
    M, seed, cap = 9, 4242, 32768
    with xyz.create(X, np.ones(257, np.int8)) as ctx:
        ctx.set_y_real(Yr)
        ctx.search(30, M, 0.5, 99)                          # leaves a threshold behind
        rc0, got0 = _noalloc(lib, ctx, M, seed, 2, cap)
        rc1, got1 = _noalloc(lib, ctx, M, seed, 3, cap)
        assert rc0 == xyz.XYZ_OK and rc1 == xyz.XYZ_OK, lib.xyz_last_error()
        want0 = ctx.run_candidates(M, seed, 2)
        want1 = ctx.run_candidates(M, seed, 3)
    o0, _ = orc.xyz_weighted_range(X, Yr, 2, 3, M, -1.0, seed)
    o1, _ = orc.xyz_weighted_range(X, Yr, 3, 4, M, -1.0, seed)
    assert len(want0) > 100 and len(want1) > 100
    assert np.array_equal(got0, want0) and np.array_equal(got0, o0[:, :2])
    assert np.array_equal(got1, want1) and np.array_equal(got1, o1[:, :2])


def test_noalloc_refuses_real_x():
    from paper_1610_05108_gb300 import xyz
    lib = xyz.load()
    rng = np.random.default_rng(26)
    Xf = rng.uniform(-1, 1, size=(64, 500)).astype(np.float32, order="F")
    Yf = rng.normal(size=64)
    with xyz.Context.from_real_unbiased(Xf, Yf) as ctx:
        rc, _ = _noalloc(lib, ctx, 6, 1, 0, 1024)
        assert rc == xyz.XYZ_EINVAL
        assert b"real X" in lib.xyz_last_error()


def test_noalloc_refuses_sizes_over_its_limits():
    from paper_1610_05108_gb300 import xyz
    lib = xyz.load()
    X, Y = _rand(40, 16385, 22)          # one column over XYZ_NOALLOC_MAX_P
    with xyz.create(X, Y) as ctx:
        rc, _ = _noalloc(lib, ctx, 5, 1, 0, 16)
        assert rc == xyz.XYZ_EINVAL
        assert b"XYZ_NOALLOC_MAX_P" in lib.xyz_last_error()
    X, Y = _rand(40, 3000, 23)
    with xyz.create(X, Y) as ctx:
        rc, _ = _noalloc(lib, ctx, 0, 1, 0, 16)              # M = 0: every pair is a candidate
        assert rc == xyz.XYZ_ENOMEM
        rc, got = _noalloc(lib, ctx, 9, 1, 0, 32768)        # still usable afterwards
        assert rc == xyz.XYZ_OK
        assert np.array_equal(got, ctx.run_candidates(9, 1, 0))
