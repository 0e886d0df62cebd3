"""Packing of X and Y (the form-Z step of Algorithm 2, "form Z"): one tiled kernel reads
every entry of X once -- from device memory, from a device copy of a
pageable host array, or in place from pinned host memory -- and writes the
bit columns and bit rows.  The bit rows are checked through the keys of
sampled rows against the oracle, the bit columns through the agreement of
every column with another, for shapes that take the 16-byte and the byte
load paths, ragged column words, several row chunks and the padding.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# (n, p): n % 16 == 0 takes 16-byte loads (for an aligned X), the others byte
# loads; n above 1024 spans row chunks; p % 32 != 0 leaves a ragged word
SHAPES = [(1, 2), (31, 33), (32, 64), (48, 100), (1000, 777), (1024, 32), (1040, 95),
          (2000, 4100), (2047, 129), (3000, 65)]


@pytest.fixture(scope="module")
def xyz():
    from paper_1610_05108_gb300 import build, xyz as mod
    build.build()
    mod.load()
    return mod


def _data(n, p, seed):
    rng = np.random.default_rng(seed)
    X = np.asfortranarray(rng.choice(np.array([-1, 1], np.int8), size=(n, p)))
    Y = rng.choice(np.array([-1, 1], np.int8), size=n)
    return X, Y


def _check_packed(ctx, X, Y, orc, seed):
    n, p = X.shape
    M = 64
    for run in range(6):                       # bit rows: keys of sampled rows
        kx, _ = ctx.run_keys(M, seed, run)
        ox, _ = orc.keys(X, Y, orc.draw_rows(seed, run, M, n))
        assert np.array_equal(kx, ox), (n, p, run)
    rng = np.random.default_rng(seed + 1)      # bit columns and response bits
    j = np.arange(p, dtype=np.int32)
    k = rng.integers(0, p, size=p).astype(np.int32)
    assert np.array_equal(ctx.agree(j, k), orc.agree_pairs(X, Y, j, k)), (n, p)


@pytest.mark.parametrize("n,p", SHAPES)
def test_pack_from_pageable_host(xyz, orc, n, p):
    X, Y = _data(n, p, n * 7 + p)
    with xyz.Context.from_host(X, Y) as ctx:
        _check_packed(ctx, X, Y, orc, 3)


@pytest.mark.parametrize("n,p", SHAPES)
def test_pack_from_pinned_host_in_place(xyz, orc, n, p):
    torch = pytest.importorskip("torch")
    X, Y = _data(n, p, n * 11 + p)
    Xh = torch.from_numpy(np.ascontiguousarray(X.T)).pin_memory()
    Yh = torch.from_numpy(Y).pin_memory()
    with xyz.Context.from_host(Xh.numpy().T, Yh.numpy()) as ctx:
        _check_packed(ctx, X, Y, orc, 4)


def test_pack_from_pinned_host_unaligned(xyz, orc):
    # X starting one byte into a pinned buffer: the byte load path reads it
    torch = pytest.importorskip("torch")
    n, p = 2000, 300
    X, Y = _data(n, p, 5)
    buf = torch.empty(n * p + 16, dtype=torch.int8).pin_memory()
    view = buf.numpy()[1:1 + n * p]
    view[:] = X.ravel(order="F")
    Xv = view.reshape((p, n)).T
    assert Xv.ctypes.data % 16 == 1
    Yh = torch.from_numpy(Y).pin_memory()
    with xyz.Context.from_host(Xv, Yh.numpy()) as ctx:
        _check_packed(ctx, X, Y, orc, 6)


@pytest.mark.parametrize("n,p", [(48, 100), (2000, 4100), (2047, 129)])
def test_pack_from_device(xyz, orc, n, p):
    torch = pytest.importorskip("torch")
    X, Y = _data(n, p, n * 13 + p)
    dX = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()    # column-major X
    dY = torch.from_numpy(Y).cuda()
    with xyz.Context.from_device(dX.data_ptr(), dY.data_ptr(), n, p) as ctx:
        _check_packed(ctx, X, Y, orc, 7)


def test_pack_rejects_bad_entries_in_place(xyz):
    torch = pytest.importorskip("torch")
    X, Y = _data(1040, 70, 8)
    X[1033, 65] = 0                            # last row chunk, ragged column word
    Xh = torch.from_numpy(np.ascontiguousarray(X.T)).pin_memory()
    Yh = torch.from_numpy(Y).pin_memory()
    with pytest.raises(xyz.XyzError) as e:
        xyz.Context.from_host(Xh.numpy().T, Yh.numpy())
    assert e.value.code == xyz.XYZ_EINVAL
    X[1033, 65] = 1
    Y[3] = 2
    Yh = torch.from_numpy(Y).pin_memory()
    Xh = torch.from_numpy(np.ascontiguousarray(X.T)).pin_memory()
    with pytest.raises(xyz.XyzError) as e:
        xyz.Context.from_host(Xh.numpy().T, Yh.numpy())
    assert e.value.code == xyz.XYZ_EINVAL
