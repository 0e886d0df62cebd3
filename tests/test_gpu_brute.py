"""Exhaustive screen (the comparator of the search): every pair j < k with
(2a - n) >= kappa*n, compared with the oracle's brute force element by
element, on ragged tiles (p not a multiple of 128), ragged words (n not a
multiple of 32), thresholds from 'all pairs' to 'none', and against the
M = 0 search, which is the same set by Algorithm 2's definition.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xyz():
    from paper_1610_05108_gb300 import build, xyz as mod
    build.build()
    mod.load()
    return mod


def _rand(n, p, seed):
    rng = np.random.default_rng(seed)
    X = np.asfortranarray((rng.integers(0, 2, size=(n, p), dtype=np.int8) * 2 - 1).astype(np.int8))
    Y = (rng.integers(0, 2, size=n, dtype=np.int8) * 2 - 1).astype(np.int8)
    return X, Y


def _arr(res):
    if len(res) == 0:
        return np.zeros((0, 3), np.int32)
    return np.stack([res["j"], res["k"], res["agree"]], axis=1).astype(np.int32)


@pytest.mark.parametrize("n,p,kappas", [
    (1, 2, (-1.0, 1.0)),
    (33, 129, (-1.0, 0.0, 0.3)),
    (200, 300, (0.1, 0.2, 1.0)),
    (95, 1000, (0.25, 0.4)),
    (1000, 517, (0.1, 0.12)),
])
def test_brute_force_equals_oracle(xyz, orc, n, p, kappas):
    X, Y = _rand(n, p, n * 7 + p)
    Y[: n // 3] = (X[: n // 3, 0] * X[: n // 3, p - 1]).astype(np.int8)   # one stronger pair
    with xyz.create(X, Y) as ctx:
        for kappa in kappas:
            got = ctx.brute_force(kappa)
            want = orc.brute_force(X, Y, kappa)
            assert np.array_equal(_arr(got), want), (n, p, kappa)
            st = ctx.stats()
            assert st["candidates"] == p * (p - 1) // 2
            assert st["unique_pairs"] == len(want)
            if len(got):
                assert np.allclose(got["strength"], (2.0 * got["agree"] - n) / n)


def test_brute_force_equals_M0_search(xyz):
    X, Y = _rand(150, 700, 5)
    Y = (X[:, 3] * X[:, 600]).astype(np.int8)
    Y[:20] = -Y[:20]
    with xyz.create(X, Y) as ctx:
        for kappa in (0.15, 0.5):
            assert np.array_equal(ctx.brute_force(kappa), ctx.search(1, 0, kappa, 9))


def test_brute_force_planted_pair_large_p(xyz):
    # p spans 40 tiles; only the planted pair reaches kappa
    X, Y = _rand(512, 5000, 11)
    Y = (X[:, 17] * X[:, 4321]).astype(np.int8)
    Y[:40] = -Y[:40]
    with xyz.create(X, Y) as ctx:
        got = ctx.brute_force(0.6)
    assert list(zip(got["j"], got["k"])) == [(17, 4321)]
    assert got["agree"][0] == 512 - 40


def test_brute_force_bad_kappa(xyz):
    X, Y = _rand(10, 5, 1)
    with xyz.create(X, Y) as ctx:
        with pytest.raises(xyz.XyzError) as e:
            ctx.brute_force(1.5)
        assert e.value.code == xyz.XYZ_EINVAL
