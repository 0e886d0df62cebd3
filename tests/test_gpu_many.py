"""Many independent searches launched as one CUDA graph: every result equals
the same search run alone (and the oracle's, where it is small), for
instances of uneven n and p that take the filter, general-sort (M >= 32)
and partitioned (p > 262144) paths, including searches whose spilled runs
and empty results finish outside the graph.
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


def _inst(n, p, seed, pair=(0, 1), flip=0.1):
    rng = np.random.default_rng(seed)
    X = np.asfortranarray((rng.integers(0, 2, size=(n, p), dtype=np.int8) * 2 - 1).astype(np.int8))
    Y = (X[:, pair[0]] * X[:, pair[1]]).astype(np.int8)
    f = rng.random(n) < flip
    Y[f] = -Y[f]
    return X, Y


def _arr(res):
    if len(res) == 0:
        return np.zeros((0, 3), np.int32)
    return np.stack([res["j"], res["k"], res["agree"]], axis=1).astype(np.int32)


def test_many_equals_alone(xyz, orc):
    specs = [  # (n, p, L, M, kappa, seed)
        (200, 2000, 30, 9, 0.5, 1),
        (77, 5000, 12, 7, 0.3, 2),
        (1000, 300, 40, 10, 0.2, 3),
        (150, 700, 10, 33, 0.1, 4),          # general sort path
        (64, 300000, 2, 10, 0.6, 5),         # partitioned grouping
        (120, 9000, 6, 4, 0.95, 6),          # c = 0 runs spill to the sort path
        (90, 400, 5, 8, 1.0, 7),             # nothing passes
    ]
    data = [_inst(n, p, 10 + i, pair=(1, p - 1)) for i, (n, p, *_rest) in enumerate(specs)]
    ctxs = [xyz.create(X, Y) for X, Y in data]
    try:
        got = xyz.search_many(ctxs, [s[2] for s in specs], [s[3] for s in specs], [s[4] for s in specs],
                              [s[5] for s in specs])
        again = xyz.search_many(ctxs, [s[2] for s in specs], [s[3] for s in specs], [s[4] for s in specs],
                                [s[5] for s in specs])
        for i, ((n, p, L, M, kappa, seed), (X, Y)) in enumerate(zip(specs, data)):
            with xyz.create(X, Y) as alone:
                want = alone.search(L, M, kappa, seed)
            assert np.array_equal(got[i], want), i
            assert np.array_equal(again[i], want), i
            if n * p <= 1_000_000 and M <= 33:
                assert np.array_equal(_arr(got[i]), orc.xyz(X, Y, L, M, kappa, seed)), i
        assert sum(len(g) for g in got) > 0 and len(got[-1]) == 0
    finally:
        for c in ctxs:
            c.close()


def test_many_rejects_shared_context(xyz):
    X, Y = _inst(64, 100, 1)
    with xyz.create(X, Y) as c:
        with pytest.raises(xyz.XyzError) as e:
            xyz.search_many([c, c], [2, 2], [5, 5], [0.3, 0.3], [1, 2])
        assert e.value.code == xyz.XYZ_EINVAL
