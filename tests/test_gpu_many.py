"""Many independent searches launched as one CUDA graph: every result equals
the same search run alone (and the oracle's, where it is small), for
instances of uneven n and p that take the filter, general-sort (M >= 32)
and partitioned (p > 262144) paths, including searches whose spilled runs
and empty results finish outside the graph, and searches whose filters
share fused persistent launches.
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


def test_fused_filter_launch_equals_alone(xyz, orc):
    # 70 searches of the key class M <= 16 (two fused launches: 64 + 6), some
    # of M in 17..24 and 25..31, one weighted response, one real X through
    # the unbiased transform and one class-split search (p > 262144), which
    # keep launches of their own; fused, unfused and alone all agree
    rng = np.random.default_rng(77)
    specs = []
    for i in range(70):
        n = int(rng.integers(40, 400))
        p = int(rng.integers(300, 6000))
        specs.append((n, p, int(rng.integers(2, 40)), int(rng.integers(4, 17)), float(rng.uniform(0.2, 0.7))))
    for i in range(6):
        specs.append((int(rng.integers(100, 600)), int(rng.integers(2000, 40000)), int(rng.integers(2, 12)),
                      int(rng.integers(17, 32)), float(rng.uniform(0.1, 0.5))))
    ctxs, data = [], []
    try:
        for i, (n, p, L, M, kappa) in enumerate(specs):
            X, Y = _inst(n, p, 500 + i, pair=(0, p - 1))
            data.append((X, Y))
            ctxs.append(xyz.create(X, Y))
        # weighted response on one binary X
        Xw, Yw = _inst(300, 3000, 999, pair=(2, 5))
        yw = Yw.astype(np.float64) * np.random.default_rng(3).uniform(0.5, 2.0, size=300)
        cw = xyz.create(Xw, Yw)
        cw.set_y_real(yw)
        ctxs.append(cw)
        specs.append((300, 3000, 20, 10, 0.3))
        # real X (unbiased transform) and a class-split search: not fused
        Xr = np.asfortranarray(np.random.default_rng(4).standard_normal((100, 800)))
        Yr = Xr[:, 3] * Xr[:, 7] + 0.1 * np.random.default_rng(5).standard_normal(100)
        ctxs.append(xyz.Context.from_real_unbiased(Xr, Yr))
        specs.append((100, 800, 10, 8, 0.3))
        Xb, Yb = _inst(64, 300000, 998, pair=(1, 2))
        ctxs.append(xyz.create(Xb, Yb))
        specs.append((64, 300000, 2, 12, 0.6))
        Ls, Ms, ks = [s[2] for s in specs], [s[3] for s in specs], [s[4] for s in specs]
        seeds = [1000 + i for i in range(len(specs))]
        fused = xyz.search_many(ctxs, Ls, Ms, ks, seeds)
        for c in ctxs:
            c.set_fused_filter(False)
        plain = xyz.search_many(ctxs, Ls, Ms, ks, seeds)
        for c in ctxs:
            c.set_fused_filter(True)
        for i, c in enumerate(ctxs):
            want = c.search(Ls[i], Ms[i], ks[i], seeds[i])
            assert np.array_equal(fused[i], want), i
            assert np.array_equal(plain[i], want), i
        for i in range(0, 70, 9):                       # oracle on a sample of the binary searches
            X, Y = data[i]
            assert np.array_equal(_arr(fused[i]), orc.xyz(X, Y, Ls[i], Ms[i], ks[i], seeds[i])), i
        assert sum(len(f) for f in fused) > 0
    finally:
        for c in ctxs:
            c.close()


def test_fused_filter_setting_checked(xyz):
    X, Y = _inst(64, 100, 1)
    with xyz.create(X, Y) as c:
        with pytest.raises(xyz.XyzError) as e:
            xyz._check(xyz.load().xyz_set_fused_filter(c.handle, 2))
        assert e.value.code == xyz.XYZ_EINVAL


def test_fused_search_that_overflows_is_redone(xyz, orc):
    # M = 13 over 30000 random columns: nearly every column survives and the
    # first attempt's groups overflow the member space reserved for them; in
    # a fused filter launch that search must be redone on its own after the
    # graph, and every result must still equal the search alone
    rng = np.random.default_rng(29)
    Xo = np.asfortranarray((rng.integers(0, 2, size=(64, 30000), dtype=np.int8) * 2 - 1).astype(np.int8))
    Yo = (rng.integers(0, 2, size=64, dtype=np.int8) * 2 - 1).astype(np.int8)
    specs = [(12, 13, 0.5, 3)] + [(20, 9, 0.3, 10 + i) for i in range(3)]
    data = [(Xo, Yo)] + [_inst(150, 3000, 60 + i, pair=(0, 2999)) for i in range(3)]
    ctxs = [xyz.create(X, Y) for X, Y in data]
    try:
        got = xyz.search_many(ctxs, [s[0] for s in specs], [s[1] for s in specs], [s[2] for s in specs],
                              [s[3] for s in specs])
        for i, ((L, M, kappa, seed), (X, Y)) in enumerate(zip(specs, data)):
            with xyz.create(X, Y) as alone:
                assert np.array_equal(got[i], alone.search(L, M, kappa, seed)), i
        assert np.array_equal(_arr(got[0]), orc.xyz(Xo, Yo, 12, 13, 0.5, 3))
    finally:
        for c in ctxs:
            c.close()
