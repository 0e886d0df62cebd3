"""Launch shapes (xyz_set_tiles, xyz_autotune_tiles): the results of a search
are the same whatever the filter CTA size, the launch-group size and the
verification's blocks per SM -- on the single survivor filter (p <= 262144)
and on the class-split filter (forced at small p) -- and equal the oracle's;
the tuner returns shapes in range and leaves them set; bad shapes are
refused."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def xyz():
    from paper_1610_05108_gb300 import build, xyz as mod
    build.build()
    mod.load()
    return mod


def _planted(n, p, seed):
    rng = np.random.default_rng(seed)
    X = np.asfortranarray((rng.integers(0, 2, size=(n, p), dtype=np.int8) * 2 - 1).astype(np.int8))
    Y = (X[:, 7] * X[:, p - 3]).astype(np.int8)
    Y[rng.random(n) < 0.1] *= -1
    return X, Y


def _arr(res):
    return np.stack([res["j"], res["k"], res["agree"]], axis=1).astype(np.int32)


SHAPES = [(0, 0, 0), (512, 1, 0), (640, 2, 7), (1024, 0, 25), (768, 3, 1)]


@pytest.mark.parametrize("mode", [1, 2])
def test_results_do_not_depend_on_launch_shapes(xyz, orc, mode):
    X, Y = _planted(180, 6000, 5 + mode)
    L, M, kappa, seed = 60, 11, 0.3, 21
    want = orc.xyz(X, Y, L, M, kappa, seed)
    assert len(want) > 0
    with xyz.create(X, Y) as ctx:
        ctx.set_filter(mode)
        for ft, vb, gr in SHAPES:
            ctx.set_tiles(ft, vb, gr)
            got = _arr(ctx.search(L, M, kappa, seed))
            assert np.array_equal(got, want), (mode, ft, vb, gr)
            if gr:
                assert ctx.stats()["chunks"] == -(-L // gr) or gr * 6000 < 64, ctx.stats()


def test_autotune_tiles_sets_shapes_in_range(xyz, orc):
    X, Y = _planted(256, 20000, 9)
    L, M, kappa, seed = 400, 12, 0.3, 4
    want = orc.xyz(X, Y, L, M, kappa, seed)
    with xyz.create(X, Y) as ctx:
        tiles, ms = ctx.autotune_tiles(M, kappa, seed=3, trial_runs=400)
        assert ms > 0
        assert tiles["filter_threads"] in (0, 640, 768, 896, 1024)
        assert tiles["verify_blocks_per_sm"] in (0, 1, 2)
        assert tiles["group_runs"] >= 0
        got = _arr(ctx.search(L, M, kappa, seed))
    assert np.array_equal(got, want)


def test_bad_shapes_are_refused(xyz):
    X, Y = _planted(64, 500, 1)
    with xyz.create(X, Y) as ctx:
        for bad in [(500, 0, 0), (1056, 0, 0), (32, 0, 0), (0, -1, 0), (0, 0, -5)]:
            with pytest.raises(xyz.XyzError) as e:
                ctx.set_tiles(*bad)
            assert e.value.code == xyz.XYZ_EINVAL


def test_block_start_table_growth_keeps_results(xyz):
    # M = 7 on 40000 random columns: about 6e6 candidates per run, 4e8 per
    # search, past the verification's first block-start table (2^22 blocks
    # of 32 candidates).  One launch group (most blocks find their bucket by
    # binary search), groups of 4 and 16 runs (the table grows after the
    # first group) and a second search on the grown table must agree, and
    # every pair must be one of the exhaustive screen's with its agreement
    rng = np.random.default_rng(77)
    X = np.asfortranarray((rng.integers(0, 2, size=(64, 40000), dtype=np.int8) * 2 - 1).astype(np.int8))
    Y = (X[:, 3] * X[:, 39000]).astype(np.int8)
    L, M, kappa, seed = 64, 7, 0.5, 5
    with xyz.create(X, Y) as ctx:
        one = ctx.search(L, M, kappa, seed)
        cand = ctx.stats()["candidates"]
        brute = ctx.brute_force(kappa)
    assert cand > 2 ** 27
    for gr in (4, 16):
        with xyz.create(X, Y) as ctx:
            ctx.set_tiles(group_runs=gr)
            a = ctx.search(L, M, kappa, seed)
            b = ctx.search(L, M, kappa, seed)
        assert np.array_equal(a, one), gr
        assert np.array_equal(b, one), gr
    bs = {(int(j), int(k)): int(g) for j, k, g in zip(brute["j"], brute["k"], brute["agree"])}
    assert len(one) > 0
    assert all(bs.get((int(j), int(k))) == int(g) for j, k, g in zip(one["j"], one["k"], one["agree"]))
