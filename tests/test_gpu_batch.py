"""Batched search: B responses on one resident X share the row stream and
each run's keys; every response's result must equal its own search (and the
oracle's), including responses whose runs spill off chip (c = 0), B = 1, and
configurations outside the batched kernels (M >= 32: one response at a time).
"""
import numpy as np
import pytest

from paper_1610_05108_gb300 import synth

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
    return X, rng


def _arr(res):
    if len(res) == 0:
        return np.zeros((0, 3), np.int32)
    return np.stack([res["j"], res["k"], res["agree"]], axis=1).astype(np.int32)


def _responses(X, rng, B):
    n, p = X.shape
    Ys = np.empty((B, n), dtype=np.int8)
    for b in range(B):
        a, c = rng.choice(p, size=2, replace=False)
        y = (X[:, a] * X[:, c]).astype(np.int8)
        flip = rng.random(n) < 0.1
        y[flip] = -y[flip]
        Ys[b] = y
    return Ys


def test_batch_equals_single_searches_and_oracle(xyz, orc):
    X, rng = _rand(150, 3000, 31)
    Ys = _responses(X, rng, 6)
    L, M, kappa, seed = 40, 9, 0.3, 1234
    with xyz.create(X, Ys[0]) as ctx:
        got = ctx.search_batch(Ys, L, M, kappa, seed)
        for b in range(len(Ys)):
            ctx.set_y(Ys[b])
            single = ctx.search(L, M, kappa, seed)
            assert np.array_equal(got[b], single), b
    for b in (0, 3, 5):
        assert np.array_equal(_arr(got[b]), orc.xyz(X, Ys[b], L, M, kappa, seed))
    assert sum(len(g) for g in got) > 0


def test_batch_with_spilled_responses(xyz, orc):
    # response 1 is all +1: c = 0 in every run, all 6500 columns survive:
    # its runs go through the sort path, or through hash partitions on chip;
    # the others stay on chip
    X, rng = _rand(100, 6500, 32)
    Ys = _responses(X, rng, 3)
    Ys[1] = 1
    L, M, kappa, seed = 6, 12, 0.9, 7
    for parts in (0, 32):                     # sort path, then partitions on chip
        with xyz.create(X, Ys[0]) as ctx:
            ctx.set_onchip_partitions(parts)
            got = ctx.search_batch(Ys, L, M, kappa, seed)
        for b in range(3):
            assert np.array_equal(_arr(got[b]), orc.xyz(X, Ys[b], L, M, kappa, seed)), (parts, b)


def test_batch_of_one_and_lsd_fallback(xyz, orc):
    X, rng = _rand(64, 800, 33)
    Ys = _responses(X, rng, 3)
    with xyz.create(X, Ys[2]) as ctx:
        one = ctx.search_batch(Ys[:1], 25, 7, 0.2, 3)
        assert np.array_equal(_arr(one[0]), orc.xyz(X, Ys[0], 25, 7, 0.2, 3))
        # the context's own response is unchanged by a batch
        assert np.array_equal(_arr(ctx.search(25, 7, 0.2, 3)), orc.xyz(X, Ys[2], 25, 7, 0.2, 3))
        big_m = ctx.search_batch(Ys, 10, 33, 0.0, 5)       # M >= 32: one response at a time
    for b in range(3):
        assert np.array_equal(_arr(big_m[b]), orc.xyz(X, Ys[b], 10, 33, 0.0, 5))


def test_batch_rejects_bad_input(xyz):
    X, rng = _rand(20, 50, 34)
    Ys = _responses(X, rng, 2)
    with xyz.create(X, Ys[0]) as ctx:
        bad = Ys.copy()
        bad[1, 3] = 0
        with pytest.raises(xyz.XyzError) as e:
            ctx.search_batch(bad, 5, 4, 0.1, 1)
        assert e.value.code == xyz.XYZ_EINVAL
        with pytest.raises(xyz.XyzError):
            ctx.search_batch(Ys, 0, 4, 0.1, 1)


def test_batch_gwas_many_responses(xyz, orc):
    # many responses on an SNP-shaped X (the batching workload's shape, smaller)
    d = synth.gwas(800, 20000, 11)
    Ys, planted, _ = synth.extra_responses(d.X, 24, 5, pairs_per_y=3)
    L, M, kappa, seed = 300, 16, 0.3, 99
    with xyz.create(d.X, d.Y) as ctx:
        got = ctx.search_batch(Ys, L, M, kappa, seed)
        for b in (0, 7, 23):
            ctx.set_y(Ys[b])
            assert np.array_equal(got[b], ctx.search(L, M, kappa, seed)), b
    for b in (0, 23):
        res = got[b]
        assert np.array_equal(res["agree"], orc.agree_pairs(d.X, Ys[b], res["j"], res["k"]))


def test_autotune_M_picks_a_measured_point(xyz):
    X, rng = _rand(300, 4000, 41)
    Y = (X[:, 10] * X[:, 20]).astype(np.int8)
    Y[:30] = -Y[:30]
    with xyz.create(X, Y) as ctx:
        before = ctx.search(200, 12, 0.3, 9)
        M, L, ms, table = ctx.autotune_M(0.3, 0.9, 0.95, 8, 14, seed=3, trial_runs=256)
        after = ctx.search(200, 12, 0.3, 9)
        assert np.array_equal(before, after)            # tuning leaves no trace in results
        assert 8 <= M <= 14 and ms > 0
        assert L == xyz.runs_for_recall(0.9 ** M, 0.95)
        assert list(table[:, 0]) == list(range(8, 15))
        assert table[M - 8, 2] == ms
        found = ctx.search(3 * L, M, 0.3, 5)
        assert (10, 20) in set(zip(found["j"].tolist(), found["k"].tolist()))
        with pytest.raises(xyz.XyzError):
            ctx.autotune_M(0.3, 1.5, 0.95, 8, 14)
