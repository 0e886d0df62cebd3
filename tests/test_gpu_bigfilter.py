"""The class-split survivor filter (keys split into 16 linear classes, one
shared-memory filter per class in turn): the search it serves must equal the
oracle's and the other paths' exactly -- at small p with the filter forced,
past the single filter's limit of p = 262144, for c = 0 runs, for runs that
overflow the on-chip capacity (hash partitions and the sort), and when a
class list overflows and the search is redone with larger ones or without
the class-split form.
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


def _pairs(res):
    if len(res) == 0:
        return np.zeros((0, 3), np.int64)
    return np.stack([res["j"], res["k"], res["agree"]], axis=1).astype(np.int64)


def _planted(n, p, seed, pairs, flip=0.1):
    X, _ = _rand(n, p, seed)
    rng = np.random.default_rng(seed + 1)
    Y = np.ones(n, np.int8)
    for a, b in pairs:
        Y = (X[:, a] * X[:, b]).astype(np.int8)
    f = rng.random(n) < flip
    Y[f] = -Y[f]
    return X, Y


@pytest.mark.parametrize("n,p,M,L,kappa", [
    (120, 9000, 10, 40, 0.2),
    (200, 4099, 14, 25, 0.3),          # ragged column word
    (64, 3000, 28, 12, 0.1),           # largest M of the class-split form
    (90, 2500, 1, 3, 0.5),             # smallest M: classes of one key bit
    (300, 20000, 12, 10, 0.3),
])
def test_class_split_matches_oracle(xyz, orc, n, p, M, L, kappa):
    X, Y = _planted(n, p, n + p + M, [(3, p - 2)])
    want = orc.xyz(X, Y, L, M, kappa, 17)
    with xyz.create(X, Y) as ctx:
        ctx.set_filter(2)
        got = _pairs(ctx.search(L, M, kappa, 17))
        st_big = ctx.stats()
        ctx.set_filter(True)
        ref = _pairs(ctx.search(L, M, kappa, 17))
        st_ref = ctx.stats()
    assert np.array_equal(got, want)
    assert np.array_equal(ref, want)
    assert st_big["candidates"] == st_ref["candidates"]


def test_class_split_c_zero_and_overflowing_runs(xyz, orc):
    # Y mostly +1, M = 10: most runs have c = 0 (every column survives) and
    # the others keep nearly every column: about 20000 survivors per run,
    # grouped in partitions on chip, or by the sort when partitions are off
    X, Y = _rand(64, 20000, 31)
    Y[:] = 1
    Y[:3] = -1
    L, M, kappa, seed = 6, 10, 0.4, 5
    want = orc.xyz(X, Y, L, M, kappa, seed)
    assert len(want) > 100
    with xyz.create(X, Y) as ctx:
        ctx.set_filter(2)
        for parts in (32, 0):
            ctx.set_onchip_partitions(parts)
            got = _pairs(ctx.search(L, M, kappa, seed))
            st = ctx.stats()
            assert np.array_equal(got, want), parts
            if parts == 0:
                assert st["survivors"] > 0


def test_class_split_above_the_single_filter(xyz, orc):
    # p past 262144: the default search takes the class-split filter
    n, p = 64, 300000
    X, Y = _planted(n, p, 41, [(5, 299990)], flip=0.05)
    L, M, kappa, seed = 6, 18, 0.5, 9
    want = orc.xyz(X, Y, L, M, kappa, seed)
    with xyz.create(X, Y) as ctx:
        got = _pairs(ctx.search(L, M, kappa, seed))
        for run in (0, 4):
            assert np.array_equal(ctx.run_candidates(M, seed, run), orc.candidates(X, Y, M, seed, run)), run
    assert np.array_equal(got, want)


def test_class_split_sub_bucket_overflow_regrows(xyz, orc):
    # two column patterns only (v and v * Y): every run has two distinct keys,
    # so all keys fall into one or two classes and overflow the class lists
    # sized for 16 balanced classes; the search is redone with larger lists
    # and then without the class-split form.  Every pair (j < 1000 <= k) is
    # a candidate in every run.
    n, p = 64, 2000
    rng = np.random.default_rng(51)
    v = (rng.integers(0, 2, size=n, dtype=np.int8) * 2 - 1).astype(np.int8)
    Y = (rng.integers(0, 2, size=n, dtype=np.int8) * 2 - 1).astype(np.int8)
    X = np.empty((n, p), np.int8, order="F")
    X[:, :1000] = v[:, None]
    X[:, 1000:] = (v * Y)[:, None]
    L, M, kappa, seed = 2, 8, 0.9, 3
    want = orc.xyz(X, Y, L, M, kappa, seed)
    with xyz.create(X, Y) as ctx:
        ctx.set_filter(2)
        got = _pairs(ctx.search(L, M, kappa, seed))
    assert len(want) > 0
    assert np.array_equal(got, want)


def test_class_split_lists_grow_for_one_class(xyz, orc):
    # 163840 identical columns: every key of a run is in one class -- more
    # than the first room of the class lists (a quarter of the columns).  The
    # lists grow to hold every key in one class and the search is redone; it
    # gives the oracle's (empty) result; c != 0 in every run (half the rows
    # of Y are -1), so no pair is a candidate.
    n, p = 64, 163840
    rng = np.random.default_rng(71)
    v = (rng.integers(0, 2, size=n, dtype=np.int8) * 2 - 1).astype(np.int8)
    Y = np.ones(n, np.int8)
    Y[::2] = -1
    X = np.empty((n, p), np.int8, order="F")
    X[:, :] = v[:, None]
    L, M, kappa, seed = 2, 20, 0.5, 4
    want = orc.xyz(X, Y, L, M, kappa, seed)
    with xyz.create(X, Y) as ctx:
        ctx.set_filter(2)
        got = _pairs(ctx.search(L, M, kappa, seed))
        again = _pairs(ctx.search(L, M, kappa, seed))
    assert np.array_equal(got, want) and np.array_equal(again, want)


def test_filter_mode_argument_check(xyz):
    X, Y = _rand(40, 100, 61)
    with xyz.create(X, Y) as ctx:
        with pytest.raises(xyz.XyzError) as e:
            ctx.set_filter(3)
        assert e.value.code == xyz.XYZ_EINVAL


def test_class_split_huge_group_grouped_from_global_memory(xyz, orc):
    # 9000 identical columns v and two columns v o Y: one group of 9002
    # members -- its hash bin is larger than the on-chip survivor array, so
    # the bin is grouped straight from the bin-sorted copy of the run's
    # survivors (its distinct keys fit the table); nothing is left for the
    # sort path, and every run's candidates equal the oracle's.
    n, p = 64, 100000
    X, Y = _rand(n, p, 81)
    rng = np.random.default_rng(82)
    v = (rng.integers(0, 2, size=n, dtype=np.int8) * 2 - 1).astype(np.int8)
    X[:, 1000:10000] = v[:, None]
    X[:, 20000] = v * Y
    X[:, 70000] = v * Y
    L, M, kappa, seed = 3, 20, 0.3, 8
    want = orc.xyz(X, Y, L, M, kappa, seed)
    with xyz.create(X, Y) as ctx:
        ctx.set_filter(2)
        got = _pairs(ctx.search(L, M, kappa, seed))
        st = ctx.stats()
        assert st["survivors"] == 0 and st["bucket_members"] >= 9002
        for run in (0, 2):
            assert np.array_equal(ctx.run_candidates(M, seed, run), orc.candidates(X, Y, M, seed, run)), run
    assert len(want) > 0
    assert np.array_equal(got, want)


@pytest.mark.parametrize("M", [18, 24])
def test_class_split_c_zero_runs_keep_repeated_keys(xyz, orc, M):
    # Y = +1: c = 0 in every run, so a pair is a candidate exactly when its
    # two columns have equal keys.  The filter keeps the columns whose key
    # occurs at least twice (with M = 24 a good share of the 600000 keys is
    # unique and dropped, with M = 18 nearly none), and the candidates equal
    # the oracle's.
    n, p = 64, 600000
    X, _ = _rand(n, p, 91)
    Y = np.ones(n, np.int8)
    seed = 12
    with xyz.create(X, Y) as ctx:
        for run in (0, 1):
            got = ctx.run_candidates(M, seed, run)
            st = ctx.stats()
            assert np.array_equal(got, orc.candidates(X, Y, M, seed, run)), run
            assert 0 < st["filter_kept"] <= p
            if M == 24:
                assert st["filter_kept"] < p
