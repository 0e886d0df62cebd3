"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer work, so the bar is bit-exact: keys of every column, the candidate
set E_l of a run, the agreement counts, and the final pair list of a
search.  Sizes span several tiles and ragged tails (n and p not multiples of
32 or of the 4096-entry sort tile), the degenerate cases (M = 0, c = 0 runs,
constant columns that make one huge bucket, empty results) and, at the end,
the full-size SNP-shaped workload the benchmark times, checked on sampled
runs and on every reported pair.
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
    Y = (rng.integers(0, 2, size=n, dtype=np.int8) * 2 - 1).astype(np.int8)
    return X, Y


def _as_set(a):
    return {tuple(int(v) for v in r) for r in a}


def _pairs_array(res):
    return np.stack([res["j"], res["k"], res["agree"]], axis=1).astype(np.int32) if len(res) else np.zeros((0, 3), np.int32)


# ------------------------------------------------------------------ keys

@pytest.mark.parametrize("n,p", [(200, 2000), (97, 333), (33, 65), (1000, 257), (1, 40)])
@pytest.mark.parametrize("M", [0, 1, 10, 31, 32, 33, 63, 64])
def test_keys_match_oracle(xyz, orc, n, p, M):
    X, Y = _rand(n, p, n * 7 + p + M)
    seed = 0xABCDEF + M
    with xyz.create(X, Y) as ctx:
        for run in (0, 1, 17):
            kx, c = ctx.run_keys(M, seed, run)
            rows = orc.draw_rows(seed, run, M, n)
            ox, oz = orc.keys(X, Y, rows)
            assert np.array_equal(kx, ox)
            assert np.array_equal(kx ^ np.uint64(c), oz)


# ------------------------------------------------------------ candidates

def _cand_cases():
    d = synth.config_small(1)
    yield "small_iid", d.X, d.Y, 10, range(3)
    X, Y = _rand(97, 333, 5)
    yield "ragged_M4", X, Y, 4, range(3)
    X, Y = _rand(64, 300, 6)
    Y[:] = 1                                   # c = 0 in every run
    yield "c_zero", X, Y, 5, range(3)
    X, Y = _rand(50, 60, 7)
    yield "M0_all_pairs", X, Y, 0, range(1)
    X, Y = _rand(80, 5000, 8)
    X[:, 100:900] = 1                          # 800 equal columns: one huge bucket
    X[:, 1000:1300] = -1
    yield "heavy_bucket", X, Y, 6, range(2)
    X, Y = _rand(2000, 4100, 9)
    yield "two_tiles_M12", X, Y, 12, range(2)
    X, Y = _rand(300, 9000, 10)
    yield "three_blocks_M9", X, Y, 9, range(2)
    X, Y = _rand(70, 3000, 17)
    X[:, 10:400] = X[:, [5]]                   # 391 equal columns: groups survive M >= 32
    X[:, 500:520] = X[:, [6]] * Y[:, None]     # X_j = Z_6: partners of column 6 in every run
    yield "lsd_path_M33", X, Y, 33, range(2)
    yield "lsd_path_M40", X, Y, 40, range(1)
    yield "part_path_M31", X, Y, 31, range(2)
    X, Y = _rand(90, 9000, 18)
    Y[:] = 1                                   # c = 0: all 9000 columns survive -> spill path
    yield "spill_c_zero", X, Y, 13, range(2)


@pytest.mark.parametrize("case", list(_cand_cases()), ids=lambda c: c[0])
def test_candidates_match_oracle(xyz, orc, case):
    name, X, Y, M, runs = case
    seed = 4242
    with xyz.create(X, Y) as ctx:
        for run in runs:
            got = ctx.run_candidates(M, seed, run)
            want = orc.candidates(X, Y, M, seed, run)
            assert got.shape == want.shape, (name, run, got.shape, want.shape)
            assert np.array_equal(got, want), (name, run)


# ---------------------------------------------------------------- agree

@pytest.mark.parametrize("n", [1, 31, 32, 33, 127, 200, 4001])
def test_agree_matches_oracle(xyz, orc, n):
    p = 50
    X, Y = _rand(n, p, n)
    rng = np.random.default_rng(n)
    j = rng.integers(0, p, size=300).astype(np.int32)
    k = rng.integers(0, p, size=300).astype(np.int32)
    with xyz.create(X, Y) as ctx:
        a = ctx.agree(j, k)
    want = orc.agree_pairs(X, Y, j, k)
    assert np.array_equal(a, want)


def test_sample_agree_matches_oracle(xyz, orc):
    X, Y = _rand(300, 700, 3)
    with xyz.create(X, Y) as ctx:
        j, k, a = ctx.sample_agree(5000, 99)
    assert np.all(j != k) and j.min() >= 0 and k.max() < 700
    assert np.array_equal(a, orc.agree_pairs(X, Y, j, k))
    # every column is drawn (uniform on 700 columns, 10000 draws)
    assert len(np.unique(np.concatenate([j, k]))) > 650


# --------------------------------------------------------------- search

def test_search_small_config_matches_oracle(xyz, orc):
    d = synth.config_small(1)
    with xyz.create(d.X, d.Y) as ctx:
        res = ctx.search(10, 10, 0.5, 2024)
    want = orc.xyz(d.X, d.Y, 10, 10, 0.5, 2024)
    got = _pairs_array(res)
    assert np.array_equal(got, want)
    assert np.allclose(res["strength"], ((2 * want[:, 2] - d.n) / d.n).astype(np.float32))
    assert (0, 1) in {(int(a), int(b)) for a, b in want[:, :2]}


@pytest.mark.parametrize("n,p,L,M,kappa", [(97, 333, 25, 4, 0.2), (33, 1000, 40, 6, 0.3),
                                           (500, 4097, 12, 9, 0.25), (64, 200, 7, 3, -0.1),
                                           (40, 700, 30, 32, 0.0), (40, 700, 30, 36, 0.0)])
def test_search_ragged_matches_oracle(xyz, orc, n, p, L, M, kappa):
    X, Y = _rand(n, p, n + p)
    Y = (X[:, 3] * X[:, p - 2]).astype(np.int8)
    Y[: n // 8] = -Y[: n // 8]
    with xyz.create(X, Y) as ctx:
        got = _pairs_array(ctx.search(L, M, kappa, 31337))
    want = orc.xyz(X, Y, L, M, kappa, 31337)
    assert np.array_equal(got, want)


def test_search_independent_of_launch_grouping(xyz):
    X, Y = _rand(120, 900, 11)
    Y = (X[:, 10] * X[:, 500]).astype(np.int8)
    Y[:20] = -Y[:20]
    with xyz.create(X, Y) as ctx:
        ref = ctx.search(37, 5, 0.1, 5)
        for entries in (10, 100, 900, 900 * 3, 900 * 8 + 5, 10**9):
            ctx.set_chunk_entries(entries)
            got = ctx.search(37, 5, 0.1, 5)
            assert np.array_equal(got, ref), entries
            st = ctx.stats()
            assert st["runs"] == 37


@pytest.mark.parametrize("M", [6, 12, 31])
def test_search_independent_of_filter(xyz, orc, M):
    d = synth.gwas(400, 6000, 7)
    with xyz.create(d.X, d.Y) as ctx:
        on = ctx.search(60, M, 0.2, 9)
        st_on = ctx.stats()
        ctx.set_filter(False)
        off = ctx.search(60, M, 0.2, 9)
        st_off = ctx.stats()
    assert np.array_equal(on, off)
    assert st_on["candidates"] == st_off["candidates"]
    assert st_on["survivors"] <= st_off["survivors"] == 60 * d.p
    assert np.array_equal(_pairs_array(on), orc.xyz(d.X, d.Y, 60, M, 0.2, 9))


def test_search_mixing_spilled_and_on_chip_runs(xyz, orc):
    # Y mostly +1: with M = 4 most runs draw only +1 rows (c = 0, every
    # column survives, p > 8192 -> general sort path), the others are grouped
    # on chip; both feed one result.
    X, Y = _rand(120, 9000, 19)
    Y[:] = 1
    Y[:6] = -1
    Y = Y * (X[:, 2] * X[:, 3]) * (X[:, 2] * X[:, 3])     # keep +-1, no change
    want = orc.xyz(X, Y, 12, 4, 0.9, 5)
    with xyz.create(X, Y) as ctx:
        ctx.set_onchip_partitions(0)               # every overflowing run spills
        got = _pairs_array(ctx.search(12, 4, 0.9, 5))
        st = ctx.stats()
        assert st["survivors"] > 0
        assert np.array_equal(got, want)
        ctx.set_onchip_partitions(32)              # hash partitions on chip
        got = _pairs_array(ctx.search(12, 4, 0.9, 5))
        st = ctx.stats()
        assert st["survivors"] == 0
        assert np.array_equal(got, want)


def test_onchip_partitions_match_oracle(xyz, orc):
    # Y mostly +1 and M = 10: most runs have c = 0, and in the others nearly
    # every key has a partner, so about 20000 columns survive per run -- three
    # or more partitions of at most 8192 on chip.  A lower limit sends the run
    # to the sort; every limit gives the oracle's result and the same E_l.
    X, Y = _rand(64, 20000, 23)
    Y[:] = 1
    Y[:3] = -1
    L, M, kappa, seed = 6, 10, 0.4, 12
    want = orc.xyz(X, Y, L, M, kappa, seed)
    assert len(want) > 100
    cands = {}
    with xyz.create(X, Y) as ctx:
        for parts in (0, 1, 2, 3, 32):
            ctx.set_onchip_partitions(parts)
            got = _pairs_array(ctx.search(L, M, kappa, seed))
            st = ctx.stats()
            assert np.array_equal(got, want), parts
            cands[parts] = st["candidates"]
            if parts == 32:
                assert st["survivors"] == 0
            if parts <= 2:
                assert st["survivors"] > 0
    assert len(set(cands.values())) == 1, cands


def test_member_space_overflow_regrows(xyz, orc):
    # M = 13 over 30000 random columns: nearly every key has a partner, so
    # almost every column survives and the on-chip groups of the first
    # attempt need about seven times the member space first reserved.  The
    # launch group is abandoned (nothing reads the bucket arrays past their
    # end), the space grows to what was asked for and the search is redone.
    X, Y = _rand(64, 30000, 29)
    L, M, kappa, seed = 12, 13, 0.5, 3
    want = orc.xyz(X, Y, L, M, kappa, seed)
    assert len(want) > 0
    with xyz.create(X, Y) as ctx:
        got = _pairs_array(ctx.search(L, M, kappa, seed))
        again = _pairs_array(ctx.search(L, M, kappa, seed))
    assert np.array_equal(got, want)
    assert np.array_equal(again, want)


def test_onchip_partitions_argument_check(xyz):
    X, Y = _rand(40, 100, 24)
    with xyz.create(X, Y) as ctx:
        for bad in (-1, 33):
            with pytest.raises(xyz.XyzError):
                ctx.set_onchip_partitions(bad)


def test_spill_flush_windows_do_not_change_results(xyz, orc):
    # spilled runs grouped through the sort once per search, after every
    # launch group, and after every third one: one result
    X, Y = _rand(120, 9000, 19)
    Y[:] = 1
    Y[:6] = -1
    want = orc.xyz(X, Y, 12, 4, 0.9, 5)
    with xyz.create(X, Y) as ctx:
        ctx.set_chunk_entries(9000 // 64)         # one run per launch group
        ctx.set_onchip_partitions(0)              # overflowing runs spill
        for flush in (0, 1, 3):
            ctx.set_spill_flush(flush)
            got = _pairs_array(ctx.search(12, 4, 0.9, 5))
            st = ctx.stats()
            assert st["chunks"] == 12 and st["survivors"] > 0, flush
            assert np.array_equal(got, want), flush
        with pytest.raises(xyz.XyzError):
            ctx.set_spill_flush(-1)


def test_search_range_union(xyz):
    X, Y = _rand(150, 1200, 12)
    Y = (X[:, 7] * X[:, 8]).astype(np.int8)
    Y[:30] = -Y[:30]
    with xyz.create(X, Y) as ctx:
        whole = ctx.search(30, 6, 0.1, 77)
        parts = [ctx.search_range(a, b, 6, 0.1, 77) for a, b in ((0, 7), (7, 19), (19, 30))]
    merged = np.unique(np.concatenate(parts))
    assert np.array_equal(np.sort(merged, order=["j", "k"]), whole)


def test_M0_search_is_brute_force(xyz, orc):
    X, Y = _rand(150, 300, 13)
    Y = (X[:, 1] * X[:, 2]).astype(np.int8)
    with xyz.create(X, Y) as ctx:
        for kappa in (0.2, 0.0, 1.0):
            got = _pairs_array(ctx.search(1, 0, kappa, 1))
            assert np.array_equal(got, orc.brute_force(X, Y, kappa))


def test_set_y_then_search(xyz, orc):
    X, Y = _rand(90, 400, 14)
    Y2 = (X[:, 5] * X[:, 6]).astype(np.int8)
    with xyz.create(X, Y) as ctx:
        ctx.set_y(Y2)
        got = _pairs_array(ctx.search(8, 5, 0.3, 3))
    assert np.array_equal(got, orc.xyz(X, Y2, 8, 5, 0.3, 3))


def test_empty_result(xyz):
    X, Y = _rand(200, 300, 15)
    with xyz.create(X, Y) as ctx:
        res = ctx.search(5, 8, 0.99, 1)
        assert len(res) == 0


def test_invalid_arguments(xyz):
    X, Y = _rand(20, 10, 16)
    Xb = X.copy(order="F")
    Xb[3, 4] = 0
    with pytest.raises(xyz.XyzError) as e:
        xyz.create(Xb, Y)
    assert e.value.code == xyz.XYZ_EINVAL
    Yb = Y.copy()
    Yb[0] = 2
    with pytest.raises(xyz.XyzError):
        xyz.create(X, Yb)
    with xyz.create(X, Y) as ctx:
        for bad in [dict(L=0, M=3, kappa=0.1), dict(L=1, M=65, kappa=0.1), dict(L=1, M=-1, kappa=0.1),
                    dict(L=1, M=3, kappa=float("nan")), dict(L=1, M=3, kappa=1.5)]:
            with pytest.raises(xyz.XyzError) as e:
                ctx.search(bad["L"], bad["M"], bad["kappa"], 0)
            assert e.value.code == xyz.XYZ_EINVAL
        with pytest.raises(xyz.XyzError):
            ctx.agree(np.array([0]), np.array([10]))
        with pytest.raises(xyz.XyzError):
            ctx.set_y(Yb)
        # a rejected Y leaves the context usable with the old response
        assert len(ctx.search(2, 2, -1.0, 0)) > 0


# --------------------------------------------------- full-size workload

@pytest.fixture(scope="module")
def gwas_full():
    return synth.config_gwas(1)


@pytest.mark.parametrize("M", [19, 21])
def test_full_size_gwas_sampled_parity(xyz, orc, gwas_full, M):
    """The SNP-shaped n=2000, p=100000 workload at the M of the gamma0 = 0.55
    rule (19) and of eq. bestM (21): exact E_l on sampled runs -- one of
    them a run whose survivors exceed one on-chip grouping and are grouped
    in hash partitions, found through the stats -- and every reported pair's
    agreement recomputed one by one by the oracle."""
    d = gwas_full
    L, kappa, seed = 400, 0.3, 2026
    with xyz.create(d.X, d.Y) as ctx:
        for run in (0, 123):
            got = ctx.run_candidates(M, seed, run)
            want = orc.candidates(d.X, d.Y, M, seed, run)
            assert np.array_equal(got, want), run
        part_run = None
        for run in range(1000, 6000):
            ctx.run_candidates(M, seed, run)
            if ctx.stats()["segment_grouped_runs"] == 1:
                part_run = run
                break
        assert part_run is not None, "no run needed the on-chip partitions"
        got = ctx.run_candidates(M, seed, part_run)
        assert np.array_equal(got, orc.candidates(d.X, d.Y, M, seed, part_run)), part_run
        res = ctx.search(L, M, kappa, seed)
    amin = orc.amin(d.n, kappa)
    assert np.all(res["agree"] >= amin)
    assert np.all(res["j"] < res["k"])
    keys = res["j"].astype(np.int64) * d.p + res["k"]
    assert np.all(np.diff(keys) > 0)
    assert np.array_equal(res["agree"], orc.agree_pairs(d.X, d.Y, res["j"], res["k"]))
    # every run range result is contained in the whole result
    with xyz.create(d.X, d.Y) as ctx:
        part = ctx.search_range(0, 50, M, kappa, seed)
    assert _as_set(_pairs_array(part)) <= _as_set(_pairs_array(res))
    want_part = orc.xyz_range(d.X, d.Y, 0, 50, M, kappa, seed)
    assert np.array_equal(_pairs_array(part), want_part)


@pytest.fixture(scope="module")
def gwas_large():
    return synth.config_gwas_large(1)


@pytest.mark.parametrize("M", [23, 26])
def test_at_scale_operating_points(xyz, orc, gwas_large, M):
    """The benchmark's workload (SNP-shaped n=4000, p=10^6, class-split
    filter) at its operating point M = 23 (gamma0 = 0.55 rule) and at eq.
    bestM's M = 26: E_l of two sampled runs equals the oracle's, a short run
    range equals the oracle's search pair for pair (agreement counts
    included), and at M = 23 the runs' survivors are grouped on chip in
    several passes rather than by the sort."""
    d = gwas_large
    kappa, seed = 0.28, 777
    with xyz.create(d.X, d.Y) as ctx:
        for run in (5, 4242):
            got = ctx.run_candidates(M, seed, run)
            want = orc.candidates(d.X, d.Y, M, seed, run)
            assert len(want) > 0
            assert np.array_equal(got, want), run
        part = ctx.search_range(0, 3, M, kappa, seed)
        st = ctx.stats()
    want_part = orc.xyz_range(d.X, d.Y, 0, 3, M, kappa, seed)
    assert np.array_equal(_pairs_array(part), want_part)
    assert st["filter_kept"] > 0 and st["bucket_members"] > 0
    if M == 23:
        assert st["segment_grouped_runs"] >= 1 and st["survivors"] == 0, st


def test_sharded_search_through_library(xyz):
    # run-range sharding as the multi-GPU path does it, ranks simulated in
    # turn on one device; the merged result equals the whole search
    from paper_1610_05108_gb300 import shard
    X, Y = _rand(200, 3000, 20)
    Y = (X[:, 11] * X[:, 1500]).astype(np.int8)
    Y[:25] = -Y[:25]
    L, M, kappa, seed = 50, 8, 0.2, 99
    with xyz.create(X, Y) as ctx:
        whole = _pairs_array(ctx.search(L, M, kappa, seed))
        world = 3
        parts = [ctx.search_range(a, b, M, kappa, seed) for a, b in shard.run_ranges(L, world)]
    merged = shard.merge_pairs(parts)
    assert np.array_equal(merged, whole.astype(np.int64))
