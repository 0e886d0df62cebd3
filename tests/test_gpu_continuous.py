"""Real-valued response (Section 3.1): the GPU search with weighted rows and
weighted verification equals the oracle's continuous-response search pair
for pair (agreement counts exact, strengths to float precision), reduces to
the binary search for Y = +-1, draws the oracle's weighted rows, and rejects
unusable responses without changing the context.
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


def _X(n, p, seed):
    rng = np.random.default_rng(seed)
    return np.asfortranarray((rng.integers(0, 2, size=(n, p), dtype=np.int8) * 2 - 1).astype(np.int8)), rng


def _arr(res):
    if len(res) == 0:
        return np.zeros((0, 3), np.int32)
    return np.stack([res["j"], res["k"], res["agree"]], axis=1).astype(np.int32)


def _check(xyz, orc, X, Y, L, M, kappa, seed):
    with xyz.create(X, np.ones(X.shape[0], np.int8)) as ctx:
        ctx.set_y_real(Y)
        got = ctx.search(L, M, kappa, seed)
    want, S = orc.xyz_weighted(X, Y, L, M, kappa, seed)
    assert np.array_equal(_arr(got), want), (X.shape, L, M, kappa)
    if len(want):
        q, _ = orc.quantize_y(Y)
        Q = float(q.sum())
        strength = (2.0 * S - Q) / Q
        assert np.allclose(got["strength"], strength.astype(np.float32), rtol=0, atol=1e-6)
    return got


@pytest.mark.parametrize("n,p,L,M,kappa", [
    (200, 2000, 40, 9, 0.25),
    (97, 513, 25, 6, 0.15),
    (1000, 3000, 30, 12, 0.3),
    (130, 400, 12, 33, -0.2),          # M >= 32: general sort path
])
def test_real_response_matches_oracle(xyz, orc, n, p, L, M, kappa):
    X, rng = _X(n, p, n + p + M)
    Y = rng.standard_t(3, size=n) + 2.0 * X[:, 5] * X[:, p - 3]
    got = _check(xyz, orc, X, Y, L, M, kappa, 17)
    if M < 30:
        assert (5, p - 3) in set(zip(got["j"].tolist(), got["k"].tolist()))


def test_real_pm1_equals_binary(xyz):
    X, rng = _X(150, 1200, 3)
    Yb = (X[:, 7] * X[:, 900]).astype(np.int8)
    Yb[:20] = -Yb[:20]
    with xyz.create(X, Yb) as ctx:
        binary = ctx.search(30, 8, 0.2, 5)
        ctx.set_y_real(Yb.astype(np.float64) * 3.5)
        real = ctx.search(30, 8, 0.2, 5)
        ctx.set_y(Yb)                                   # back to the binary mode
        again = ctx.search(30, 8, 0.2, 5)
    assert np.array_equal(_arr(binary), _arr(real))
    assert np.allclose(binary["strength"], real["strength"], atol=1e-6)
    assert np.array_equal(binary, again)


def test_weighted_rows_and_candidates(xyz, orc):
    X, rng = _X(300, 700, 8)
    Y = rng.exponential(size=300) * np.where(rng.random(300) < 0.3, -1.0, 1.0)
    Y[10:20] = 0.0
    q, sgn = orc.quantize_y(Y)
    with xyz.create(X, np.ones(300, np.int8)) as ctx:
        ctx.set_y_real(Y)
        for run in (0, 5, 77):
            kx, c = ctx.run_keys(10, 123, run)
            rows = orc.draw_rows_weighted(q, 123, run, 10)
            assert not set(rows.tolist()) & set(range(10, 20))       # weight 0: never drawn
            ox, oz = orc.keys(X, sgn, rows)
            assert np.array_equal(kx, ox)
            assert c == int(ox[0] ^ oz[0])
            got = ctx.run_candidates(10, 123, run)
            want, _ = orc.xyz_weighted_range(X, Y, run, run + 1, 10, -1.0, 123)
            assert np.array_equal(got, want[:, :2])


def test_section31_model_pair_found(xyz, orc):
    # Y_i = X_i1 X_i2 + eps_i, sigma^2 = 0.5: the weighted strength of (1, 2)
    # is about 0.94 while the rest stay near 0.5
    X, rng = _X(2000, 5000, 21)
    Y = X[:, 1].astype(np.float64) * X[:, 2] + rng.normal(0, np.sqrt(0.5), size=2000)
    with xyz.create(X, np.ones(2000, np.int8)) as ctx:
        ctx.set_y_real(Y)
        got = ctx.search(20, 14, 0.6, 4)
    assert list(zip(got["j"].tolist(), got["k"].tolist())) == [(1, 2)]
    a, S = orc.weighted_agree(X, Y, 1, 2)
    q, _ = orc.quantize_y(Y)
    assert got["agree"][0] == a
    assert abs(got["strength"][0] - (2 * S - q.sum()) / q.sum()) < 1e-6


def test_unusable_real_response(xyz):
    X, rng = _X(64, 300, 2)
    Y = rng.normal(size=64)
    with xyz.create(X, np.ones(64, np.int8)) as ctx:
        ctx.set_y_real(Y)
        before = ctx.search(10, 6, 0.1, 1)
        for bad in (np.zeros(64), np.where(np.arange(64) == 3, np.nan, 1.0),
                    np.where(np.arange(64) == 9, np.inf, 1.0)):
            with pytest.raises(xyz.XyzError) as e:
                ctx.set_y_real(bad)
            assert e.value.code == xyz.XYZ_EINVAL
        assert np.array_equal(ctx.search(10, 6, 0.1, 1), before)
        with pytest.raises(xyz.XyzError):
            ctx.brute_force(0.1)
        with pytest.raises(xyz.XyzError):
            ctx.search_batch(np.ones((2, 64), np.int8), 5, 6, 0.1, 1)


def test_abs_search_matches_oracle(xyz, orc):
    X, rng = _X(160, 500, 21)
    Y = (X[:, 3] * X[:, 300]).astype(np.int8)
    Y[:20] = -Y[:20]
    Y[80:] = (-(X[80:, 40] * X[80:, 41])).astype(np.int8)
    with xyz.create(X, Y) as ctx:
        got = ctx.search_abs(20, 5, 0.2, 3)
        plain = ctx.search(20, 5, 0.2, 3)              # signs restored afterwards
    want = orc.xyz_abs(X, Y, 20, 5, 0.2, 3)
    assert np.array_equal(_arr(got), want)
    assert np.allclose(got["strength"], (2.0 * want[:, 2] - 160) / 160)
    assert np.array_equal(_arr(plain), orc.xyz(X, Y, 20, 5, 0.2, 3))
    s = dict(zip(zip(got["j"].tolist(), got["k"].tolist()), got["strength"].tolist()))
    assert s[(40, 41)] < 0 < s[(3, 300)]


def test_kkt_screen_matches_oracle(xyz, orc):
    X, rng = _X(300, 900, 22)
    r = rng.normal(size=300) + 1.5 * X[:, 2] * X[:, 600] - 1.2 * X[:, 10] * X[:, 11]
    r = r - r.mean()
    with xyz.create(X, np.ones(300, np.int8)) as ctx:
        for lam in (0.5, 0.8):
            got = ctx.kkt_screen(r, lam, 40, 6, 9)
            want, d = orc.kkt_xyz(X, r, 40, 6, lam, 9)
            assert np.array_equal(_arr(got), want), lam
            _, e = np.frexp(np.abs(r).max())
            assert np.allclose(got["strength"], d * 2.0 ** (int(e) - 24) / 300, atol=1e-6)
            assert {(2, 600), (10, 11)} <= set(zip(got["j"].tolist(), got["k"].tolist()))
        with pytest.raises(xyz.XyzError):
            ctx.kkt_screen(r, -1.0, 10, 6, 1)


def test_sign_transform_search_matches_oracle(xyz, orc):
    rng = np.random.default_rng(40)
    n, p = 500, 1500
    X = rng.standard_t(5, size=(n, p)).astype(np.float32)
    X[rng.random((n, p)) < 0.02] = 0.0                 # exact zeros take the coin
    Y = X[:, 4].astype(np.float64) * X[:, 1000] + rng.normal(0, 0.7, size=n)
    T = orc.sign_transform(X, coin_seed=5)
    with xyz.Context.from_real_sign(X, coin_seed=5) as ctx:
        kx, _ = ctx.run_keys(20, 1, 0)
        ox, _ = orc.keys(T, np.ones(n, np.int8), orc.draw_rows(1, 0, 20, n))
        assert np.array_equal(kx, ox)                  # the packed X is the transform
        ctx.set_y_real(Y)
        got = ctx.search(30, 10, 0.3, 2)
    want, S = orc.xyz_weighted(T, Y, 30, 10, 0.3, 2)
    assert np.array_equal(_arr(got), want)
    assert (4, 1000) in set(zip(got["j"].tolist(), got["k"].tolist()))
    with pytest.raises(xyz.XyzError):
        xyz.Context.from_real_sign(np.full((4, 3), np.nan, np.float32))


def _unbiased_data(n, p, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1.5, 1.5, size=(n, p)).astype(np.float32)
    X[rng.random((n, p)) < 0.01] = 0.0
    Y = X[:, 2].astype(np.float64) * X[:, p - 5] + rng.normal(0, 0.1, size=n)
    return X, Y


def test_unbiased_candidates_exact(xyz, orc):
    X, Y = _unbiased_data(160, 900, 60)
    with xyz.Context.from_real_unbiased(X, Y) as ctx:
        for run in (0, 3, 11):
            got = ctx.run_candidates(8, 21, run)
            want, _ = orc.xyz_unbiased_range(X, Y, run, run + 1, 8, -1.0, 21)
            assert np.array_equal(got, want), run


@pytest.mark.parametrize("n,p,L,M,kappa", [(160, 900, 40, 8, 0.2), (301, 2500, 30, 10, 0.25)])
def test_unbiased_search_matches_oracle(xyz, orc, n, p, L, M, kappa):
    X, Y = _unbiased_data(n, p, n + p)
    with xyz.Context.from_real_unbiased(X, Y) as ctx:
        got = ctx.search(L, M, kappa, 8)
    pairs, dots = orc.xyz_unbiased_range(X, Y, 0, L, M, -1.0, 8)     # every candidate with its dot
    Xs, Ys = orc.unbiased_scale(X, Y)
    norm1 = np.abs(Ys).sum()
    # Both sides sum the same double terms Y'_i (X'_ij X'_ik) (a product of
    # two floats is exact in double); only the order of the additions
    # differs, so the sums agree to n 2^-52 ||Y'||_1 and the pass decisions
    # are identical for every candidate farther than that from the threshold.
    thr, tol = kappa * norm1, n * 2.0**-52 * norm1
    cand = {(int(j), int(k)): d for (j, k), d in zip(pairs, dots)}
    gotset = set(zip(got["j"].tolist(), got["k"].tolist()))
    near = [d for d in cand.values() if abs(d - thr) <= tol]
    assert not near                                  # no candidate this close: decisions must match
    assert gotset == {pk_ for pk_, d in cand.items() if d >= thr}
    for pk_, s_ in zip(zip(got["j"].tolist(), got["k"].tolist()), got["strength"].tolist()):
        assert abs(s_ - np.float32(cand[pk_] / norm1)) <= 2.5e-7 * abs(s_)     # a float ulp
    assert (got["agree"] == -1).all()
    assert (2, p - 5) in gotset


def test_unbiased_context_limits(xyz):
    X, Y = _unbiased_data(64, 200, 3)
    with xyz.Context.from_real_unbiased(X, Y) as ctx:
        with pytest.raises(xyz.XyzError):
            ctx.set_y(np.ones(64, np.int8))
        with pytest.raises(xyz.XyzError):
            ctx.search_abs(5, 6, 0.3, 1)
        with pytest.raises(xyz.XyzError):
            ctx.search(5, 40, 0.3, 1)                   # M >= 32: no real-X path
        ctx.set_y_real(-Y)                              # a new response is scaled too
        assert len(ctx.search(20, 6, 0.2, 1)) >= 0
    Xn = X.copy()
    Xn[5, 7] = np.nan
    with pytest.raises(xyz.XyzError):
        xyz.Context.from_real_unbiased(Xn, Y)
