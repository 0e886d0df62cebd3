"""Pins of the oracle's continuous-response search (Section 3.1 with the
readings R9-R11 stated in oracle/xyz_oracle.c) against things other than
itself: the binary search it must reduce to for Y = +-1, the sampling
distribution q_i / Q, the printed table of Section 3.1 and the closed form
of the weighted strength in that example, and numpy matrix products.
"""
import json
import math
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _X(n, p, seed):
    rng = np.random.default_rng(seed)
    return np.asfortranarray((rng.integers(0, 2, size=(n, p), dtype=np.int8) * 2 - 1).astype(np.int8)), rng


def test_quantize_fixed_point_rule(orc):
    Y = np.array([0.5, -1.25, 0.0, 3.0, -0.001, 2.9999999])
    q, sgn = orc.quantize_y(Y)
    # max |Y| = 3 = 0.75 * 2^2 -> q_i = round(|Y_i| * 2^22)
    assert list(q) == [round(abs(v) * 2**22) for v in Y]
    assert list(sgn) == [1, -1, 1, 1, -1, 1]
    assert q.max() <= 2**24
    with pytest.raises(ValueError):
        orc.quantize_y(np.zeros(4))
    with pytest.raises(ValueError):
        orc.quantize_y(np.array([1.0, np.nan]))


def test_equal_weights_reduce_to_uniform_draw(orc):
    q, _ = orc.quantize_y(np.where(np.arange(37) % 3 == 0, -1.0, 1.0))
    for run in range(50):
        assert np.array_equal(orc.draw_rows_weighted(q, 99, run, 13), orc.draw_rows(99, run, 13, 37))


def test_weighted_draw_frequencies(orc):
    rng = np.random.default_rng(4)
    Y = rng.standard_cauchy(40)
    Y[5] = 0.0
    q, _ = orc.quantize_y(Y)
    draws = np.concatenate([orc.draw_rows_weighted(q, 2024, r, 64) for r in range(400)])
    counts = np.bincount(draws, minlength=40)
    N = len(draws)
    prob = q / q.sum()
    assert counts[5] == 0                      # weight 0: never drawn
    sd = np.sqrt(N * prob * (1 - prob)) + 1e-9
    assert np.all(np.abs(counts - N * prob) <= 5 * sd + 1)


def test_pm1_response_equals_binary_search(orc):
    X, rng = _X(120, 400, 5)
    Yb = (X[:, 3] * X[:, 77]).astype(np.int8)
    Yb[:15] = -Yb[:15]
    for kappa in (0.1, 0.3, 0.55):
        got, S = orc.xyz_weighted(X, Yb.astype(np.float64), 12, 6, kappa, 31)
        want = orc.xyz(X, Yb, 12, 6, kappa, 31)
        assert np.array_equal(got, want)
        assert np.all(S == got[:, 2].astype(np.int64) * 2**23)     # q_i = 2^23 for |Y_i| = 1


def test_sigma_table_and_weighted_closed_form(orc):
    """Section 3.1's example: the unweighted sign agreement of the pair
    (1, 2) reproduces the printed table; the |Y|-weighted strength matches
    its closed form [Phi(1/s) + s phi(1/s)] / [2 Phi(1/s) - 1 + 2 s phi(1/s)]."""
    from scipy.stats import norm
    table = json.load(open(os.path.join(HERE, "golden", "sec31_sigma_table.json")))
    n = 200000
    X, rng = _X(n, 2, 8)
    for s2, printed in zip(table["sigma2"], table["gamma12"]):
        s = math.sqrt(s2)
        Y = X[:, 0].astype(np.float64) * X[:, 1] + rng.normal(0.0, s, size=n)
        a, S = orc.weighted_agree(X, Y, 0, 1)
        q, _ = orc.quantize_y(Y)
        uniform = 0.5 * (1 + (norm.cdf(1 / s) - norm.cdf(-1 / s)))
        assert abs(a / n - uniform) < 5 * math.sqrt(uniform * (1 - uniform) / n)
        assert abs(a / n - printed) < 0.011
        weighted = (norm.cdf(1 / s) + s * norm.pdf(1 / s)) / (2 * norm.cdf(1 / s) - 1 + 2 * s * norm.pdf(1 / s))
        assert abs(S / q.sum() - weighted) < 0.01, (s2, S / q.sum(), weighted)
        assert weighted > uniform - 1e-12       # heavier rows agree more often


def test_weighted_brute_force_matches_matrix_product(orc):
    X, rng = _X(90, 60, 9)
    Y = rng.normal(size=90) + 2.0 * X[:, 4] * X[:, 50]
    q, sgn = orc.quantize_y(Y)
    Q = int(q.sum())
    G = X.T.astype(np.int64) @ (X.astype(np.int64) * (sgn.astype(np.int64) * q)[:, None])   # 2S - Q
    for kappa in (0.0, 0.2, 0.4):
        got, S = orc.brute_force_weighted(X, Y, kappa)
        want = [(j, k) for j in range(60) for k in range(j + 1, 60) if float(G[j, k]) >= kappa * Q]
        assert [tuple(r[:2]) for r in got] == want
        for (j, k, a), s_ in zip(got, S):
            assert 2 * s_ - Q == G[j, k]
            assert a == int(np.sum(X[:, j] * X[:, k] == sgn))


def test_weighted_search_is_subset_with_weighted_rows(orc):
    X, rng = _X(150, 300, 12)
    Y = rng.normal(size=150) + 3.0 * X[:, 10] * X[:, 200]
    got, S = orc.xyz_weighted(X, Y, 30, 7, 0.3, 5)
    bf, Sb = orc.brute_force_weighted(X, Y, 0.3)
    bset = {(int(j), int(k)): (int(a), int(s)) for (j, k, a), s in zip(bf, Sb)}
    for (j, k, a), s in zip(got, S):
        assert bset[(int(j), int(k))] == (int(a), int(s))
    assert (10, 200) in {(int(j), int(k)) for j, k, _ in got}
    # candidates of one run: the pairs equal on the weighted rows, Z = sgn(Y) X
    q, sgn = orc.quantize_y(Y)
    rows = orc.draw_rows_weighted(q, 5, 3, 7)
    Xs = X[rows, :]
    Zs = Xs * sgn[rows][:, None]
    eq = {(min(j, k), max(j, k)) for j in range(300) for k in range(300)
          if j != k and np.array_equal(Xs[:, j], Zs[:, k])}
    one, _ = orc.xyz_weighted_range(X, Y, 3, 4, 7, -1.0, 5)
    assert {(int(j), int(k)) for j, k, _ in one} == eq


def test_abs_search_is_union_of_signs(orc):
    X, rng = _X(160, 500, 21)
    Y = (X[:, 3] * X[:, 300]).astype(np.int8)
    Y[:20] = -Y[:20]
    Yn = (-(X[:, 40] * X[:, 41])).astype(np.int8)       # a negative interaction
    Y[80:] = Yn[80:]
    got = orc.xyz_abs(X, Y, 20, 5, 0.2, 3)
    bf = orc.brute_force(X, Y, -1.0)                      # every pair with its a
    n = 160
    strong = {(int(j), int(k)): int(a) for j, k, a in bf if abs(2 * a - n) >= 0.2 * n}
    for j, k, a in got:
        assert strong[(int(j), int(k))] == int(a)
    pairs = {(int(j), int(k)) for j, k, _ in got}
    assert (40, 41) in pairs and (3, 300) in pairs
    s = {(int(j), int(k)): (2 * int(a) - n) / n for j, k, a in got}
    assert s[(40, 41)] < 0 < s[(3, 300)]


def test_kkt_rule_matches_float_definition(orc):
    X, rng = _X(120, 70, 22)
    r = rng.normal(size=120) + 1.5 * X[:, 2] * X[:, 60] - 1.2 * X[:, 10] * X[:, 11]
    r = r - r.mean()                                       # a centred residual
    dots = (X.T.astype(np.float64) @ (X.astype(np.float64) * r[:, None])) / 120
    for lam in (0.2, 0.4, 0.7):
        got, d = orc.kkt_brute(X, r, lam)
        want = [(j, k) for j in range(70) for k in range(j + 1, 70) if abs(dots[j, k]) > lam]
        # the fixed-point rule agrees with the float definition except within
        # 2^-24 max|r| n of the boundary (none here)
        near = [abs(abs(dots[j, k]) - lam) for j in range(70) for k in range(j + 1, 70)]
        assert min(near) > 1e-5
        assert [tuple(v[:2]) for v in got] == want
        _, e = np.frexp(np.abs(r).max())
        assert np.allclose(d * 2.0 ** (int(e) - 24) / 120, [dots[j, k] for j, k, _ in got], atol=1e-5)
    xs, dx = orc.kkt_xyz(X, r, 40, 4, 0.4, 9)
    bf, db = orc.kkt_brute(X, r, 0.4)
    bset = {(int(j), int(k)): int(v) for (j, k, _), v in zip(bf, db)}
    for (j, k, _), v in zip(xs, dx):
        assert bset[(int(j), int(k))] == int(v)
    assert {(2, 60), (10, 11)} <= {(int(j), int(k)) for j, k, _ in xs}


def test_sign_transform_definition(orc):
    rng = np.random.default_rng(30)
    X = rng.normal(size=(50, 40)).astype(np.float32)
    X[rng.random((50, 40)) < 0.3] = 0.0
    T = orc.sign_transform(X, coin_seed=77)
    nz = X != 0
    assert np.array_equal(T[nz], np.sign(X[nz]).astype(np.int8))
    # zeros: the top bit of splitmix64 output t = j*n + i
    ii, jj = np.nonzero(~nz)
    want = [(-1 if orc.splitmix64_at(77, int(j) * 50 + int(i)) >> 63 else 1) for i, j in zip(ii, jj)]
    assert list(T[ii, jj]) == want
    assert 0.35 < np.mean(np.array(want) == -1) < 0.65
    with pytest.raises(ValueError):
        orc.sign_transform(np.full((3, 3), np.nan, np.float32))


def test_sign_transform_strength(orc):
    """Section 3.2: with the sign transform the weighted strength of (j, k) is
    1/2 + sum_i Y_i sgn(X_ij) sgn(X_ik) / (2 ||Y||_1)."""
    rng = np.random.default_rng(31)
    X = rng.standard_t(4, size=(400, 30)).astype(np.float32)
    Y = X[:, 3].astype(np.float64) * X[:, 7] + rng.normal(0, 0.5, size=400)
    T = orc.sign_transform(X)
    for j, k in ((3, 7), (0, 1), (5, 20)):
        _, S = orc.weighted_agree(T, Y, j, k)
        q, _ = orc.quantize_y(Y)
        g = 0.5 + np.sum(Y * np.sign(X[:, j]) * np.sign(X[:, k])) / (2 * np.abs(Y).sum())
        assert abs(S / q.sum() - g) < 1e-6


def test_unbiased_transform_is_unbiased_and_matches_proposition(orc):
    """Section 3.2: the transform has E X~ = X' (Proposition 'unbiased') and a
    match probability 1/2 + sum_i Y'_i X'_ij X'_ik / (2 ||Y'||_1) under
    |Y'|-weighted row draws (the proposition on transformed strengths)."""
    rng = np.random.default_rng(50)
    n, p = 6, 3
    X = rng.uniform(-2, 2, size=(n, p)).astype(np.float32)
    Y = rng.normal(size=n)
    Xs, Ys = orc.unbiased_scale(X, Y)
    assert np.all(np.abs(Xs) <= 1) and np.allclose(np.abs(Xs).max(axis=1), 1)
    nu = np.abs(X).max(axis=1).astype(np.float64)
    assert np.allclose(Ys, Y * nu * nu)
    # unbiasedness of the per-draw transform, entry by entry
    R = 6000
    for i, j in ((0, 0), (3, 1), (5, 2)):
        v = [orc.unbiased_draw(Xs, 9, r, 1, 0, i, j) for r in range(R)]
        assert abs(np.mean(v) - Xs[i, j]) < 5 / np.sqrt(R)
    # match probability of (0, 1) with |Y'| weighted rows
    q, sgn = orc.quantize_y(Ys)
    hits = 0
    T = 20000
    rows = orc.draw_rows_weighted(q, 11, 0, T)
    for t, i in enumerate(rows):
        a = orc.unbiased_draw(Xs, 11, 0, T, t, int(i), 0)
        b = orc.unbiased_draw(Xs, 11, 0, T, t, int(i), 1)
        hits += int(a * b == sgn[i])
    gamma = 0.5 + np.sum(Ys * Xs[:, 0].astype(np.float64) * Xs[:, 1]) / (2 * np.abs(Ys).sum())
    assert abs(hits / T - gamma) < 5 * np.sqrt(gamma * (1 - gamma) / T)


def test_unbiased_search_subset_of_exact_screen(orc):
    rng = np.random.default_rng(51)
    n, p = 200, 120
    X = rng.uniform(-1, 1, size=(n, p)).astype(np.float32)
    Y = X[:, 3].astype(np.float64) * X[:, 90] + rng.normal(0, 0.05, size=n)
    pairs, dots = orc.xyz_unbiased_range(X, Y, 0, 60, 6, 0.3, 4)
    Xs, Ys = orc.unbiased_scale(X, Y)
    G = Xs.T.astype(np.float64) @ (Xs.astype(np.float64) * Ys[:, None])
    thr = 0.3 * np.abs(Ys).sum()
    for (j, k), d in zip(pairs, dots):
        assert abs(G[j, k] - d) < 1e-9 * np.abs(Ys).sum() and d >= thr
    assert (3, 90) in {(int(j), int(k)) for j, k in pairs}
