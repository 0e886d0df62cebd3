"""Pins of the CPU oracle against facts fixed by the paper or by mathematics.

Each test checks the oracle against something other than itself: a worked
example printed in the paper, a closed form, an identity evaluated with a
library routine (numpy matrix products), a brute-force definition on tiny
inputs, or a binomial law the paper states.  A plausible slip in the oracle
(a dropped term, a wrong sign or index, sampling without replacement, a
transposed operand, a missing colour check) fails at least one of them.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_pm1(rng, *shape):
    return (rng.integers(0, 2, size=shape, dtype=np.int8) * 2 - 1).astype(np.int8)


def _pairs_set(arr):
    return {tuple(int(v) for v in row[:2]) for row in arr}


# ------------------------------------------------------------------ stream

def test_splitmix64_published_first_outputs(orc):
    # splitmix64 (Steele, Lea & Flood 2014) started from state 0: the first
    # outputs of the published reference generator.
    assert orc.splitmix64_at(0, 0) == 0xE220A8397B1DCDAF
    assert orc.splitmix64_at(0, 1) == 0x6E789E6AA1B965F4
    assert orc.splitmix64_at(0, 2) == 0x06C45D188009454F


def test_rows_uniform_with_replacement(orc):
    # eq. projR, subsampling class: i.i.d. uniform indices with replacement.
    n, M, runs = 37, 16, 4000
    rows = np.concatenate([orc.draw_rows(12345, l, M, n) for l in range(runs)])
    assert rows.min() >= 0 and rows.max() < n
    counts = np.bincount(rows, minlength=n)
    exp = len(rows) / n
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    # chi-square with n-1 = 36 dof: mean 36, sd ~8.5; 5 sd bound
    assert chi2 < 36 + 5 * math.sqrt(72)
    # with replacement: a run of M draws from n rows repeats a row with
    # probability 1 - n!/((n-M)! n^M)
    p_nodup = math.prod((n - m) / n for m in range(M))
    dup = np.mean([len(set(orc.draw_rows(999, l, M, n).tolist())) < M for l in range(runs)])
    sd = math.sqrt(p_nodup * (1 - p_nodup) / runs)
    assert abs(dup - (1 - p_nodup)) < 5 * sd


# ---------------------------------------------------------------- strength

@pytest.mark.parametrize("n,p,seed", [(97, 23, 1), (64, 17, 2), (1, 5, 3), (33, 2, 4)])
def test_agreement_equivalence_identity(orc, n, p, seed):
    # eq. equiv: 2 gamma_jk - 1 = Y^T(X_j o X_k)/n = Z_j^T X_k / n
    #            = 1 - ||Z_j - X_k||^2 / (2n), with Z = Y o X.
    rng = np.random.default_rng(seed)
    X = np.asfortranarray(_rand_pm1(rng, n, p))
    Y = _rand_pm1(rng, n)
    Xf = X.astype(np.float64)
    Z = Xf * Y[:, None]
    G = Xf.T @ (Y[:, None] * Xf)           # Y^T (X_j o X_k)
    H = Z.T @ Xf                           # Z_j^T X_k
    for j in range(p):
        for k in range(p):
            a = orc.agree(X, Y, j, k)
            assert 2 * a - n == G[j, k] == H[j, k]
            dist2 = float(((Z[:, j] - Xf[:, k]) ** 2).sum())
            assert 2 * a - n == n - dist2 / 2


@pytest.mark.parametrize("kappa", [0.0, 0.25, 0.5, -0.5, 1.0, -1.0])
def test_brute_force_matches_matrix_product(orc, kappa):
    # eq. inter_search1 (with >=): keep j < k with Y^T(X_j o X_k)/n >= kappa.
    rng = np.random.default_rng(7)
    n, p = 80, 30
    X = np.asfortranarray(_rand_pm1(rng, n, p))
    Y = _rand_pm1(rng, n)
    # plant a strong pair so the high thresholds are not empty
    Y[:] = X[:, 3] * X[:, 11]
    Y[:8] = -Y[:8]
    Xf = X.astype(np.float64)
    G = Xf.T @ (Y[:, None] * Xf)
    want = {(j, k) for j in range(p) for k in range(j + 1, p)
            if Fraction(int(G[j, k])) >= Fraction(kappa) * n}
    got = orc.brute_force(X, Y, kappa)
    assert _pairs_set(got) == want
    for j, k, a in got:
        assert 2 * a - n == G[j, k]
    assert np.all(got[:, 0] < got[:, 1])


def test_amin_matches_exact_rational_rule(orc):
    # reading R5: least a with 2a - n >= kappa * n.  For dyadic kappa the
    # product kappa*n is exact in binary64, so the rule equals the exact one.
    for n in [1, 2, 7, 200, 859, 2000, 4001]:
        for kappa in [-1.0, -0.75, -0.5, -0.125, 0.0, 0.0625, 0.25, 0.5, 0.75, 0.96875, 1.0]:
            exact = next((a for a in range(n + 1)
                          if Fraction(2 * a - n) >= Fraction(kappa) * n), n + 1)
            assert orc.amin(n, kappa) == exact, (n, kappa)
    rng = np.random.default_rng(1)
    for _ in range(300):
        n = int(rng.integers(1, 5000))
        kappa = float(rng.uniform(-1, 1))
        exact = math.ceil((Fraction(kappa) * n + n) / 2)
        exact = min(max(exact, 0), n + 1)
        got = orc.amin(n, kappa)
        if got != exact:  # may differ only where kappa*n rounds across an integer
            assert abs(kappa * n - round(kappa * n)) < 1e-9


# ------------------------------------------------------ equal-pairs search

def test_figure2_worked_example(orc):
    fx = json.load(open(os.path.join(GOLDEN, "fig2_equal_pairs.json")))
    want = {tuple(e) for e in fx["expected_pairs_1based"]}
    x = np.array(fx["x"], dtype=np.float64)
    z = np.array(fx["z"], dtype=np.float64)
    got = orc.equal_pairs(x, z)
    assert {(int(j) + 1, int(k) + 1) for j, k in got} == want
    assert len(got) == len(want)
    # the same placement as integer keys
    xi = np.round(x * 100).astype(np.uint64)
    zi = np.round(z * 100).astype(np.uint64)
    got = orc.equal_pairs(xi, zi)
    assert {(int(j) + 1, int(k) + 1) for j, k in got} == want


def test_equal_pairs_brute_force(orc):
    rng = np.random.default_rng(3)
    for _ in range(20):
        p = int(rng.integers(1, 40))
        x = rng.integers(0, 6, size=p).astype(np.uint64)
        z = rng.integers(0, 6, size=p).astype(np.uint64)
        want = {(j, k) for j in range(p) for k in range(p) if x[j] == z[k]}
        got = orc.equal_pairs(x, z)
        assert len(got) == len(want)
        assert {tuple(map(int, r)) for r in got} == want


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_candidates_are_pairs_equal_on_sampled_rows(orc, seed):
    # Section 2 (remark on minimal subsampling with tau = 0): the close pairs
    # are exactly the (j, k) with X_{i_m j} = Z_{i_m k} for all m.
    rng = np.random.default_rng(seed)
    n, p, M = 50, 30, 4
    X = np.asfortranarray(_rand_pm1(rng, n, p))
    Y = _rand_pm1(rng, n)
    X[:, 5] = X[:, 9] * Y           # a perfect pair
    for run in range(6):
        rows = orc.draw_rows(seed * 100, run, M, n)
        Xs = X[rows, :].astype(np.int64)            # M x p
        Zs = Xs * Y[rows, None]
        eq = np.all(Xs[:, :, None] == Zs[:, None, :], axis=0)   # eq[j,k]: X_j = Z_k on S
        want = {(min(j, k), max(j, k)) for j, k in zip(*np.nonzero(eq)) if j != k}
        got = orc.candidates(X, Y, M, seed * 100, run)
        assert _pairs_set(got) == want
        assert (5, 9) in want


@pytest.mark.parametrize("seed", [4, 5])
def test_real_projection_gives_the_same_equal_pairs(orc, seed):
    # the projection step of Algorithm 2 with F = U[0,1]: the real projection and the integer
    # keys of the sampled bits give the same equal pairs (Section 2.2: any
    # continuous F gives identical results).
    rng = np.random.default_rng(seed)
    n, p, M = 40, 25, 3
    X = np.asfortranarray(_rand_pm1(rng, n, p))
    Y = _rand_pm1(rng, n)
    for run in range(8):
        rows = orc.draw_rows(seed, run, M, n)
        D = rng.uniform(0, 1, size=M)
        xr, zr = orc.project_real(X, Y, rows, D)
        xi, zi = orc.keys(X, Y, rows)
        a = {tuple(map(int, r)) for r in orc.equal_pairs(xr, zr)}
        b = {tuple(map(int, r)) for r in orc.equal_pairs(xi, zi)}
        assert a == b


# ---------------------------------------------------------- whole search

def test_M0_reduces_to_brute_force(orc):
    # eq. projR with M = 0 gives R = 0, so every pair is an equal pair and one
    # run verifies all of them: xyz(M=0, L=1) is the naive search.
    rng = np.random.default_rng(11)
    n, p = 70, 40
    X = np.asfortranarray(_rand_pm1(rng, n, p))
    Y = _rand_pm1(rng, n)
    for kappa in [0.0, 0.2, -0.3]:
        a = orc.xyz(X, Y, 1, 0, kappa, 5)
        b = orc.brute_force(X, Y, kappa)
        assert np.array_equal(a, b)


def test_perfect_interaction_found_every_run(orc):
    # Section 2: if Y = X_j o X_k then X_j = Z_k and the pair collides under
    # every projection (gamma = 1 is retained with probability 1).
    rng = np.random.default_rng(12)
    n, p = 60, 50
    X = np.asfortranarray(_rand_pm1(rng, n, p))
    Y = (X[:, 7] * X[:, 31]).astype(np.int8)
    assert orc.agree(X, Y, 7, 31) == n
    for run in range(40):
        assert (7, 31) in _pairs_set(orc.candidates(X, Y, 12, 77, run))
    res = orc.xyz(X, Y, 3, 12, 0.99, 77)
    assert (7, 31) in _pairs_set(res)


def test_xyz_is_subset_of_brute_force(orc):
    # the verification step of Algorithm 2: I only holds verified pairs, with their exact counts.
    rng = np.random.default_rng(13)
    n, p = 100, 120
    X = np.asfortranarray(_rand_pm1(rng, n, p))
    Y = (X[:, 0] * X[:, 1]).astype(np.int8)
    Y[:15] = -Y[:15]
    bf = {(j, k): a for j, k, a in orc.brute_force(X, Y, 0.2)}
    res = orc.xyz(X, Y, 30, 6, 0.2, 3)
    assert len(res) > 0
    for j, k, a in res:
        assert bf[(j, k)] == a
    assert np.all(np.diff(res[:, 0].astype(np.int64) * p + res[:, 1]) > 0)


def test_single_run_retention_is_gamma_to_the_M(orc):
    # Section 2.3: a pair of strength gamma is in E_1 with probability gamma^M,
    # and E|E_1| = sum_{j,k} gamma_jk^M (proof of Theorem 2).  Checked over
    # many runs with a 5-sigma binomial / CLT bound.
    rng = np.random.default_rng(14)
    n, p, M, R = 40, 8, 3, 4000
    X = np.asfortranarray(_rand_pm1(rng, n, p))
    Y = _rand_pm1(rng, n)
    Y[:30] = X[:30, 0] * X[:30, 1]
    gam = {(j, k): orc.agree(X, Y, j, k) / n for j in range(p) for k in range(j + 1, p)}
    hits = {jk: 0 for jk in gam}
    sizes = []
    for run in range(R):
        cand = _pairs_set(orc.candidates(X, Y, M, 2024, run))
        sizes.append(len(cand))
        for jk in cand:
            hits[jk] += 1
    for jk, g in gam.items():
        q = g ** M
        sd = math.sqrt(R * q * (1 - q)) + 1e-9
        assert abs(hits[jk] - R * q) <= 5 * sd + 1, (jk, hits[jk], R * q)
    # unordered pairs j < k: E|E_1| = sum_{j<k} gamma_jk^M
    mean_size = float(np.mean(sizes))
    exp_size = sum(g ** M for g in gam.values())
    sd = float(np.std(sizes)) / math.sqrt(R)
    assert abs(mean_size - exp_size) <= 5 * sd + 1e-6


def test_discovery_probability_eta(orc):
    # eq. eta: a pair of strength gamma is in I with probability
    # 1 - (1 - gamma^M)^L.  Checked over independent seeds (5 sigma).
    rng = np.random.default_rng(15)
    n, p, M, L = 50, 12, 6, 4
    X = np.asfortranarray(_rand_pm1(rng, n, p))
    Y = (X[:, 2] * X[:, 9]).astype(np.int8)
    Y[:10] = -Y[:10]                                  # gamma = 0.8
    g = orc.agree(X, Y, 2, 9) / n
    eta = 1 - (1 - g ** M) ** L
    S = 600
    found = sum((2, 9) in _pairs_set(orc.xyz(X, Y, L, M, 0.5, s)) for s in range(S))
    sd = math.sqrt(S * eta * (1 - eta))
    assert abs(found - S * eta) <= 5 * sd


def test_range_union_equals_whole_search(orc):
    # Runs are independent (Algorithm 2 loop): the union of two run ranges is
    # the whole search.
    rng = np.random.default_rng(16)
    n, p = 60, 80
    X = np.asfortranarray(_rand_pm1(rng, n, p))
    Y = (X[:, 4] * X[:, 40]).astype(np.int8)
    Y[:6] = -Y[:6]
    whole = orc.xyz(X, Y, 12, 5, 0.1, 9)
    a = orc.xyz_range(X, Y, 0, 5, 5, 0.1, 9)
    b = orc.xyz_range(X, Y, 5, 12, 5, 0.1, 9)
    merged = sorted({tuple(r) for r in np.concatenate([a, b]).tolist()})
    assert merged == [tuple(r) for r in whole.tolist()]


def test_rejects_non_pm1(orc):
    X = np.asfortranarray(np.ones((5, 3), dtype=np.int8))
    Y = np.ones(5, dtype=np.int8)
    X[2, 1] = 0
    with pytest.raises(ValueError):
        orc.brute_force(X, Y, 0.0)


def test_agree_pairs_matches_single(orc):
    rng = np.random.default_rng(17)
    n, p = 45, 20
    X = np.asfortranarray(_rand_pm1(rng, n, p))
    Y = _rand_pm1(rng, n)
    j = rng.integers(0, p, size=50)
    k = rng.integers(0, p, size=50)
    Xf = X.astype(np.int64)
    want = [int(((Xf[:, a] * Xf[:, b]) == Y).sum()) for a, b in zip(j, k)]
    assert orc.agree_pairs(X, Y, j, k).tolist() == want
