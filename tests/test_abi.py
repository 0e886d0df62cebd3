"""The C ABI library: builds, loads without a GPU, exports every symbol that
include/xyz.h declares, and its host-only planner matches the paper's
printed arithmetic."""
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1610_05108_gb300 import build, xyz
    build.build()
    return xyz


def _declared():
    src = open(os.path.join(ROOT, "include", "xyz.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(xyz_[A-Za-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    so = lib.load()
    for name in names:
        assert hasattr(so, name), name
        assert name in lib.SIGNATURES, name
    assert set(lib.SIGNATURES) == set(names)


def test_amin_matches_oracle(lib, orc):
    rng = np.random.default_rng(0)
    for _ in range(500):
        n = int(rng.integers(1, 10000))
        kappa = float(rng.uniform(-1, 1)) if rng.random() < 0.8 else float(rng.choice([-1, 0, 0.5, 1]))
        assert lib.amin(n, kappa) == orc.amin(n, kappa)


def test_eta_luric_arithmetic(lib):
    # Section 5.3: with M* = 21 and L = 100 a pair of strength 0.85 is missed
    # with probability (1 - 0.85^21)^100, printed as "about 0.03" (0.0351).
    miss = 1 - lib.eta(0.85, 21, 100)
    assert abs(miss - 0.0351) < 5e-4
    assert round(miss, 2) in (0.03, 0.04)
    # gamma = 1 is always found (Section 2); gamma^0 = 1 too
    assert lib.eta(1.0, 30, 1) == 1.0
    assert lib.eta(0.3, 0, 1) == 1.0


def test_runs_for_recall_is_least_L(lib):
    # eq. L_choice: least L with 1 - (1 - beta)^L >= eta, checked by search
    for beta in [0.5, 0.1, 0.0123, 1e-3, 2.5e-5]:
        for eta_t in [0.5, 0.9, 0.95, 0.99]:
            L = lib.runs_for_recall(beta, eta_t)
            assert 1 - (1 - beta) ** L >= eta_t - 1e-12
            assert L == 1 or 1 - (1 - beta) ** (L - 1) < eta_t
    assert lib.runs_for_recall(0.0, 0.9) == -1
    assert lib.runs_for_recall(1.0, 0.9) == 1


def test_M_for_gamma0(lib):
    # Section 5.2 sets M so that gamma_0 = p^(-1/M) is about 0.55
    for p in [1000, 5000, 30000, 10**6]:
        M = lib.M_for_gamma0(p, 0.55)
        g0 = p ** (-1.0 / M)
        for Mo in (M - 1, M + 1):
            if Mo >= 1:
                assert abs(g0 - 0.55) <= abs(p ** (-1.0 / Mo) - 0.55) + 1e-12


def test_runtime_exponents_printed(lib):
    # Section 2.3: gamma = 0.9, gamma_0 = 0.55 gives exponent ~1.17; Section
    # 5.3: gamma = 0.85 gives p^1.27.  (Planner inputs, checked here so the
    # gamma_0 convention of M_for_gamma0 matches the paper's.)
    assert abs(1 + math.log(0.9) / math.log(0.55) - 1.176) < 1e-3
    assert abs(1 + math.log(0.85) / math.log(0.55) - 1.272) < 1e-3


def test_best_M_is_pareto_optimal(lib):
    # Proposition (Pareto): for any (M', L') with eta(M', L') >= eta(M*, L),
    # the cost C(M', L') is not smaller.  Checked over a grid with the same
    # plug-in strengths the planner used.
    rng = np.random.default_rng(1)
    n, p = 2000, 100000
    agree = (n * np.clip(rng.normal(0.5, 0.02, size=20000), 0, 1)).astype(np.int32)
    gamma = 0.7
    M, cost = lib.best_M(n, p, gamma, agree)
    assert 1 <= M <= 64

    def C(Mx, Lx):
        S = p * (p - 1) * np.mean((agree / n) ** Mx)
        return Lx * (Mx * p + p * math.log(p) + n * S)

    for L in [10, 100, 1000]:
        target = lib.eta(gamma, M, L)
        base = C(M, L)
        for Mo in range(1, 41):
            Lo = lib.runs_for_recall(gamma ** Mo, target) if target < 1 else 1
            if Lo < 0:
                continue
            # L' is the least with eta(M', L') >= target
            assert C(Mo, Lo) >= base * (1 - 1e-9) - (Mo * p + p * math.log(p)) * 2
