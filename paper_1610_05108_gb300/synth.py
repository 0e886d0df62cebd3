"""Seeded synthetic inputs for the xyz search.

This module only makes inputs: +-1 matrices X (n x p, column-major int8) and
responses Y (n int8) with planted interaction pairs.  It holds none of the
search's arithmetic (no keys, no grouping, no verification), and both the
CUDA path and the CPU oracle are fed from it.

Workload recipes (all values +-1, bit(v) = 1 iff v = -1 is never used here):

* ``iid``: X_ij i.i.d. uniform on {-1, +1}; Y_i = X_i0 X_i1 flipped with
  probability ``flip`` (the binary example of Section 1 with label noise).
* ``gwas``: SNP-shaped columns.  Per row, a latent AR(1) chain over columns
  u_j = rho u_{j-1} + sqrt(1 - rho^2) e_j, restarted at every block of
  ``block`` columns; each column has a minor frequency f_j ~ U[fmin, fmax] and
  X_ij = -1 iff Phi(u_ij) < f_j.  Planted pairs take their columns from
  distinct blocks among columns with f_j >= 0.35.  The response is chosen so
  that the planted products P_t = X_a_t o X_b_t reach strengths
  lambda * target_t with the largest feasible lambda: a linear programme over
  the 2^T sign patterns of (P_1..P_T) gives the fraction of +1 responses in
  each pattern, which is then allocated exactly (the targets of a stated set
  can exceed what one response can realise, because near-orthogonal products
  obey Bessel's inequality sum_t s_t^2 <= 1).  Main effects are planted last
  by copying Y into a random fraction beta_m of the rows of a few other
  columns.  Realised strengths s_t = Y^T P_t / n are recorded.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_STREAMS = {"X": 1, "Y": 2, "plant": 3, "main": 4, "multi": 5, "inst": 6, "serve": 7}


def rng_for(seed: int, stream: str) -> np.random.Generator:
    """Independent numpy generator for (seed, named stream)."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), _STREAMS[stream]])))


@dataclass
class Dataset:
    """One synthetic problem: X (n, p) column-major int8, Y (n,) int8."""

    X: np.ndarray
    Y: np.ndarray
    planted: list = field(default_factory=list)     # [(j, k)] with j < k
    strengths: list = field(default_factory=list)   # realised Y^T(X_j o X_k)/n
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.X.shape[0]

    @property
    def p(self) -> int:
        return self.X.shape[1]


def _realised(X: np.ndarray, Y: np.ndarray, pairs) -> list:
    y = Y.astype(np.int64)
    n = X.shape[0]
    return [float(np.dot(y, X[:, a].astype(np.int64) * X[:, b].astype(np.int64)) / n) for a, b in pairs]


# --------------------------------------------------------------------- iid

def iid(n: int, p: int, seed: int, flip: float = 0.1, pair=(0, 1)) -> Dataset:
    """X iid uniform +-1; Y = X_a o X_b with each sign flipped w.p. ``flip``."""
    rx = rng_for(seed, "X")
    X = np.asfortranarray((rx.integers(0, 2, size=(n, p), dtype=np.int8) * 2 - 1).astype(np.int8))
    ry = rng_for(seed, "Y")
    a, b = pair
    Y = (X[:, a].astype(np.int16) * X[:, b]).astype(np.int8)
    flips = ry.random(n) < flip
    Y[flips] = -Y[flips]
    Y = np.ascontiguousarray(Y, dtype=np.int8)
    planted = [tuple(sorted(pair))]
    return Dataset(X, Y, planted, _realised(X, Y, planted),
                   {"recipe": "iid", "flip": flip, "seed": seed})


def iid_noise_only(n: int, p: int, seed: int) -> Dataset:
    """X and Y i.i.d. uniform +-1 with nothing planted."""
    rx = rng_for(seed, "X")
    X = np.asfortranarray((rx.integers(0, 2, size=(n, p), dtype=np.int8) * 2 - 1).astype(np.int8))
    Y = (rng_for(seed, "Y").integers(0, 2, size=n, dtype=np.int8) * 2 - 1).astype(np.int8)
    return Dataset(X, Y, [], [], {"recipe": "iid_noise", "seed": seed})


# -------------------------------------------------------------------- gwas

def _ndtri(f: np.ndarray) -> np.ndarray:
    from scipy.special import ndtri
    return ndtri(f)


def gwas_X(n: int, p: int, rng: np.random.Generator, block: int = 20, rho: float = 0.6,
           fmin: float = 0.05, fmax: float = 0.5, chunk_cols: int = 10000, workers: int = 0):
    """SNP-shaped +-1 matrix (latent AR(1) in blocks, minor frequency f_j).

    Columns are made in chunks of whole blocks; chunk i draws its normals
    from its own generator, seeded by the i-th of a list of seeds drawn from
    ``rng``, so the chunks are made by ``workers`` threads (0: one per core)
    and the result depends only on ``rng``."""
    import concurrent.futures as cf
    import os

    f = rng.uniform(fmin, fmax, size=p)
    thr = _ndtri(f).astype(np.float32)
    X = np.empty((n, p), dtype=np.int8, order="F")
    s = np.float32(math.sqrt(1.0 - rho * rho))
    rho32 = np.float32(rho)
    chunk_cols = max(block, (chunk_cols // block) * block)
    starts = list(range(0, p, chunk_cols))
    seeds = rng.integers(0, 2**63 - 1, size=len(starts), dtype=np.int64)

    def one(i):
        c0 = starts[i]
        c1 = min(p, c0 + chunk_cols)
        g = np.random.Generator(np.random.PCG64(int(seeds[i])))
        e = g.standard_normal(size=(c1 - c0, n), dtype=np.float32)  # column-major rows
        # the chain restarts at every block start (c0 is one); step all blocks
        # of the chunk together, one position within the block at a time
        nb = -(-(c1 - c0) // block)
        u = np.zeros((nb * block, n), dtype=np.float32)
        u[: c1 - c0] = e
        del e
        u = u.reshape(nb, block, n)
        for t in range(1, block):
            u[:, t] = rho32 * u[:, t - 1] + s * u[:, t]
        u = u.reshape(nb * block, n)[: c1 - c0]
        X[:, c0:c1] = np.where(u < thr[c0:c1, None], np.int8(-1), np.int8(1)).T

    nw = workers or min(16, os.cpu_count() or 1)
    if nw <= 1 or len(starts) == 1:
        for i in range(len(starts)):
            one(i)
    else:
        with cf.ThreadPoolExecutor(max_workers=nw) as ex:
            list(ex.map(one, range(len(starts))))
    return X, f


def _pick_planted(f: np.ndarray, count: int, block: int, rng: np.random.Generator, exclude=()):
    """``count`` disjoint pairs whose 2*count columns lie in distinct blocks
    and have minor frequency >= 0.35."""
    p = len(f)
    ok = np.flatnonzero(f >= 0.35)
    ok = np.setdiff1d(ok, np.asarray(list(exclude), dtype=np.int64))
    rng.shuffle(ok)
    used_blocks, cols = set(), []
    for c in ok:
        b = int(c) // block
        if b in used_blocks:
            continue
        used_blocks.add(b)
        cols.append(int(c))
        if len(cols) == 2 * count:
            break
    if len(cols) < 2 * count:
        raise ValueError(f"p={p} too small to plant {count} pairs")
    return [tuple(sorted((cols[2 * t], cols[2 * t + 1]))) for t in range(count)]


def plant_response(X: np.ndarray, pairs, targets, rng: np.random.Generator, balance: bool = False):
    """Response whose products with the planted pairs reach lambda * targets
    for the largest feasible lambda (<= 1), allocated exactly per pattern.

    ``balance`` adds the constraint sum_i Y_i = 0 (up to rounding): on
    SNP-shaped columns an unbalanced response makes every pair of nearly
    constant columns (both of low minor frequency) look like an interaction
    of strength about mean(Y)."""
    from scipy.optimize import linprog

    n = X.shape[0]
    T = len(pairs)
    targets = np.asarray(targets, dtype=np.float64)
    P = np.stack([X[:, a].astype(np.int8) * X[:, b] for a, b in pairs], axis=1)  # n x T
    code = ((P < 0).astype(np.int64) << np.arange(T)).sum(axis=1)
    counts = np.bincount(code, minlength=1 << T).astype(np.float64)
    # pattern index c has bit t set iff P_t = -1
    pats = np.array([[(-1.0 if (c >> t) & 1 else 1.0) for t in range(T)] for c in range(1 << T)])
    mu = counts / n
    nv = 1 << T
    # variables: y(c) in [-1, 1] for each pattern, lambda in [0, 1]
    c_obj = np.zeros(nv + 1)
    c_obj[-1] = -1.0
    A_eq = np.zeros((T + int(balance), nv + 1))
    A_eq[:T, :nv] = (pats * mu[:, None]).T
    A_eq[:T, nv] = -targets
    if balance:
        A_eq[T, :nv] = mu
    bounds = [(-1.0, 1.0)] * nv + [(0.0, 1.0)]
    res = linprog(c_obj, A_eq=A_eq, b_eq=np.zeros(len(A_eq)), bounds=bounds, method="highs")
    if not res.success:
        raise RuntimeError("planting LP failed: " + str(res.message))
    yv = res.x[:nv]
    lam = float(res.x[-1])
    Y = np.empty(n, dtype=np.int8)
    for c in range(nv):
        rows = np.flatnonzero(code == c)
        if len(rows) == 0:
            continue
        plus = int(round(len(rows) * (1.0 + yv[c]) / 2.0))
        perm = rng.permutation(rows)
        Y[perm[:plus]] = 1
        Y[perm[plus:]] = -1
    return Y, lam


def plant_main_effects(X: np.ndarray, Y: np.ndarray, cols, betas, rng: np.random.Generator):
    """Copy Y into a fraction beta_m of the rows of column m (in place)."""
    n = X.shape[0]
    for m, beta in zip(cols, betas):
        rows = rng.random(n) < beta
        X[rows, m] = Y[rows]


def gwas(n: int, p: int, seed: int, targets=(0.2, 0.3, 0.4, 0.5, 0.6), n_main: int = 10,
         main_range=(0.1, 0.3), block: int = 20, rho: float = 0.6,
         fmin: float = 0.05, fmax: float = 0.5) -> Dataset:
    """GWAS-shaped binary problem with planted pairs and main effects."""
    rx = rng_for(seed, "X")
    X, f = gwas_X(n, p, rx, block=block, rho=rho, fmin=fmin, fmax=fmax)
    rp = rng_for(seed, "plant")
    pairs = _pick_planted(f, len(targets), block, rp)
    Y, lam = plant_response(X, pairs, targets, rng_for(seed, "Y"))
    planted_cols = {c for pr in pairs for c in pr}
    rm = rng_for(seed, "main")
    cand = np.setdiff1d(np.arange(p), np.asarray(sorted(planted_cols)))
    main_cols = rm.choice(cand, size=min(n_main, len(cand)), replace=False)
    betas = rm.uniform(main_range[0], main_range[1], size=len(main_cols))
    plant_main_effects(X, Y, main_cols, betas, rm)
    Y = np.ascontiguousarray(Y, dtype=np.int8)
    return Dataset(X, Y, pairs, _realised(X, Y, pairs),
                   {"recipe": "gwas", "seed": seed, "targets": list(map(float, targets)),
                    "lambda": lam, "main_cols": [int(c) for c in main_cols],
                    "main_betas": [float(b) for b in betas], "block": block, "rho": rho,
                    "fmin": fmin, "fmax": fmax})


# ------------------------------------------------------------ named configs

def config_small(seed: int = 1) -> Dataset:
    """n=200, p=2000, X iid +-1, Y = X_0 o X_1 flipped w.p. 0.1."""
    return iid(200, 2000, seed, flip=0.1, pair=(0, 1))


def config_gwas(seed: int = 1) -> Dataset:
    """n=2000, p=100000 SNP-shaped columns, 5 planted pairs, 10 main effects."""
    return gwas(2000, 100000, seed)


def config_gwas_large(seed: int = 1) -> Dataset:
    """n=4000, p=1,000,000 SNP-shaped columns, 10 planted pairs U[0.15,0.5]."""
    r = rng_for(seed, "plant")
    targets = tuple(float(t) for t in r.uniform(0.15, 0.5, size=10))
    return gwas(4000, 1000000, seed, targets=targets)


def extra_responses(X: np.ndarray, count: int, seed: int, pairs_per_y: int = 3,
                    target_range=(0.3, 0.5), flip_noise: float = 0.0, balance: bool = False):
    """``count`` further responses for one X, each with its own planted pairs.

    Returns (Ys (count, n) int8, planted [[(j, k)]], realised [[s]])."""
    n, p = X.shape
    r = rng_for(seed, "multi")
    Ys = np.empty((count, n), dtype=np.int8)
    planted, real = [], []
    for b in range(count):
        cols = r.choice(p, size=2 * pairs_per_y, replace=False)
        pairs = [tuple(sorted((int(cols[2 * t]), int(cols[2 * t + 1])))) for t in range(pairs_per_y)]
        targets = r.uniform(target_range[0], target_range[1], size=pairs_per_y)
        Y, _ = plant_response(X, pairs, targets, r, balance=balance)
        if flip_noise > 0:
            fl = r.random(n) < flip_noise
            Y[fl] = -Y[fl]
        Ys[b] = Y
        planted.append(pairs)
        real.append(_realised(X, Y, pairs))
    return Ys, planted, real


def instance_sizes(count: int, seed: int, n_range=(500, 8000), p_range=(10000, 500000)):
    """Log-uniform (n, p) for independent instances."""
    r = rng_for(seed, "inst")
    ns = np.exp(r.uniform(math.log(n_range[0]), math.log(n_range[1]), size=count)).astype(np.int64)
    ps = np.exp(r.uniform(math.log(p_range[0]), math.log(p_range[1]), size=count)).astype(np.int64)
    return [(int(a), int(b)) for a, b in zip(ns, ps)]


def poisson_arrivals(count: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson stream with mean ``rate`` per second."""
    r = rng_for(seed, "serve")
    return np.cumsum(r.exponential(1.0 / rate, size=count))


def single_pair_responses(X: np.ndarray, f: np.ndarray, count: int, seed: int,
                          gammas=(0.7, 0.8, 0.9), block: int = 20):
    """``count`` balanced responses for one X, each with one planted pair
    whose interaction strength gamma = a/n is drawn from ``gammas`` (the
    scaling experiment of Section 5.2 plants one pair of gamma in {0.7, 0.8,
    0.9}).

    Returns (Ys (count, n) int8, pairs [(j, k)], realised [Y^T(X_j o X_k)/n])."""
    n, _ = X.shape
    r = rng_for(seed, "multi")
    Ys = np.empty((count, n), dtype=np.int8)
    pairs, real = [], []
    for b in range(count):
        pr = _pick_planted(f, 1, block, r)
        g = float(r.choice(np.asarray(gammas, dtype=np.float64)))
        Y, _ = plant_response(X, pr, [2.0 * g - 1.0], r, balance=True)
        Ys[b] = Y
        pairs.append(pr[0])
        real.append(_realised(X, Y, pr)[0])
    return Ys, pairs, real


def serve_requests(count: int, rate: float, seed: int, datasets: int, responses: int,
                   L_range=(20, 200), kappa_range=(0.2, 0.6)):
    """A Poisson request stream over resident datasets: per request the
    arrival time (s), dataset index, response index, L (uniform integer in
    L_range), kappa (uniform in kappa_range) and search seed."""
    r = rng_for(seed, "serve")
    t = np.cumsum(r.exponential(1.0 / rate, size=count))
    ds = r.integers(0, datasets, size=count)
    ys = r.integers(0, responses, size=count)
    Ls = r.integers(L_range[0], L_range[1] + 1, size=count)
    ks = r.uniform(kappa_range[0], kappa_range[1], size=count)
    seeds = r.integers(0, 2**62, size=count)
    return [dict(t=float(t[i]), dataset=int(ds[i]), response=int(ys[i]), L=int(Ls[i]),
                 kappa=float(ks[i]), seed=int(seeds[i])) for i in range(count)]
