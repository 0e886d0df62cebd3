"""Seeded synthetic inputs: shapes, +-1 values, determinism, and that the
recorded planted strengths are what the oracle measures."""
import numpy as np

from paper_1610_05108_gb300 import synth


def test_small_config_shape_and_strength(orc):
    d = synth.config_small(1)
    assert d.X.shape == (200, 2000) and d.X.flags.f_contiguous and d.X.dtype == np.int8
    assert set(np.unique(d.X)) == {-1, 1} and set(np.unique(d.Y)) <= {-1, 1}
    (j, k), = d.planted
    assert (j, k) == (0, 1)
    a = orc.agree(d.X, d.Y, j, k)
    assert abs((2 * a - d.n) / d.n - d.strengths[0]) < 1e-12
    # flips w.p. 0.1: strength near 0.8
    assert 0.6 < d.strengths[0] < 0.95


def test_generators_are_deterministic():
    a = synth.gwas(300, 4000, 5)
    b = synth.gwas(300, 4000, 5)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.Y, b.Y)
    assert a.planted == b.planted


def test_gwas_planted_strengths_recorded(orc):
    d = synth.gwas(600, 6000, 3)
    assert len(d.planted) == 5
    for (j, k), s in zip(d.planted, d.strengths):
        a = orc.agree(d.X, d.Y, j, k)
        assert abs((2 * a - d.n) / d.n - s) < 1e-12
    # realised strengths follow the targets' order (lambda-scaled)
    assert d.strengths == sorted(d.strengths)
    lam = d.meta["lambda"]
    for s, t in zip(d.strengths, d.meta["targets"]):
        assert abs(s - lam * t) < 0.05
    # columns of a block are positively correlated, minor allele is -1
    assert (d.X == -1).mean() < 0.5
