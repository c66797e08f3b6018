"""The seeded input recipes (paper_2604_23826_gb300/inputs.py) on the host: they hold no
statistics of the method, only the draws both sides read, so what is checked here is that
they are reproducible and have the structure they claim."""
import numpy as np
import pytest

from paper_2604_23826_gb300 import inputs


def test_correlated_rows_do_not_depend_on_chunking():
    """Any row range equals the same rows of one long draw (row blocks are seeded by (seed, b))."""
    L, mu = inputs.wide_factor(6, 10)
    whole = inputs.gen_correlated_host(200_000, L, mu, seed=9)
    cuts = [0, 1, 65_535, 65_536, 65_537, 131_072, 150_001, 200_000]
    parts = [inputs.gen_correlated_host(b - a, L, mu, seed=9, row0=a) for a, b in zip(cuts, cuts[1:])]
    assert np.array_equal(np.concatenate(parts, axis=1), whole)
    assert not np.array_equal(inputs.gen_correlated_host(1000, L, mu, seed=10), whole[:, :1000])


@pytest.mark.parametrize("p", [4, 24])
def test_wide_factor_spectrum_and_sample_covariance(p):
    """L L^T has eigenvalues exactly 1/k (k = 1..p) up to rounding, and the sample covariance of
    the generated rows approaches it within a few standard errors."""
    L, mu = inputs.wide_factor(3, p)
    ev = np.sort(np.linalg.eigvalsh(L @ L.T))[::-1]
    assert np.allclose(ev, 1.0 / np.arange(1, p + 1), rtol=0, atol=1e-12)
    assert np.all((mu >= 0) & (mu <= 1e3))
    n = 400_000
    X = inputs.gen_correlated_host(n, L, mu, seed=1)
    C = np.cov(X)
    se = np.sqrt((np.diag(L @ L.T)[:, None] * np.diag(L @ L.T)[None, :] + (L @ L.T) ** 2) / n)
    assert np.all(np.abs(C - L @ L.T) <= 6 * se)
    assert np.all(np.abs(X.mean(axis=1) - mu) <= 6 * np.sqrt(np.diag(L @ L.T) / n))


def test_many_tables_shapes():
    """Row counts log-uniform in [1e3, 1e7), widths from {8, 16, 32, 64}, means and spreads in
    their ranges; the same seed gives the same shapes."""
    a = inputs.many_tables_shapes(3, 512)
    b = inputs.many_tables_shapes(3, 512)
    assert all(x[0] == y[0] and x[1] == y[1] and np.array_equal(x[2], y[2]) and np.array_equal(x[3], y[3])
               for x, y in zip(a, b))
    ns = np.array([t[0] for t in a])
    ps = {t[1] for t in a}
    assert ns.min() >= 1000 and ns.max() < 10 ** 7 and ps <= {8, 16, 32, 64} and len(ps) == 4
    assert abs(np.median(np.log10(ns)) - 5.0) < 0.3
    for n, p, mu, sd in a[:20]:
        assert mu.shape == (p,) and np.all((mu >= 1e3) & (mu <= 1e5)) and np.all((sd >= 0.1) & (sd <= 10))
    groups = inputs.waves(a, 4 * 10 ** 9)
    assert sorted(t for g in groups for t in g) == list(range(512))
