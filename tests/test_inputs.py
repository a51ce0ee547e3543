"""The synthetic workload recipes, pinned to what they are stated to be: counts and sizes of the
uneven batch, the distributions and layout order of the right-hand sides, boundaries, and
reproducibility from the seed. These generators are the only code the oracle and the GPU path
share; they hold no multigrid arithmetic."""

import numpy as np
import pytest

from paper_1108_2045_gb300 import inputs


def test_uneven_batch_recipe():
    ks, fs = inputs.uneven_batch(1024, seed=1)
    counts = [ks.count(k) for k in range(6, 11)]
    assert counts == [204, 206, 205, 202, 207]
    assert sum((2 ** k - 1) ** 2 for k in ks) == 286_840_320
    # exponents first, then each problem's interior in layout order, from one stream
    rng = np.random.default_rng(1)
    assert ks == [int(k) for k in rng.integers(6, 11, size=1024)]
    for k, f in zip(ks[:5], fs[:5]):
        n = 2 ** k
        assert f.shape == (n + 1, n + 1)
        np.testing.assert_array_equal(f[1:-1, 1:-1], rng.standard_normal((n - 1, n - 1)))
        assert not f[(0, -1), :].any() and not f[:, (0, -1)].any()
    big = np.concatenate([f[1:-1, 1:-1].ravel() for f in fs[:50]])
    assert abs(big.mean()) < 5e-3 and abs(big.std() - 1.0) < 5e-3


@pytest.mark.parametrize("ndim,n", [(2, 64), (3, 16)])
def test_uniform_and_normal_rhs_layout(ndim, n):
    inner = (slice(1, -1),) * ndim
    f = inputs.uniform_rhs(n, ndim, seed=7)
    np.testing.assert_array_equal(f[inner], np.random.default_rng(7).uniform(-1.0, 1.0, (n - 1,) * ndim))
    g = inputs.normal_rhs(n, ndim, seed=7)
    np.testing.assert_array_equal(g[inner], np.random.default_rng(7).standard_normal((n - 1,) * ndim))
    for a in (f, g):
        assert a.shape == (n + 1,) * ndim
        mask = np.ones(a.shape, dtype=bool)
        mask[inner] = False
        assert not a[mask].any()
    assert np.abs(f).max() <= 1.0


def test_benchmark_rhs_is_reproducible():
    a = inputs.uniform_rhs(256, 2, seed=0)
    b = inputs.uniform_rhs(256, 2, seed=0)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, inputs.uniform_rhs(256, 2, seed=1))


@pytest.mark.parametrize("ndim", [2, 3])
def test_sine_rhs_is_d_pi_squared_times_the_solution(ndim):
    n = 16
    u = inputs.sine_solution(n, ndim)
    f = inputs.sine_rhs(n, ndim)
    np.testing.assert_allclose(f, ndim * np.pi ** 2 * u, rtol=0, atol=1e-13)
    x = np.arange(n + 1) / n
    if ndim == 2:
        np.testing.assert_allclose(u, np.outer(np.sin(np.pi * x), np.sin(np.pi * x)), atol=1e-15)


def test_paper_poly_rhs_is_minus_the_laplacian_of_its_solution():
    # the continuous -Laplacian of u = -x^2 y^2 (1 - x^2)(1 - y^2), by symbolic-free central
    # differences on a fine grid: agreement to O(h^2)
    n = 256
    u = inputs.paper_poly_solution(n)
    f = inputs.paper_poly_rhs(n)
    h = 1.0 / n
    lap = (u[1:-1, 2:] + u[1:-1, :-2] + u[2:, 1:-1] + u[:-2, 1:-1] - 4 * u[1:-1, 1:-1]) / h ** 2
    assert np.abs(-lap - f[1:-1, 1:-1]).max() < 1e-4
