"""Seeded synthetic inputs for the HOMG solver and its tests.

This module holds no multigrid arithmetic: it only produces right-hand sides (and, for tests, the
continuous solutions they come from) on node grids of (n+1)^d nodes, n = 2^K, h = 1/n, indexed
[j, i] / [k, j, i] with x fastest. Boundary nodes are 0. Both the GPU path and the CPU oracle
consume these arrays; neither produces them.

Workloads (stand-ins for the paper's Poisson experiments of Sec. 4; the paper uses no dataset):
* ``sine_rhs``     f = d pi^2 prod_k sin(pi x_k), whose continuous solution is prod_k sin(pi x_k).
* ``uniform_rhs``  f iid uniform[-1, 1] over the interior nodes in layout order, numpy
                   ``default_rng(seed)`` (seed 0 for the 4097^2 benchmark grid).
* ``normal_rhs``   f iid N(0, 1), same ordering.
* ``grf_coefficient`` k = exp(g) on the node grid, g a stationary Gaussian random field with
                   variance sigma^2 and squared-exponential correlation exp(-r^2 / (2 ell^2)),
                   sampled exactly by circulant embedding (seed 2 and sigma = 1, ell = 0.05 for
                   the 2049^2 variable-coefficient workload).
* ``uneven_batch`` a batch of 2-D problems with sides 2^k + 1, k uniform on 6..10, f iid N(0, 1)
                   (seed 1 for the 1024-problem batch benchmark).
* ``paper_poly_rhs`` / ``paper_poly_solution``: the polynomial test problem of Sec. 4, converted
                   to A = -Laplacian (the paper states Laplacian(u) = f, so f here is minus the
                   paper's source and the solution is the paper's u).
"""

import numpy as np


def node_coords(n, ndim):
    """Coordinates x_k of every node, as a list of ndim broadcastable arrays ([..., i] = x)."""
    x = np.arange(n + 1, dtype=np.float64) / n
    if ndim == 2:
        return [x[None, :], x[:, None]]
    return [x[None, None, :], x[None, :, None], x[:, None, None]]


def _zero_boundary(a):
    a[(0, -1), ...] = 0.0
    a[:, (0, -1)] = 0.0
    if a.ndim == 3:
        a[:, :, (0, -1)] = 0.0
    return a


def sine_solution(n, ndim=2):
    xs = node_coords(n, ndim)
    u = np.ones((n + 1,) * ndim)
    for x in xs:
        u = u * np.sin(np.pi * x)
    return _zero_boundary(np.ascontiguousarray(u))


def sine_rhs(n, ndim=2):
    """f = d pi^2 prod sin(pi x_k) (cfg: 129^2 with 7 levels; 513^3 with 9 levels)."""
    return _zero_boundary(ndim * np.pi ** 2 * sine_solution(n, ndim))


def uniform_rhs(n, ndim=2, seed=0):
    """f iid uniform[-1, 1] on interior nodes in layout order from ``default_rng(seed)``."""
    rng = np.random.default_rng(seed)
    f = np.zeros((n + 1,) * ndim)
    f[(slice(1, -1),) * ndim] = rng.uniform(-1.0, 1.0, size=(n - 1,) * ndim)
    return f


def normal_rhs(n, ndim=2, seed=0):
    """f iid N(0, 1) on interior nodes in layout order from ``default_rng(seed)``."""
    rng = np.random.default_rng(seed)
    f = np.zeros((n + 1,) * ndim)
    f[(slice(1, -1),) * ndim] = rng.standard_normal(size=(n - 1,) * ndim)
    return f


def paper_poly_solution(n):
    """u = -x^2 y^2 (1 - x^2)(1 - y^2), the analytic solution of the paper's test problem (Sec. 4)."""
    x, y = node_coords(n, 2)
    return np.ascontiguousarray(-(x ** 2) * y ** 2 * (1 - x ** 2) * (1 - y ** 2))


def paper_poly_rhs(n):
    """Right-hand side for A = -Laplacian whose solution is ``paper_poly_solution`` (Sec. 4, Eq. for the source, sign flipped)."""
    x, y = node_coords(n, 2)
    f_paper = -2.0 * (y ** 2 * (1 - 6 * x ** 2) * (1 - y ** 2) + x ** 2 * (1 - 6 * y ** 2) * (1 - x ** 2))
    return _zero_boundary(np.ascontiguousarray(-f_paper + 0.0 * x * y))


def uneven_batch(count, seed=1, kmin=6, kmax=10):
    """A batch of 2-D problems of uneven sizes: `count` exponents k uniform on kmin..kmax (sides
    2^k + 1), then for each problem in turn f iid N(0, 1) over its interior in layout order, all
    drawn in that order from numpy's default_rng(seed). Returns (ks, fs)."""
    rng = np.random.default_rng(seed)
    ks = [int(k) for k in rng.integers(kmin, kmax + 1, size=count)]
    fs = []
    for k in ks:
        n = 2 ** k
        f = np.zeros((n + 1, n + 1))
        f[1:-1, 1:-1] = rng.standard_normal((n - 1, n - 1))
        fs.append(f)
    return ks, fs


def grf_coefficient(n, sigma=1.0, ell=0.05, seed=2):
    """k = exp(g) on the (n+1)^2 nodes of the unit square (h = 1/n), g a stationary Gaussian random field
    with mean 0, variance sigma^2 and correlation exp(-r^2 / (2 ell^2)).

    Circulant embedding: the covariance is laid out on a periodic (2(n+1))^2 grid (periodic distance,
    so the embedding is at least twice the domain), its FFT gives the eigenvalues (clipped at 0; for
    ell well below the embedding period they are non-negative to rounding), and g is the inverse FFT
    of sqrt(eigenvalues) times the FFT of real white noise N(0, 1) drawn from default_rng(seed) over
    the periodic grid in layout order; the (n+1)^2 corner block is kept."""
    N = 2 * (n + 1)
    h = 1.0 / n
    d = np.minimum(np.arange(N), N - np.arange(N)) * h
    cov = sigma ** 2 * np.exp(-(d[:, None] ** 2 + d[None, :] ** 2) / (2.0 * ell ** 2))
    lam = np.maximum(np.fft.fft2(cov).real, 0.0)
    w = np.random.default_rng(seed).standard_normal((N, N))
    g = np.fft.ifft2(np.sqrt(lam) * np.fft.fft2(w)).real
    return np.ascontiguousarray(np.exp(g[: n + 1, : n + 1]))
