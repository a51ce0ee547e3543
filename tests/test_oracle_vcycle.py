"""Pins of the oracle's classic V(nu1, nu2) comparator (CPU): its explicit prolongation against
(bi/tri)linear reproduction and the full-weighting adjoint identity, its coarse solve against the
Jacobi closed form, and its restarted solves against dense LAPACK solutions."""

import numpy as np
import pytest

import oracle
from paper_1108_2045_gb300 import inputs

import test_oracle_pins as pins


@pytest.mark.parametrize("ndim,nc", [(2, 8), (2, 32), (3, 4), (3, 8)])
def test_prolong_reproduces_multilinear(ndim, nc):
    rng = np.random.default_rng(21)
    c = rng.standard_normal(8)
    nf = 2 * nc
    x = np.arange(nf + 1) / nf
    if ndim == 2:
        X, Y = x[None, :], x[:, None]
        g = c[0] + c[1] * X + c[2] * Y + c[3] * X * Y
    else:
        X, Y, Z = x[None, None, :], x[None, :, None], x[:, None, None]
        g = c[0] + c[1] * X + c[2] * Y + c[3] * Z + c[4] * X * Y + c[5] * Y * Z + c[6] * X * Z + c[7] * X * Y * Z
    g = np.ascontiguousarray(np.broadcast_to(g, (nf + 1,) * ndim))
    Ec = np.ascontiguousarray(g[(slice(None, None, 2),) * ndim])
    Ef = oracle.prolong(Ec)
    inside = (slice(1, -1),) * ndim
    np.testing.assert_allclose(Ef[inside], g[inside], rtol=0, atol=1e-13)


@pytest.mark.parametrize("ndim,nf", [(2, 16), (2, 64), (3, 8)])
def test_full_weighting_is_adjoint_of_prolong(ndim, nf):
    rng = np.random.default_rng(3)
    xf = np.zeros((nf + 1,) * ndim)
    pins.interior(xf)[...] = rng.standard_normal((nf - 1,) * ndim)
    yc = np.zeros((nf // 2 + 1,) * ndim)
    pins.interior(yc)[...] = rng.standard_normal((nf // 2 - 1,) * ndim)
    lhs = np.sum(pins.interior(oracle.restrict(xf)) * pins.interior(yc))
    rhs = np.sum(pins.interior(xf) * pins.interior(oracle.prolong(yc))) / 2 ** ndim
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1)


@pytest.mark.parametrize("ndim,n", [(2, 4), (2, 8), (3, 4)])
def test_coarsest_solve_is_undamped_jacobi(ndim, n):
    # one level: the cycle is max(1, n^2) undamped Jacobi sweeps from zero; on an eigenmode F = v
    # the result is (1 - g^t) v / lambda with g = 1 - lambda h^2 / (2d)
    ks = (1, 2, 1)[:ndim]
    v = pins.sine_mode(n, ndim, *ks)
    lam = pins.eig(n, ks)
    g = 1 - lam / n ** 2 / (2 * ndim)
    t = n * n
    e = oracle.vcycle(v, 1)
    np.testing.assert_allclose(e, (1 - g ** t) * v / lam, rtol=0, atol=1e-13 * np.abs(v / lam).max())


def test_single_interior_node_is_solved_in_one_cycle():
    f = np.zeros((3, 3))
    f[1, 1] = 5.0
    u, status, cycles, hist = oracle.solve_vcycle(f, 1, tol=1e-14)
    assert status == oracle.OK and cycles == 1
    assert u[1, 1] == pytest.approx(5.0 * 0.5 ** 2 / 4, rel=1e-15)  # 4u / h^2 = f, h = 1/2


@pytest.mark.parametrize("ndim,K", [(2, 2), (2, 3), (2, 4), (2, 5), (3, 2), (3, 3)])
def test_vcycle_solution_matches_dense_direct_solve(ndim, K):
    n = 2 ** K
    f = inputs.uniform_rhs(n, ndim, seed=K + 10)
    ref = np.linalg.solve(pins.dense_matrix(n, ndim), pins.interior(f).ravel())
    for levels in sorted({1, K} if K <= 3 else {K - 1, K}):
        u, status, cycles, hist = oracle.solve_vcycle(f, levels, tol=1e-13, max_cycles=500)
        assert status == oracle.OK, (levels, hist[-3:])
        np.testing.assert_allclose(pins.interior(u).ravel(), ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_vcycle_contraction_is_resolution_independent():
    rates = []
    for K in (6, 7, 8, 9):
        n = 2 ** K
        u, status, cycles, hist = oracle.solve_vcycle(inputs.uniform_rhs(n, 2, 0), K, tol=1e-10)
        assert status == oracle.OK and np.all(np.diff(hist) < 0)
        rates.append(hist[-1] / hist[-2])
    assert max(rates) - min(rates) < 0.02
    assert 0.05 < np.mean(rates) < 0.3  # Jacobi-smoothed V(2,2) with full weighting and bilinear transfer
