"""Pins of the oracle's power-of-two grids (Sec. 3): N = 2^K nodes per side, four quadrant lattices
marked from the external corners, one row/column just outside each quadrant, interpolation from the
node's own quadrant only.

Independent references: the nested full weighting of the Poisson oracle (``oracle.restrict``) on a
quadrant's own nested sub-grid, a dense Poisson matrix, bilinear functions, and symmetry.
"""

import numpy as np
import pytest

import oracle

OMEGA = 0.8 / 4


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def fine_rhs(N, seed):
    f = np.zeros((N, N))
    f[1:-1, 1:-1] = np.random.default_rng(seed).uniform(-1, 1, (N - 2, N - 2))
    return f


def marked_at(N, m):
    """Nodes a level-m relaxation from e = 0 with F = 1 moves: exactly the marked nodes."""
    s = oracle.pow2_local_side(N, m)
    F = np.ones((N, N)) if m == 0 else np.ones((4, s, s))
    e, _ = oracle.pow2_iteration(N, m, -1, OMEGA, F, None, np.zeros((N, N)))
    return e != 0


@pytest.mark.parametrize("N", [16, 32])
def test_lattice_structure(N):
    K = int(np.log2(N))
    H = N // 2
    for m in range(1, K):
        l, nm = 1 << m, H >> m
        want = np.zeros((N, N), dtype=bool)
        for q in range(4):
            for a in range(1, nm + 1):
                for b in range(1, nm + 1):
                    x = (N - 1 - a * l) if q & 1 else a * l
                    y = (N - 1 - b * l) if q >> 1 else b * l
                    assert not want[y, x]  # the four lattices are disjoint
                    want[y, x] = True
        got = marked_at(N, m)
        np.testing.assert_array_equal(got, want)
        assert got.sum() == 4 * nm * nm
    # the coarsest level holds exactly the four central points
    got = marked_at(N, K - 1)
    assert sorted(zip(*np.nonzero(got))) == [(H - 1, H - 1), (H - 1, H), (H, H - 1), (H, H)]
    assert marked_at(N, 0)[1:-1, 1:-1].all()


@pytest.mark.parametrize("N,m", [(32, 1), (32, 2), (64, 3), (64, 4)])
def test_restriction_is_nested_full_weighting(N, m):
    # on each quadrant's own nested sub-grid of N/2 + 1 nodes (anchored at its external corner), the
    # restriction equals m nested full weightings wherever those see only that sub-grid
    r = fine_rhs(N, 1)
    H = N // 2
    Fm = oracle.pow2_restrict(r, m)
    nm = H >> m
    for q in range(4):
        sub = r
        if q & 1:
            sub = sub[:, ::-1]
        if q >> 1:
            sub = sub[::-1, :]
        nested = np.ascontiguousarray(sub[:H + 1, :H + 1])
        for _ in range(m):
            nested = oracle.restrict(nested)
        inner = slice(1, nm)  # a, b < n_m: stencil inside the sub-grid
        np.testing.assert_allclose(Fm[q][inner, inner], nested[inner, inner], rtol=1e-13, atol=1e-15)
        assert np.all(Fm[q][0, :] == 0) and np.all(Fm[q][:, 0] == 0)


def test_restriction_of_a_constant_is_that_constant_inside():
    # the hat weights sum to 1: interior points of a constant residual see the constant
    N, m = 64, 3
    r = np.ones((N, N))
    Fm = oracle.pow2_restrict(r, m)
    l, nm = 1 << m, (N // 2) >> m
    for q in range(4):
        assert np.allclose(Fm[q][1:nm, 1:nm], 1.0, rtol=1e-14)


@pytest.mark.parametrize("iters", [1, 4])
def test_single_level_cycle_is_damped_jacobi(iters):
    N = 16
    n = N - 1
    m1 = N - 2
    T = 2 * np.eye(m1) - np.eye(m1, k=1) - np.eye(m1, k=-1)
    A = (np.kron(np.eye(m1), T) + np.kron(T, np.eye(m1))) * n * n
    F = fine_rhs(N, 2)
    x = np.zeros(m1 * m1)
    Dinv = 1.0 / np.diag(A)
    for _ in range(iters):
        x = x + 0.8 * Dinv * (F[1:-1, 1:-1].ravel() - A @ x)
    e = oracle.pow2_cycle(F, 1, schedule=[0] * iters)
    np.testing.assert_allclose(e[1:-1, 1:-1].ravel(), x, rtol=1e-12, atol=1e-14 * np.abs(x).max())


@pytest.mark.parametrize("N,mp", [(32, 1), (32, 2), (64, 3)])
def test_interpolation_uses_the_nodes_own_quadrant(N, mp):
    # a different bilinear function on each quadrant's lattice: every node not marked at level mp gets
    # the function of the quadrant that contains it, exactly
    H, l = N // 2, 1 << mp
    s = oracle.pow2_local_side(N, mp)
    coef = np.random.default_rng(3).standard_normal((4, 4))

    def g(q, x, y):
        a, b, c, d = coef[q]
        return a + b * x + c * y + d * x * y

    dprev = np.zeros((4, s, s))
    for q in range(4):
        for b in range(s):
            for a in range(s):
                x = (N - 1 - a * l) if q & 1 else a * l
                y = (N - 1 - b * l) if q >> 1 else b * l
                dprev[q, b, a] = g(q, x, y)
    e, _ = oracle.pow2_iteration(N, 0, mp, OMEGA, np.zeros((N, N)), dprev, np.zeros((N, N)))
    marked = marked_at(N, mp)
    for y in range(1, N - 1):
        for x in range(1, N - 1):
            q = int(x >= H) | (int(y >= H) << 1)
            want = 0.0 if marked[y, x] else g(q, x, y)
            assert abs(e[y, x] - want) <= 1e-12 * max(1.0, abs(want)), (x, y)


@pytest.mark.parametrize("N", [8, 16, 32])
def test_solution_matches_dense_direct_solve(N):
    n, m1 = N - 1, N - 2
    T = 2 * np.eye(m1) - np.eye(m1, k=1) - np.eye(m1, k=-1)
    A = (np.kron(np.eye(m1), T) + np.kron(T, np.eye(m1))) * n * n
    f = fine_rhs(N, 4)
    x = np.linalg.solve(A, f[1:-1, 1:-1].ravel())
    K = int(np.log2(N))
    u, st, cyc, hist = oracle.pow2_solve(f, K, tol=1e-13)
    assert st == oracle.OK
    assert np.abs(u[1:-1, 1:-1].ravel() - x).max() <= 1e-11 * np.abs(x).max() * np.linalg.cond(A)


def test_contraction_is_resolution_independent(Ks=(6, 7, 8)):
    rates = []
    for K in Ks:
        N = 2 ** K
        _, st, cyc, hist = oracle.pow2_solve(fine_rhs(N, 5), K, tol=1e-11)
        assert st == oracle.OK and np.all(np.diff(hist) < 0)
        rates.append(np.median(hist[2:] / hist[1:-1]))
    assert max(rates) < 0.2 and max(rates) / min(rates) < 1.3, rates


def test_mirror_symmetry():
    # a right-hand side symmetric under x -> N-1-x (and y) gives a symmetric cycle: the quadrants are
    # mirror images of one another
    N = 64
    f = fine_rhs(N, 6)
    f = f + f[:, ::-1]
    f = f + f[::-1, :]
    e = oracle.pow2_cycle(f, 6)
    assert np.abs(e - e[:, ::-1]).max() <= 1e-14 * np.abs(e).max()
    assert np.abs(e - e[::-1, :]).max() <= 1e-14 * np.abs(e).max()
    g = f + f.T
    e = oracle.pow2_cycle(g, 6)
    assert np.abs(e - e.T).max() <= 1e-14 * np.abs(e).max()
