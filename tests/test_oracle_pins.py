"""Pins of the CPU oracle to facts fixed by the paper and by the mathematics (no GPU).

Each test checks the oracle against something other than itself: a closed form, a dense direct
solve through LAPACK, an algebraic identity between two independently written operators, or a
value the paper prints. A plausible slip in the oracle (dropped term, wrong sign, stride, weight,
index order or delay) fails at least one of them.
"""

import json
import os

import numpy as np
import pytest

import oracle
from paper_1108_2045_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def sine_mode(n, ndim, kx=1, ky=1, kz=1):
    """prod_k sin(k pi x) sampled on the node grid (0 on the boundary)."""
    x = np.arange(n + 1) / n
    if ndim == 2:
        return np.ascontiguousarray(np.sin(ky * np.pi * x)[:, None] * np.sin(kx * np.pi * x)[None, :])
    return np.ascontiguousarray(np.sin(kz * np.pi * x)[:, None, None] * np.sin(ky * np.pi * x)[None, :, None]
                                * np.sin(kx * np.pi * x)[None, None, :])


def eig(n, ks):
    """Eigenvalue of A_h = -Laplacian_h (5/7-point) for the sine mode with wave numbers ks."""
    h = 1.0 / n
    return sum(4.0 / h ** 2 * np.sin(k * np.pi * h / 2) ** 2 for k in ks)


def dense_matrix(n, ndim):
    """A_h as a Kronecker sum of 1-D second differences over interior nodes (independent of the stencil code)."""
    h = 1.0 / n
    m = n - 1
    T = (2 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)) / h ** 2
    I = np.eye(m)
    if ndim == 2:
        return np.kron(I, T) + np.kron(T, I)
    return np.kron(np.kron(I, I), T) + np.kron(np.kron(I, T), I) + np.kron(np.kron(T, I), I)


def interior(a):
    return a[(slice(1, -1),) * a.ndim]


# --------------------------------------------------------------------------------------------
# Schedule (Sec. 2, MFMG paragraph)
# --------------------------------------------------------------------------------------------

def test_mfmg_schedule_rule():
    with open(os.path.join(GOLDEN, "paper_values.json")) as fh:
        rule = json.load(fh)["mfmg_rule"]
    s = oracle.mfmg_schedule(7, 32)
    levels = sorted(set(s), reverse=True)
    assert s == sorted(s, reverse=True), "coarse to fine"
    counts = [s.count(m) for m in levels]
    assert counts[0] == rule["coarsest_iterations"]
    for a, b in zip(counts, counts[1:]):
        assert b == min(a * rule["growth_factor"], 32)
    assert s[-1] == 0
    # whole-grid operations per cycle for the benchmark grids (2-D: 7, 9, 11, 12 levels)
    assert [len(oracle.mfmg_schedule(L, 32)) for L in (7, 9, 11, 12)] == [126, 190, 254, 286]
    assert oracle.mfmg_schedule(5, 2) == [4, 4, 3, 3, 2, 2, 1, 1, 0, 0]
    assert oracle.mfmg_schedule(3, 1) == [2, 1, 0]


# --------------------------------------------------------------------------------------------
# Residual operator: closed-form eigen-pairs and the dense matrix
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("ndim,n", [(2, 16), (2, 64), (3, 8), (3, 16)])
def test_residual_closed_form(ndim, n):
    ks = (1, 3, 2)[:ndim]
    v = sine_mode(n, ndim, *ks)
    r = oracle.residual(np.zeros_like(v), v)
    # r = f - A v with f = 0 and A v = lambda v exactly for a discrete sine mode
    np.testing.assert_allclose(r, -eig(n, ks) * v, rtol=0, atol=1e-9 * eig(n, ks))
    assert np.all(r[(0, -1), ...] == 0)


@pytest.mark.parametrize("ndim,n", [(2, 8), (3, 4)])
def test_residual_matches_dense(ndim, n):
    rng = np.random.default_rng(7)
    u = np.zeros((n + 1,) * ndim)
    interior(u)[...] = rng.standard_normal((n - 1,) * ndim)
    f = inputs.normal_rhs(n, ndim, seed=8)
    r = oracle.residual(f, u)
    ref = interior(f).ravel() - dense_matrix(n, ndim) @ interior(u).ravel()
    np.testing.assert_allclose(interior(r).ravel(), ref, rtol=1e-12, atol=1e-10)


# --------------------------------------------------------------------------------------------
# Restriction (full weighting) and interpolation
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("ndim,nf", [(2, 32), (2, 128), (3, 16)])
def test_restrict_sine_closed_form(ndim, nf):
    # FW of sin(k pi x) at spacing H: sin(k pi x) * cos^2(k pi H / 2) per dimension
    ks = (1, 2, 3)[:ndim]
    F = sine_mode(nf, ndim, *ks)
    Fc = oracle.restrict(F)
    H = 1.0 / nf
    factor = np.prod([np.cos(k * np.pi * H / 2) ** 2 for k in ks])
    np.testing.assert_allclose(Fc, factor * sine_mode(nf // 2, ndim, *ks), rtol=0, atol=1e-14)


def prolong(y, n_fine, ndim):
    """Bilinear/trilinear prolongation of a compact stride-2 array, through the oracle's iteration.

    With e_old = 0 and F_m = 0 the relaxation contributes exactly 0, so one iteration at level 0
    returns y's interpolant on the nodes off the stride-2 lattice; the lattice nodes keep y.
    """
    e0 = np.zeros((n_fine + 1,) * ndim)
    e1, _ = oracle.iteration(n_fine, 0, 1, 0.25, np.zeros_like(e0), np.ascontiguousarray(y), e0)
    e1[(slice(None, None, 2),) * ndim] += y
    return e1


@pytest.mark.parametrize("ndim,nf", [(2, 16), (2, 64), (3, 8)])
def test_restrict_is_adjoint_of_interpolation(ndim, nf):
    # full weighting = P^T / 2^d (interior nodes, zero boundaries): <R x, y>_c = <x, P y>_f / 2^d
    rng = np.random.default_rng(11)
    x = np.zeros((nf + 1,) * ndim)
    interior(x)[...] = rng.standard_normal((nf - 1,) * ndim)
    y = np.zeros((nf // 2 + 1,) * ndim)
    interior(y)[...] = rng.standard_normal((nf // 2 - 1,) * ndim)
    lhs = np.sum(interior(oracle.restrict(x)) * interior(y))
    rhs = np.sum(interior(x) * interior(prolong(y, nf, ndim))) / 2 ** ndim
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1)


@pytest.mark.parametrize("ndim,n,mp", [(2, 32, 1), (2, 32, 3), (2, 64, 5), (3, 16, 1), (3, 16, 2)])
def test_interpolation_reproduces_multilinear(ndim, n, mp):
    # S reproduces any (bi/tri)linear function from its lattice samples (dyadic weights)
    rng = np.random.default_rng(5)
    c = rng.standard_normal(8)
    x = np.arange(n + 1) / n
    if ndim == 2:
        X, Y = x[None, :], x[:, None]
        g = c[0] + c[1] * X + c[2] * Y + c[3] * X * Y
    else:
        X, Y, Z = x[None, None, :], x[None, :, None], x[:, None, None]
        g = (c[0] + c[1] * X + c[2] * Y + c[3] * Z + c[4] * X * Y + c[5] * Y * Z + c[6] * X * Z
             + c[7] * X * Y * Z)
    g = np.ascontiguousarray(np.broadcast_to(g, (n + 1,) * ndim))
    lp = 2 ** mp
    d = np.ascontiguousarray(g[(slice(None, None, lp),) * ndim])
    # level mp+1 relaxation has F = 0 and e_old = 0, so only the interpolation of d acts
    e0 = np.zeros((n + 1,) * ndim)
    Fm = np.zeros(((n >> (mp + 1)) + 1,) * ndim)
    e1, _ = oracle.iteration(n, mp + 1, mp, 0.2, Fm, d, e0)
    off = np.ones((n + 1,) * ndim, bool)
    off[(slice(None, None, lp),) * ndim] = False
    inside = np.zeros_like(off)
    inside[(slice(1, -1),) * ndim] = True
    np.testing.assert_allclose(e1[off & inside], g[off & inside], rtol=0, atol=1e-13)
    assert np.all(e1[~off] == 0) and np.all(e1[~inside] == 0)


# --------------------------------------------------------------------------------------------
# Relaxation: damped Jacobi (explicit Euler of Eq. "heat") at level m
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("ndim,n,m", [(2, 64, 0), (2, 64, 2), (2, 64, 4), (3, 16, 0), (3, 16, 1)])
def test_level_relaxation_closed_form(ndim, n, m):
    # one iteration at level m on a sine mode: delta = omega (h_m^2 F - (2d - 2 sum cos(k pi h_m)) e)
    ks = (1, 2, 1)[:ndim]
    l = 2 ** m
    hm = l / n
    omega = 0.2 if ndim == 2 else 1.0 / 7.0
    e_old = sine_mode(n, ndim, *ks)
    Fm = 3.0 * sine_mode(n >> m, ndim, *ks)
    e_new, d = oracle.iteration(n, m, -1, omega, Fm, None, e_old)
    lam = 2 * ndim - 2 * sum(np.cos(k * np.pi * hm) for k in ks)
    lat = (slice(None, None, l),) * ndim
    expect_d = omega * (hm ** 2 * Fm - lam * e_old[lat])
    np.testing.assert_allclose(d, expect_d, rtol=0, atol=1e-13)
    expect = e_old.copy()
    expect[lat] += expect_d
    np.testing.assert_allclose(e_new, expect, rtol=0, atol=1e-13)


@pytest.mark.parametrize("ndim,n,t", [(2, 32, 1), (2, 32, 7), (2, 64, 20), (3, 8, 5)])
def test_single_level_cycle_is_damped_jacobi(ndim, n, t):
    # with one level, a cycle is t damped-Jacobi sweeps from e = 0; on an eigenmode F = v:
    # e_t = (1 - g^t) v / lambda, g = 1 - omega_J lambda h^2 / (2d)
    ks = (3, 1, 2)[:ndim]
    v = sine_mode(n, ndim, *ks)
    lam = eig(n, ks)
    omj = oracle.default_omega_j(ndim)
    g = 1 - omj * lam / n ** 2 / (2 * ndim)
    e = oracle.cycle(v, levels=1, schedule=[0] * t)
    np.testing.assert_allclose(e, (1 - g ** t) * v / lam, rtol=0, atol=1e-14 * np.abs(v / lam).max() * 10)


# --------------------------------------------------------------------------------------------
# The paper's Fig. 3 narrative (Sec. 4): spike, stalled relaxation, pyramid
# --------------------------------------------------------------------------------------------

def test_fig3_spike_stall_pyramid():
    with open(os.path.join(GOLDEN, "paper_values.json")) as fh:
        omj = json.load(fh)["fig3_narrative"]["stall_requires_omega_j"]
    n, L = 128, 7
    M = L - 1
    F0 = inputs.paper_poly_rhs(n)
    F = [F0]
    for _ in range(1, L):
        F.append(oracle.restrict(F[-1]))
    omega = omj / 4
    e0 = np.zeros_like(F0)
    # iteration 1 at the coarsest level: only the middle node changes (spike)
    e1, d1 = oracle.iteration(n, M, -1, omega, F[M], None, e0)
    c = n // 2
    hM = 2 ** M / n
    assert e1[c, c] == pytest.approx(omega * hM ** 2 * F[M][1, 1], rel=1e-15)
    mask = np.ones_like(e1, bool)
    mask[c, c] = False
    assert np.all(e1[mask] == 0)
    # iteration 2: the relaxation has stalled (one-point problem solved exactly with omega_J = 1)
    e2, d2 = oracle.iteration(n, M, M, omega, F[M], d1, e1)
    assert d2[1, 1] == 0.0
    # ... while the interpolation of iteration 1's variation forms a pyramid (bilinear hat)
    x = np.arange(n + 1) / n
    hat = (1 - np.abs(x - 0.5) / 0.5)
    np.testing.assert_allclose(e2, e1[c, c] * hat[:, None] * hat[None, :], rtol=0, atol=1e-16)
    # iteration 3 relaxes on the next finer level: exactly the 3x3 interior nodes of stride 32 move
    # by their relaxation, and the rest receives no new interpolation (the stalled variation is 0)
    e3, d3 = oracle.iteration(n, M - 1, M, omega, F[M - 1], d2, e2)
    changed = e3 != e2
    lat = np.zeros_like(changed)
    lat[32:97:32, 32:97:32] = True
    assert not np.any(changed & ~lat)
    np.testing.assert_array_equal(changed[32:97:32, 32:97:32], d3[1:4, 1:4] != 0)
    assert np.count_nonzero(d3) == 9


# --------------------------------------------------------------------------------------------
# Converged solutions: closed form, dense LU, O(h^2), residual decrease
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("ndim,K", [(2, 5), (2, 7), (3, 4)])
def test_solution_matches_discrete_eigen_closed_form(ndim, K):
    n = 2 ** K
    f = inputs.sine_rhs(n, ndim)
    u, status, cycles, hist = oracle.solve(f, K, tol=1e-12, max_cycles=60)
    assert status == oracle.OK
    h = 1.0 / n
    ch = np.pi ** 2 * h ** 2 / (4 * np.sin(np.pi * h / 2) ** 2)
    uh = ch * inputs.sine_solution(n, ndim)
    # f is the lowest eigenmode, so ||u - u_h|| / ||u_h|| <= relres
    assert np.linalg.norm(u - uh) / np.linalg.norm(uh) < 1e-12 * 1.01 + 1e-15


@pytest.mark.parametrize("ndim,K", [(2, 2), (2, 3), (2, 4), (2, 5), (3, 2), (3, 3)])
def test_solution_matches_dense_direct_solve(ndim, K):
    n = 2 ** K
    f = inputs.uniform_rhs(n, ndim, seed=K)
    ref = np.linalg.solve(dense_matrix(n, ndim), interior(f).ravel())
    # a single level is plain damped Jacobi, which needs O(n^2) sweeps: only on the smallest grids
    for levels in sorted({max(1, K - 1), K} | ({1} if K <= 3 else set())):
        u, status, cycles, hist = oracle.solve(f, levels, tol=1e-13, max_cycles=2000)
        assert status == 0, (levels, hist[-3:])
        np.testing.assert_allclose(interior(u).ravel(), ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_discretisation_error_is_second_order():
    errs = []
    for K in (4, 5, 6, 7):
        n = 2 ** K
        u, status, _, _ = oracle.solve(inputs.sine_rhs(n), K, tol=1e-12, max_cycles=60)
        assert status == 0
        errs.append(np.abs(u - inputs.sine_solution(n)).max())
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all(np.abs(ratios - 4) < 0.05), ratios
    # max|u_h - u| = (c_h - 1) for the sine mode: pi^2 h^2 / 12 + O(h^4)
    assert errs[-1] == pytest.approx(np.pi ** 2 / 128 ** 2 / 12, rel=2e-3)


@pytest.mark.parametrize("rhs", ["uniform", "sine"])
def test_residual_decreases_every_cycle(rhs):
    n = 128
    f = inputs.uniform_rhs(n, 2, 0) if rhs == "uniform" else inputs.sine_rhs(n)
    u, status, cycles, hist = oracle.solve(f, 7, tol=1e-10)
    assert status == 0 and hist[-1] <= 1e-10 and hist[0] == 1.0
    assert np.all(np.diff(hist) < 0)
    # resolution-independent contraction (Sec. 4, Fig. 4 discussion)
    assert np.all(hist[2:] / hist[1:-1] < 0.2)


def test_zero_rhs_and_max_cycles_zero():
    f = np.zeros((33, 33))
    u0 = np.ones((33, 33))
    u, status, cycles, hist = oracle.solve(f, 5, u0=u0)
    assert status == 0 and cycles == 0 and np.all(interior(u) == 0) and np.all(u[0] == 1)
    f = inputs.uniform_rhs(32, 2, 1)
    u, status, cycles, hist = oracle.solve(f, 5, max_cycles=0)
    assert status == oracle.NOT_CONVERGED and cycles == 0 and hist[0] == 1.0 and np.all(u == 0)


def test_nan_rhs_diverges():
    f = inputs.uniform_rhs(32, 2, 1)
    f[5, 7] = np.nan
    u, status, cycles, hist = oracle.solve(f, 5)
    assert status == oracle.DIVERGED


def test_invalid_arguments_rejected():
    f = np.zeros((33, 33))
    with pytest.raises(ValueError):
        oracle.solve(f, 6)  # more levels than 2^5 allows
    with pytest.raises(ValueError):
        oracle.cycle(f, 3, schedule=[2, 1])  # must end on the finest level
    with pytest.raises(ValueError):
        oracle.cycle(np.zeros((31, 31)), 2)  # not 2^K + 1 nodes


# --------------------------------------------------------------------------------------------
# The paper's printed error levels (Sec. 4, Fig. 4): order of magnitude only
# --------------------------------------------------------------------------------------------

def test_tpaper_one_cycle_error_order_of_magnitude():
    with open(os.path.join(GOLDEN, "paper_values.json")) as fh:
        ref = json.load(fh)["tpaper_l1_error_one_cycle"]
    errs = {}
    for maxi in (4, 32):
        per_n = []
        for K in (6, 7, 8):
            n = 2 ** K
            u, _, _, _ = oracle.solve(inputs.paper_poly_rhs(n), K, tol=0, max_cycles=1, max_i=maxi)
            ue = inputs.paper_poly_solution(n)
            per_n.append(np.abs(u - ue).sum() / np.abs(ue).sum())
        # "cycles with the same MaxI descend over the same convergence path for different resolutions"
        assert max(per_n) - min(per_n) < 0.01
        errs[maxi] = per_n[-1]
    assert errs[32] < errs[4]  # larger MaxI reaches a lower error
    for maxi in (4, 32):
        ratio = errs[maxi] / ref["max_i_%d" % maxi]
        assert 0.1 < ratio < 10, (maxi, errs[maxi])
