"""Pins of the oracle's variable-coefficient operator A u = -div(k grad u) (2-D, five-point flux form,
harmonic-mean face coefficients, k injected on coarser lattices) and of the HOMG solver on it.

The independent reference here is a dense matrix assembled face by face: every interior face adds
its coefficient to the two diagonal entries and subtracts it from the two off-diagonal ones, every
face to a boundary node adds it to the interior node's diagonal. It is built from the definition,
not from the oracle's node-wise stencil code.
"""

import numpy as np
import pytest

import oracle
from paper_1108_2045_gb300 import inputs

OMEGA_J = 0.8


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def lognormal_k(n, seed, s=1.0):
    return np.exp(s * np.random.default_rng(seed).standard_normal((n + 1, n + 1)))


def face(a, b):
    return 2.0 * a * b / (a + b)


def assemble(kc, n_lattice, stride, h):
    """Dense matrix of -div(k grad .) on the interior nodes of a lattice with n_lattice intervals per
    side, neighbour spacing h, node coefficients kc[j*stride, i*stride] (injection)."""
    kk = kc[::stride, ::stride]
    m = n_lattice - 1
    idx = lambda i, j: (j - 1) * m + (i - 1)
    A = np.zeros((m * m, m * m))
    inside = lambda i, j: 0 < i < n_lattice and 0 < j < n_lattice
    # x-faces between (i, j) and (i+1, j), y-faces between (i, j) and (i, j+1)
    for j in range(0, n_lattice + 1):
        for i in range(0, n_lattice + 1):
            for di, dj in ((1, 0), (0, 1)):
                i2, j2 = i + di, j + dj
                if i2 > n_lattice or j2 > n_lattice:
                    continue
                a, b = inside(i, j), inside(i2, j2)
                if not (a or b):
                    continue
                kf = face(kk[j, i], kk[j2, i2]) / h ** 2
                if a:
                    A[idx(i, j), idx(i, j)] += kf
                if b:
                    A[idx(i2, j2), idx(i2, j2)] += kf
                if a and b:
                    A[idx(i, j), idx(i2, j2)] -= kf
                    A[idx(i2, j2), idx(i, j)] -= kf
    return A


def interior(v):
    return v[1:-1, 1:-1].reshape(-1)


def embed(x, n):
    out = np.zeros((n + 1, n + 1))
    out[1:-1, 1:-1] = x.reshape(n - 1, n - 1)
    return out


@pytest.mark.parametrize("n", [8, 16])
def test_residual_matches_face_assembly(n):
    kc = lognormal_k(n, 1)
    f = inputs.normal_rhs(n, 2, seed=2)
    u = embed(np.random.default_rng(3).standard_normal((n - 1) ** 2), n)
    A = assemble(kc, n, 1, 1.0 / n)
    r = oracle.residual_vc(kc, f, u)
    ref = interior(f) - A @ interior(u)
    np.testing.assert_allclose(interior(r), ref, rtol=1e-12, atol=1e-12 * np.abs(A @ interior(u)).max())
    assert np.all(r[0] == 0) and np.all(r[-1] == 0) and np.all(r[:, 0] == 0) and np.all(r[:, -1] == 0)
    # the assembled operator is symmetric positive definite
    assert np.allclose(A, A.T) and np.linalg.eigvalsh(A).min() > 0


def test_unit_coefficient_is_the_poisson_operator():
    n = 64
    kc = np.ones((n + 1, n + 1))
    f = inputs.uniform_rhs(n, 2, seed=4)
    u = embed(np.random.default_rng(5).standard_normal((n - 1) ** 2), n)
    r0, r1 = oracle.residual(f, u), oracle.residual_vc(kc, f, u)
    assert np.abs(r1 - r0).max() <= 1e-13 * np.abs(r0).max()
    e0, e1 = oracle.cycle(f, 6), oracle.cycle_vc(kc, f, 6)
    assert np.abs(e1 - e0).max() <= 1e-13 * np.abs(e0).max()
    e0l, e1l = oracle.cycle_lp(f, 6, "fp32"), oracle.cycle_vc(kc, f, 6, precision="fp32")
    assert np.abs(e1l - e0l).max() <= 1e-5 * np.abs(e0l).max()
    _, s0, c0, _ = oracle.solve(f, 6)
    _, s1, c1, _ = oracle.solve_vc(kc, f, 6)
    assert (s0, c0) == (s1, c1) == (oracle.OK, c0)


def test_constant_coefficient_scales_the_iterates():
    # k = c: A = c A_Poisson, the relaxation weight is omega_J / (4c), so every iterate is the Poisson
    # iterate of F / c
    n, c = 32, 3.75
    f = inputs.normal_rhs(n, 2, seed=6)
    e0 = oracle.cycle(f, 5)
    e1 = oracle.cycle_vc(np.full((n + 1, n + 1), c), f, 5)
    assert np.abs(c * e1 - e0).max() <= 1e-13 * np.abs(e0).max()


@pytest.mark.parametrize("iters", [1, 5])
def test_single_level_cycle_is_damped_jacobi(iters):
    # levels = 1: every iteration is damped Jacobi on A with the weight omega_J / D, D = diag(A) h^2
    n = 16
    h = 1.0 / n
    kc = lognormal_k(n, 7)
    F = inputs.normal_rhs(n, 2, seed=8)
    A = assemble(kc, n, 1, h)
    Dinv = 1.0 / np.diag(A)
    x = np.zeros((n - 1) ** 2)
    for _ in range(iters):
        x = x + OMEGA_J * Dinv * (interior(F) - A @ x)
    e = oracle.cycle_vc(kc, F, 1, schedule=[0] * iters)
    np.testing.assert_allclose(interior(e), x, rtol=1e-12, atol=1e-13 * np.abs(x).max())


@pytest.mark.parametrize("m", [1, 2])
def test_coarse_level_relaxation_uses_injected_coefficients(m):
    # two relaxations on the level-m lattice from e = 0: damped Jacobi for the operator assembled on
    # the lattice (spacing 2^m h) from the node coefficients at the lattice nodes
    n = 32
    l = 1 << m
    nm = n >> m
    hm = l / n
    kc = lognormal_k(n, 9)
    Fm = inputs.normal_rhs(nm, 2, seed=10)
    A = assemble(kc, nm, l, hm)
    Dinv = 1.0 / np.diag(A)
    x = np.zeros((nm - 1) ** 2)
    for _ in range(2):
        x = x + OMEGA_J * Dinv * (interior(Fm) - A @ x)
    e = np.zeros((n + 1, n + 1))
    d = None
    mp = -1
    for _ in range(2):
        e, d2 = oracle.iteration_vc(n, m, mp, OMEGA_J, kc, Fm, d, e)
        d, mp = d2, m
    got = interior(e[::l, ::l])
    np.testing.assert_allclose(got, x, rtol=1e-12, atol=1e-13 * np.abs(x).max())
    # off-lattice nodes still hold the interpolation of the first variation only (delayed by one)
    assert np.abs(e[1::2, :]).max() > 0


@pytest.mark.parametrize("n,levels", [(16, 4), (32, 5)])
def test_solution_matches_dense_direct_solve(n, levels):
    kc = inputs.grf_coefficient(n, sigma=1.0, ell=0.1, seed=11)
    f = inputs.normal_rhs(n, 2, seed=12)
    A = assemble(kc, n, 1, 1.0 / n)
    x = np.linalg.solve(A, interior(f))
    u, status, cycles, hist = oracle.solve_vc(kc, f, levels, tol=1e-13, max_cycles=80)
    assert status == oracle.OK
    cond = np.linalg.cond(A)
    assert np.abs(interior(u) - x).max() <= 1e-13 * cond * np.abs(x).max()


def test_residual_decreases_every_cycle_on_a_random_field():
    n = 128
    kc = inputs.grf_coefficient(n)
    f = inputs.normal_rhs(n, 2, seed=13)
    _, status, cycles, hist = oracle.solve_vc(kc, f, 7, tol=1e-10, max_cycles=60)
    assert status == oracle.OK and cycles <= 30
    assert np.all(np.diff(hist) < 0)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_low_precision_cycles_reach_the_same_solution(precision):
    n = 64
    kc = inputs.grf_coefficient(n, ell=0.1, seed=14)
    f = inputs.normal_rhs(n, 2, seed=15)
    u64, s64, c64, _ = oracle.solve_vc(kc, f, 6, tol=1e-11)
    ulp, slp, clp, hist = oracle.solve_vc(kc, f, 6, precision=precision, tol=1e-11, max_cycles=80)
    assert s64 == slp == oracle.OK and hist[-1] <= 1e-11
    A = assemble(kc, n, 1, 1.0 / n)
    assert np.abs(ulp - u64).max() <= 2e-11 * np.linalg.cond(A) * np.abs(u64).max()
    e64 = oracle.cycle_vc(kc, f, 6)
    elp = oracle.cycle_vc(kc, f, 6, precision=precision)
    bound = 1e-5 if precision == "fp32" else 5e-2
    assert np.abs(elp - e64).max() <= bound * np.abs(e64).max()


def test_grf_coefficient_statistics():
    # variance sigma^2 of g = log k and the squared-exponential correlation at one correlation length
    n, ell = 256, 0.05
    gs = [np.log(inputs.grf_coefficient(n, sigma=1.0, ell=ell, seed=s)) for s in range(6)]
    var = np.mean([np.mean(g * g) for g in gs])
    lag = int(round(ell * n))
    cor = np.mean([np.mean(g[:, :-lag] * g[:, lag:]) for g in gs]) / var
    assert abs(var - 1.0) < 0.15
    assert abs(cor - np.exp(-0.5)) < 0.1
    k = inputs.grf_coefficient(n)
    assert k.shape == (n + 1, n + 1) and np.all(k > 0) and np.all(np.isfinite(k))
