"""Variable-coefficient operator -div(k grad u) on the GPU vs the CPU oracle (GB300 only).

Bar: FP64 cycles within ||u_gpu - u_oracle|| / ||u_oracle|| <= 1e-12 after every cycle; FP32 and
bfloat16 cycles against the oracle's cycles of the same precision (1e-5, 5e-2 after one cycle), and
every converged solution checked with the oracle's own FP64 residual. Sides 2^K + 1 give ragged
tails against the kernels' tiles; coefficients are lognormal Gaussian random fields.
"""

import numpy as np
import pytest

import oracle
from paper_1108_2045_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def homg():
    import torch

    import __graft_entry__

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    __graft_entry__.build()
    oracle.build()
    from paper_1108_2045_gb300 import homg as binding

    return binding


def gpu_solve_vc(homg, kc, f_np, levels, tol=0.0, max_cycles=1, u0=None, **kw):
    import torch

    with homg.Solver(2, f_np.shape[0], levels, **kw) as s:
        k = torch.from_numpy(np.ascontiguousarray(kc)).cuda()
        s.set_coefficient(k)
        del k  # the handle keeps its own derived coefficients
        f = torch.from_numpy(np.ascontiguousarray(f_np)).cuda()
        u = torch.zeros_like(f) if u0 is None else torch.from_numpy(np.ascontiguousarray(u0)).cuda()
        status, cycles, relres = s.solve(f, u, tol=tol, max_cycles=max_cycles)
        return u.cpu().numpy(), status, cycles, relres, s.history()


def rel(a, b):
    """The larger of two relative errors of a against b: in the 2-norm over the grid, and at the
    worst single node against the largest |b| (so no single node can hide in a large grid's norm)."""
    nb = np.linalg.norm(b)
    mb = np.max(np.abs(b)) if b.size else 0.0
    return max(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0),
               (np.max(np.abs(a - b)) if b.size else 0.0) / (mb if mb > 0 else 1.0))


def oracle_relres(kc, f, u):
    return oracle.norm_interior(oracle.residual_vc(kc, f, u)) / oracle.norm_interior(f)


@pytest.mark.parametrize("K,levels", [(3, 3), (5, 5), (6, 4), (7, 7), (8, 8), (9, 6)])
def test_fp64_cycles_match_oracle(homg, K, levels):
    n = 2 ** K
    kc = inputs.grf_coefficient(n, ell=0.1, seed=K)
    f = inputs.normal_rhs(n, 2, seed=K + 1)
    for k in (1, 2, 3):
        ref, _, _, rhist = oracle.solve_vc(kc, f, levels, tol=0.0, max_cycles=k)
        got, st, cyc, rr, hist = gpu_solve_vc(homg, kc, f, levels, max_cycles=k)
        assert st == homg.HOMG_NOT_CONVERGED and cyc == k
        assert rel(got, ref) <= 1e-12, (k, rel(got, ref))
        np.testing.assert_allclose(hist, rhist, rtol=1e-9)


@pytest.mark.parametrize("precision,bound", [("fp32", 1e-5), ("bf16", 5e-2)])
@pytest.mark.parametrize("K,levels", [(5, 5), (7, 7), (8, 6)])
def test_low_precision_cycle_matches_oracle(homg, precision, bound, K, levels):
    n = 2 ** K
    kc = inputs.grf_coefficient(n, ell=0.1, seed=20 + K)
    f = inputs.normal_rhs(n, 2, seed=21 + K)
    ref, _, _, _ = oracle.solve_vc(kc, f, levels, precision=precision, tol=0.0, max_cycles=1)
    got, st, cyc, rr, _ = gpu_solve_vc(homg, kc, f, levels, max_cycles=1, precision=precision)
    assert rel(got, ref) <= bound, rel(got, ref)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_converged_solution_passes_the_oracle_residual(homg, precision):
    n, levels = 256, 8
    kc = inputs.grf_coefficient(n, seed=3)
    f = inputs.normal_rhs(n, 2, seed=4)
    got, st, cyc, rr, hist = gpu_solve_vc(homg, kc, f, levels, tol=1e-10, max_cycles=80, precision=precision)
    assert st == homg.HOMG_OK and rr <= 1e-10
    assert oracle_relres(kc, f, got) <= 1.0001e-10
    _, ost, ocyc, _ = oracle.solve_vc(kc, f, levels, precision=precision, tol=1e-10, max_cycles=80)
    assert ost == oracle.OK and abs(ocyc - cyc) <= 1


def test_unit_coefficient_matches_poisson_handle(homg):
    import torch

    n, levels = 128, 7
    f_np = inputs.uniform_rhs(n, 2, seed=5)
    f = torch.from_numpy(f_np).cuda()
    with homg.Solver(2, n + 1, levels) as s:
        u0 = torch.zeros_like(f)
        s.solve(f, u0, tol=0.0, max_cycles=2)
        s.set_coefficient(torch.ones_like(f))
        u1 = torch.zeros_like(f)
        s.solve(f, u1, tol=0.0, max_cycles=2)
        assert rel(u1.cpu().numpy(), u0.cpu().numpy()) <= 1e-13
        # back to the Poisson operator: bit-identical to the first solve
        s.set_coefficient(None)
        u2 = torch.zeros_like(f)
        s.solve(f, u2, tol=0.0, max_cycles=2)
        assert torch.equal(u2, u0)


def test_residual_norm_uses_the_coefficient(homg):
    import torch

    n = 64
    kc = inputs.grf_coefficient(n, ell=0.1, seed=6)
    f_np = inputs.normal_rhs(n, 2, seed=7)
    u_np = inputs.normal_rhs(n, 2, seed=8)
    with homg.Solver(2, n + 1, 6) as s:
        s.set_coefficient(torch.from_numpy(kc).cuda())
        rr = s.residual_norm(torch.from_numpy(f_np).cuda(), torch.from_numpy(u_np).cuda())
    ref = oracle_relres(kc, f_np, u_np)
    assert abs(rr - ref) <= 1e-13 * ref


def test_invalid_coefficients_are_rejected(homg):
    import torch

    n = 32
    f = torch.from_numpy(inputs.uniform_rhs(n, 2, seed=9)).cuda()
    with homg.Solver(2, n + 1, 5) as s:
        for bad in (0.0, -1.0, float("nan"), float("inf")):
            k = torch.ones(n + 1, n + 1, dtype=torch.float64, device="cuda")
            k[3, 4] = bad
            with pytest.raises(homg.HomgError) as ei:
                s.set_coefficient(k)
            assert ei.value.code == homg.HOMG_EINVAL
        # still the Poisson operator and usable
        u = torch.zeros_like(f)
        st, cyc, rr = s.solve(f, u, tol=1e-10, max_cycles=40)
        assert st == homg.HOMG_OK
    for kw in [dict(strict_fp=True), dict(exec_mode="wholegrid"), dict(cycle="v")]:
        with homg.Solver(2, n + 1, 5, **kw) as s:
            with pytest.raises(homg.HomgError):
                s.set_coefficient(torch.ones(n + 1, n + 1, dtype=torch.float64, device="cuda"))
    with homg.Solver(3, 17, 4) as s:
        with pytest.raises(homg.HomgError):
            s.set_coefficient(torch.ones(17, 17, 17, dtype=torch.float64, device="cuda"))


_FULL = {}


def full_inputs():
    # the 2049^2 variable-coefficient workload: k = exp(g), g a Gaussian random field (sigma 1,
    # squared-exponential correlation length 0.05, seed 2), f iid N(0, 1) (seed 0), 11 levels
    if not _FULL:
        n = 2048
        _FULL.update(k=inputs.grf_coefficient(n, sigma=1.0, ell=0.05, seed=2), f=inputs.normal_rhs(n, 2, seed=0))
    return _FULL["k"], _FULL["f"]


def test_full_size_first_cycle_matches_oracle(homg):
    kc, f = full_inputs()
    ref, _, _, rhist = oracle.solve_vc(kc, f, 11, tol=0.0, max_cycles=1)
    got, st, cyc, rr, hist = gpu_solve_vc(homg, kc, f, 11, max_cycles=1)
    assert rel(got, ref) <= 1e-12, rel(got, ref)
    np.testing.assert_allclose(hist, rhist, rtol=1e-9)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_full_size_solve(homg, precision):
    kc, f = full_inputs()
    got, st, cyc, rr, hist = gpu_solve_vc(homg, kc, f, 11, tol=1e-10, max_cycles=100, precision=precision)
    assert st == homg.HOMG_OK and rr <= 1e-10
    assert oracle_relres(kc, f, got) <= 1.0001e-10
    assert np.all(np.diff(hist) < 0)
