"""Mixed precision on the GPU (GB300 only): cycles in binary32 or bfloat16 storage inside an FP64
restart loop (iterative refinement), against the oracle's single-precision cycle.

Bars: strict whole-grid form is bit-identical to the oracle's low-precision cycle (same operation
order and the same storage rounding). The fast forms reassociate binary32 arithmetic: after each
cycle ||u_gpu - u_oracle|| / ||u_oracle|| <= 1e-5 (binary32; the cycle itself differs from FP64 by
~1e-7) and <= 5e-2 (bfloat16 storage: one bfloat16 rounding is 2^-9 relative, and the oracle's
bfloat16 cycle differs from FP64 by ~3e-2). Every form must reach relres 1e-10 through the FP64
residual.
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
    from paper_1108_2045_gb300 import homg as binding

    return binding


def gpu_solve(homg, f_np, levels, tol=0.0, max_cycles=1, **kw):
    import torch

    with homg.Solver(f_np.ndim, f_np.shape[0], levels, **kw) as s:
        f = torch.from_numpy(np.ascontiguousarray(f_np)).cuda()
        u = torch.zeros_like(f)
        status, cycles, relres = s.solve(f, u, tol=tol, max_cycles=max_cycles)
        return u.cpu().numpy(), status, cycles, relres, s.history()


def rel(a, b):
    """The larger of two relative errors of a against b: in the 2-norm over the grid, and at the
    worst single node against the largest |b| (so no single node can hide in a large grid's norm)."""
    nb = np.linalg.norm(b)
    mb = np.max(np.abs(b)) if b.size else 0.0
    return max(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0),
               (np.max(np.abs(a - b)) if b.size else 0.0) / (mb if mb > 0 else 1.0))


TOL = {"fp32": 1e-5, "bf16": 5e-2}


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("ndim,K,levels", [(2, 5, 5), (2, 7, 7), (2, 8, 6), (3, 4, 4), (3, 5, 5)])
def test_strict_wholegrid_is_bit_identical_to_oracle(homg, precision, ndim, K, levels):
    n = 2 ** K
    f = inputs.uniform_rhs(n, ndim, seed=K)
    for k in (1, 2):
        ref, _, _, rhist = oracle.solve_mixed(f, levels, precision, tol=0.0, max_cycles=k)
        got, st, cyc, rr, hist = gpu_solve(homg, f, levels, max_cycles=k, exec_mode="wholegrid", strict_fp=True,
                                           precision=precision)
        assert cyc == k
        np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("mode", ["lattice", "wholegrid"])
@pytest.mark.parametrize("strict", [True, False])
@pytest.mark.parametrize("ndim,K,levels", [(2, 7, 7), (2, 10, 10), (3, 5, 5)])
def test_cycles_follow_oracle(homg, precision, mode, strict, ndim, K, levels):
    n = 2 ** K
    f = inputs.uniform_rhs(n, ndim, seed=K + 1)
    for k in (1, 2):
        ref, _, _, _ = oracle.solve_mixed(f, levels, precision, tol=0.0, max_cycles=k)
        got, st, cyc, rr, hist = gpu_solve(homg, f, levels, max_cycles=k, exec_mode=mode, strict_fp=strict,
                                           precision=precision)
        assert cyc == k
        assert rel(got, ref) <= TOL[precision], (k, rel(got, ref))


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("ndim,K", [(2, 7), (2, 10), (3, 5)])
def test_mixed_solve_reaches_tolerance(homg, precision, ndim, K):
    n = 2 ** K
    f = inputs.uniform_rhs(n, ndim, seed=3) if ndim == 2 else inputs.normal_rhs(n, 3, seed=3)
    got, st, cyc, rr, hist = gpu_solve(homg, f, K, tol=1e-10, max_cycles=60, precision=precision)
    assert st == homg.HOMG_OK and rr <= 1e-10
    r = oracle.residual(f, got)
    assert oracle.norm_interior(r) / oracle.norm_interior(f) <= 1e-10
    _, _, ocyc, _ = oracle.solve_mixed(f, K, precision, tol=1e-10, max_cycles=60)
    assert abs(cyc - ocyc) <= (0 if precision == "fp32" else 2), (cyc, ocyc)
    # two solutions with relative residuals <= 1e-10 differ by at most cond(A) * 2e-10 relative
    u64, _, c64, _ = oracle.solve(f, K, tol=1e-10)
    cond = (np.sin(np.pi * (n - 1) / (2 * n)) / np.sin(np.pi / (2 * n))) ** 2
    assert rel(got, u64) <= 2e-10 * cond


@pytest.mark.parametrize("precision,strict,want", [("fp32", False, 17), ("bf16", False, 17), ("fp32", True, 32),
                                                   ("fp64", False, 32)])
def test_plain_sweeps_fuse_two_per_launch(homg, precision, strict, want):
    # binary32 fast lattice cycles fuse consecutive plain level-0 sweeps: of the 32 sweeps, the first
    # (level change) and the last stay single launches, the 30 in between run as 15 two-sweep launches
    import torch

    with homg.Solver(2, 129, 7, precision=precision, strict_fp=strict, exec_mode="lattice") as s:
        f = torch.from_numpy(inputs.uniform_rhs(128, 2, seed=5)).cuda()
        u = torch.zeros_like(f)
        s.solve(f, u, tol=0.0, max_cycles=1)
        st = s.stats()
    assert st["fine_iterations_per_cycle"] == 32 and st["fine_launches_per_cycle"] == want


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("schedule", [[3, 3, 3, 2, 2, 1, 1, 1, 1, 1, 0, 0, 0], [2, 1, 1, 0, 0, 0, 0, 0, 0, 0, 0]])
def test_fused_sweeps_follow_oracle_on_short_runs(homg, precision, schedule):
    # runs of 2 to 9 sweeps per level: fused pairs plus single leftovers follow the oracle's cycle
    n, levels = 256, 8
    f = inputs.uniform_rhs(n, 2, seed=3)
    for k in (1, 2):
        ref, _, _, _ = oracle.solve_mixed(f, levels, precision, tol=0.0, max_cycles=k, schedule=schedule)
        got, st, cyc, rr, hist = gpu_solve(homg, f, levels, max_cycles=k, exec_mode="lattice", precision=precision,
                                           schedule=schedule)
        assert cyc == k
        assert rel(got, ref) <= TOL[precision], (k, rel(got, ref))


@pytest.mark.parametrize("precision,want", [("fp32", 17), ("bf16", 17), ("fp64", 32)])
def test_3d_plain_sweeps_fuse_two_per_launch(homg, precision, want):
    # 3-D binary32 lattice cycles pair plain level-0 sweeps too (k_jacobi3_x2); the iterates still
    # follow the oracle's low-precision cycle
    import torch

    n, levels = 64, 6
    f_np = inputs.normal_rhs(n, 3, seed=7)
    with homg.Solver(3, n + 1, levels, precision=precision, exec_mode="lattice") as s:
        f = torch.from_numpy(f_np).cuda()
        u = torch.zeros_like(f)
        s.solve(f, u, tol=0.0, max_cycles=2)
        st = s.stats()
        got = u.cpu().numpy()
    assert st["fine_iterations_per_cycle"] == 32 and st["fine_launches_per_cycle"] == want
    if precision != "fp64":
        ref, _, _, _ = oracle.solve_mixed(f_np, levels, precision, tol=0.0, max_cycles=2)
        assert rel(got, ref) <= TOL[precision], rel(got, ref)
