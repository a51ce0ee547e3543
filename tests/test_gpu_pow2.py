"""Power-of-two grids (Sec. 3) on the GPU vs the CPU oracle (GB300 only).

Bar: FP64 cycles within ||u_gpu - u_oracle|| / ||u_oracle|| <= 1e-12 after every cycle (the fast
whole-grid form); every converged solution, FP64 and FP32 cycles, passes the oracle's own FP64
residual test.
"""

import numpy as np
import pytest

import oracle

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


def rhs(N, seed):
    f = np.zeros((N, N))
    f[1:-1, 1:-1] = np.random.default_rng(seed).uniform(-1, 1, (N - 2, N - 2))
    return f


def gpu_solve(homg, f_np, levels, tol=0.0, max_cycles=1, **kw):
    import torch

    N = f_np.shape[0]
    with homg.Solver(2, N, levels, geometry="pow2", **kw) as s:
        f = torch.from_numpy(np.ascontiguousarray(f_np)).cuda()
        u = torch.zeros_like(f)
        st, cyc, rr = s.solve(f, u, tol=tol, max_cycles=max_cycles)
        return u.cpu().numpy(), st, cyc, rr, s.history()


def rel(a, b):
    """The larger of two relative errors of a against b: in the 2-norm over the grid, and at the
    worst single node against the largest |b| (so no single node can hide in a large grid's norm)."""
    nb = np.linalg.norm(b)
    mb = np.max(np.abs(b)) if b.size else 0.0
    return max(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0),
               (np.max(np.abs(a - b)) if b.size else 0.0) / (mb if mb > 0 else 1.0))


@pytest.mark.parametrize("K,levels", [(2, 2), (3, 3), (4, 4), (6, 6), (6, 3), (8, 8), (9, 5)])
def test_cycles_match_oracle(homg, K, levels):
    N = 2 ** K
    f = rhs(N, K)
    for k in (1, 2, 3):
        ref, _, _, rhist = oracle.pow2_solve(f, levels, tol=0.0, max_cycles=k)
        got, st, cyc, rr, hist = gpu_solve(homg, f, levels, max_cycles=k)
        assert st == homg.HOMG_NOT_CONVERGED and cyc == k
        assert rel(got, ref) <= 1e-12, (k, rel(got, ref))
        np.testing.assert_allclose(hist, rhist, rtol=1e-9)


@pytest.mark.parametrize("schedule", [[3, 1, 2, 0, 0], [0, 2, 2, 1, 0]])
def test_custom_schedules_match_oracle(homg, schedule):
    N, levels = 64, 4
    f = rhs(N, 11)
    ref, _, _, _ = oracle.pow2_solve(f, levels, tol=0.0, max_cycles=2, schedule=schedule)
    got, *_ = gpu_solve(homg, f, levels, max_cycles=2, schedule=schedule)
    assert rel(got, ref) <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("launch", ["graph", "stream"])
def test_converged_solution_passes_the_oracle_residual(homg, precision, launch):
    N, levels = 512, 9
    f = rhs(N, 12)
    got, st, cyc, rr, hist = gpu_solve(homg, f, levels, tol=1e-10, max_cycles=60, precision=precision,
                                       launch_mode=launch)
    assert st == homg.HOMG_OK and rr <= 1e-10 and np.all(np.diff(hist) < 0)
    assert oracle.norm_interior(oracle.residual(f, got)) / oracle.norm_interior(f) <= 1.0001e-10


def test_benchmark_grid_first_cycle_matches_oracle(homg):
    # 4096^2 nodes, 12 levels: the power-of-two workload the benchmark times
    N, K = 4096, 12
    f = rhs(N, 0)
    ref, _, _, rhist = oracle.pow2_solve(f, K, tol=0.0, max_cycles=1)
    got, st, cyc, rr, hist = gpu_solve(homg, f, K, max_cycles=1)
    assert rel(got, ref) <= 1e-12, rel(got, ref)
    np.testing.assert_allclose(hist, rhist, rtol=1e-9)
