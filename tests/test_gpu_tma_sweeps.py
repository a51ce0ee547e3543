"""Two-sweep launches with the tile staged by TMA (k_jacobi2_x2t, GB300 only): binary32 and
bfloat16 lattice-form cycles, one problem per handle.

Bars: the iterates, cycle counts and residual histories are bit-identical to the same cycles with
the marching two-sweep kernels (tma_min_n = -1), on lattices whose sides are not multiples of the
block's 240 output columns or its 16 / 32 output rows; the converged solution meets the FP64
oracle's residual. Agreement with the oracle's low-precision cycle itself is covered by the
mixed-precision tests, which run with the default threshold.
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


def solve(homg, f_np, levels, cycles, tol=0.0, **kw):
    import torch

    with homg.Solver(2, f_np.shape[0], levels, exec_mode="lattice", **kw) as s:
        f = torch.from_numpy(f_np).cuda()
        u = torch.zeros_like(f)
        st, cyc, rr = s.solve(f, u, tol=tol, max_cycles=cycles)
        return u, st, cyc, rr, s.history()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("K,levels", [(8, 8), (10, 10), (12, 12)])
def test_tma_sweeps_are_bit_identical_to_marching_sweeps(homg, precision, K, levels):
    import torch

    f_np = inputs.uniform_rhs(2 ** K, 2, seed=50 + K)
    cycles = 1 if K == 12 else 2
    u1, _, c1, r1, h1 = solve(homg, f_np, levels, cycles, precision=precision, tma_min_n=256)
    u0, _, c0, r0, h0 = solve(homg, f_np, levels, cycles, precision=precision, tma_min_n=-1)
    assert c1 == c0 == cycles and r1 == r0 and h1 == h0
    assert torch.equal(u1, u0)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_tma_sweeps_converge_to_the_oracle_residual(homg, precision):
    n, levels = 1024, 10
    f_np = inputs.normal_rhs(n, 2, seed=61)
    u, st, cyc, rr, _ = solve(homg, f_np, levels, 60, tol=1e-10, precision=precision, tma_min_n=256)
    assert st == homg.HOMG_OK and rr <= 1e-10
    got = u.cpu().numpy()
    assert oracle.norm_interior(oracle.residual(f_np, got)) / oracle.norm_interior(f_np) <= 1.0001e-10


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_3d_tma_sweeps_are_bit_identical_to_marching_sweeps(homg, precision):
    # 3-D: the planes staged by TMA in rings, the block marching down z (k_jacobi3_x2t); 257^3 nodes:
    # the level-0 lattice of 256 intervals is not a multiple of the blocks' 240 columns, 4 rows or
    # 32 planes
    import torch

    n, levels = 256, 8
    f_np = inputs.normal_rhs(n, 3, seed=71)
    out = {}
    for tma in (256, -1):
        with homg.Solver(3, n + 1, levels, exec_mode="lattice", precision=precision, tma_min_n=tma) as s:
            f = torch.from_numpy(f_np).cuda()
            u = torch.zeros_like(f)
            st, cyc, rr = s.solve(f, u, tol=0.0, max_cycles=2)
            out[tma] = (u, cyc, rr, s.history())
    assert out[256][1:] == out[-1][1:]
    assert torch.equal(out[256][0], out[-1][0])
