"""Level runs in shared memory (k_level_run2, GB300 only): in binary32 and bfloat16 lattice-form
cycles, each level run on a lattice of at most run_max_n (default 128) intervals per side -- the
level change and all of the level's sweeps -- is one launch of one block per problem.

Bars: the iterates, cycle counts and residual histories are bit-identical to the same cycles run
as separate launches (run_max_n = -1), for single problems and batches; the launches per cycle
drop by the sweeps the runs absorb. Agreement with the oracle's low-precision cycle is covered by
the mixed-precision and batch tests, which run with the default.
"""

import numpy as np
import pytest

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


def solve(homg, f_np, levels, cycles, **kw):
    import torch

    with homg.Solver(2, f_np.shape[0], levels, exec_mode="lattice", **kw) as s:
        f = torch.from_numpy(f_np).cuda()
        u = torch.zeros_like(f)
        st, cyc, rr = s.solve(f, u, tol=0.0, max_cycles=cycles)
        return u, cyc, rr, s.history(), s.stats()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("K,levels", [(10, 10), (8, 8), (7, 5), (9, 4)])
def test_level_runs_are_bit_identical_to_separate_launches(homg, precision, K, levels):
    import torch

    f_np = inputs.uniform_rhs(2 ** K, 2, seed=K)
    for cycles in (1, 3):
        u1, c1, r1, h1, s1 = solve(homg, f_np, levels, cycles, precision=precision)
        u0, c0, r0, h0, s0 = solve(homg, f_np, levels, cycles, precision=precision, run_max_n=-1)
        assert c1 == c0 == cycles and r1 == r0 and h1 == h0
        assert torch.equal(u1, u0)
    # lattices of 32..128 intervals below the finest level run as one launch each, except the
    # coarsest level's run (no level change) and lattices of at most 16 (the coarse-lattice block)
    runs = sum(1 for m in range(1, levels) if 16 < (2 ** K >> m) <= 128 and m < levels - 1)
    assert s1["kernels_per_cycle"] < s0["kernels_per_cycle"] if runs else s1["kernels_per_cycle"] == s0["kernels_per_cycle"]


def test_level_runs_with_short_and_skipped_runs(homg):
    # explicit schedules: runs of 1 and 2 sweeps, and a level change that skips a level (stride 4,
    # not a level run); every variant bit-identical to separate launches
    import torch

    f_np = inputs.normal_rhs(256, 2, seed=21)
    for schedule in ([4, 4, 3, 2, 2, 1, 0, 0, 0], [5, 3, 3, 3, 1, 1, 0, 0], [3, 2, 1, 1, 1, 1, 1, 0, 0]):
        for precision in ("fp32", "bf16"):
            u1, c1, r1, h1, _ = solve(homg, f_np, 8, 2, precision=precision, schedule=schedule)
            u0, c0, r0, h0, _ = solve(homg, f_np, 8, 2, precision=precision, schedule=schedule, run_max_n=-1)
            assert h1 == h0 and torch.equal(u1, u0), (schedule, precision)


def test_run_max_n_bounds_the_fused_lattices(homg):
    f_np = inputs.uniform_rhs(1024, 2, seed=3)
    st = {r: solve(homg, f_np, 10, 1, precision="fp32", run_max_n=r)[4]["kernels_per_cycle"] for r in (-1, 32, 64, 0)}
    assert st[-1] > st[32] > st[64] > st[0]
    with pytest.raises(homg.HomgError):
        homg.homg_create(2, 1025, 10, precision="fp32", run_max_n=129)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_level_runs_in_batches(homg, precision):
    # one block per problem of a size group; converged problems skip the run
    import torch

    sides = [65, 129, 257, 65, 513, 129]
    f_np = [inputs.normal_rhs(s - 1, 2, seed=40 + i) for i, s in enumerate(sides)]
    out = {}
    for r in (0, -1):
        with homg.BatchSolver(sides, precision=precision, run_max_n=r) as b:
            fs = [torch.from_numpy(f).cuda() for f in f_np]
            us = [torch.zeros_like(f) for f in fs]
            rc, status, cycles, relres, ms = b.solve(fs, us, tol=1e-10, max_cycles=40)
        assert all(s == homg.HOMG_OK for s in status)
        out[r] = (us, cycles, relres)
    assert out[0][1] == out[-1][1] and out[0][2] == out[-1][2]
    for a, c in zip(out[0][0], out[-1][0]):
        assert torch.equal(a, c)
    assert np.all(np.array(out[0][2]) <= 1e-10)
