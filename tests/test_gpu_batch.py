"""Batched solves on the GPU (GB300 only): every problem of a batch must come out bit-identical to
solving it alone (the batched launches run the same per-node arithmetic and reduction order), and
problems must not influence each other's outcome."""

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


def single(homg, f_np, tol, max_cycles, precision):
    import torch

    K = int(np.log2(f_np.shape[0] - 1))
    with homg.Solver(2, f_np.shape[0], K, precision=precision) as s:
        f = torch.from_numpy(f_np).cuda()
        u = torch.zeros_like(f)
        st, cyc, rr = s.solve(f, u, tol=tol, max_cycles=max_cycles)
        return u.cpu().numpy(), st, cyc, rr


@pytest.mark.parametrize("precision", ["fp32", "fp64", "bf16"])
def test_batch_matches_single_solves(homg, precision):
    import torch

    rng = np.random.default_rng(2)
    ks = [5, 6, 7, 8, 6, 5, 7, 9, 6, 8, 5, 7]
    fs_np = [inputs.normal_rhs(2 ** k, 2, seed=int(rng.integers(1 << 30))) for k in ks]
    with homg.BatchSolver([2 ** k + 1 for k in ks], precision=precision) as b:
        st = b.stats()
        assert st["groups"] == 5 and sorted(st["counts"]) == [1, 2, 3, 3, 3] and all(r >= 1 for r in st["rows"])
        fs = [torch.from_numpy(f).cuda() for f in fs_np]
        us = [torch.zeros_like(f) for f in fs]
        rc, status, cycles, relres, ms = b.solve(fs, us, tol=1e-10, max_cycles=40)
        assert rc == homg.HOMG_OK and all(s == homg.HOMG_OK for s in status)
        assert all(t > 0 for t in ms)
        for p, f_np in enumerate(fs_np):
            ref, st1, cyc1, rr1 = single(homg, f_np, 1e-10, 40, precision)
            assert (status[p], cycles[p]) == (st1, cyc1)
            assert relres[p] == rr1
            np.testing.assert_array_equal(us[p].cpu().numpy(), ref)
        # a second solve on the same handle reuses its graphs and gives the same answer
        us2 = [torch.zeros_like(f) for f in fs]
        rc2, status2, cycles2, relres2, _ = b.solve(fs, us2, tol=1e-10, max_cycles=40)
        assert cycles2 == cycles and relres2 == relres
        for a, c in zip(us, us2):
            assert torch.equal(a, c)


def test_batch_problems_are_independent(homg):
    import torch

    n = 64
    good = inputs.uniform_rhs(n, 2, seed=1)
    zero = np.zeros_like(good)
    bad = good.copy()
    bad[7, 9] = np.nan
    f_np = [good, zero, bad, good]
    with homg.BatchSolver([n + 1] * 4, precision="fp32") as b:
        fs = [torch.from_numpy(f).cuda() for f in f_np]
        us = [torch.zeros_like(f) for f in fs]
        rc, status, cycles, relres, ms = b.solve(fs, us, tol=1e-10, max_cycles=40)
    assert status == [homg.HOMG_OK, homg.HOMG_OK, homg.HOMG_DIVERGED, homg.HOMG_OK]
    assert rc == homg.HOMG_DIVERGED
    assert cycles[1] == 0 and relres[1] == 0.0 and torch.count_nonzero(us[1]) == 0
    assert torch.equal(us[0], us[3]) and cycles[0] == cycles[3]
    ref, _, cyc1, _ = single(homg, good, 1e-10, 40, "fp32")
    np.testing.assert_array_equal(us[0].cpu().numpy(), ref)


def test_batch_continuation_beyond_one_graph(homg):
    # an unreachable tolerance runs to max_cycles, past the cycles one graph launch unrolls
    import torch

    n = 32
    f_np = [inputs.uniform_rhs(n, 2, seed=s) for s in (3, 4)]
    with homg.BatchSolver([n + 1] * 2, precision="fp64") as b:
        fs = [torch.from_numpy(f).cuda() for f in f_np]
        us = [torch.zeros_like(f) for f in fs]
        rc, status, cycles, relres, ms = b.solve(fs, us, tol=0.0, max_cycles=30)
    assert status == [homg.HOMG_NOT_CONVERGED] * 2 and cycles == [30, 30]
    ref, st1, cyc1, rr1 = single(homg, f_np[0], 0.0, 30, "fp64")
    assert cyc1 == 30 and relres[0] == rr1
    np.testing.assert_array_equal(us[0].cpu().numpy(), ref)


def test_batch_rejects_unsupported_options(homg):
    for kw in [dict(strict_fp=True), dict(exec_mode="wholegrid"), dict(cycle="v"), dict(launch_mode="stream")]:
        with pytest.raises(homg.HomgError):
            homg.homg_batch_create([33, 65], **kw)
    with pytest.raises(homg.HomgError):
        homg.homg_batch_create([33, 64])


def test_full_uneven_batch_sampled_against_oracle(homg):
    # the benchmarked launch configuration: 1024 problems, sides 2^k + 1 with k ~ U{6..10} (seed 1),
    # FP32 cycles; every problem converges, sampled solutions pass the oracle's own FP64 residual
    # test and equal a solve of the same problem alone, bit for bit
    import torch

    import oracle

    oracle.build()
    ks, fs_np = inputs.uneven_batch(1024, seed=1)
    fs = [torch.from_numpy(f).cuda() for f in fs_np]
    us = [torch.zeros_like(f) for f in fs]
    with homg.BatchSolver([2 ** k + 1 for k in ks], precision="fp32") as b:
        rc, status, cycles, relres, ms = b.solve(fs, us, tol=1e-10, max_cycles=40)
    assert rc == homg.HOMG_OK and all(s == homg.HOMG_OK for s in status) and max(relres) <= 1e-10
    ks_arr = np.array(ks)
    for k in range(6, 11):
        for i in np.flatnonzero(ks_arr == k)[:2]:
            un = us[i].cpu().numpy()
            rr = oracle.norm_interior(oracle.residual(fs_np[i], un)) / oracle.norm_interior(fs_np[i])
            # r = f - A u cancels to ~1e-10 of f, so the two FP64 residuals agree to ~1e-6 relative
            assert rr <= 1.0001e-10 and abs(rr - relres[i]) <= 1e-4 * rr, (k, rr, relres[i])
        i = int(np.flatnonzero(ks_arr == k)[-1])
        ref, st1, cyc1, rr1 = single(homg, fs_np[i], 1e-10, 40, "fp32")
        assert (st1, cyc1, rr1) == (status[i], cycles[i], relres[i])
        np.testing.assert_array_equal(us[i].cpu().numpy(), ref)


def _rel(a, b):
    """Larger of the relative 2-norm error and the worst node's error against max |b|."""
    return max(np.linalg.norm(a - b) / np.linalg.norm(b), np.max(np.abs(a - b)) / np.max(np.abs(b)))


BATCH_ITERATE_TOL = {"fp64": 1e-12, "fp32": 1e-5, "bf16": 5e-2}


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_batch_iterates_match_oracle(homg, precision):
    """The iterates of a batch after one and two cycles against the oracle's own solve of each
    problem (FP64 cycles: oracle.solve; binary32 / bfloat16 cycles: oracle.solve_mixed), one problem
    of every side class 65..1025 of the benchmark batch plus repeats, so that every group of the
    batched launches is checked, not only the batch against the GPU's single solves. Tolerances are
    those of the single-problem parity tests."""
    import torch

    import oracle

    oracle.build()
    ks = [6, 7, 8, 9, 10, 7, 6]
    fs_np = [inputs.normal_rhs(2 ** k, 2, seed=40 + i) for i, k in enumerate(ks)]
    fs = [torch.from_numpy(f).cuda() for f in fs_np]
    with homg.BatchSolver([2 ** k + 1 for k in ks], precision=precision) as b:
        for cycles in (1, 2):
            us = [torch.zeros_like(f) for f in fs]
            rc, status, cyc, relres, _ = b.solve(fs, us, tol=0.0, max_cycles=cycles)
            assert rc == homg.HOMG_NOT_CONVERGED and cyc == [cycles] * len(ks)
            for p, (k, f_np) in enumerate(zip(ks, fs_np)):
                if precision == "fp64":
                    ref, _, _, rhist = oracle.solve(f_np, k, tol=0.0, max_cycles=cycles)
                else:
                    ref, _, _, rhist = oracle.solve_mixed(f_np, k, precision, tol=0.0, max_cycles=cycles)
                err = _rel(us[p].cpu().numpy(), ref)
                assert err <= BATCH_ITERATE_TOL[precision], (precision, cycles, k, err)
                if precision == "fp64":
                    assert abs(relres[p] - rhist[-1]) <= 1e-9 * rhist[-1], (cycles, k, relres[p], rhist[-1])


def test_persistent_batch_matches_graph_batch(homg):
    """The persistent kernel runs the same ops with the same arithmetic as the per-group graphs:
    after a fixed number of cycles the iterates are bit-identical (only the order of the final norm
    sums differs, so the relative residuals agree to rounding), and a solve to 1e-10 takes the same
    cycles and ends on the same solution."""
    import torch

    rng = np.random.default_rng(3)
    ks = [5, 6, 7, 8, 6, 5, 7, 9, 6, 8, 5, 10]
    fs_np = [inputs.normal_rhs(2 ** k, 2, seed=int(rng.integers(1 << 30))) for k in ks]
    sides = [2 ** k + 1 for k in ks]
    fs = [torch.from_numpy(f).cuda() for f in fs_np]
    for precision in ("fp32", "fp64", "bf16"):
        with homg.BatchSolver(sides, precision=precision) as bg, \
                homg.BatchSolver(sides, precision=precision, launch_mode="persistent") as bp:
            for tol, cyc in ((0.0, 2), (1e-10, 40)):
                ug = [torch.zeros_like(f) for f in fs]
                up = [torch.zeros_like(f) for f in fs]
                rg = bg.solve(fs, ug, tol=tol, max_cycles=cyc)
                rp = bp.solve(fs, up, tol=tol, max_cycles=cyc)
                assert rp[0] == rg[0] and rp[1] == rg[1] and rp[2] == rg[2], (precision, tol, rp[:3], rg[:3])
                for a, b in zip(rp[3], rg[3]):
                    assert abs(a - b) <= 1e-12 * b, (precision, a, b)
                for a, b in zip(up, ug):
                    assert torch.equal(a, b), precision


def test_persistent_batch_iterates_match_oracle(homg):
    import torch

    import oracle

    oracle.build()
    ks = [6, 7, 8, 9, 10, 7]
    fs_np = [inputs.normal_rhs(2 ** k, 2, seed=60 + i) for i, k in enumerate(ks)]
    fs = [torch.from_numpy(f).cuda() for f in fs_np]
    with homg.BatchSolver([2 ** k + 1 for k in ks], precision="fp32", launch_mode="persistent") as b:
        us = [torch.zeros_like(f) for f in fs]
        rc, status, cyc, relres, _ = b.solve(fs, us, tol=0.0, max_cycles=2)
        assert cyc == [2] * len(ks)
        for p, (k, f_np) in enumerate(zip(ks, fs_np)):
            ref, _, _, _ = oracle.solve_mixed(f_np, k, "fp32", tol=0.0, max_cycles=2)
            assert _rel(us[p].cpu().numpy(), ref) <= BATCH_ITERATE_TOL["fp32"], k
        us = [torch.zeros_like(f) for f in fs]
        rc, status, cyc, relres, ms = b.solve(fs, us, tol=1e-10, max_cycles=40)
        assert rc == homg.HOMG_OK and all(t > 0 for t in ms)
        for p, f_np in enumerate(fs_np):
            rr = oracle.norm_interior(oracle.residual(f_np, us[p].cpu().numpy())) / oracle.norm_interior(f_np)
            assert rr <= 1.0001e-10, (p, rr)


def test_persistent_batch_problems_are_independent(homg):
    import torch

    n = 64
    good = inputs.uniform_rhs(n, 2, seed=1)
    bad = good.copy()
    bad[7, 9] = np.nan
    f_np = [good, np.zeros_like(good), bad, good, inputs.uniform_rhs(32, 2, seed=2)]
    with homg.BatchSolver([f.shape[0] for f in f_np], precision="fp32", launch_mode="persistent") as b:
        fs = [torch.from_numpy(f).cuda() for f in f_np]
        us = [torch.zeros_like(f) for f in fs]
        rc, status, cycles, relres, ms = b.solve(fs, us, tol=1e-10, max_cycles=40)
    assert status == [homg.HOMG_OK, homg.HOMG_OK, homg.HOMG_DIVERGED, homg.HOMG_OK, homg.HOMG_OK]
    assert rc == homg.HOMG_DIVERGED and cycles[1] == 0 and torch.count_nonzero(us[1]) == 0
    assert torch.equal(us[0], us[3])
    ref, _, _, _ = single(homg, good, 1e-10, 40, "fp32")
    np.testing.assert_array_equal(us[0].cpu().numpy(), ref)


def test_persistent_barrier_wait_gives_up_and_context_stays_usable(homg):
    """A grid barrier that can never complete (it waits for one block more than the launch has):
    every block's bounded wait gives up after 0.25 s, the call reports HOMG_TIMEOUT, and the same
    batch then solves normally."""
    import torch

    n = 32
    f_np = [inputs.uniform_rhs(n, 2, seed=s) for s in (5, 6)]
    with homg.BatchSolver([n + 1] * 2, precision="fp32", launch_mode="persistent") as b:
        rc, ms = b.check_barrier_timeout()
        assert rc == homg.HOMG_TIMEOUT and "gave up" in homg.homg_last_error(None)
        assert 200.0 <= ms <= 5000.0, ms
        fs = [torch.from_numpy(f).cuda() for f in f_np]
        us = [torch.zeros_like(f) for f in fs]
        rc, status, cycles, relres, _ = b.solve(fs, us, tol=1e-10, max_cycles=40)
    assert rc == homg.HOMG_OK
    ref, _, cyc1, _ = single(homg, f_np[0], 1e-10, 40, "fp32")
    assert cycles[0] == cyc1
    np.testing.assert_array_equal(us[0].cpu().numpy(), ref)
