"""The classic V(2,2) comparator on the GPU against the oracle's V-cycle (GB300 only).

Same bar as the HOMG path: strict mode bit-identical after each cycle, fast mode within 1e-12
relative; full solves reach 1e-10 with the oracle's cycle count."""

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

    with homg.Solver(f_np.ndim, f_np.shape[0], levels, cycle="v", **kw) as s:
        f = torch.from_numpy(np.ascontiguousarray(f_np)).cuda()
        u = torch.zeros_like(f)
        status, cycles, relres = s.solve(f, u, tol=tol, max_cycles=max_cycles)
        return u.cpu().numpy(), status, cycles, relres, s.history(), s.stats()


def rel(a, b):
    """The larger of two relative errors of a against b: in the 2-norm over the grid, and at the
    worst single node against the largest |b| (so no single node can hide in a large grid's norm)."""
    nb = np.linalg.norm(b)
    mb = np.max(np.abs(b)) if b.size else 0.0
    return max(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0),
               (np.max(np.abs(a - b)) if b.size else 0.0) / (mb if mb > 0 else 1.0))


@pytest.mark.parametrize("ndim,K,levels", [(2, 3, 3), (2, 5, 5), (2, 7, 7), (2, 8, 4), (2, 10, 10), (3, 4, 4), (3, 5, 5), (3, 6, 4)])
@pytest.mark.parametrize("strict", [True, False])
def test_vcycle_matches_oracle(homg, ndim, K, levels, strict):
    n = 2 ** K
    f = inputs.uniform_rhs(n, ndim, seed=K + 20)
    for k in (1, 2, 3):
        ref, _, _, rhist = oracle.solve_vcycle(f, levels, tol=0.0, max_cycles=k)
        got, st, cyc, rr, hist, _ = gpu_solve(homg, f, levels, max_cycles=k, strict_fp=strict)
        assert cyc == k
        if strict:
            np.testing.assert_array_equal(got, ref)
        else:
            assert rel(got, ref) <= 1e-12, (k, rel(got, ref))
        np.testing.assert_allclose(hist, rhist, rtol=1e-9)


@pytest.mark.parametrize("v", [(1, 1), (3, 1), (2, 4)])
def test_vcycle_smoothing_counts(homg, v):
    n, K = 64, 6
    f = inputs.uniform_rhs(n, 2, seed=5)
    ref, _, _, _ = oracle.solve_vcycle(f, K, nu1=v[0], nu2=v[1], tol=0.0, max_cycles=2)
    got, st, cyc, rr, hist, _ = gpu_solve(homg, f, K, max_cycles=2, v_pre=v[0], v_post=v[1])
    assert rel(got, ref) <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_vcycle_full_solve(homg, precision):
    n, K = 1024, 10
    f = inputs.uniform_rhs(n, 2, seed=0)
    ref, rst, rcyc, rhist = oracle.solve_vcycle(f, K, tol=1e-10, max_cycles=60)
    got, st, cyc, rr, hist, stats = gpu_solve(homg, f, K, tol=1e-10, max_cycles=60, precision=precision)
    assert st == homg.HOMG_OK and rr <= 1e-10
    r = oracle.residual(f, got)
    assert oracle.norm_interior(r) / oracle.norm_interior(f) <= 1e-10
    if precision == "fp64":
        assert cyc == rcyc and rel(got, ref) <= 1e-12
    else:
        assert abs(cyc - rcyc) <= 3
