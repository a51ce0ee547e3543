"""The largest grids the library accepts (2-D 2^15 + 1 = 32769 nodes per side, 3-D 2^10 + 1 = 1025)
and the smallest inputs (GB300 only).

At the maximum sizes the oracle is far too slow, so the checks are properties that hold at any size:
one cycle lowers the relative residual by the resolution-independent HOMG factor (below 0.2), the
library's own residual norm of the returned iterate equals the solve's last relative residual, and
the boundary stays 0. Inputs are drawn on the device from a seeded generator.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def homg():
    import torch

    import __graft_entry__

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    __graft_entry__.build()
    from paper_1108_2045_gb300 import homg as binding

    return binding


def device_rhs(ndim, n1, seed):
    import torch

    g = torch.Generator(device="cuda").manual_seed(seed)
    f = torch.rand((n1,) * ndim, generator=g, device="cuda", dtype=torch.float64) * 2 - 1
    idx = (slice(1, -1),) * ndim
    out = torch.zeros_like(f)
    out[idx] = f[idx]
    del f
    return out


@pytest.mark.parametrize("ndim,K,precision", [(2, 15, "fp32"), (2, 15, "fp64"), (3, 10, "fp32")])
def test_maximum_grid_one_cycle(homg, ndim, K, precision):
    import torch

    n1 = 2 ** K + 1
    f = device_rhs(ndim, n1, seed=K)
    u = torch.zeros_like(f)
    with homg.Solver(ndim, n1, K, precision=precision) as s:
        st, cyc, rr = s.solve(f, u, tol=0.0, max_cycles=2)
        hist = s.history()
        assert st == homg.HOMG_NOT_CONVERGED and cyc == 2
        assert hist[0] == pytest.approx(1.0, rel=1e-12)  # u0 = 0: r = f
        assert hist[1] < 0.2 and hist[2] < 0.2 * hist[1], hist
        rr2 = s.residual_norm(f, u)
        assert abs(rr2 - rr) <= 1e-6 * rr
    edge = [u[0], u[-1]] if ndim == 2 else [u[0], u[-1], u[:, 0], u[:, -1]]
    assert all(float(torch.abs(e).max()) == 0.0 for e in edge)
    del f, u
    torch.cuda.empty_cache()


def test_one_interior_node(homg):
    # 3 x 3 nodes: A = 4/h^2 on the single unknown; a damped-Jacobi cycle with omega_J = 1 is exact
    import torch

    f = torch.zeros(3, 3, dtype=torch.float64, device="cuda")
    f[1, 1] = 2.0
    u = torch.zeros_like(f)
    with homg.Solver(2, 3, 1, omega_j=1.0) as s:
        st, cyc, rr = s.solve(f, u, tol=1e-14, max_cycles=5)
    assert st == homg.HOMG_OK and cyc == 1
    assert float(u[1, 1]) == pytest.approx(2.0 / (4.0 * 4.0), rel=1e-15)


def test_empty_and_oversized_requests_are_rejected(homg):
    import ctypes

    lib = homg.load()
    h = ctypes.c_void_p()
    assert lib.homg_batch_create(0, (ctypes.c_int64 * 1)(33), None, ctypes.byref(h)) == homg.HOMG_EINVAL
    with pytest.raises(homg.HomgError) as ei:
        homg.homg_create(2, 2 ** 16 + 1, 3)
    assert ei.value.code == homg.HOMG_ESHAPE
