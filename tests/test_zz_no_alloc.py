"""The allocation-free residual entry point (homg_residual_norm_noalloc) against homg_residual_norm.

The allocation-free call serves callers that cannot call cudaMalloc and so cannot create a handle.
Its scratch is a static device array shared by every call and left holding the previous call's
data, so the check runs two calls in a row on different inputs and compares each with the handle
entry point, within the 1e-12 relative tolerance of the other parity tests. This file is named to
be collected last.
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


@pytest.mark.parametrize("ndim,n,levels", [(2, 256, 8), (2, 4096, 12), (3, 64, 6)])
def test_noalloc_matches_handle_entry_point_twice(homg, ndim, n, levels):
    import torch

    f = torch.from_numpy(inputs.uniform_rhs(n, ndim, seed=11)).cuda()
    us = []
    for seed in (12, 13):
        u = inputs.normal_rhs(n, ndim, seed=seed) * 1e-4
        us.append(torch.from_numpy(u).cuda())
    with homg.Solver(ndim, n + 1, levels) as s:
        expect = [s.residual_norm(f, u) for u in us]
    got = [homg.homg_residual_norm_noalloc(f, u) for u in us]  # two calls in a row
    for g, e in zip(got, expect):
        assert abs(g - e) <= 1e-12 * abs(e), (g, e)
    assert got[0] != got[1]


def test_noalloc_rejects_grids_beyond_its_scratch(homg):
    import ctypes

    lib = homg.load()
    dims = (ctypes.c_int64 * 2)(16385, 16385)  # needs 131072 partial sums: rejected before any device access
    rr = ctypes.c_double(0.0)
    rc = lib.homg_residual_norm_noalloc(2, dims, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.byref(rr), None)
    assert rc == homg.HOMG_ESHAPE
    assert "static scratch" in homg.homg_last_error(None)
