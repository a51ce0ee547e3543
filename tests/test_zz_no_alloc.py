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


# 8193^2 (35,328 partial sums) and 513^3 (exactly HOMG_NOALLOC_MAX_BLOCKS = 65,536) are the largest
# grids the header promises; a change of the residual kernel's launch shape that shrinks that range
# fails here.
@pytest.mark.parametrize("ndim,n,levels", [(2, 256, 8), (2, 4096, 12), (3, 64, 6), (2, 8192, 13), (3, 512, 9)])
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
    # 16385^2 needs 137 x 1024 = 140,288 partial sums and 1025^3 needs 32 x 256 x 64 = 524,288: both
    # are rejected by the size check, before any device access
    for ndim, side, parts in ((2, 16385, 140288), (3, 1025, 524288)):
        dims = (ctypes.c_int64 * ndim)(*([side] * ndim))
        rr = ctypes.c_double(0.0)
        rc = lib.homg_residual_norm_noalloc(ndim, dims, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.byref(rr), None)
        assert rc == homg.HOMG_ESHAPE
        msg = homg.homg_last_error(None)
        assert "static scratch" in msg and ("needs %d partial sums" % parts) in msg, msg
