"""The two kernels of two fused plain damped-Jacobi sweeps (Sec. 2, the relaxation formula; binary32
cycles fuse consecutive plain sweeps two per launch) against each other and against two sweeps
evaluated here.

`homg_check_sweep_pair` runs the packed kernel (two columns per lane, packed binary32 pairs) and
the per-column kernel on the same lattice. They must agree bit for bit on every node: the interior
they write and the boundary and padding they must leave alone. The input's padding columns hold
NaN, so a padding value that reached a stored result would show. Both must also match two sweeps
computed with NumPy in binary32 (each sum correctly rounded; the fused multiply-adds through
binary64, which can differ from a fused result by one unit in the last place, rarely).
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
    from paper_1108_2045_gb300 import homg as h

    return h


OM, C1 = 0.2, 0.2  # fast-form scalars for omega_J = 4/5 in 2-D


def fma32(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def sweep32(E, G, n, to_store):
    """One sweep in binary32 on the interior, rounded to the storage type; boundary kept."""
    om, c1 = np.float32(OM), np.float32(C1)
    s = (E[1:n, 0:n - 1] + E[1:n, 2:n + 1]) + (E[0:n - 1, 1:n] + E[2:n + 1, 1:n])
    O = E.copy()
    O[1:n, 1:n] = to_store(fma32(np.full_like(s, c1), E[1:n, 1:n], fma32(np.full_like(s, om), s, G[1:n, 1:n])))
    return O


def lattice(n, dtype, seed):
    import torch

    pitch = -(-(n + 1) // 16) * 16
    rng = np.random.default_rng(seed)
    E = np.zeros((n + 1, pitch), np.float32)
    G = np.zeros_like(E)
    E[1:n, 1:n] = rng.standard_normal((n - 1, n - 1))
    G[1:n, 1:n] = 0.1 * rng.standard_normal((n - 1, n - 1))
    E[:, n + 1:] = np.nan
    G[:, n + 1:] = np.nan
    e = torch.from_numpy(E).to(dtype).cuda()
    g = torch.from_numpy(G).to(dtype).cuda()
    return e, g


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("n,rows", [(2, 0), (4, 1), (16, 0), (60, 3), (64, 0), (120, 7), (128, 16), (256, 0),
                                    (1024, 16), (4096, 16)])
def test_packed_pairs_equal_per_column_pairs(homg, precision, n, rows):
    import torch

    dtype = torch.float32 if precision == "fp32" else torch.bfloat16
    e, g = lattice(n, dtype, seed=n + (7 if precision == "bf16" else 0))
    sentinel = 3.0
    out_p = torch.full_like(e, sentinel)
    out_c = torch.full_like(e, sentinel)
    homg.homg_check_sweep_pair(e, g, out_p, out_c, n, OM, C1, rows)
    torch.cuda.synchronize()
    bits = torch.int32 if precision == "fp32" else torch.int16
    assert torch.equal(out_p.view(bits), out_c.view(bits))
    got = out_p.float().cpu().numpy()
    untouched = np.ones(got.shape, bool)
    untouched[1:n, 1:n] = False
    assert (got[untouched] == sentinel).all()
    assert np.isfinite(got[1:n, 1:n]).all()

    if precision == "fp32":
        to_store = lambda x: x  # noqa: E731
    else:
        to_store = lambda x: torch.from_numpy(x).to(torch.bfloat16).float().numpy()  # noqa: E731
    E = e.float().cpu().numpy()[:, :n + 1]
    G = g.float().cpu().numpy()[:, :n + 1]
    want = sweep32(sweep32(E, G, n, to_store), G, n, to_store)[1:n, 1:n]
    have = got[1:n, 1:n]
    if precision == "fp32":
        ulp = np.abs(have.view(np.int32).astype(np.int64) - want.view(np.int32).astype(np.int64))
        assert ulp.max() <= 2 and np.count_nonzero(ulp) <= max(4, 1e-5 * have.size)
    else:
        assert np.allclose(have, want, rtol=2.0 ** -7, atol=2.0 ** -7 * np.abs(want).max())


def test_sweep_pair_rejects_bad_layouts(homg):
    import torch

    n = 64
    e, g = lattice(n, torch.float32, seed=1)
    out = torch.zeros_like(e)
    short = torch.zeros((n + 1, n + 1), dtype=torch.float32, device="cuda")  # pitch n + 1 < n + 2
    import ctypes

    lib = homg.load()
    vp = ctypes.c_void_p
    rc = lib.homg_check_sweep_pair(homg.HOMG_PREC_FP32, n, ctypes.c_int64(n + 1), vp(short.data_ptr()),
                                   vp(short.data_ptr()), vp(short.data_ptr()), vp(short.data_ptr()), 0.2, 0.2, 0)
    assert rc == homg.HOMG_EINVAL
    rc = lib.homg_check_sweep_pair(homg.HOMG_PREC_FP64, n, ctypes.c_int64(e.shape[1]), vp(e.data_ptr()),
                                   vp(g.data_ptr()), vp(out.data_ptr()), vp(out.data_ptr()), 0.2, 0.2, 0)
    assert rc == homg.HOMG_EINVAL
    odd = vp(e.data_ptr() + 4)  # a float pair that starts on an odd element
    rc = lib.homg_check_sweep_pair(homg.HOMG_PREC_FP32, n, ctypes.c_int64(e.shape[1]), odd, vp(g.data_ptr()),
                                   vp(out.data_ptr()), vp(out.data_ptr()), 0.2, 0.2, 0)
    assert rc == homg.HOMG_EINVAL
