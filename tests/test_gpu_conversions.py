"""The library's integer binary64 <-> binary32 conversions (used by the fast residual kernels to keep
conversions off the FP64 pipe) against the hardware conversions, bit for bit: random bit patterns of
every class, ties to even, the overflow and underflow edges, signed zeros."""

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


def doubles():
    rng = np.random.default_rng(11)
    parts = [rng.integers(0, 2 ** 64, 1 << 20, dtype=np.uint64)]  # every class, NaNs and infinities
    # binary32 normal range, random fractions
    e = rng.integers(1023 - 126, 1023 + 128, 1 << 18, dtype=np.uint64)
    f = rng.integers(0, 1 << 52, 1 << 18, dtype=np.uint64)
    s = rng.integers(0, 2, 1 << 18, dtype=np.uint64) << np.uint64(63)
    parts.append(s | (e << np.uint64(52)) | f)
    # exact ties and their neighbours: dropped 29 bits = 2^28 (+-1), kept fraction odd and even
    m = rng.integers(0, 1 << 23, 1 << 16, dtype=np.uint64)
    e = rng.integers(1023 - 126, 1023 + 128, 1 << 16, dtype=np.uint64)
    base = (e << np.uint64(52)) | (m << np.uint64(29))
    for d in (0, 1, -1):
        parts.append(base + np.uint64((1 << 28) + d))
    parts.append(base | np.uint64((1 << 29) - 1))
    # edges: largest binary32 and the tie above it, the smallest normal and below, zeros, subnormals
    edge = [0x47EFFFFFE0000000, 0x47EFFFFFF0000000, 0x47EFFFFFEFFFFFFF, 0x47F0000000000000,
            0x3810000000000000, 0x380FFFFFF0000000, 0x380FFFFFFFFFFFFF, 0x3800000000000000,
            0x0, 0x8000000000000000, 0x1, 0x800FFFFFFFFFFFFF, 0x7FF0000000000000, 0xFFF0000000000000,
            0x7FF8000000000000, 0x3FF0000000000000, 0xBFF0000010000000, 0x3FF0000030000000]
    parts.append(np.array(edge, dtype=np.uint64))
    return np.concatenate(parts).view(np.float64)


def floats(n):
    rng = np.random.default_rng(12)
    bits = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    bits[:12] = [0, 0x80000000, 1, 0x807FFFFF, 0x00800000, 0x7F7FFFFF, 0x7F800000, 0xFF800000, 0x7FC00000,
                 0x3F800000, 0xBF800001, 0x33800000]
    return bits.view(np.float32)


def test_conversions_match_hardware(homg):
    import torch

    d = torch.from_numpy(doubles()).cuda()
    f = torch.from_numpy(floats(d.numel())).cuda()
    f_out, d_out = homg.homg_check_conversions(d, f)
    want_f = d.to(torch.float32)
    want_d = f.to(torch.float64)
    got_fb = f_out.cpu().numpy().view(np.uint32)
    want_fb = want_f.cpu().numpy().view(np.uint32)
    bad = np.flatnonzero(got_fb != want_fb)
    assert bad.size == 0, [(hex(int(x)), hex(int(y))) for x, y in zip(d.cpu().numpy().view(np.uint64)[bad[:5]], got_fb[bad[:5]])]
    assert np.array_equal(d_out.cpu().numpy().view(np.uint64), want_d.cpu().numpy().view(np.uint64))


def test_conversion_arguments_are_checked(homg):
    import ctypes

    lib = homg.load()
    assert lib.homg_check_conversions(None, None, None, None, ctypes.c_int64(-1)) == homg.HOMG_EINVAL
    assert lib.homg_check_conversions(None, None, None, None, ctypes.c_int64(4)) == homg.HOMG_EINVAL
    assert lib.homg_check_conversions(None, None, None, None, ctypes.c_int64(0)) == homg.HOMG_OK
