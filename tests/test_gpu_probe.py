"""The FP64 issue-rate probe the benchmark uses as the denominator of the FP64 ALU fraction."""

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


def test_probe_counts_and_results(homg):
    import torch

    blocks, iters = 4, 1000
    sink = torch.full((blocks * homg.HOMG_PROBE_THREADS,), float("nan"), dtype=torch.float64, device="cuda")
    instr = homg.homg_fp64_issue_probe(1, blocks, iters, sink)
    torch.cuda.synchronize()
    assert instr == blocks * homg.HOMG_PROBE_THREADS * iters * 8
    # op 1: every chain adds b = 1e-7 to x0 = 1 + 1e-3 (thread + c), `iters` times
    t = torch.arange(homg.HOMG_PROBE_THREADS, dtype=torch.float64, device="cuda")
    expect = sum(1.0 + 1.0e-3 * (t + c) + iters * 1.0e-7 for c in range(8)).repeat(blocks)
    assert torch.allclose(sink, expect, rtol=1e-12, atol=0.0)
    homg.homg_fp64_issue_probe(0, blocks, iters, sink)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(sink).all())


def test_probe_rate_is_plausible(homg):
    """The measured rate lies between 0.1x and 1.2x the nominal 0.625e12 FP64 instructions/s."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks, iters = 8 * sms, 1024
    sink = torch.empty(blocks * homg.HOMG_PROBE_THREADS, dtype=torch.float64, device="cuda")
    for _ in range(2):
        homg.homg_fp64_issue_probe(0, blocks, iters, sink)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    instr = homg.homg_fp64_issue_probe(0, blocks, iters, sink)
    e1.record()
    torch.cuda.synchronize()
    rate = instr / (e0.elapsed_time(e1) * 1e-3)
    assert 0.1 * 0.625e12 < rate < 1.2 * 0.625e12, rate


def test_probe_rejects_bad_arguments(homg):
    import ctypes

    lib = homg.load()
    out = ctypes.c_double(0.0)
    assert lib.homg_fp64_issue_probe(2, 1, 1, ctypes.c_void_p(16), None, ctypes.byref(out)) == homg.HOMG_EINVAL
    assert lib.homg_fp64_issue_probe(0, 0, 1, ctypes.c_void_p(16), None, ctypes.byref(out)) == homg.HOMG_EINVAL
    assert lib.homg_fp64_issue_probe(0, 1, 1, None, None, ctypes.byref(out)) == homg.HOMG_EINVAL
