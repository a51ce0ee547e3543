"""The C ABI library loads and exports every entry point ``include/homg.h`` declares; host-side
argument validation runs without a GPU (no compute call is made)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include"))) if h.endswith(".h")]


@pytest.fixture(scope="module")
def homg():
    import __graft_entry__

    from paper_1108_2045_gb300 import build

    build.build()
    from paper_1108_2045_gb300 import homg as binding

    binding.load()
    return binding


def declared_functions():
    src = "\n".join(open(h).read() for h in HEADERS)
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(homg_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("homg_create", "homg_solve", "homg_residual_norm", "homg_destroy", "homg_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(homg):
    lib = ctypes.CDLL(homg.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(homg.EXPORTS) == declared_functions()


def test_default_options(homg):
    o = homg.homg_default_options()
    assert o.max_i == 32 and o.exec_mode == homg.HOMG_EXEC_AUTO and o.diverge_factor == 1e3 and o.n_schedule == 0
    assert o.launch_mode == homg.HOMG_LAUNCH_GRAPH and o.precision == homg.HOMG_PREC_FP64


@pytest.mark.parametrize(
    "args,code",
    [
        ((1, 129, 7, 5), -1),          # ndim
        ((2, 129, 7, 7), -1),          # stencil of the wrong dimension
        ((3, 65, 6, 5), -1),
        ((2, 128, 7, 5), -2),          # not 2^K + 1
        ((2, 2, 1, 5), -2),            # K = 0
        ((2, 129, 8, 5), -1),          # levels > K
        ((2, 129, 0, 5), -1),          # levels < 1
        ((2, (1 << 16) + 1, 3, 5), -2),  # beyond the 2-D maximum
        ((3, (1 << 11) + 1, 3, 7), -2),  # beyond the 3-D maximum
    ],
)
def test_create_rejects_invalid_arguments(homg, args, code):
    with pytest.raises(homg.HomgError) as ei:
        homg.homg_create(*args)
    assert ei.value.code == code
    assert homg.homg_last_error(None)


def test_create_rejects_unequal_sides_and_bad_options(homg):
    lib = homg.load()
    dims = (ctypes.c_int64 * 2)(129, 65)
    h = ctypes.c_void_p()
    assert lib.homg_create(2, dims, 3, 5, None, ctypes.byref(h)) == homg.HOMG_ESHAPE
    assert h.value is None
    for kw in [dict(omega_j=-1.0), dict(max_i=-3), dict(exec_mode=7), dict(diverge_factor=0.5),
               dict(schedule=[1, 2]), dict(schedule=[3, 0]), dict(schedule=[0, 1, 0], exec_mode="lattice"),
               dict(launch_mode=5), dict(precision=7), dict(cycle=3), dict(cycle="v", v_pre=-1),
               dict(cycle="v", schedule=[1, 0]), dict(cycle="v", exec_mode="wholegrid")]:
        with pytest.raises(homg.HomgError) as ei:
            homg.homg_create(2, 33, 3, **kw)
        assert ei.value.code == homg.HOMG_EINVAL, kw


def test_vcycle_coarsest_level_limit(homg):
    with pytest.raises(homg.HomgError) as ei:
        homg.homg_create(2, 1025, 3, cycle="v")  # coarsest lattice 256 intervals per side
    assert ei.value.code == homg.HOMG_EINVAL and "coarsest" in str(ei.value)


def test_null_handle_calls_are_rejected(homg):
    lib = homg.load()
    assert lib.homg_solve(None, None, None, 1e-10, 5, None, None) == homg.HOMG_EINVAL
    assert lib.homg_residual_norm(None, None, None, None) == homg.HOMG_EINVAL
    assert lib.homg_set_stream(None, None) == homg.HOMG_EINVAL
    lib.homg_destroy(None)


def test_binding_refuses_host_tensors_for_device_calls(homg):
    import torch

    with pytest.raises(TypeError):
        homg._devptr(torch.zeros(3, dtype=torch.float64), "f")


def test_power_of_two_geometry_argument_checks(homg):
    cases = [((2, 129, 5), {}, homg.HOMG_ESHAPE),          # 2^K + 1 is the nested geometry's side
             ((2, 2, 1), {}, homg.HOMG_ESHAPE),            # K >= 2
             ((2, 64, 7), {}, homg.HOMG_EINVAL),           # levels <= K
             ((3, 64, 3), {}, homg.HOMG_EINVAL),           # 2-D only
             ((2, 64, 4), dict(strict_fp=True), homg.HOMG_EINVAL),
             ((2, 64, 4), dict(exec_mode="lattice"), homg.HOMG_EINVAL),
             ((2, 64, 4), dict(cycle="v"), homg.HOMG_EINVAL)]
    for args, kw, code in cases:
        with pytest.raises(homg.HomgError) as ei:
            homg.homg_create(*args, geometry="pow2", **kw)
        assert ei.value.code == code, (args, kw)
    with pytest.raises(homg.HomgError):
        homg.homg_create(2, 33, 3, geometry=7)
    with pytest.raises(homg.HomgError):
        homg.homg_batch_create([33, 65], geometry="pow2")


def test_noalloc_binding_rejects_mismatched_tensors_before_the_device(homg):
    """The allocation-free residual's binding checks shapes, devices and dtypes before it hands any
    pointer to the library (a smaller u would otherwise be read past its end)."""
    import torch

    f = torch.zeros(9, 9, dtype=torch.float64)
    cases = [torch.zeros(5, 5, dtype=torch.float64),                    # smaller u
             torch.zeros(9, 9, 9, dtype=torch.float64),                 # other dimension
             torch.zeros(9, 9, dtype=torch.float64, device="meta"),     # other device
             torch.zeros(9, 9, dtype=torch.float32)]                    # other dtype
    for u in cases:
        with pytest.raises(TypeError):
            homg.homg_residual_norm_noalloc(f, u)
    with pytest.raises(TypeError):
        homg.homg_residual_norm_noalloc(torch.zeros(9, 5, dtype=torch.float64), torch.zeros(9, 5, dtype=torch.float64))
    with pytest.raises(TypeError):  # host tensors never reach the library
        homg.homg_residual_norm_noalloc(f, torch.zeros(9, 9, dtype=torch.float64))


def test_noalloc_rejects_grids_beyond_its_scratch_on_the_host(homg):
    """Grids needing more partial sums than the static scratch holds are refused by the size check,
    which runs before any device access."""
    lib = homg.load()
    for ndim, side, parts in ((2, 16385, 140288), (3, 1025, 524288)):
        dims = (ctypes.c_int64 * ndim)(*([side] * ndim))
        rr = ctypes.c_double(0.0)
        rc = lib.homg_residual_norm_noalloc(ndim, dims, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.byref(rr), None)
        assert rc == homg.HOMG_ESHAPE
        assert ("needs %d partial sums" % parts) in homg.homg_last_error(None)


def test_persistent_launch_mode_is_for_batches_only(homg):
    with pytest.raises(homg.HomgError) as ei:
        homg.homg_create(2, 33, 3, launch_mode="persistent")
    assert ei.value.code == homg.HOMG_EINVAL and "batches" in str(ei.value)
    lib = homg.load()
    assert lib.homg_batch_check_barrier_timeout(None, None) == homg.HOMG_EINVAL
