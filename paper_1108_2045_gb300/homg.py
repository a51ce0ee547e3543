"""Python binding of the HOMG C ABI (``include/homg.h``): argument marshalling only.

Every function has the name of the C entry point it calls. Grid arrays passed as device pointers
are torch CUDA tensors (float64, contiguous, shape (n+1,)*ndim); host arrays are numpy arrays or
CPU tensors. All arithmetic runs in ``lib/libhomg.so``; there is no fallback: if the library is
missing, loading raises.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libhomg.so")

HOMG_OK, HOMG_NOT_CONVERGED, HOMG_DIVERGED, HOMG_TIMEOUT = 0, 1, 2, 3
HOMG_EINVAL, HOMG_ESHAPE, HOMG_ECUDA, HOMG_ENOMEM = -1, -2, -3, -4
HOMG_EXEC_AUTO, HOMG_EXEC_WHOLEGRID, HOMG_EXEC_LATTICE = 0, 1, 2
HOMG_LAUNCH_GRAPH, HOMG_LAUNCH_STREAM, HOMG_LAUNCH_PERSISTENT = 0, 1, 2
HOMG_PREC_FP64, HOMG_PREC_FP32, HOMG_PREC_BF16 = 0, 1, 2
HOMG_MAX_CYCLES = 200

EXEC_MODES = {"auto": HOMG_EXEC_AUTO, "wholegrid": HOMG_EXEC_WHOLEGRID, "lattice": HOMG_EXEC_LATTICE}
LAUNCH_MODES = {"graph": HOMG_LAUNCH_GRAPH, "stream": HOMG_LAUNCH_STREAM, "persistent": HOMG_LAUNCH_PERSISTENT}
PRECISIONS = {"fp64": HOMG_PREC_FP64, "fp32": HOMG_PREC_FP32, "bf16": HOMG_PREC_BF16}
HOMG_CYCLE_HOMG, HOMG_CYCLE_V = 0, 1
CYCLES = {"homg": HOMG_CYCLE_HOMG, "v": HOMG_CYCLE_V}

# Every entry point declared in include/homg.h (checked by the symbol test).
EXPORTS = [
    "homg_default_options",
    "homg_create",
    "homg_set_stream",
    "homg_solve",
    "homg_solve_host",
    "homg_residual_norm",
    "homg_set_coefficient",
    "homg_get_history",
    "homg_get_stats",
    "homg_last_error",
    "homg_destroy",
    "homg_residual_norm_noalloc",
    "homg_check_conversions",
    "homg_check_sweep_pair",
    "homg_fp64_issue_probe",
    "homg_batch_create",
    "homg_batch_set_stream",
    "homg_batch_solve",
    "homg_batch_get_stats",
    "homg_batch_destroy",
    "homg_batch_check_barrier_timeout",
    "homg_net_param_count",
    "homg_net_create",
    "homg_net_set_stream",
    "homg_net_set_params",
    "homg_net_get_params",
    "homg_net_get_grads",
    "homg_net_forward",
    "homg_net_train_step",
    "homg_net_gather_patches",
    "homg_net_check_barrier_timeout",
    "homg_net_last_error",
    "homg_net_destroy",
    "homg_features",
    "homg_solve_learned",
    "homg_net_set_loss",
    "homg_set_learned_judge",
    "homg_net_set_tile_rows",
]

HOMG_BATCH_MAX_GROUPS = 16


class homg_options(ctypes.Structure):
    _fields_ = [
        ("omega_j", ctypes.c_double),
        ("max_i", ctypes.c_int),
        ("n_schedule", ctypes.c_int),
        ("schedule", ctypes.POINTER(ctypes.c_int)),
        ("exec_mode", ctypes.c_int),
        ("strict_fp", ctypes.c_int),
        ("diverge_factor", ctypes.c_double),
        ("launch_mode", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("cycle", ctypes.c_int),
        ("v_pre", ctypes.c_int),
        ("v_post", ctypes.c_int),
        ("geometry", ctypes.c_int),
        ("run_max_n", ctypes.c_int),
        ("tma_min_n", ctypes.c_int),
    ]


class homg_stats(ctypes.Structure):
    _fields_ = [
        ("cycles", ctypes.c_int),
        ("status", ctypes.c_int),
        ("exec_mode", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("iterations_per_cycle", ctypes.c_int),
        ("fine_iterations_per_cycle", ctypes.c_int),
        ("kernels_per_cycle", ctypes.c_int),
        ("kernels_fixed", ctypes.c_int),
        ("kernel_launches", ctypes.c_longlong),
        ("solve_ms", ctypes.c_double),
        ("coarse_ms", ctypes.c_double),
        ("fine_ms", ctypes.c_double),
        ("residual_ms", ctypes.c_double),
        ("setup_ms", ctypes.c_double),
        ("fine_bytes_per_iteration", ctypes.c_double),
        ("fine_flops_per_iteration", ctypes.c_double),
        ("coarse_bytes_per_cycle", ctypes.c_double),
        ("coarse_fp64_ops_per_cycle", ctypes.c_double),
        ("fine_launches_per_cycle", ctypes.c_int),
    ]


class homg_batch_stats(ctypes.Structure):
    _fields_ = [
        ("groups", ctypes.c_int),
        ("solve_ms", ctypes.c_double),
        ("sides", ctypes.c_int64 * HOMG_BATCH_MAX_GROUPS),
        ("counts", ctypes.c_int * HOMG_BATCH_MAX_GROUPS),
        ("rows", ctypes.c_int * HOMG_BATCH_MAX_GROUPS),
        ("tuned_us", ctypes.c_double * HOMG_BATCH_MAX_GROUPS),
    ]


_lib = None


def load(path=LIB_PATH):
    """Load ``libhomg.so`` (raises if it has not been built: there is no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("HOMG CUDA library not built (%s missing): run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    lib.homg_default_options.argtypes = [ctypes.POINTER(homg_options)]
    lib.homg_default_options.restype = None
    lib.homg_create.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.c_int,
                                ctypes.POINTER(homg_options), ctypes.POINTER(vp)]
    lib.homg_set_stream.argtypes = [vp, vp]
    lib.homg_solve.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_int, ip, dp]
    lib.homg_solve_host.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_int, ip, dp]
    lib.homg_residual_norm.argtypes = [vp, vp, vp, dp]
    lib.homg_set_coefficient.argtypes = [vp, vp]
    fp = ctypes.POINTER(ctypes.c_float)
    lib.homg_net_param_count.restype = ctypes.c_int64
    lib.homg_net_create.argtypes = [ctypes.POINTER(vp)]
    lib.homg_net_set_stream.argtypes = [vp, vp]
    lib.homg_net_set_params.argtypes = [vp, fp, ctypes.c_int64]
    lib.homg_net_get_params.argtypes = [vp, fp, ctypes.c_int64]
    lib.homg_net_get_grads.argtypes = [vp, fp, ctypes.c_int64]
    lib.homg_net_forward.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]
    lib.homg_net_train_step.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float, fp]
    lib.homg_net_gather_patches.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int,
                                            vp, vp]
    lib.homg_net_check_barrier_timeout.argtypes = [vp, dp]
    lib.homg_net_last_error.argtypes = [vp]
    lib.homg_net_last_error.restype = ctypes.c_char_p
    lib.homg_net_destroy.argtypes = [vp]
    lib.homg_features.argtypes = [vp, vp, vp, vp, vp, vp, dp]
    lib.homg_solve_learned.argtypes = [vp, vp, vp, vp, ctypes.c_double, ctypes.c_int, ip, dp, ip]
    lib.homg_net_set_loss.argtypes = [vp, ctypes.c_int]
    lib.homg_net_set_tile_rows.argtypes = [vp, ctypes.c_int]
    lib.homg_set_learned_judge.argtypes = [vp, ctypes.c_int]
    lib.homg_get_history.argtypes = [vp, dp, ctypes.c_int]
    lib.homg_get_stats.argtypes = [vp, ctypes.POINTER(homg_stats)]
    lib.homg_last_error.argtypes = [vp]
    lib.homg_last_error.restype = ctypes.c_char_p
    lib.homg_residual_norm_noalloc.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), vp, vp, dp, vp]
    lib.homg_fp64_issue_probe.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, dp]
    lib.homg_check_sweep_pair.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, vp, vp, vp, vp, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int]
    lib.homg_destroy.argtypes = [vp]
    lib.homg_destroy.restype = None
    vpp = ctypes.POINTER(ctypes.c_void_p)
    lib.homg_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(homg_options),
                                      ctypes.POINTER(vp)]
    lib.homg_batch_set_stream.argtypes = [vp, vp]
    lib.homg_batch_solve.argtypes = [vp, vpp, vpp, ctypes.c_double, ctypes.c_int, ip, ip, dp, dp]
    lib.homg_batch_get_stats.argtypes = [vp, ctypes.POINTER(homg_batch_stats)]
    lib.homg_batch_check_barrier_timeout.argtypes = [vp, dp]
    lib.homg_batch_destroy.argtypes = [vp]
    lib.homg_batch_destroy.restype = None
    lib.homg_net_destroy.restype = None
    not_int = ("homg_default_options", "homg_last_error", "homg_destroy", "homg_batch_destroy", "homg_net_last_error",
               "homg_net_destroy", "homg_net_param_count")
    for name in EXPORTS:
        if name not in not_int:
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class HomgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("HOMG error %d: %s" % (code, msg))
        self.code = code


def homg_last_error(handle=None):
    return load().homg_last_error(handle).decode(errors="replace")


def homg_default_options():
    o = homg_options()
    load().homg_default_options(ctypes.byref(o))
    return o


def _check(rc, handle):
    if rc < 0:
        raise HomgError(rc, homg_last_error(handle))
    return rc


GEOMETRIES = {"nested": 0, "pow2": 1}
HOMG_GEOM_NESTED, HOMG_GEOM_POW2 = 0, 1


def _options(omega_j=0.0, max_i=32, schedule=None, exec_mode="auto", strict_fp=False, diverge_factor=0.0,
             launch_mode="graph", precision="fp64", cycle="homg", v_pre=0, v_post=0, geometry="nested", run_max_n=0,
             tma_min_n=0):
    o = homg_default_options()
    o.omega_j = omega_j
    o.max_i = max_i
    o.exec_mode = EXEC_MODES[exec_mode] if isinstance(exec_mode, str) else int(exec_mode)
    o.strict_fp = 1 if strict_fp else 0
    o.diverge_factor = diverge_factor
    o.launch_mode = LAUNCH_MODES[launch_mode] if isinstance(launch_mode, str) else int(launch_mode)
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.cycle = CYCLES[cycle] if isinstance(cycle, str) else int(cycle)
    o.v_pre = v_pre
    o.v_post = v_post
    o.geometry = GEOMETRIES[geometry] if isinstance(geometry, str) else int(geometry)
    o.run_max_n = int(run_max_n)
    o.tma_min_n = int(tma_min_n)
    keep = None
    if schedule is not None:
        keep = (ctypes.c_int * len(schedule))(*schedule)
        o.n_schedule = len(schedule)
        o.schedule = ctypes.cast(keep, ctypes.POINTER(ctypes.c_int))
    return o, keep


def homg_batch_create(sides, **opts):
    """Create a batch of 2-D problems with the given nodes per side; returns an opaque handle."""
    lib = load()
    o, _keep = _options(**opts)
    arr = (ctypes.c_int64 * len(sides))(*sides)
    h = ctypes.c_void_p()
    _check(lib.homg_batch_create(len(sides), arr, ctypes.byref(o), ctypes.byref(h)), None)
    return h.value


def homg_batch_set_stream(handle, stream):
    raw = getattr(stream, "cuda_stream", stream) or 0
    return _check(load().homg_batch_set_stream(handle, ctypes.c_void_p(raw)), None)


def homg_batch_solve(handle, fs, us, tol=1e-10, max_cycles=50):
    """Solve every problem in place (lists of device tensors). Returns (rc, status, cycles, relres, solve_ms)."""
    n = len(fs)
    fp = (ctypes.c_void_p * n)(*[_devptr(f, "f").value for f in fs])
    up = (ctypes.c_void_p * n)(*[_devptr(u, "u").value for u in us])
    st, cy = (ctypes.c_int * n)(), (ctypes.c_int * n)()
    rr, ms = (ctypes.c_double * n)(), (ctypes.c_double * n)()
    rc = load().homg_batch_solve(handle, fp, up, tol, max_cycles, st, cy, rr, ms)
    _check(rc, None)
    return rc, list(st), list(cy), list(rr), list(ms)


def homg_batch_get_stats(handle):
    s = homg_batch_stats()
    _check(load().homg_batch_get_stats(handle, ctypes.byref(s)), None)
    g = s.groups
    return {"groups": g, "solve_ms": s.solve_ms, "sides": list(s.sides[:g]), "counts": list(s.counts[:g]),
            "rows": list(s.rows[:g]), "tuned_us": list(s.tuned_us[:g])}


def homg_batch_destroy(handle):
    if handle:
        load().homg_batch_destroy(handle)


class BatchSolver:
    """Owner of a batch handle (same options as homg_create)."""

    def __init__(self, sides, **opts):
        self.sides = list(sides)
        self.handle = homg_batch_create(self.sides, **opts)

    def set_stream(self, stream):
        return homg_batch_set_stream(self.handle, stream)

    def solve(self, fs, us, tol=1e-10, max_cycles=50):
        return homg_batch_solve(self.handle, fs, us, tol, max_cycles)

    def stats(self):
        return homg_batch_get_stats(self.handle)

    def check_barrier_timeout(self):
        """Persistent batches: run the grid barrier's failure-path self-test; returns (return code,
        milliseconds the launch took)."""
        ms = ctypes.c_double(0.0)
        rc = load().homg_batch_check_barrier_timeout(self.handle, ctypes.byref(ms))
        return rc, ms.value

    def close(self):
        homg_batch_destroy(self.handle)
        self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False


def homg_create(ndim, n_nodes, levels, stencil=None, **opts):
    """Create a handle for an (n_nodes)^ndim grid; returns an opaque handle (int). Options as in
    homg_options (omega_j, max_i, schedule, exec_mode, strict_fp, diverge_factor, launch_mode,
    precision, cycle, v_pre, v_post, geometry, run_max_n, tma_min_n)."""
    lib = load()
    o, _keep = _options(**opts)
    dims = (ctypes.c_int64 * ndim)(*([n_nodes] * ndim))
    h = ctypes.c_void_p()
    stencil = stencil if stencil is not None else (5 if ndim == 2 else 7)
    _check(lib.homg_create(ndim, dims, levels, stencil, ctypes.byref(o), ctypes.byref(h)), None)
    return h.value


def homg_set_stream(handle, stream):
    """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None (legacy default stream)."""
    raw = getattr(stream, "cuda_stream", stream) or 0
    return _check(load().homg_set_stream(handle, ctypes.c_void_p(raw)), handle)


def _devptr(t, name):
    if not (hasattr(t, "is_cuda") and t.is_cuda):
        raise TypeError("%s must be a CUDA tensor" % name)
    if str(t.dtype) != "torch.float64" or not t.is_contiguous():
        raise TypeError("%s must be a contiguous float64 tensor" % name)
    return ctypes.c_void_p(t.data_ptr())


def _devptr_any(t, name):
    """Device pointer of a contiguous CUDA tensor of any dtype (network images, targets, corners)."""
    if not (hasattr(t, "is_cuda") and t.is_cuda):
        raise TypeError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise TypeError("%s must be contiguous" % name)
    return ctypes.c_void_p(t.data_ptr())


def homg_solve(handle, f, u, tol=1e-10, max_cycles=50):
    """Solve in place on device tensors; returns (status, cycles, relres)."""
    cyc, rr = ctypes.c_int(0), ctypes.c_double(0.0)
    rc = load().homg_solve(handle, _devptr(f, "f"), _devptr(u, "u"), tol, max_cycles, ctypes.byref(cyc), ctypes.byref(rr))
    return _check(rc, handle), cyc.value, rr.value


def _hostptr(a, name):
    import numpy as np

    if hasattr(a, "is_cuda"):
        if a.is_cuda or str(a.dtype) != "torch.float64" or not a.is_contiguous():
            raise TypeError("%s must be a contiguous float64 CPU tensor" % name)
        return ctypes.c_void_p(a.data_ptr())
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise TypeError("%s must be a contiguous float64 array" % name)
    return ctypes.c_void_p(a.ctypes.data)


def homg_solve_host(handle, f, u, tol=1e-10, max_cycles=50):
    """Solve with host arrays (copies in and out inside the call); returns (status, cycles, relres)."""
    cyc, rr = ctypes.c_int(0), ctypes.c_double(0.0)
    rc = load().homg_solve_host(handle, _hostptr(f, "f"), _hostptr(u, "u"), tol, max_cycles, ctypes.byref(cyc),
                                ctypes.byref(rr))
    return _check(rc, handle), cyc.value, rr.value


def homg_residual_norm(handle, f, u):
    rr = ctypes.c_double(0.0)
    _check(load().homg_residual_norm(handle, _devptr(f, "f"), _devptr(u, "u"), ctypes.byref(rr)), handle)
    return rr.value


def homg_set_coefficient(handle, k):
    """Switch the handle to A u = -div(k grad u) with the FP64 device tensor k of node coefficients
    (None: back to the Poisson operator)."""
    _check(load().homg_set_coefficient(handle, None if k is None else _devptr(k, "k")), handle)


def homg_residual_norm_noalloc(f, u, stream=None):
    """||f - A u|| / ||f|| of device tensors without a handle; the library allocates nothing for it
    (its scratch is a fixed static device array shared by all calls: do not overlap calls).

    f and u must be contiguous float64 tensors of the same (2^K+1)^ndim shape on the same GPU; the
    call runs with that GPU current. Mismatches raise TypeError before anything reaches the device."""
    import torch

    ndim = f.dim()
    if ndim not in (2, 3) or any(d != f.shape[0] for d in f.shape):
        raise TypeError("f must be a square (2-D) or cubic (3-D) node grid, got shape %s" % (tuple(f.shape),))
    if tuple(u.shape) != tuple(f.shape):
        raise TypeError("u must have f's shape %s, got %s" % (tuple(f.shape), tuple(u.shape)))
    if u.device != f.device:
        raise TypeError("u and f must be on the same device, got %s and %s" % (u.device, f.device))
    if f.dtype != torch.float64 or u.dtype != torch.float64:
        raise TypeError("f and u must be float64")
    dims = (ctypes.c_int64 * ndim)(*f.shape)
    rr = ctypes.c_double(0.0)
    raw = getattr(stream, "cuda_stream", stream) or 0
    fp, up = _devptr(f, "f"), _devptr(u, "u")
    with torch.cuda.device(f.device):
        _check(load().homg_residual_norm_noalloc(ndim, dims, fp, up, ctypes.byref(rr), ctypes.c_void_p(raw)), None)
    return rr.value


HOMG_PROBE_THREADS = 256


def homg_fp64_issue_probe(op, blocks, iters, sink, stream=None):
    """Enqueue the FP64 issue-rate probe kernel (op 0: fused multiply-adds, op 1: additions) on
    `stream`; sink is a float64 CUDA tensor of at least blocks * HOMG_PROBE_THREADS elements.
    Returns the FP64 instructions the launch executes (time it with CUDA events on `stream`)."""
    if sink.numel() < blocks * HOMG_PROBE_THREADS:
        raise TypeError("sink must hold blocks * %d doubles" % HOMG_PROBE_THREADS)
    raw = getattr(stream, "cuda_stream", stream) or 0
    instr = ctypes.c_double(0.0)
    _check(load().homg_fp64_issue_probe(op, blocks, iters, _devptr(sink, "sink"), ctypes.c_void_p(raw),
                                        ctypes.byref(instr)), None)
    return instr.value


def homg_check_sweep_pair(e_old, g, e_packed, e_column, n, omega, c1, rows=0):
    """Both two-sweep kernels of binary32 cycles on one lattice of n intervals (the library's
    self-test): two damped-Jacobi sweeps of e_old with source g, by the packed kernel into e_packed
    and by the per-column kernel into e_column (interiors only). All four are device tensors of
    shape (n + 1, pitch), float32 or bfloat16 alike, pitch >= n + 2 and even."""
    import torch

    kinds = {torch.float32: HOMG_PREC_FP32, torch.bfloat16: HOMG_PREC_BF16}
    ts = (e_old, g, e_packed, e_column)
    if e_old.dtype not in kinds or any(t.dtype != e_old.dtype for t in ts):
        raise TypeError("e_old, g, e_packed and e_column must all be float32 or all bfloat16")
    if any(t.dim() != 2 or t.shape != e_old.shape or not t.is_contiguous() or t.device != e_old.device for t in ts):
        raise TypeError("e_old, g, e_packed and e_column must be contiguous 2-D tensors of one shape and device")
    if e_old.shape[0] != n + 1:
        raise TypeError("the tensors must have n + 1 rows")
    with torch.cuda.device(e_old.device):
        _check(load().homg_check_sweep_pair(kinds[e_old.dtype], int(n), ctypes.c_int64(e_old.shape[1]),
                                            *(_devptr_any(t, nm) for t, nm in zip(ts, ("e_old", "g", "e_packed", "e_column"))),
                                            float(omega), float(c1), int(rows)), None)


def homg_check_conversions(d_in, f_in):
    """The library's integer binary64 -> binary32 (round to nearest even) and binary32 -> binary64
    conversions of device tensors d_in (float64) and f_in (float32, same element count): returns
    (f_out, d_out)."""
    import torch

    if d_in.dtype != torch.float64 or f_in.dtype != torch.float32 or d_in.numel() != f_in.numel():
        raise TypeError("d_in must be float64 and f_in float32 with the same element count")
    f_out = torch.empty(d_in.shape, dtype=torch.float32, device=d_in.device)
    d_out = torch.empty(f_in.shape, dtype=torch.float64, device=f_in.device)
    _check(load().homg_check_conversions(_devptr_any(d_in, "d_in"), _devptr_any(f_out, "f_out"),
                                         _devptr_any(f_in, "f_in"), _devptr_any(d_out, "d_out"),
                                         ctypes.c_int64(d_in.numel())), None)
    return f_out, d_out


def homg_get_history(handle, cap=HOMG_MAX_CYCLES + 1):
    buf = (ctypes.c_double * cap)()
    cnt = _check(load().homg_get_history(handle, buf, cap), handle)
    return list(buf[:cnt])


def homg_get_stats(handle):
    s = homg_stats()
    _check(load().homg_get_stats(handle, ctypes.byref(s)), handle)
    return {name: getattr(s, name) for name, _ in homg_stats._fields_}


def homg_destroy(handle):
    if handle:
        load().homg_destroy(handle)


class Solver:
    """Convenience owner of a handle (same arguments as ``homg_create``)."""

    def __init__(self, ndim, n_nodes, levels, **kw):
        self.ndim, self.n_nodes, self.levels = ndim, n_nodes, levels
        self.handle = homg_create(ndim, n_nodes, levels, **kw)

    def set_stream(self, stream):
        return homg_set_stream(self.handle, stream)

    def solve(self, f, u, tol=1e-10, max_cycles=50):
        return homg_solve(self.handle, f, u, tol, max_cycles)

    def solve_host(self, f, u, tol=1e-10, max_cycles=50):
        return homg_solve_host(self.handle, f, u, tol, max_cycles)

    def residual_norm(self, f, u):
        return homg_residual_norm(self.handle, f, u)

    def set_coefficient(self, k):
        return homg_set_coefficient(self.handle, k)

    def history(self):
        return homg_get_history(self.handle)

    def stats(self):
        return homg_get_stats(self.handle)

    def close(self):
        homg_destroy(self.handle)
        self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            if self.handle:
                self.close()
        except Exception:
            pass


# ---- learned corrector (include/homg_net.h) -------------------------------------------------------
def _net_check(rc, net):
    if rc < 0:
        raise HomgError(rc, homg_net_last_error(net))
    return rc


def homg_net_last_error(net):
    """Message of the last hard error on a network handle (None: of the last failed creation)."""
    msg = load().homg_net_last_error(net)
    return msg.decode() if msg else ""


def image_channels_first_to_device_layout(x):
    """[C, H, W] (C = 2 or 16) array -> the library's row-chunked 16-channel layout [H][2][W][8] (numpy, same dtype)."""
    import numpy as np

    C, H, W = x.shape
    full = np.zeros((16, H, W), dtype=x.dtype)
    full[:C] = x
    return np.ascontiguousarray(full.reshape(2, 8, H, W).transpose(2, 0, 3, 1))


def image_device_layout_to_channels_first(xr):
    """Inverse of image_channels_first_to_device_layout for one image: [H][2][W][8] -> [16, H, W]."""
    import numpy as np

    H, G, W, E = xr.shape
    return np.ascontiguousarray(xr.transpose(1, 3, 0, 2).reshape(G * E, H, W))


NET_LOSSES = {"error": 0, "residual": 1}
JUDGES = {"proposal": 0, "after_cycle": 1}


def homg_set_learned_judge(handle, judge):
    """How homg_solve_learned judges proposals on this handle: "proposal" (the proposal's own
    residual) or "after_cycle" (the residuals after one HOMG cycle from each candidate)."""
    _check(load().homg_set_learned_judge(handle, JUDGES[judge] if isinstance(judge, str) else judge), handle)


class Net:
    """Owner of a learned-corrector network handle (include/homg_net.h)."""

    def __init__(self):
        lib = load()
        h = ctypes.c_void_p()
        _net_check(lib.homg_net_create(ctypes.byref(h)), None)
        self.handle = h.value
        self.count = lib.homg_net_param_count()

    def set_stream(self, stream):
        raw = getattr(stream, "cuda_stream", stream) or 0
        _net_check(load().homg_net_set_stream(self.handle, ctypes.c_void_p(raw)), self.handle)

    def set_params(self, flat):
        import numpy as np

        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == self.count
        _net_check(load().homg_net_set_params(self.handle, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size),
                   self.handle)

    def get_params(self):
        import numpy as np

        a = np.empty(self.count, dtype=np.float32)
        _net_check(load().homg_net_get_params(self.handle, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size),
                   self.handle)
        return a

    def get_grads(self):
        import numpy as np

        a = np.empty(self.count, dtype=np.float32)
        _net_check(load().homg_net_get_grads(self.handle, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size),
                   self.handle)
        return a

    def forward(self, x, y):
        """x: device bfloat16 tensor [B, H, 2, W, 8]; y: device float32 tensor [B, H, W]."""
        B, H, _, W, _ = x.shape
        _net_check(load().homg_net_forward(self.handle, _devptr_any(x, "x"), B, H, W, _devptr_any(y, "y")), self.handle)

    def set_loss(self, kind):
        """Training loss: "error" (mean squared error against the scaled error target) or "residual"
        (the residual the proposal leaves on each patch; the target is then not used)."""
        _net_check(load().homg_net_set_loss(self.handle, NET_LOSSES[kind] if isinstance(kind, str) else kind), self.handle)

    def set_tile_rows(self, rows):
        """Output rows per convolution tile (4 or 8); results do not depend on it."""
        _net_check(load().homg_net_set_tile_rows(self.handle, int(rows)), self.handle)

    def train_step(self, x, t, lr):
        B, H, _, W, _ = x.shape
        loss = ctypes.c_float(0.0)
        _net_check(load().homg_net_train_step(self.handle, _devptr_any(x, "x"), _devptr_any(t, "t"), B, H, W, float(lr),
                                              ctypes.byref(loss)), self.handle)
        return loss.value

    def gather_patches(self, x, t, corners, P, xp, tp):
        """x: [1, H, 2, W, 8] image, t: [H, W]; corners: device int32 [B, 2]; writes xp [B, P, 2, P, 8], tp [B, P, P]."""
        H, W = t.shape
        B = corners.shape[0]
        _net_check(load().homg_net_gather_patches(self.handle, _devptr_any(x, "x"), _devptr_any(t, "t"), H, W,
                                                  _devptr_any(corners, "corners"), B, P, _devptr_any(xp, "xp"),
                                                  _devptr_any(tp, "tp")), self.handle)

    def check_barrier_timeout(self):
        """Run the failure-path self-test; returns (return code, milliseconds the kernel took)."""
        ms = ctypes.c_double(0.0)
        rc = load().homg_net_check_barrier_timeout(self.handle, ctypes.byref(ms))
        return rc, ms.value

    def close(self):
        if self.handle:
            load().homg_net_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False


def homg_features(handle, f, u, x_out, u_ref=None, t_out=None):
    """Network features of iterate u (device FP64) on a variable-coefficient handle; returns rho."""
    rho = ctypes.c_double(0.0)
    _check(load().homg_features(handle, _devptr(f, "f"), _devptr(u, "u"),
                                None if u_ref is None else _devptr(u_ref, "u_ref"), _devptr_any(x_out, "x_out"),
                                None if t_out is None else _devptr_any(t_out, "t_out"), ctypes.byref(rho)), handle)
    return rho.value


def homg_solve_learned(handle, net, f, u, tol=1e-10, max_cycles=50):
    """Learned-corrector solve; returns (status, cycles, relres, accepted list)."""
    cyc = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    acc = (ctypes.c_int * max(1, max_cycles))()
    st = _check(load().homg_solve_learned(handle, net.handle, _devptr(f, "f"), _devptr(u, "u"), tol, max_cycles,
                                          ctypes.byref(cyc), ctypes.byref(rr), acc), handle)
    return st, cyc.value, rr.value, [bool(acc[i]) for i in range(cyc.value)]
