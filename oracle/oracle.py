"""numpy wrappers around the C oracle (``homg_oracle.c``) -- TEST INFRASTRUCTURE ONLY.

Arrays are FP64, C-contiguous, node grids of shape (n+1, n+1) or (n+1, n+1, n+1) indexed
[j, i] / [k, j, i] (x fastest), n = 2^K. Compact level-m arrays have side n/2^m + 1.
"""

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "homg_oracle.c")
_LIB = os.path.join(_HERE, "libhomg_oracle.so")
_lib = None

OK, NOT_CONVERGED, DIVERGED = 0, 1, 2


def build(force=False):
    """Compile the oracle with gcc into ``oracle/libhomg_oracle.so`` (plain -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fno-fast-math", "-ffp-contract=off",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load(path=None):
    global _lib
    if _lib is None or path is not None:
        lib = ctypes.CDLL(path or build())
        P = ctypes.POINTER(ctypes.c_double)
        IP = ctypes.POINTER(ctypes.c_int)
        i64 = ctypes.c_int64
        lib.homg_oracle_mfmg_schedule.argtypes = [ctypes.c_int, ctypes.c_int, IP, ctypes.c_int]
        lib.homg_oracle_residual.argtypes = [ctypes.c_int, i64, P, P, P]
        lib.homg_oracle_norm_interior.argtypes = [ctypes.c_int, i64, P]
        lib.homg_oracle_norm_interior.restype = ctypes.c_double
        lib.homg_oracle_restrict.argtypes = [ctypes.c_int, i64, P, P]
        lib.homg_oracle_iteration.argtypes = [ctypes.c_int, i64, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                              P, P, P, P, P]
        lib.homg_oracle_cycle.argtypes = [ctypes.c_int, i64, ctypes.c_int, IP, ctypes.c_int, ctypes.c_double, P, P]
        lib.homg_oracle_solve.argtypes = [ctypes.c_int, i64, ctypes.c_int, IP, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double, P, P, ctypes.c_double, ctypes.c_int, P, IP, P]
        lib.homg_oracle_cycle_lp.argtypes = [ctypes.c_int, i64, ctypes.c_int, IP, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_int, P, P]
        lib.homg_oracle_solve_mixed.argtypes = [ctypes.c_int, i64, ctypes.c_int, IP, ctypes.c_int, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_int, P, P, ctypes.c_double, ctypes.c_int,
                                                P, IP, P]
        lib.homg_oracle_prolong.argtypes = [ctypes.c_int, i64, P, P]
        lib.homg_oracle_vcycle.argtypes = [ctypes.c_int, i64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           P, P]
        lib.homg_oracle_solve_vcycle.argtypes = [ctypes.c_int, i64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_double, ctypes.c_double, P, P, ctypes.c_double,
                                                 ctypes.c_int, P, IP, P]
        lib.homg_oracle_residual_vc.argtypes = [i64, P, P, P, P]
        lib.homg_oracle_iteration_vc.argtypes = [i64, ctypes.c_int, ctypes.c_int, ctypes.c_double, P, P, P, P, P, P]
        lib.homg_oracle_cycle_vc.argtypes = [i64, ctypes.c_int, IP, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                             P, P, P]
        lib.homg_oracle_solve_vc.argtypes = [i64, ctypes.c_int, IP, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_int, P, P, P, ctypes.c_double, ctypes.c_int, P, IP, P]
        lib.homg_oracle_pow2_restrict.argtypes = [i64, ctypes.c_int, P, P]
        lib.homg_oracle_pow2_iteration.argtypes = [i64, ctypes.c_int, ctypes.c_int, ctypes.c_double, P, P, P, P, P]
        lib.homg_oracle_pow2_cycle.argtypes = [i64, ctypes.c_int, IP, ctypes.c_int, ctypes.c_double, P, P]
        lib.homg_oracle_pow2_solve.argtypes = [i64, ctypes.c_int, IP, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                               P, P, ctypes.c_double, ctypes.c_int, P, IP, P]
        lib.homg_oracle_bf16_round.argtypes = [ctypes.c_float]
        lib.homg_oracle_bf16_round.restype = ctypes.c_float
        _lib = lib
    return _lib


class using_library:
    """Context manager: route every wrapper through another build of ``homg_oracle.c`` (used by the
    mutation test, which plants mistakes in copies of the oracle to show that the pins catch them)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _lib
        _load(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _p(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _grid_n(a):
    n = a.shape[0] - 1
    assert all(s == n + 1 for s in a.shape) and a.ndim in (2, 3), a.shape
    return a.ndim, n


def default_omega_j(ndim):
    """Reading A2: the classic optimal smoothing weight of damped Jacobi, 4/5 (2-D) or 6/7 (3-D)."""
    return 4.0 / 5.0 if ndim == 2 else 6.0 / 7.0


def mfmg_schedule(levels, max_i=32):
    """Level of every iteration of one MFMG cycle (Sec. 2): coarsest first, 2 iterations, doubling, capped."""
    lib = _load()
    cnt = lib.homg_oracle_mfmg_schedule(levels, max_i, None, 0)
    if cnt < 0:
        raise ValueError("invalid levels/max_i")
    out = (ctypes.c_int * cnt)()
    lib.homg_oracle_mfmg_schedule(levels, max_i, out, cnt)
    return list(out)


def residual(f, u):
    """r = f - A_h u on interior nodes, 0 on the boundary."""
    ndim, n = _grid_n(f)
    r = np.empty_like(f)
    _load().homg_oracle_residual(ndim, n, _p(f), _p(u), _p(r))
    return r


def norm_interior(v):
    ndim, n = _grid_n(v)
    return _load().homg_oracle_norm_interior(ndim, n, _p(v))


def restrict(Ff):
    """Full weighting of a compact array with nf intervals per side onto nf/2 intervals."""
    ndim, nf = _grid_n(Ff)
    Fc = np.empty((nf // 2 + 1,) * ndim)
    _load().homg_oracle_restrict(ndim, nf, _p(Ff), _p(Fc))
    return Fc


def iteration(n, m, mprev, omega, Fm, dprev, e_old):
    """One HOMG iteration at level m with the pending variation of level mprev (None: none).

    Returns (e_new, d_new) where d_new is the compact level-m variation.
    """
    ndim = e_old.ndim
    e_new = np.empty_like(e_old)
    d_new = np.empty(((n >> m) + 1,) * ndim)
    if dprev is None:
        dprev = np.zeros(1)
        mprev = -1
    _load().homg_oracle_iteration(ndim, n, m, mprev, omega, _p(Fm), _p(dprev), _p(e_old), _p(e_new), _p(d_new))
    return e_new, d_new


def cycle(F0, levels, schedule=None, max_i=32, omega_j=None):
    """One HOMG cycle on A e = F0 from e = 0; returns e."""
    ndim, n = _grid_n(F0)
    if omega_j is None:
        omega_j = default_omega_j(ndim)
    sched = mfmg_schedule(levels, max_i) if schedule is None else list(schedule)
    cs = (ctypes.c_int * len(sched))(*sched)
    e = np.empty_like(F0)
    rc = _load().homg_oracle_cycle(ndim, n, levels, cs, len(sched), omega_j, _p(np.ascontiguousarray(F0)), _p(e))
    if rc != 0:
        raise ValueError("oracle cycle rejected its arguments (rc=%d)" % rc)
    return e


PRECISIONS = {"fp32": 1, "bf16": 2}


def prolong(Ec):
    """Bilinear/trilinear prolongation of a compact coarse array onto the grid with twice the intervals."""
    ndim, nc = _grid_n(Ec)
    Ef = np.empty((2 * nc + 1,) * ndim)
    _load().homg_oracle_prolong(ndim, 2 * nc, _p(np.ascontiguousarray(Ec)), _p(Ef))
    return Ef


def vcycle(F0, levels, nu1=2, nu2=2, omega_j=None):
    """One classic V(nu1, nu2) cycle on A e = F0 from e = 0."""
    ndim, n = _grid_n(F0)
    if omega_j is None:
        omega_j = default_omega_j(ndim)
    e = np.empty_like(F0)
    rc = _load().homg_oracle_vcycle(ndim, n, levels, nu1, nu2, omega_j, _p(np.ascontiguousarray(F0)), _p(e))
    if rc != 0:
        raise ValueError("oracle V-cycle rejected its arguments (rc=%d)" % rc)
    return e


def solve_vcycle(f, levels, nu1=2, nu2=2, u0=None, tol=1e-10, max_cycles=100, omega_j=None, div_factor=1e3):
    """Restarted V(nu1, nu2) solve. Returns (u, status, cycles, hist)."""
    ndim, n = _grid_n(f)
    if omega_j is None:
        omega_j = default_omega_j(ndim)
    u = np.zeros_like(f) if u0 is None else np.array(u0, dtype=np.float64, order="C", copy=True)
    hist = np.zeros(max_cycles + 1)
    cyc = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    status = _load().homg_oracle_solve_vcycle(ndim, n, levels, nu1, nu2, omega_j, div_factor,
                                              _p(np.ascontiguousarray(f)), _p(u), tol, max_cycles, _p(hist),
                                              ctypes.byref(cyc), ctypes.byref(rr))
    if status < 0:
        raise ValueError("oracle V-cycle solve rejected its arguments (rc=%d)" % status)
    return u, status, cyc.value, hist[: cyc.value + 1]


def bf16_round(x):
    """Round a binary32 value to bfloat16 (round to nearest even), as the low-precision cycle stores."""
    return _load().homg_oracle_bf16_round(float(x))


def cycle_lp(F0, levels, precision="fp32", schedule=None, max_i=32, omega_j=None):
    """One low-precision HOMG cycle (binary32 arithmetic; fp32 or bf16 storage) on A e = F0."""
    ndim, n = _grid_n(F0)
    if omega_j is None:
        omega_j = default_omega_j(ndim)
    sched = mfmg_schedule(levels, max_i) if schedule is None else list(schedule)
    cs = (ctypes.c_int * len(sched))(*sched)
    e = np.empty_like(F0)
    rc = _load().homg_oracle_cycle_lp(ndim, n, levels, cs, len(sched), omega_j, PRECISIONS[precision],
                                      _p(np.ascontiguousarray(F0)), _p(e))
    if rc != 0:
        raise ValueError("oracle cycle rejected its arguments (rc=%d)" % rc)
    return e


def solve_mixed(f, levels, precision="fp32", u0=None, tol=1e-10, max_cycles=100, schedule=None, max_i=32,
                omega_j=None, div_factor=1e3):
    """Restarted solve with binary64 residual/update/norms around low-precision cycles."""
    ndim, n = _grid_n(f)
    if omega_j is None:
        omega_j = default_omega_j(ndim)
    sched = mfmg_schedule(levels, max_i) if schedule is None else list(schedule)
    cs = (ctypes.c_int * len(sched))(*sched)
    u = np.zeros_like(f) if u0 is None else np.array(u0, dtype=np.float64, order="C", copy=True)
    hist = np.zeros(max_cycles + 1)
    cyc = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    status = _load().homg_oracle_solve_mixed(ndim, n, levels, cs, len(sched), omega_j, div_factor,
                                             PRECISIONS[precision], _p(np.ascontiguousarray(f)), _p(u), tol,
                                             max_cycles, _p(hist), ctypes.byref(cyc), ctypes.byref(rr))
    if status < 0:
        raise ValueError("oracle solve rejected its arguments (rc=%d)" % status)
    return u, status, cyc.value, hist[: cyc.value + 1]


def solve(f, levels, u0=None, tol=1e-10, max_cycles=100, schedule=None, max_i=32, omega_j=None,
          div_factor=1e3):
    """Restarted HOMG solve. Returns (u, status, cycles, hist) with hist[k] = ||r_k|| / ||f||."""
    ndim, n = _grid_n(f)
    if omega_j is None:
        omega_j = default_omega_j(ndim)
    sched = mfmg_schedule(levels, max_i) if schedule is None else list(schedule)
    cs = (ctypes.c_int * len(sched))(*sched)
    u = np.zeros_like(f) if u0 is None else np.array(u0, dtype=np.float64, order="C", copy=True)
    hist = np.zeros(max_cycles + 1)
    cyc = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    status = _load().homg_oracle_solve(ndim, n, levels, cs, len(sched), omega_j, div_factor,
                                       _p(np.ascontiguousarray(f)), _p(u), tol, max_cycles, _p(hist),
                                       ctypes.byref(cyc), ctypes.byref(rr))
    if status < 0:
        raise ValueError("oracle solve rejected its arguments (rc=%d)" % status)
    return u, status, cyc.value, hist[: cyc.value + 1]


# ---- variable-coefficient diffusion, 2-D: A u = -div(k grad u), harmonic-mean face coefficients ----
VC_PRECISIONS = {"fp64": 0, "fp32": 1, "bf16": 2}


def _k(kc, n):
    kc = np.ascontiguousarray(kc, dtype=np.float64)
    assert kc.shape == (n + 1, n + 1), kc.shape
    return kc


def residual_vc(kc, f, u):
    """r = f - A u for A = -div(k grad .) (flux form, harmonic-mean faces); 0 on the boundary."""
    ndim, n = _grid_n(f)
    assert ndim == 2
    kc = _k(kc, n)
    r = np.empty_like(f)
    _load().homg_oracle_residual_vc(n, _p(kc), _p(np.ascontiguousarray(f)), _p(np.ascontiguousarray(u)), _p(r))
    return r


def iteration_vc(n, m, mprev, omega_j, kc, Fm, dprev, e_old):
    """One variable-coefficient HOMG iteration at level m (k injected on the lattice); returns (e_new, d_new)."""
    kc = _k(kc, n)
    e_new = np.empty_like(e_old)
    d_new = np.empty(((n >> m) + 1,) * 2)
    if dprev is None:
        dprev = np.zeros(1)
        mprev = -1
    _load().homg_oracle_iteration_vc(n, m, mprev, omega_j, _p(kc), _p(Fm), _p(dprev), _p(e_old), _p(e_new),
                                     _p(d_new))
    return e_new, d_new


def cycle_vc(kc, F0, levels, precision="fp64", schedule=None, max_i=32, omega_j=None):
    """One variable-coefficient HOMG cycle on A e = F0 from e = 0 (fp64, or fp32 / bf16 storage)."""
    ndim, n = _grid_n(F0)
    assert ndim == 2
    kc = _k(kc, n)
    if omega_j is None:
        omega_j = default_omega_j(2)
    sched = mfmg_schedule(levels, max_i) if schedule is None else list(schedule)
    cs = (ctypes.c_int * len(sched))(*sched)
    e = np.empty_like(F0)
    rc = _load().homg_oracle_cycle_vc(n, levels, cs, len(sched), omega_j, VC_PRECISIONS[precision], _p(kc),
                                      _p(np.ascontiguousarray(F0)), _p(e))
    if rc != 0:
        raise ValueError("oracle cycle rejected its arguments (rc=%d)" % rc)
    return e


def solve_vc(kc, f, levels, precision="fp64", u0=None, tol=1e-10, max_cycles=100, schedule=None, max_i=32,
             omega_j=None, div_factor=1e3):
    """Restarted variable-coefficient solve (binary64 residual/update/norms). Returns (u, status, cycles, hist)."""
    ndim, n = _grid_n(f)
    assert ndim == 2
    kc = _k(kc, n)
    if omega_j is None:
        omega_j = default_omega_j(2)
    sched = mfmg_schedule(levels, max_i) if schedule is None else list(schedule)
    cs = (ctypes.c_int * len(sched))(*sched)
    u = np.zeros_like(f) if u0 is None else np.array(u0, dtype=np.float64, order="C", copy=True)
    hist = np.zeros(max_cycles + 1)
    cyc = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    status = _load().homg_oracle_solve_vc(n, levels, cs, len(sched), omega_j, div_factor, VC_PRECISIONS[precision],
                                          _p(kc), _p(np.ascontiguousarray(f)), _p(u), tol, max_cycles, _p(hist),
                                          ctypes.byref(cyc), ctypes.byref(rr))
    if status < 0:
        raise ValueError("oracle solve rejected its arguments (rc=%d)" % status)
    return u, status, cyc.value, hist[: cyc.value + 1]


# ---- power-of-two grids (Sec. 3), 2-D: N = 2^K nodes per side, four quadrant lattices per level ----
def pow2_local_side(N, m):
    """Nodes per side of one quadrant's level-m local lattice (m >= 1)."""
    return (N // 2 >> m) + 1


def pow2_restrict(r, m):
    """Level-m sources of the four quadrants [4, s, s] from the fine N x N residual r (m >= 1)."""
    N = r.shape[0]
    s = pow2_local_side(N, m)
    Fc = np.empty((4, s, s))
    _load().homg_oracle_pow2_restrict(N, m, _p(np.ascontiguousarray(r, dtype=np.float64)), _p(Fc))
    return Fc


def pow2_iteration(N, m, mprev, omega, Fm, dprev, e_old):
    """One power-of-two HOMG iteration; returns (e_new, d_new) (d_new: [4, s, s] for m >= 1, None for m = 0)."""
    e_new = np.empty_like(e_old)
    d_new = np.empty((4, pow2_local_side(N, m), pow2_local_side(N, m))) if m >= 1 else np.zeros(1)
    if dprev is None:
        dprev, mprev = np.zeros(1), -1
    _load().homg_oracle_pow2_iteration(N, m, mprev, omega, _p(np.ascontiguousarray(Fm, dtype=np.float64)),
                                       _p(np.ascontiguousarray(dprev, dtype=np.float64)), _p(e_old), _p(e_new),
                                       _p(d_new))
    return e_new, (d_new if m >= 1 else None)


def pow2_cycle(F0, levels, schedule=None, max_i=32, omega_j=None):
    """One power-of-two HOMG cycle on A e = F0 (N x N, N = 2^K) from e = 0."""
    N = F0.shape[0]
    if omega_j is None:
        omega_j = default_omega_j(2)
    sched = mfmg_schedule(levels, max_i) if schedule is None else list(schedule)
    cs = (ctypes.c_int * len(sched))(*sched)
    e = np.empty_like(F0)
    rc = _load().homg_oracle_pow2_cycle(N, levels, cs, len(sched), omega_j, _p(np.ascontiguousarray(F0)), _p(e))
    if rc != 0:
        raise ValueError("oracle cycle rejected its arguments (rc=%d)" % rc)
    return e


def pow2_solve(f, levels, u0=None, tol=1e-10, max_cycles=100, schedule=None, max_i=32, omega_j=None, div_factor=1e3):
    """Restarted power-of-two HOMG solve on the N x N node grid. Returns (u, status, cycles, hist)."""
    N = f.shape[0]
    if omega_j is None:
        omega_j = default_omega_j(2)
    sched = mfmg_schedule(levels, max_i) if schedule is None else list(schedule)
    cs = (ctypes.c_int * len(sched))(*sched)
    u = np.zeros_like(f) if u0 is None else np.array(u0, dtype=np.float64, order="C", copy=True)
    hist = np.zeros(max_cycles + 1)
    cyc = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    status = _load().homg_oracle_pow2_solve(N, levels, cs, len(sched), omega_j, div_factor,
                                            _p(np.ascontiguousarray(f)), _p(u), tol, max_cycles, _p(hist),
                                            ctypes.byref(cyc), ctypes.byref(rr))
    if status < 0:
        raise ValueError("oracle solve rejected its arguments (rc=%d)" % status)
    return u, status, cyc.value, hist[: cyc.value + 1]
