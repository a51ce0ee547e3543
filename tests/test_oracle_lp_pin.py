"""Independent pin of the oracle's binary32 / bfloat16 HOMG cycle (``oracle.cycle_lp``).

The low-precision cycle follows the paper's single-precision runs (Sec. 4): every value of a cycle
(restricted sources, iterates, variations) is computed in IEEE binary32, and with bfloat16 storage
every stored value is rounded to bfloat16 while the arithmetic stays binary32. The C oracle and the
GPU's strict kernels agree bit for bit, so a rounding put in the wrong place (an intermediate kept
in binary32 where the stored value should be bfloat16, or the reverse) would pass both. This test
restates the cycle once more, in NumPy float32 arrays, from the method's definition alone (Sec. 2:
full-weighting restriction, the relaxation formula on the level-m lattice, the interpolation of the
previous iteration's variation, delayed one iteration as in the Sec. 4 discussion of Fig. 3), and
requires the two to agree bit for bit. NumPy float32 operations round every operation to binary32
and never contract a multiply and an add, which is the arithmetic the definition asks for.

The operation order inside each formula is the one fixed for the oracle (residual-free here):
  restriction   ((4 c + 2 (((w + e) + s) + n)) + (((sw + se) + nw) + ne)) / 16
  relaxation    lap = (((4 v - w) - e) - s) - n;  delta = omega (h_m^2 F - lap)
  update        v' = (v + delta) + S(d_prev)  with S = ((wx0 wy0) d00 + (wx1 wy0) d10) + ((wx0 wy1) d01 + (wx1 wy1) d11)
Stored values (F, d, e) are rounded to the storage format; delta enters v unrounded.
"""

import numpy as np
import pytest

import oracle
from paper_1108_2045_gb300 import inputs

F32 = np.float32


def to_bf16(x):
    """Round binary32 values to bfloat16 (nearest, ties to even on the 16 dropped bits), written from
    the format: bfloat16 is the top half of the binary32 encoding."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    keep = (b >> 16) & 1
    r = ((b + 0x7FFF + keep) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32)


def store(x, precision):
    x = np.asarray(x, dtype=np.float32)
    return to_bf16(x) if precision == "bf16" else x


def restrict(Ff, precision):
    nf = Ff.shape[0] - 1
    nc = nf // 2
    Fc = np.zeros((nc + 1, nc + 1), dtype=np.float32)
    J = np.arange(1, nc) * 2
    I = np.arange(1, nc) * 2
    c = Ff[np.ix_(J, I)]
    w, e = Ff[np.ix_(J, I - 1)], Ff[np.ix_(J, I + 1)]
    s, nn = Ff[np.ix_(J - 1, I)], Ff[np.ix_(J + 1, I)]
    sw, se = Ff[np.ix_(J - 1, I - 1)], Ff[np.ix_(J - 1, I + 1)]
    nw, ne = Ff[np.ix_(J + 1, I - 1)], Ff[np.ix_(J + 1, I + 1)]
    edges = ((w + e) + s) + nn
    corners = ((sw + se) + nw) + ne
    Fc[1:-1, 1:-1] = store((F32(4) * c + F32(2) * edges + corners) / F32(16), precision)
    return Fc


def interp_weights(n, mp):
    """Per axis: lower/upper lattice index and the dyadic weights (lp - a)/lp, a/lp in binary32."""
    lp = 1 << mp
    idx = np.arange(n + 1)
    a = idx & (lp - 1)
    lo = idx >> mp
    hi = np.where(a == 0, lo, lo + 1)
    w0 = (lp - a).astype(np.float32) / F32(lp)
    w1 = a.astype(np.float32) / F32(lp)
    return lo, hi, w0, w1


def iteration(n, m, mp, omega, Fm, dprev, e_old, precision):
    l = 1 << m
    nm = n >> m
    h = F32(1) / F32(n)
    hm = h * F32(l)
    hm2 = hm * hm
    v = e_old.copy()
    d_new = np.zeros((nm + 1, nm + 1), dtype=np.float32)
    J = np.arange(1, nm) * l
    I = np.arange(1, nm) * l
    if len(I):
        c = e_old[np.ix_(J, I)]
        lap = F32(4) * c
        lap = lap - e_old[np.ix_(J, I - l)]
        lap = lap - e_old[np.ix_(J, I + l)]
        lap = lap - e_old[np.ix_(J - l, I)]
        lap = lap - e_old[np.ix_(J + l, I)]
        delta = omega * (hm2 * Fm[1:-1, 1:-1] - lap)
        d_new[1:-1, 1:-1] = store(delta, precision)
        v[np.ix_(J, I)] = c + delta
    if mp >= 0:
        lp = 1 << mp
        xl, xh, wx0, wx1 = interp_weights(n, mp)
        yl, yh, wy0, wy1 = interp_weights(n, mp)
        d00 = dprev[np.ix_(yl, xl)]
        d10 = dprev[np.ix_(yl, xh)]
        d01 = dprev[np.ix_(yh, xl)]
        d11 = dprev[np.ix_(yh, xh)]
        t00 = (wx0[None, :] * wy0[:, None]) * d00
        t10 = (wx1[None, :] * wy0[:, None]) * d10
        t01 = (wx0[None, :] * wy1[:, None]) * d01
        t11 = (wx1[None, :] * wy1[:, None]) * d11
        s = (t00 + t10) + (t01 + t11)
        off = ~(((np.arange(n + 1)[:, None] % lp) == 0) & ((np.arange(n + 1)[None, :] % lp) == 0))
        v = np.where(off, v + s, v)
    v = store(v, precision)
    v[0, :] = v[-1, :] = v[:, 0] = v[:, -1] = 0
    return v, d_new


def cycle(F0, levels, precision, schedule, omega_j=0.8):
    n = F0.shape[0] - 1
    omega = F32(omega_j / 4.0)
    F = [store(F0.astype(np.float32), precision)]
    for m in range(1, levels):
        F.append(restrict(F[-1], precision))
    e = np.zeros((n + 1, n + 1), dtype=np.float32)
    d, mp = None, -1
    for m in schedule:
        e, d = iteration(n, m, mp, omega, F[m], d, e, precision)
        mp = m
    return e.astype(np.float64)


def test_bf16_rounding_of_the_pin():
    # ties to even, and a value that rounds up into the next binade
    vals = np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, 2.0 - 2 ** -9, -3.0], dtype=np.float32)
    np.testing.assert_array_equal(to_bf16(vals), np.array([1.0, 1.0 + 2 ** -6, 1.0, 2.0, -3.0], dtype=np.float32))


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("K,levels,schedule", [
    (3, 3, None),                                   # 9^2, the MFMG schedule (2, 4, 8 iterations)
    (4, 4, None),                                   # 17^2
    (4, 4, [3, 1, 2, 0, 1, 0, 0]),                  # back to coarser levels: pending variations of finer levels
    (5, 3, [2, 2, 1, 0, 0]),                        # fewer levels than K
])
def test_low_precision_cycle_bit_exact(precision, K, levels, schedule):
    n = 2 ** K
    F0 = inputs.uniform_rhs(n, 2, seed=30 + K) * 100.0  # values spread over several binades
    sched = oracle.mfmg_schedule(levels, 32) if schedule is None else schedule
    got = oracle.cycle_lp(F0, levels, precision=precision, schedule=sched)
    ref = cycle(F0, levels, precision, sched)
    np.testing.assert_array_equal(got, ref)


def test_pin_detects_a_misplaced_rounding():
    """The pin is sharp: storing the unrounded binary32 iterate in a bfloat16 cycle (one plausible
    slip) changes the result, so the bit-exact comparison above would catch it."""
    n, levels = 16, 4
    F0 = inputs.uniform_rhs(n, 2, seed=3) * 100.0
    sched = oracle.mfmg_schedule(levels, 32)
    good = cycle(F0, levels, "bf16", sched)
    global store
    saved = store
    try:
        store = lambda x, p: np.asarray(x, dtype=np.float32)  # noqa: E731  no bfloat16 rounding anywhere
        slip = cycle(F0, levels, "bf16", sched)
    finally:
        store = saved
    assert not np.array_equal(good, slip)
