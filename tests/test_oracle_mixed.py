"""Pins of the oracle's low-precision cycle (binary32 arithmetic, binary32 or bfloat16 storage)
and of the mixed-precision restarted solve (CPU, no GPU).

The binary32 cycle restates the pinned binary64 cycle step for step; a structural slip in the
copy would show as an O(1) difference, while binary32 rounding over a cycle of a few hundred
iterations stays near 1e-6 relative. bfloat16 rounding is checked against published values of the
format. The mixed solve must reach the same tolerance as the FP64 solve.
"""

import math

import numpy as np
import pytest

import oracle
from paper_1108_2045_gb300 import inputs


def test_bf16_rounding_known_values():
    assert oracle.bf16_round(1.0) == 1.0
    assert oracle.bf16_round(math.pi) == 3.140625            # 0x4049
    assert oracle.bf16_round(1.0 / 3.0) == 0.333984375         # 0x3EAB
    assert oracle.bf16_round(1.0 + 2.0 ** -8) == 1.0           # tie, to even
    assert oracle.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # tie, to even (up)
    assert oracle.bf16_round(-2.0 ** -130) == -2.0 ** -130     # subnormal kept when representable
    assert math.isinf(oracle.bf16_round(3.4e38))               # rounds past the largest finite value
    assert math.isnan(oracle.bf16_round(float("nan")))


@pytest.mark.parametrize("ndim,K,levels", [(2, 6, 6), (2, 8, 8), (2, 8, 5), (3, 4, 4), (3, 5, 5)])
def test_fp32_cycle_follows_fp64_cycle(ndim, K, levels):
    n = 2 ** K
    F0 = inputs.uniform_rhs(n, ndim, seed=K)
    e64 = oracle.cycle(F0, levels)
    e32 = oracle.cycle_lp(F0, levels, "fp32")
    rel = np.linalg.norm(e32 - e64) / np.linalg.norm(e64)
    assert rel < 1e-5, rel
    assert rel > 0  # really computed in binary32
    eb = oracle.cycle_lp(F0, levels, "bf16")
    relb = np.linalg.norm(eb - e64) / np.linalg.norm(e64)
    assert relb < 5e-2, relb
    assert relb > rel


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_mixed_solve_reaches_fp64_tolerance(precision):
    n, K = 128, 7
    f = inputs.uniform_rhs(n, 2, seed=0)
    u64, s64, c64, h64 = oracle.solve(f, K, tol=1e-10)
    u, s, c, h = oracle.solve_mixed(f, K, precision, tol=1e-10, max_cycles=60)
    assert s == oracle.OK and h[-1] <= 1e-10
    assert np.all(np.diff(h) < 0)
    assert c <= c64 + (0 if precision == "fp32" else 6)
    # both are converged solutions of the same system: they agree to about tol * condition
    assert np.linalg.norm(u - u64) / np.linalg.norm(u64) < 1e-8
