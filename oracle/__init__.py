"""HOMG CPU oracle -- TEST INFRASTRUCTURE ONLY.

Plain FP64 restatement of the high-occupancy multigrid of arXiv:1108.2045, in C
(``homg_oracle.c``) behind thin numpy wrappers. Only ``tests/``, the package smoke check and the
benchmark's CPU-baseline leg may import this package. The GPU library shares no code with it and
never calls it.
"""

from .oracle import (  # noqa: F401
    DIVERGED,
    NOT_CONVERGED,
    OK,
    bf16_round,
    build,
    cycle_lp,
    cycle,
    cycle_vc,
    default_omega_j,
    iteration,
    iteration_vc,
    mfmg_schedule,
    norm_interior,
    pow2_cycle,
    pow2_iteration,
    pow2_local_side,
    pow2_restrict,
    pow2_solve,
    prolong,
    residual,
    residual_vc,
    restrict,
    solve,
    solve_mixed,
    solve_vc,
    solve_vcycle,
    vcycle,
)
