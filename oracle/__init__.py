"""FP64 CPU oracle for the dust drag-coupling step (test infrastructure only).

Only the tests, the smoke check and the CPU-baseline leg of the benchmark
import this package.  The product library never loads it.
"""
from .oracle import (  # noqa: F401
    OG_CARTESIAN, OG_SHEARING_BOX, OG_CYLINDRICAL, OG_SPHERICAL,
    OB_PERIODIC, OB_OUTFLOW, OW_CIC, OW_TSC, OW_VOLUME, OT_CONST, OT_STOKES, OT_EPSTEIN,
    OP_EM, OP_SEMI_IMPLICIT,
    W1_CART_CIC, W1_CART_TSC, W1_CYL_R_CIC, W1_CYL_R_TSC, W1_SPH_R_CIC,
    W1_SPH_R_TSC, W1_SPH_TH_CIC, W1_SPH_TH_TSC, W1_CYL_R_VOL, W1_SPH_R_VOL, W1_SPH_TH_VOL,
    build, weights_1d, weights_vol, locate, Problem, step, step_fixed, gas_momentum, gas_predictor,
    deposit_mass,
)
