// Rollout + CVaR kernels of the kinematic bicycle model.
#define RA_MODEL 0
#include "ra_rollout_inst.inc"
