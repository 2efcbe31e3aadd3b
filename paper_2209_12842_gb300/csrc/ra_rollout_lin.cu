// Rollout + CVaR kernels of the linear test system model.
#define RA_MODEL 2
#include "ra_rollout_inst.inc"
