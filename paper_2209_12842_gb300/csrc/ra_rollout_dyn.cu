// Rollout + CVaR kernels of the dynamic single-track model.
#define RA_MODEL 1
#include "ra_rollout_inst.inc"
