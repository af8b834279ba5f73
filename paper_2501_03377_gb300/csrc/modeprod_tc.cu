// Tensor-core (tcgen05) form of the mode products -- placeholder until the
// BF16 kernels land.
#include "tpcg_dev.cuh"

namespace tpcg {
int tc_plan_setup(tpcg_plan*) { return TPCG_ERR_UNSUPPORTED; }
void tc_plan_release(tpcg_plan*) {}
int run_precond_tc(const tpcg_plan*, float*, SolveState*) { return TPCG_ERR_UNSUPPORTED; }
}  // namespace tpcg
