// Rollout kernel instantiations: CLEAR = false, GRID = false.
#include "rollout_inst.cuh"

namespace gmapp {
RolloutKernel rollout_kernel_noclear(int ag, int nt) { return rollout_table<false, false>(ag, nt); }
}  // namespace gmapp
