// Rollout kernel instantiations: CLEAR = true, GRID = false.
#include "rollout_inst.cuh"

namespace gmapp {
RolloutKernel rollout_kernel_clear(int ag, int nt) { return rollout_table<true, false>(ag, nt); }
}  // namespace gmapp
