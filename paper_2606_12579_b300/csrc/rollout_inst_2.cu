// Rollout kernel instantiations: CLEAR = false, GRID = true.
#include "rollout_inst.cuh"

namespace gmapp {
RolloutKernel rollout_kernel_grid_noclear(int ag, int nt) {
    return rollout_table<false, true>(ag, nt);
}
}  // namespace gmapp
