// Rollout kernel instantiations: CLEAR = true, GRID = true.
#include "rollout_inst.cuh"

namespace gmapp {
RolloutKernel rollout_kernel_grid_clear(int ag, int nt) {
    return rollout_table<true, true>(ag, nt);
}
}  // namespace gmapp
