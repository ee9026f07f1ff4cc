// Rollout kernel instantiations: heterogeneous ensemble (MFI + projected
// current + APF), CLEAR = true, GRID = true.
#include "rollout_inst.cuh"

namespace gmapp {
RolloutKernel rollout_kernel_ens3_grid_clear(int ag, int nt) {
    return rollout_table<true, true, 2>(ag, nt);
}
}  // namespace gmapp
