// Rollout kernel instantiations: heterogeneous ensemble (MFI + projected
// current + APF), CLEAR = false, GRID = true.
#include "rollout_inst.cuh"

namespace gmapp {
RolloutKernel rollout_kernel_ens3_grid_noclear(int ag, int nt) {
    return rollout_table<false, true, 2>(ag, nt);
}
}  // namespace gmapp
