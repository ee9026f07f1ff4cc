// Rollout kernel instantiations: heterogeneous ensemble (MFI + APF), CLEAR = false, GRID = true.
#include "rollout_inst.cuh"

namespace gmapp {
RolloutKernel rollout_kernel_ens_grid_noclear(int ag, int nt) {
    return rollout_table<false, true, 1>(ag, nt);
}
}  // namespace gmapp
