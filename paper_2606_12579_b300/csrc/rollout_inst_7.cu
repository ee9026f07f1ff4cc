// Rollout kernel instantiations: heterogeneous ensemble (MFI + APF), CLEAR = true, GRID = true.
#include "rollout_inst.cuh"

namespace gmapp {
RolloutKernel rollout_kernel_ens_grid_clear(int ag, int nt) {
    return rollout_table<true, true, 1>(ag, nt);
}
}  // namespace gmapp
