// Rollout kernel instantiations: heterogeneous ensemble (MFI + projected
// current + APF), CLEAR = true, GRID = false.
#include "rollout_inst.cuh"

namespace gmapp {
RolloutKernel rollout_kernel_ens3_clear(int ag, int nt) {
    return rollout_table<true, false, 2>(ag, nt);
}
}  // namespace gmapp
