// Rollout kernel instantiations: heterogeneous ensemble (MFI + projected
// current + APF), CLEAR = false, GRID = false.
#include "rollout_inst.cuh"

namespace gmapp {
RolloutKernel rollout_kernel_ens3_noclear(int ag, int nt) {
    return rollout_table<false, false, 2>(ag, nt);
}
}  // namespace gmapp
