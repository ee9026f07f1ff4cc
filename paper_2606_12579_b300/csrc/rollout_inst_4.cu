// Rollout kernel instantiations: heterogeneous ensemble (MFI + APF), CLEAR = false, GRID = false.
#include "rollout_inst.cuh"

namespace gmapp {
RolloutKernel rollout_kernel_ens_noclear(int ag, int nt) {
    return rollout_table<false, false, 1>(ag, nt);
}
}  // namespace gmapp
