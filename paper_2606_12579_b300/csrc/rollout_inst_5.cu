// Rollout kernel instantiations: heterogeneous ensemble (MFI + APF), CLEAR = true, GRID = false.
#include "rollout_inst.cuh"

namespace gmapp {
RolloutKernel rollout_kernel_ens_clear(int ag, int nt) {
    return rollout_table<true, false, 1>(ag, nt);
}
}  // namespace gmapp
