// Rollout kernel instantiations: heterogeneous ensemble, CLEAR = false, GRID = false.
#include "rollout_inst.cuh"

namespace gmapp {
RolloutKernel rollout_kernel_ens_noclear(int ag, int nt) {
    return rollout_table<false, false, true>(ag, nt);
}
}  // namespace gmapp
