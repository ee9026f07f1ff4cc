// Instantiations of the rollout kernel template with CLEAR = false.
#include "rollout_kernel.cuh"

namespace gmapp {
namespace {

template <int AG>
RolloutKernel by_threads(int nt) {
    // register budget: with 512 threads a CTA gets at most 128 registers per
    // thread, enough for 8 agents in registers; 384 threads allow 10
    switch (nt) {
        case 128: return k_rollout<AG, sfu_agents(AG), 128, false>;
        case 256: return k_rollout<AG, sfu_agents(AG), 256, false>;
        case 384:
            if constexpr (AG <= 10) return k_rollout<AG, sfu_agents(AG), 384, false>;
            return nullptr;
        case 512:
            if constexpr (AG <= 8) return k_rollout<AG, sfu_agents(AG), 512, false>;
            return nullptr;
        default: return nullptr;
    }
}

}  // namespace

RolloutKernel rollout_kernel_noclear(int ag, int nt) {
    switch (ag) {
        case 1: return by_threads<1>(nt);
        case 2: return by_threads<2>(nt);
        case 3: return by_threads<3>(nt);
        case 4: return by_threads<4>(nt);
        case 5: return by_threads<5>(nt);
        case 6: return by_threads<6>(nt);
        case 7: return by_threads<7>(nt);
        case 8: return by_threads<8>(nt);
        case 9: return by_threads<9>(nt);
        case 10: return by_threads<10>(nt);
        case 11: return by_threads<11>(nt);
        case 12: return by_threads<12>(nt);
        case 13: return by_threads<13>(nt);
        case 14: return by_threads<14>(nt);
        case 15: return by_threads<15>(nt);
        case 16: return by_threads<16>(nt);
        default: return nullptr;
    }
}

}  // namespace gmapp
