// Instantiation table of the rollout kernel template: agents per group
// 1..16 x compute threads 128..512 for one (CLEAR, GRID, ENS) triple; each
// rollout_inst_*.cu compiles one triple, so the eight build in parallel.
#pragma once

#include "rollout_kernel.cuh"

namespace gmapp {
namespace {

template <int AG, bool CLEAR, bool GRID, bool ENS>
RolloutKernel by_threads(int nt) {
    // register budget (compute threads + the exchange warp, allocated per
    // 128 threads): 384 + 32 threads get at most 128 registers per thread,
    // enough for 14 agents in registers without spills; 512 + 32 get 96,
    // enough for 10.  The ensemble kernel (both pair loops; an APF agent
    // holds three force accumulators) stops at kMaxEnsembleAgents and 384.
    if constexpr (ENS && AG > kMaxEnsembleAgents) {
        return nullptr;
    } else {
        switch (nt) {
            case 128: return k_rollout<AG, sfu_agents(AG), 128, CLEAR, GRID, ENS>;
            case 256: return k_rollout<AG, sfu_agents(AG), 256, CLEAR, GRID, ENS>;
            case 384:
                if constexpr (AG <= 14) return k_rollout<AG, sfu_agents(AG), 384, CLEAR, GRID, ENS>;
                return nullptr;
            case 512:
                if constexpr (AG <= 10 && !ENS)
                    return k_rollout<AG, sfu_agents(AG), 512, CLEAR, GRID, ENS>;
                return nullptr;
            default: return nullptr;
        }
    }
}

template <bool CLEAR, bool GRID, bool ENS = false>
RolloutKernel rollout_table(int ag, int nt) {
    switch (ag) {
        case 1: return by_threads<1, CLEAR, GRID, ENS>(nt);
        case 2: return by_threads<2, CLEAR, GRID, ENS>(nt);
        case 3: return by_threads<3, CLEAR, GRID, ENS>(nt);
        case 4: return by_threads<4, CLEAR, GRID, ENS>(nt);
        case 5: return by_threads<5, CLEAR, GRID, ENS>(nt);
        case 6: return by_threads<6, CLEAR, GRID, ENS>(nt);
        case 7: return by_threads<7, CLEAR, GRID, ENS>(nt);
        case 8: return by_threads<8, CLEAR, GRID, ENS>(nt);
        case 9: return by_threads<9, CLEAR, GRID, ENS>(nt);
        case 10: return by_threads<10, CLEAR, GRID, ENS>(nt);
        case 11: return by_threads<11, CLEAR, GRID, ENS>(nt);
        case 12: return by_threads<12, CLEAR, GRID, ENS>(nt);
        case 13: return by_threads<13, CLEAR, GRID, ENS>(nt);
        case 14: return by_threads<14, CLEAR, GRID, ENS>(nt);
        case 15: return by_threads<15, CLEAR, GRID, ENS>(nt);
        case 16: return by_threads<16, CLEAR, GRID, ENS>(nt);
        default: return nullptr;
    }
}

}  // namespace
}  // namespace gmapp
