// Instantiation table of the rollout kernel template: agents per group
// 1..16 x compute threads 128..512 for one (CLEAR, GRID, EK) triple; each
// rollout_inst_*.cu compiles one triple, so the twelve build in parallel.
#pragma once

#include "rollout_kernel.cuh"

namespace gmapp {
namespace {

template <int AG, bool CLEAR, bool GRID, int EK>
RolloutKernel by_threads(int nt) {
    // register budget (compute threads + the exchange warp, allocated per
    // 128 threads): 384 + 32 threads get at most 128 registers per thread,
    // enough for 14 agents in registers without spills; 512 + 32 get 96,
    // enough for 10.  The ensemble kernel (both pair loops; an APF agent
    // holds three force accumulators) stops at kMaxEnsembleAgents and 384.
    if constexpr (EK > 0 && AG > kMaxEnsembleAgents) {
        return nullptr;
    } else {
        switch (nt) {
            case 128: return k_rollout<AG, sfu_agents(AG), 128, CLEAR, GRID, EK>;
            case 256: return k_rollout<AG, sfu_agents(AG), 256, CLEAR, GRID, EK>;
            case 384:
                if constexpr (AG <= 14) return k_rollout<AG, sfu_agents(AG), 384, CLEAR, GRID, EK>;
                return nullptr;
            case 512:
                if constexpr (AG <= 10 && EK == 0)
                    return k_rollout<AG, sfu_agents(AG), 512, CLEAR, GRID, EK>;
                return nullptr;
            default: return nullptr;
        }
    }
}

template <bool CLEAR, bool GRID, int EK = 0>
RolloutKernel rollout_table(int ag, int nt) {
    switch (ag) {
        case 1: return by_threads<1, CLEAR, GRID, EK>(nt);
        case 2: return by_threads<2, CLEAR, GRID, EK>(nt);
        case 3: return by_threads<3, CLEAR, GRID, EK>(nt);
        case 4: return by_threads<4, CLEAR, GRID, EK>(nt);
        case 5: return by_threads<5, CLEAR, GRID, EK>(nt);
        case 6: return by_threads<6, CLEAR, GRID, EK>(nt);
        case 7: return by_threads<7, CLEAR, GRID, EK>(nt);
        case 8: return by_threads<8, CLEAR, GRID, EK>(nt);
        case 9: return by_threads<9, CLEAR, GRID, EK>(nt);
        case 10: return by_threads<10, CLEAR, GRID, EK>(nt);
        case 11: return by_threads<11, CLEAR, GRID, EK>(nt);
        case 12: return by_threads<12, CLEAR, GRID, EK>(nt);
        case 13: return by_threads<13, CLEAR, GRID, EK>(nt);
        case 14: return by_threads<14, CLEAR, GRID, EK>(nt);
        case 15: return by_threads<15, CLEAR, GRID, EK>(nt);
        case 16: return by_threads<16, CLEAR, GRID, EK>(nt);
        default: return nullptr;
    }
}

}  // namespace
}  // namespace gmapp
