// Device body of score_and_select (Sec. IV-A cost and selection), shared by
// the single-query entry point (score.cu) and the batched queries (batch.cu).
#pragma once

#include <math.h>

#include "gmapp_internal.cuh"

namespace gmapp {
namespace {


constexpr int kScoreThreads = 1024;

struct ScoreArgs {
    const float *p_final, *path_len, *clear_pen, *traj;
    int32_t n, n_steps;
    float goal[3];
    float w_path, w_goal, w_clear;
    float prev_best, alpha;
    float *costs;
    int32_t *best;
    float *best_traj;
};

__device__ __forceinline__ void better(float &bv, int &bi, float ov, int oi) {
    if (ov < bv || (ov == bv && oi < bi)) {
        bv = ov;
        bi = oi;
    }
}

__device__ __forceinline__ void score_select_block(const ScoreArgs &S) {
    __shared__ float wv[kScoreThreads / 32];
    __shared__ int wi[kScoreThreads / 32];
    __shared__ int s_best;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool has_prev = !isnan(S.prev_best);
    const float thr = S.alpha * S.prev_best;
    float bv = INFINITY;
    int bi = INT_MAX;
    for (int i = tid; i < S.n; i += kScoreThreads) {
        const float dx = S.p_final[i] - S.goal[0];
        const float dy = S.p_final[S.n + i] - S.goal[1];
        const float dz = S.p_final[2 * S.n + i] - S.goal[2];
        const float dist = sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
        const float pen = S.clear_pen ? S.clear_pen[i] : 0.0f;
        const float C = S.w_path * S.path_len[i] + S.w_goal * dist + S.w_clear * pen;
        S.costs[i] = C;
        const bool ok = !isnan(C) && (!has_prev || C < thr);
        if (ok && C < bv) {  // i ascends within a thread: strict < keeps the lowest index
            bv = C;
            bi = i;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float ov = __shfl_xor_sync(0xffffffffu, bv, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        better(bv, bi, ov, oi);
    }
    if (lane == 0) {
        wv[warp] = bv;
        wi[warp] = bi;
    }
    __syncthreads();
    if (warp == 0) {
        bv = lane < kScoreThreads / 32 ? wv[lane] : INFINITY;
        bi = lane < kScoreThreads / 32 ? wi[lane] : INT_MAX;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            better(bv, bi, ov, oi);
        }
        if (lane == 0) {
            s_best = bi == INT_MAX ? -1 : bi;
            *S.best = s_best;
        }
    }
    __syncthreads();
    const int b = s_best;
    if (b >= 0 && S.best_traj) {
        const int m = (S.n_steps + 1) * 3;
        const float *src = S.traj + (size_t)b * m;
        for (int j = tid; j < m; j += kScoreThreads) S.best_traj[j] = src[j];
    }
}


__global__ void __launch_bounds__(kScoreThreads) k_score_select(const ScoreArgs S) { score_select_block(S); }

}  // namespace
}  // namespace gmapp
