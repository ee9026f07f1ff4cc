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
    // four-term cost (score_and_select4): the rollout's sums [5][n], the
    // weights w_1..w_4 and 1 / (N_k dt^4 a_max^2); terms == NULL selects the
    // cost above
    const float *terms = nullptr;
    float w4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    float smooth_scale = 0.0f;
    // current-plan cost C_best on the device (read as the previous best,
    // replaced by the chosen agent's cost), or NULL
    float *c_best = nullptr;
};

// Eq. (cost_function) from the rollout's sums: C_goal = S_goal / N_k,
// C_obs = S_obs / N_k, C_path of Eq. (cost_path) (0 when L = d1 = 0),
// C_smooth = min(1, J / (N_k dt^4 a_max^2)).
__device__ __forceinline__ float four_term_cost(const ScoreArgs &S, int i) {
    const float nk = static_cast<float>(S.n_steps);
    const float sg = S.terms[i], so = S.terms[S.n + i], L = S.terms[2 * S.n + i];
    const float J = S.terms[3 * S.n + i], d1 = S.terms[4 * S.n + i];
    const float cpath = L >= d1 ? (L > 0.0f ? 1.0f - d1 / L : 0.0f) : 1.0f - L / d1;
    const float csmooth = fminf(1.0f, J * S.smooth_scale);
    return S.w4[0] * (sg / nk) + S.w4[1] * (so / nk) + S.w4[2] * cpath + S.w4[3] * csmooth;
}

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
    const float prev = S.c_best ? *S.c_best : S.prev_best;
    const bool has_prev = !isnan(prev);
    const float thr = S.alpha * prev;
    float bv = INFINITY;
    int bi = INT_MAX;
    for (int i = tid; i < S.n; i += kScoreThreads) {
        float C;
        if (S.terms) {
            C = four_term_cost(S, i);
        } else {
            const float dx = S.p_final[i] - S.goal[0];
            const float dy = S.p_final[S.n + i] - S.goal[1];
            const float dz = S.p_final[2 * S.n + i] - S.goal[2];
            const float dist = sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
            const float pen = S.clear_pen ? S.clear_pen[i] : 0.0f;
            C = S.w_path * S.path_len[i] + S.w_goal * dist + S.w_clear * pen;
        }
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
            if (S.c_best && s_best >= 0) *S.c_best = bv;
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
