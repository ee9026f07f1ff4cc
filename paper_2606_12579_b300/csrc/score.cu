// score_and_select: per-agent cost and the best agent i* (Sec. IV-A "Cost
// Functions" and "Selection Mechanism").
//
// One CTA: each thread scores a strided set of agents and keeps its best
// (cost, index) with ties to the lower index; a warp-shuffle argmin and one
// more over the warp winners give i*; the CTA then copies the winner's
// trajectory so the caller can hand it to the controller with one read.
#include <math.h>

#include "gmapp_internal.cuh"

namespace gmapp {
namespace {

constexpr int kThreads = 1024;

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

__global__ void __launch_bounds__(kThreads) k_score_select(const ScoreArgs S) {
    __shared__ float wv[kThreads / 32];
    __shared__ int wi[kThreads / 32];
    __shared__ int s_best;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool has_prev = !isnan(S.prev_best);
    const float thr = S.alpha * S.prev_best;
    float bv = INFINITY;
    int bi = INT_MAX;
    for (int i = tid; i < S.n; i += kThreads) {
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
        bv = lane < kThreads / 32 ? wv[lane] : INFINITY;
        bi = lane < kThreads / 32 ? wi[lane] : INT_MAX;
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
        for (int j = tid; j < m; j += kThreads) S.best_traj[j] = src[j];
    }
}

}  // namespace
}  // namespace gmapp

using namespace gmapp;

extern "C" gmapp_status score_and_select(gmapp_ctx *ctx, const gmapp_rollout_out *ro,
                                         int32_t n_agents, const gmapp_rollout_params *prm,
                                         const gmapp_cost_weights *w, float prev_best_cost,
                                         float alpha, float *costs, int32_t *best,
                                         float *best_traj, gmapp_stream stream) {
    if (!ctx || !ro || !prm || !w || !costs || !best || n_agents < 1) {
        set_error("score_and_select: NULL argument or n_agents < 1");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (!ro->p_final || !ro->path_len || (best_traj && !ro->traj) ||
        (w->w_clear != 0.0f && !ro->clear_pen)) {
        set_error("score_and_select: rollout outputs missing (best_traj needs ro->traj, "
                  "w_clear != 0 needs ro->clear_pen)");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (!isnan(prev_best_cost) && !isfinite(alpha)) {
        set_error("score_and_select: alpha must be finite");
        return GMAPP_ERR_INVALID_ARG;
    }
    ScoreArgs S;
    S.p_final = ro->p_final;
    S.path_len = ro->path_len;
    S.clear_pen = ro->clear_pen;
    S.traj = ro->traj;
    S.n = n_agents;
    S.n_steps = prm->n_steps;
    for (int d = 0; d < 3; ++d) S.goal[d] = prm->goal[d];
    S.w_path = w->w_path;
    S.w_goal = w->w_goal;
    S.w_clear = w->w_clear;
    S.prev_best = prev_best_cost;
    S.alpha = alpha;
    S.costs = costs;
    S.best = best;
    S.best_traj = best_traj;
    k_score_select<<<1, kThreads, 0, stream>>>(S);
    GMAPP_CHECK_CUDA(cudaGetLastError());
    return GMAPP_OK;
}
