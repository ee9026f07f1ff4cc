// score_and_select: per-agent cost and the best agent i* (Sec. IV-A "Cost
// Functions" and "Selection Mechanism").
//
// One CTA: each thread scores a strided set of agents and keeps its best
// (cost, index) with ties to the lower index; a warp-shuffle argmin and one
// more over the warp winners give i*; the CTA then copies the winner's
// trajectory so the caller can hand it to the controller with one read.
#include <math.h>

#include "score_device.cuh"



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
    k_score_select<<<1, kScoreThreads, 0, stream>>>(S);
    GMAPP_CHECK_CUDA(cudaGetLastError());
    return GMAPP_OK;
}

extern "C" gmapp_status score_and_select4(gmapp_ctx *ctx, const gmapp_rollout_out *ro,
                                          int32_t n_agents, const gmapp_rollout_params *prm,
                                          const gmapp_cost4 *w, float *c_best, float alpha,
                                          float *costs, int32_t *best, float *best_traj,
                                          gmapp_stream stream) {
    if (!ctx || !ro || !prm || !w || !costs || !best || n_agents < 1 || prm->n_steps < 1) {
        set_error("score_and_select4: NULL argument, n_agents < 1 or n_steps < 1");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (!ro->cost_terms || (best_traj && !ro->traj)) {
        set_error("score_and_select4: needs ro->cost_terms (and ro->traj for best_traj)");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (!(w->a_max > 0.0f) || !isfinite(w->a_max) || !(prm->dt > 0.0f) || !isfinite(alpha) ||
        !isfinite(w->w_goal) || !isfinite(w->w_obs) || !isfinite(w->w_path) ||
        !isfinite(w->w_smooth)) {
        set_error("score_and_select4: weights, alpha must be finite, a_max and dt > 0");
        return GMAPP_ERR_INVALID_ARG;
    }
    ScoreArgs S{};
    S.traj = ro->traj;
    S.n = n_agents;
    S.n_steps = prm->n_steps;
    S.prev_best = __builtin_nanf("");
    S.alpha = alpha;
    S.costs = costs;
    S.best = best;
    S.best_traj = best_traj;
    S.terms = ro->cost_terms;
    S.w4[0] = w->w_goal;
    S.w4[1] = w->w_obs;
    S.w4[2] = w->w_path;
    S.w4[3] = w->w_smooth;
    const double dt = prm->dt, am = w->a_max;
    S.smooth_scale = static_cast<float>(1.0 / (prm->n_steps * dt * dt * dt * dt * am * am));
    S.c_best = c_best;
    k_score_select<<<1, kScoreThreads, 0, stream>>>(S);
    GMAPP_CHECK_CUDA(cudaGetLastError());
    return GMAPP_OK;
}
