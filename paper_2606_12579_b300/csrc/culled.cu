// Rollout with spatial culling (neighbour grid): the voxel grid of the
// filter serves as the neighbour structure of S_W, so each agent visits only
// the obstacles within its detection radius instead of all N_O.
//
// Alg. 1's gate makes every pair with s_j > r_d (|d_j| > r_d + R) contribute
// nothing to W, so summing over the obstacles within r_d + R of the agent
// gives the same W as the sum over S_W (the order of the FP32 additions
// differs).  The clearance m_k is exact when the nearest obstacle lies
// within the visited rows; otherwise it is the smallest distance among the
// visited obstacles (at least r_d, or +inf when none was visited).
//
// Neighbour index (culled_device.cuh): wr[w] = the number of obstacles whose
// key is below 32 w, one binary search per 32-cell word of the grid
// (k_grid_index).
//
// k_rollout_culled: one CTA per agent.  Each step its threads take the grid
// rows of the box around the agent (rows whose (y, z) cell is farther than
// the radius are skipped), evaluate the Alg. 1 terms of their obstacles,
// reduce (W, min |d|^2) over the CTA in a fixed order, and thread 0
// integrates (Sec. IV-A) and publishes the new position.
#include <math.h>

#include <algorithm>

#include "culled_device.cuh"

namespace gmapp {
namespace {

constexpr int kCullThreads = 128;

__global__ void k_grid_index(const uint32_t *__restrict__ keys, const int32_t *n_obs, int64_t cap,
                             int64_t n_words, uint32_t *__restrict__ wr) {
    const int64_t n = std::min<int64_t>(std::max<int32_t>(*n_obs, 0), cap);
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t w = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; w <= n_words;
         w += stride) {
        const uint64_t target = static_cast<uint64_t>(w) * 32u;
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (static_cast<uint64_t>(keys[mid]) < target) lo = mid + 1;
            else hi = mid;
        }
        wr[w] = static_cast<uint32_t>(lo);
    }
}

struct CulledArgs {
    const float *ox, *oy, *oz;
    const int32_t *n_obs;
    int64_t cap;
    float r_O;
    NeighbourGrid grid;
    const float *p0, *v0, *c, *k_r, *k_a, *r_d, *r_a;
    int32_t n_agents;
    float goal[3];
    float dt;
    int32_t n_steps;
    float damping, inv_mass, rho, eps, vel_half, clear_margin, clear_beta;
    float *traj, *p_final, *v_final, *path_len, *clear_pen, *min_clear, *w_trace, *m_trace;
    uint32_t *err;
};

template <bool CLEAR>
__global__ void __launch_bounds__(kCullThreads) k_rollout_culled(const CulledArgs A) {
    constexpr int NW = kCullThreads / 32;
    __shared__ float s_w[NW], s_m[NW];
    __shared__ float s_p[3];
    const int i = blockIdx.x, tid = threadIdx.x;
    const int n = A.n_agents;
    const int32_t n_obs = *A.n_obs;
    if (n_obs < 0 || n_obs > A.cap) {
        if (tid == 0 && i == 0) raise_error(A.err, GMAPP_DEVERR_CAPACITY);
        return;
    }
    const float R = A.r_a[i] + A.r_O, rd = A.r_d[i];
    if (!isfinite(rd)) {  // no gate: nothing to cull by
        if (tid == 0) raise_error(A.err, GMAPP_DEVERR_BOUNDS);
        return;
    }
    // gate s <= r_d  <=>  d^2 <= (r_d + R)^2 (as in the all-pairs kernel)
    const float G2 = rd >= A.eps ? (rd + R) * (rd + R) : -1.0f;
    const float reach = culled_reach(rd, R, A.eps, A.grid.voxel);
    float p[3], v[3], cc[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        p[d] = A.p0[d * n + i];
        v[d] = A.v0[d * n + i];
        cc[d] = A.c[d * n + i];
    }
    const float k_r = A.k_r[i], k_a = A.k_a[i];
    const float h = A.vel_half * A.dt * A.inv_mass;
    float L = 0.0f, pen = 0.0f, minc = INFINITY;
    if (tid == 0 && A.traj) {
        float *t = A.traj + static_cast<size_t>(i) * (A.n_steps + 1) * 3;
        t[0] = p[0];
        t[1] = p[1];
        t[2] = p[2];
    }
    for (int k = 0; k < A.n_steps; ++k) {
        float W, md2;
        culled_terms<kCullThreads, CLEAR>(p, reach, G2, R, A.eps, A.grid, A.ox, A.oy, A.oz, tid,
                                          W, md2);
        culled_reduce<kCullThreads, CLEAR>(W, md2, s_w, s_m);
        if (tid == 0) {
            float g[3], kf, m;
            agent_step<CLEAR>(p, v, cc, k_r, k_a, R, A.goal, h, A.dt, A.rho, A.damping,
                              A.clear_margin, A.clear_beta, W, md2, L, pen, minc, m, g, kf);
            s_p[0] = p[0];
            s_p[1] = p[1];
            s_p[2] = p[2];
            if (A.traj) {
                float *t = A.traj + (static_cast<size_t>(i) * (A.n_steps + 1) + k + 1) * 3;
                t[0] = p[0];
                t[1] = p[1];
                t[2] = p[2];
            }
            if (A.w_trace) A.w_trace[static_cast<size_t>(i) * A.n_steps + k] = W;
            if (A.m_trace) A.m_trace[static_cast<size_t>(i) * A.n_steps + k] = m;
        }
        __syncthreads();
        p[0] = s_p[0];
        p[1] = s_p[1];
        p[2] = s_p[2];
    }
    if (tid == 0) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            A.p_final[d * n + i] = p[d];
            A.v_final[d * n + i] = v[d];
        }
        A.path_len[i] = L;
        if (A.clear_pen) A.clear_pen[i] = pen;
        if (A.min_clear) A.min_clear[i] = minc;
    }
}

int64_t grid_words(const gmapp_workspace *ws) {
    const uint64_t cells = static_cast<uint64_t>(ws->dims[0]) * ws->dims[1] * ws->dims[2];
    return static_cast<int64_t>((cells + 31) / 32);
}

bool valid_grid(const gmapp_workspace *ws) {
    if (!ws || !(ws->voxel > 0.0f) || !isfinite(ws->voxel)) return false;
    uint64_t cells = 1;
    for (int a = 0; a < 3; ++a) {
        if (ws->dims[a] < 1 || ws->dims[a] > (1 << 24) || !isfinite(ws->lo[a])) return false;
        cells *= static_cast<uint64_t>(ws->dims[a]);
    }
    return cells < 0xFFFFFFFFull;
}

}  // namespace
}  // namespace gmapp

using namespace gmapp;

extern "C" size_t gmapp_grid_index_bytes(const gmapp_workspace *ws) {
    if (!valid_grid(ws)) return 0;
    return static_cast<size_t>(grid_words(ws) + 1) * sizeof(uint32_t);
}

extern "C" gmapp_status gmapp_grid_index(gmapp_ctx *ctx, const gmapp_obstacles *obs,
                                         const gmapp_workspace *ws, uint32_t *index,
                                         size_t index_bytes, gmapp_stream stream) {
    if (!ctx || !obs || !obs->keys || !obs->n || obs->cap < 0 || !index || !valid_grid(ws)) {
        set_error("gmapp_grid_index: NULL argument, obstacle keys missing or invalid grid");
        return GMAPP_ERR_INVALID_ARG;
    }
    const int64_t nw = grid_words(ws);
    if (index_bytes < static_cast<size_t>(nw + 1) * sizeof(uint32_t)) {
        set_error("gmapp_grid_index: index of %zu bytes, %zu needed", index_bytes,
                  static_cast<size_t>(nw + 1) * sizeof(uint32_t));
        return GMAPP_ERR_CAPACITY;
    }
    const int grid = static_cast<int>(std::min<int64_t>((nw + 1 + 255) / 256, ctx->sm_count * 16));
    k_grid_index<<<std::max(grid, 1), 256, 0, stream>>>(obs->keys, obs->n, obs->cap, nw, index);
    GMAPP_CHECK_CUDA(cudaGetLastError());
    return GMAPP_OK;
}

extern "C" gmapp_status rollout_agents_culled(gmapp_ctx *ctx, const gmapp_obstacles *obs,
                                              const gmapp_workspace *ws, const uint32_t *index,
                                              const gmapp_agents *ag,
                                              const gmapp_rollout_params *prm,
                                              gmapp_rollout_out *out, gmapp_stream stream) {
    if (!ctx || !obs || !ag || !prm || !out || !index || !valid_grid(ws)) {
        set_error("rollout_agents_culled: NULL argument or invalid grid");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (!obs->x || !obs->y || !obs->z || !obs->n || obs->cap < 0) {
        set_error("rollout_agents_culled: obstacle arrays must be set");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (ag->n < 1 || !ag->p0 || !ag->v0 || !ag->c || !ag->k_r || !ag->k_a || !ag->r_d || !ag->r_a) {
        set_error("rollout_agents_culled: agent arrays must be set and n >= 1");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (prm->n_steps < 1 || !(prm->dt > 0.0f) || !isfinite(prm->dt) || !(prm->eps > 0.0f) ||
        !(prm->clear_beta > 0.0f) || !isfinite(prm->rho) || !isfinite(prm->damping)) {
        set_error("rollout_agents_culled: invalid rollout parameters");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (!out->p_final || !out->v_final || !out->path_len || out->ckpt || out->f_trace ||
        out->cost_terms) {
        set_error("rollout_agents_culled: p_final, v_final, path_len required; checkpoints, "
                  "force traces and cost sums are not produced");
        return GMAPP_ERR_INVALID_ARG;
    }
    CulledArgs A;
    A.ox = obs->x;
    A.oy = obs->y;
    A.oz = obs->z;
    A.n_obs = obs->n;
    A.cap = obs->cap;
    A.r_O = obs->r_O;
    A.grid.wr = index;
    for (int a = 0; a < 3; ++a) A.grid.lo[a] = ws->lo[a];
    A.grid.voxel = ws->voxel;
    A.grid.nx = ws->dims[0];
    A.grid.ny = ws->dims[1];
    A.grid.nz = ws->dims[2];
    A.p0 = ag->p0;
    A.v0 = ag->v0;
    A.c = ag->c;
    A.k_r = ag->k_r;
    A.k_a = ag->k_a;
    A.r_d = ag->r_d;
    A.r_a = ag->r_a;
    A.n_agents = ag->n;
    for (int d = 0; d < 3; ++d) A.goal[d] = prm->goal[d];
    A.dt = prm->dt;
    A.n_steps = prm->n_steps;
    A.damping = prm->damping;
    A.inv_mass = prm->inv_mass;
    A.rho = prm->rho;
    A.eps = prm->eps;
    A.vel_half = prm->vel_half;
    A.clear_margin = prm->clear_margin;
    A.clear_beta = prm->clear_beta;
    A.traj = out->traj;
    A.p_final = out->p_final;
    A.v_final = out->v_final;
    A.path_len = out->path_len;
    A.clear_pen = out->clear_pen;
    A.min_clear = out->min_clear;
    A.w_trace = out->w_trace;
    A.m_trace = out->m_trace;
    A.err = ctx->d_err;
    const bool clear = out->clear_pen || out->min_clear || out->m_trace;
    if (clear) k_rollout_culled<true><<<ag->n, kCullThreads, 0, stream>>>(A);
    else k_rollout_culled<false><<<ag->n, kCullThreads, 0, stream>>>(A);
    GMAPP_CHECK_CUDA(cudaGetLastError());
    return GMAPP_OK;
}
