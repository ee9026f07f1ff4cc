// rollout_agents: N_a point-mass agents x N_k steps in one launch
// (Sec. IV-A agent dynamics, Eq. (mfi) circular-field force, Alg. 1 clamp,
// gate and obstacle sum).
//
// Design (B300): a thread-block cluster of C CTAs owns a group of A agents
// for the whole rollout.  CTA r of the cluster keeps obstacle shard r of S_W
// resident in shared memory (loaded once by the TMA bulk-copy engine) and,
// every step, sums the Alg. 1 terms of its shard for all A agents
// (agents in registers, one obstacle per thread per iteration, rsqrt and rcp
// on the SFU).  Per-step partial sums are reduced with warp shuffles, across
// warps in shared memory, and across the cluster by DSMEM stores into every
// CTA's double-buffered receive slots plus one cluster barrier; every CTA then
// integrates the same agents identically, so no grid-wide synchronisation
// and no global-memory round trip happen inside the N_k loop.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "gmapp_internal.cuh"

namespace gmapp {
namespace {

constexpr int kMaxCluster = 16;
constexpr int kMaxAgents = 16;

struct RolloutArgs {
    const float *ox, *oy, *oz;
    const int32_t *n_obs;
    int64_t cap;
    float r_O;
    const float *p0, *v0, *c, *k_r, *k_a, *r_d, *r_a;
    int32_t n_agents;
    float goal[3];
    float dt;
    int32_t n_steps;
    float damping, inv_mass, rho, eps, vel_half, clear_margin, clear_beta;
    int32_t ckpt_every;
    float *traj, *p_final, *v_final, *path_len, *clear_pen, *min_clear, *w_trace, *m_trace,
        *f_trace, *ckpt;
    int32_t shard_cap;           // obstacles one CTA can hold (multiple of 4)
    int32_t agents_per_cluster;  // A <= AG
    uint32_t *err;
};

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__device__ __forceinline__ float warp_min(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fminf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// softplus_beta(x) = log(1 + exp(beta x)) / beta without overflow.
__device__ __forceinline__ float softplus(float x, float beta) {
    float bx = beta * x;
    float r = bx > 0.0f ? bx + log1pf(expf(-bx)) : log1pf(expf(bx));
    return r / beta;
}

template <int AG, int NT>
__global__ void __launch_bounds__(NT, 1) k_rollout(const RolloutArgs A) {
    constexpr int NW = NT / 32;
    extern __shared__ __align__(128) float shard[];  // [3][shard_cap] SoA obstacle centres
    __shared__ float red_w[NW][AG], red_m[NW][AG];
    __shared__ float recv_w[2][kMaxCluster][AG], recv_m[2][kMaxCluster][AG];
    __shared__ float4 pos[AG];
    __shared__ float2 gate[AG];  // (R = r_a + r_O, r_d) per agent slot
    __shared__ __align__(8) uint64_t bar;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t rank = cluster_rank();
    uint32_t C;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(C));
    const int a0 = static_cast<int>(cluster_id_x()) * A.agents_per_cluster;
    const int na = min(A.agents_per_cluster, A.n_agents - a0);

    // N_O comes from the device (written by filter_cloud on this stream).
    // Every CTA of the cluster reads the same value, so an early exit is
    // taken by the whole cluster before any DSMEM access.
    const int32_t n_obs = *A.n_obs;
    const int32_t shard_len = ((n_obs + (int32_t)C - 1) / (int32_t)C + 3) & ~3;
    if (n_obs < 0 || n_obs > A.cap || shard_len > A.shard_cap || na <= 0) {
        if (tid == 0 && rank == 0 && na > 0) raise_error(A.err, GMAPP_DEVERR_CAPACITY);
        return;
    }
    const int32_t start = static_cast<int32_t>(rank) * shard_len;
    int32_t cnt = min(shard_len, max(0, n_obs - start));
    float *sx = shard, *sy = shard + A.shard_cap, *sz = shard + 2 * A.shard_cap;

    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (cnt > 0) {
        const uint32_t bytes = static_cast<uint32_t>((cnt + 3) & ~3) * 4u;
        if (tid == 0) {
            mbar_arrive_expect_tx(&bar, 3 * bytes);
            bulk_g2s(sx, A.ox + start, bytes, &bar);
            bulk_g2s(sy, A.oy + start, bytes, &bar);
            bulk_g2s(sz, A.oz + start, bytes, &bar);
        }
    }

    // Agent state: thread t < na owns agent a0 + t (identically in every CTA).
    float p[3] = {0, 0, 0}, v[3] = {0, 0, 0}, cc[3] = {0, 0, 0};
    float k_r = 0, k_a = 0, R = 0, L = 0, pen = 0, minc = INFINITY;
    if (tid < AG) {
        float rd = -1.0f;  // empty slot: the gate never passes
        if (tid < na) {
            const int i = a0 + tid, n = A.n_agents;
            for (int d = 0; d < 3; ++d) {
                p[d] = A.p0[d * n + i];
                v[d] = A.v0[d * n + i];
                cc[d] = A.c[d * n + i];
            }
            k_r = A.k_r[i];
            k_a = A.k_a[i];
            R = A.r_a[i] + A.r_O;
            rd = A.r_d[i];
            if (rank == 0 && A.traj) {
                float *t = A.traj + (size_t)i * (A.n_steps + 1) * 3;
                t[0] = p[0];
                t[1] = p[1];
                t[2] = p[2];
            }
        }
        pos[tid] = make_float4(p[0], p[1], p[2], 0.0f);
        gate[tid] = make_float2(R, rd);
    }
    if (cnt > 0 && !mbar_wait(&bar, 0)) {
        if (tid == 0) raise_error(A.err, GMAPP_DEVERR_TIMEOUT);
        cnt = 0;  // keep the barrier sequence identical; results are flagged invalid
    }
    __syncthreads();
    float gR[AG], gD[AG];
#pragma unroll
    for (int a = 0; a < AG; ++a) {
        float2 g = gate[a];
        gR[a] = g.x;
        gD[a] = g.y;
    }
    const float eps = A.eps;
    // All CTAs of the cluster are running before anyone stores into their
    // shared memory.
    cluster_sync_all();

    const float h = A.vel_half * A.dt * A.inv_mass;
    for (int k = 0; k < A.n_steps; ++k) {
        float px[AG], py[AG], pz[AG], accw[AG], accm[AG];
#pragma unroll
        for (int a = 0; a < AG; ++a) {
            float4 q = pos[a];
            px[a] = q.x;
            py[a] = q.y;
            pz[a] = q.z;
            accw[a] = 0.0f;
            accm[a] = INFINITY;
        }
        for (int j = tid; j < cnt; j += NT) {
            const float ox = sx[j], oy = sy[j], oz = sz[j];
#pragma unroll
            for (int a = 0; a < AG; ++a) {
                const float dx = px[a] - ox, dy = py[a] - oy, dz = pz[a] - oz;
                const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                // d = d2 * rsqrt(d2); d2 == 0 gives NaN, which max() maps to eps.
                const float s = fmaxf(fmaf(d2, rsqrt_approx(d2), -gR[a]), eps);
                const float u = rcp_approx(s);
                accw[a] += (s <= gD[a]) ? u : 0.0f;
                accm[a] = fminf(accm[a], d2);
            }
        }
#pragma unroll
        for (int a = 0; a < AG; ++a) {
            accw[a] = warp_sum(accw[a]);
            accm[a] = warp_min(accm[a]);
        }
        if (lane == 0) {
#pragma unroll
            for (int a = 0; a < AG; ++a) {
                red_w[warp][a] = accw[a];
                red_m[warp][a] = accm[a];
            }
        }
        __syncthreads();
        const int par = k & 1;
        if (tid < AG) {
            float w = 0.0f, m = INFINITY;
#pragma unroll
            for (int ww = 0; ww < NW; ++ww) {
                w += red_w[ww][tid];
                m = fminf(m, red_m[ww][tid]);
            }
            const uint32_t lw = smem_u32(&recv_w[par][rank][tid]);
            const uint32_t lm = smem_u32(&recv_m[par][rank][tid]);
            for (uint32_t r = 0; r < C; ++r) {
                st_cluster_f32(map_smem(lw, r), w);
                st_cluster_f32(map_smem(lm, r), m);
            }
        }
        cluster_sync_all();
        if (tid < na) {
            float W = 0.0f, md2 = INFINITY;
            for (uint32_t r = 0; r < C; ++r) {
                W += recv_w[par][r][tid];
                md2 = fminf(md2, recv_m[par][r][tid]);
            }
            const float m = sqrtf(md2) - R;
            float g[3] = {0.0f, 0.0f, 0.0f};
            const float vv = fmaf(v[2], v[2], fmaf(v[1], v[1], v[0] * v[0]));
            if (vv >= 1e-30f) {
                const float inv = 1.0f / sqrtf(vv);
                const float vc = fmaf(v[2], cc[2], fmaf(v[1], cc[1], v[0] * cc[0]));
#pragma unroll
                for (int d = 0; d < 3; ++d) g[d] = (vv * cc[d] - v[d] * vc) * inv;
            }
            const float kf = A.rho * k_r * W;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float F = k_a * (A.goal[d] - p[d]) - A.damping * v[d] + kf * g[d];
                v[d] = fmaf(h, F, v[d]);
            }
            const float sp = sqrtf(fmaf(v[2], v[2], fmaf(v[1], v[1], v[0] * v[0])));
            L = fmaf(A.dt, sp, L);
#pragma unroll
            for (int d = 0; d < 3; ++d) p[d] = fmaf(A.dt, v[d], p[d]);
            pen += softplus(A.clear_margin - m, A.clear_beta);
            minc = fminf(minc, m);
            pos[tid] = make_float4(p[0], p[1], p[2], 0.0f);
            if (rank == 0) {
                const int i = a0 + tid;
                if (A.traj) {
                    float *t = A.traj + ((size_t)i * (A.n_steps + 1) + k + 1) * 3;
                    t[0] = p[0];
                    t[1] = p[1];
                    t[2] = p[2];
                }
                if (A.w_trace) A.w_trace[(size_t)i * A.n_steps + k] = W;
                if (A.m_trace) A.m_trace[(size_t)i * A.n_steps + k] = m;
                if (A.f_trace) {
                    float *f = A.f_trace + ((size_t)i * A.n_steps + k) * 3;
                    f[0] = kf * g[0];
                    f[1] = kf * g[1];
                    f[2] = kf * g[2];
                }
            }
        }
        __syncthreads();
    }
    if (rank == 0 && tid < na) {
        const int i = a0 + tid, n = A.n_agents;
        for (int d = 0; d < 3; ++d) {
            A.p_final[d * n + i] = p[d];
            A.v_final[d * n + i] = v[d];
        }
        A.path_len[i] = L;
        A.clear_pen[i] = pen;
        A.min_clear[i] = minc;
    }
}

// ---------------------------------------------------------------------------
// Host side: launch-shape table, validation, launch.
// ---------------------------------------------------------------------------

using KernelFn = void (*)(const RolloutArgs);

template <int AG>
KernelFn pick_kernel_nt(int nt) {
    switch (nt) {
        case 128: return k_rollout<AG, 128>;
        case 256: return k_rollout<AG, 256>;
        case 384: return k_rollout<AG, 384>;
        case 512: return k_rollout<AG, 512>;
        default: return nullptr;
    }
}

KernelFn pick_kernel(int ag, int nt) {
    switch (ag) {
        case 1: return pick_kernel_nt<1>(nt);
        case 2: return pick_kernel_nt<2>(nt);
        case 3: return pick_kernel_nt<3>(nt);
        case 4: return pick_kernel_nt<4>(nt);
        case 5: return pick_kernel_nt<5>(nt);
        case 6: return pick_kernel_nt<6>(nt);
        case 7: return pick_kernel_nt<7>(nt);
        case 8: return pick_kernel_nt<8>(nt);
        case 9: return pick_kernel_nt<9>(nt);
        case 10: return pick_kernel_nt<10>(nt);
        case 11: return pick_kernel_nt<11>(nt);
        case 12: return pick_kernel_nt<12>(nt);
        case 13: return pick_kernel_nt<13>(nt);
        case 14: return pick_kernel_nt<14>(nt);
        case 15: return pick_kernel_nt<15>(nt);
        case 16: return pick_kernel_nt<16>(nt);
        default: return nullptr;
    }
}

int32_t shard_cap_for(int64_t cap, int cluster) {
    int64_t s = (cap + cluster - 1) / cluster;
    return static_cast<int32_t>((s + 3) & ~int64_t(3));
}

gmapp_status static_smem(KernelFn fn, size_t *bytes) {
    cudaFuncAttributes fa;
    GMAPP_CHECK_CUDA(cudaFuncGetAttributes(&fa, reinterpret_cast<const void *>(fn)));
    *bytes = fa.sharedSizeBytes;
    return GMAPP_OK;
}

gmapp_status prepare(KernelFn fn, int cluster, size_t dyn) {
    GMAPP_CHECK_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          static_cast<int>(dyn)));
    if (cluster > 8)
        GMAPP_CHECK_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                              cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    return GMAPP_OK;
}

gmapp_status max_active_clusters(gmapp_ctx *ctx, KernelFn fn, int cluster, int threads,
                                 size_t dyn, int *out) {
    gmapp_status st = prepare(fn, cluster, dyn);
    if (st != GMAPP_OK) return st;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster * ctx->sm_count, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = dyn;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = cluster;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    GMAPP_CHECK_CUDA(cudaOccupancyMaxActiveClusters(out, reinterpret_cast<const void *>(fn), &cfg));
    return GMAPP_OK;
}

// Shared-memory need of one CTA for a shape; 0 when it cannot fit.
size_t shape_smem(gmapp_ctx *ctx, int64_t cap, const gmapp_tuning &t, KernelFn fn) {
    size_t st = 0;
    if (static_smem(fn, &st) != GMAPP_OK) return 0;
    size_t dyn = static_cast<size_t>(shard_cap_for(cap, t.cluster)) * 3 * sizeof(float);
    if (dyn + st > static_cast<size_t>(ctx->max_smem_optin)) return 0;
    return dyn;
}

bool shape_ok(const gmapp_tuning &t) {
    return t.cluster >= 1 && t.cluster <= kMaxCluster && t.agents_per_cta >= 1 &&
           t.agents_per_cta <= kMaxAgents &&
           (t.threads == 128 || t.threads == 256 || t.threads == 384 || t.threads == 512);
}

gmapp_status validate(const gmapp_obstacles *obs, const gmapp_agents *ag,
                      const gmapp_rollout_params *prm, const gmapp_rollout_out *out) {
    if (!obs || !ag || !prm || !out) {
        set_error("rollout_agents: NULL argument");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (!obs->x || !obs->y || !obs->z || !obs->n || obs->cap < 0 || obs->cap % 4 ||
        obs->cap > (int64_t(1) << 30)) {
        set_error("rollout_agents: obstacle arrays must be set, cap a multiple of 4");
        return GMAPP_ERR_INVALID_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(obs->x) | reinterpret_cast<uintptr_t>(obs->y) |
         reinterpret_cast<uintptr_t>(obs->z)) % 16) {
        set_error("rollout_agents: obstacle arrays must be 16-byte aligned");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (!(obs->r_O >= 0.0f) || !isfinite(obs->r_O)) {
        set_error("rollout_agents: r_O must be finite and >= 0");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (ag->n < 1 || !ag->p0 || !ag->v0 || !ag->c || !ag->k_r || !ag->k_a || !ag->r_d || !ag->r_a) {
        set_error("rollout_agents: agent arrays must be set and n >= 1");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (prm->n_steps < 1 || !(prm->dt > 0.0f) || !isfinite(prm->dt) || !(prm->eps > 0.0f) ||
        !isfinite(prm->eps) || !(prm->clear_beta > 0.0f) || !isfinite(prm->damping) ||
        !isfinite(prm->inv_mass) || !isfinite(prm->rho) || !isfinite(prm->vel_half) ||
        !isfinite(prm->clear_margin) || !isfinite(prm->goal[0]) || !isfinite(prm->goal[1]) ||
        !isfinite(prm->goal[2]) || prm->ckpt_every < 0) {
        set_error("rollout_agents: invalid rollout parameters (n_steps >= 1, dt > 0, eps > 0, "
                  "clear_beta > 0, all finite)");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (!out->p_final || !out->v_final || !out->path_len || !out->clear_pen || !out->min_clear) {
        set_error("rollout_agents: p_final, v_final, path_len, clear_pen, min_clear are required");
        return GMAPP_ERR_INVALID_ARG;
    }
    return GMAPP_OK;
}

gmapp_status launch(gmapp_ctx *ctx, const gmapp_obstacles *obs, const gmapp_agents *ag,
                    const gmapp_rollout_params *prm, gmapp_rollout_out *out,
                    const gmapp_tuning &t, gmapp_stream stream) {
    KernelFn fn = pick_kernel(t.agents_per_cta, t.threads);
    size_t dyn = shape_smem(ctx, obs->cap, t, fn);
    if (!fn || dyn == 0) {
        set_error("rollout_agents: launch shape (cluster %d, agents %d, threads %d) does not fit "
                  "an obstacle capacity of %lld",
                  t.cluster, t.agents_per_cta, t.threads, (long long)obs->cap);
        return GMAPP_ERR_INVALID_ARG;
    }
    gmapp_status st = prepare(fn, t.cluster, dyn);
    if (st != GMAPP_OK) return st;
    RolloutArgs A;
    A.ox = obs->x;
    A.oy = obs->y;
    A.oz = obs->z;
    A.n_obs = obs->n;
    A.cap = obs->cap;
    A.r_O = obs->r_O;
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
    A.ckpt_every = prm->ckpt_every;
    A.traj = out->traj;
    A.p_final = out->p_final;
    A.v_final = out->v_final;
    A.path_len = out->path_len;
    A.clear_pen = out->clear_pen;
    A.min_clear = out->min_clear;
    A.w_trace = out->w_trace;
    A.m_trace = out->m_trace;
    A.f_trace = out->f_trace;
    A.ckpt = out->ckpt;
    A.shard_cap = shard_cap_for(obs->cap, t.cluster);
    A.agents_per_cluster = t.agents_per_cta;
    A.err = ctx->d_err;

    const int n_clusters = (ag->n + t.agents_per_cta - 1) / t.agents_per_cta;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_clusters * t.cluster, 1, 1);
    cfg.blockDim = dim3(t.threads, 1, 1);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = stream;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = t.cluster;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    GMAPP_CHECK_CUDA(cudaLaunchKernelEx(&cfg, fn, A));
    return GMAPP_OK;
}

}  // namespace

// Cost model for the launch shape: the slowest CTA processes A agents x one
// shard per step; clusters beyond the co-resident maximum run in further
// waves; every step also pays a fixed reduction/barrier cost.
gmapp_status pick_tuning_impl(gmapp_ctx *ctx, int64_t cap, int32_t n_agents, gmapp_tuning *best) {
    double best_cost = 1e300;
    bool found = false;
    const int threads = 256;
    const int clusters[] = {1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 14, 16};
    for (int C : clusters) {
        // Occupancy does not depend on AG much; probe with AG = 16.
        gmapp_tuning probe{C, kMaxAgents, threads};
        KernelFn fn = pick_kernel(probe.agents_per_cta, threads);
        size_t dyn = shape_smem(ctx, cap, probe, fn);
        if (dyn == 0) continue;
        int m = 0;
        if (max_active_clusters(ctx, fn, C, threads, dyn, &m) != GMAPP_OK || m <= 0) continue;
        const double shard = static_cast<double>(shard_cap_for(cap, C));
        for (int a = 1; a <= kMaxAgents; ++a) {
            const int nc = (n_agents + a - 1) / a;
            const int waves = (nc + m - 1) / m;
            // per step: a * shard pair evaluations + ~3000 pair-equivalents of
            // reduction and cluster-barrier cost
            const double cost = waves * (a * std::max(shard, 256.0) + 3000.0 + 150.0 * C);
            if (cost < best_cost) {
                best_cost = cost;
                *best = gmapp_tuning{C, a, threads};
                found = true;
            }
        }
    }
    if (!found) {
        set_error("rollout_agents: no launch shape fits an obstacle capacity of %lld",
                  (long long)cap);
        return GMAPP_ERR_CAPACITY;
    }
    return GMAPP_OK;
}

}  // namespace gmapp

using namespace gmapp;

extern "C" gmapp_status gmapp_pick_tuning(gmapp_ctx *ctx, int64_t obs_cap, int32_t n_agents,
                                          gmapp_tuning *tune) {
    if (!ctx || !tune || obs_cap < 0 || n_agents < 1) {
        set_error("gmapp_pick_tuning: invalid argument");
        return GMAPP_ERR_INVALID_ARG;
    }
    return pick_tuning_impl(ctx, obs_cap, n_agents, tune);
}

extern "C" gmapp_status rollout_agents_tuned(gmapp_ctx *ctx, const gmapp_obstacles *obs,
                                             const gmapp_agents *agents,
                                             const gmapp_rollout_params *prm,
                                             gmapp_rollout_out *out, const gmapp_tuning *tune,
                                             gmapp_stream stream) {
    if (!ctx || !tune) {
        set_error("rollout_agents_tuned: NULL ctx or tuning");
        return GMAPP_ERR_INVALID_ARG;
    }
    gmapp_status st = validate(obs, agents, prm, out);
    if (st != GMAPP_OK) return st;
    if (!shape_ok(*tune)) {
        set_error("rollout_agents_tuned: launch shape out of range");
        return GMAPP_ERR_INVALID_ARG;
    }
    return launch(ctx, obs, agents, prm, out, *tune, stream);
}

extern "C" gmapp_status rollout_agents(gmapp_ctx *ctx, const gmapp_obstacles *obs,
                                       const gmapp_agents *agents,
                                       const gmapp_rollout_params *prm, gmapp_rollout_out *out,
                                       gmapp_stream stream) {
    if (!ctx) {
        set_error("rollout_agents: NULL ctx");
        return GMAPP_ERR_INVALID_ARG;
    }
    gmapp_status st = validate(obs, agents, prm, out);
    if (st != GMAPP_OK) return st;
    gmapp_tuning t;
    st = pick_tuning_impl(ctx, obs->cap, agents->n, &t);
    if (st != GMAPP_OK) return st;
    return launch(ctx, obs, agents, prm, out, t, stream);
}
