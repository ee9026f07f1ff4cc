// rollout_adjoint: gradient of each agent's plan cost with respect to its
// initial velocity v0, field gain k_r, attractive gain k_a and current
// vector c, by the discrete adjoint of the rollout (Sec. IV-A step map with
// the Alg. 1 obstacle sum, Eq. (mfi) force and the cost sums).
//
// Design (B300): the same cluster layout as the forward kernel -- CTA r of a
// cluster keeps obstacle shard r resident in shared memory (TMA bulk copy),
// a cluster owns a group of agents.  The forward rollout stored the state
// (p_k, v_{k-1}) every K steps.  Segments are processed from the last to
// the first: the cluster recomputes the segment's steps (all pairs again,
// now also the gradient of W and the nearest obstacle, reduced over warps
// and over the cluster by DSMEM), rank 0 stores one record per step in a
// global scratch buffer (L2-resident: N_a x K x 64 B), then its agent
// threads run the reverse sweep over the segment's records.  Memory grows
// with K, not with N_k.
#include <math.h>

#include <algorithm>

#include "gmapp_internal.cuh"

namespace gmapp {
namespace {

constexpr int kAdjMaxCluster = 16;
constexpr int kRec = 16;  // floats per step record: p(3) v(3) W gW(3) m gm(3) pad(2)

struct AdjArgs {
    const float *ox, *oy, *oz;
    const int32_t *n_obs;
    int64_t cap;
    float r_O;
    const float *c, *k_r, *k_a, *r_d, *r_a;
    int32_t n_agents;
    float goal[3];
    float dt;
    int32_t n_steps;
    float damping, inv_mass, rho, eps, vel_half, clear_margin, clear_beta;
    int32_t K;
    float w_path, w_goal, w_clear;
    const float *ckpt, *grad_cost;
    float *g_v0, *g_kr, *g_ka, *g_c, *cost;
    float *rec;
    int32_t shard_cap, n_groups;
    uint32_t *err;
};

__device__ __forceinline__ void adj_group_range(int q, int n_agents, int n_groups, int &a0, int &na) {
    const int base = n_agents / n_groups, rem = n_agents % n_groups;
    a0 = q * base + min(q, rem);
    na = base + (q < rem ? 1 : 0);
}

__device__ __forceinline__ void argmin_merge(float &bd, int &bj, float od, int oj) {
    if (od < bd || (od == bd && oj < bj)) {
        bd = od;
        bj = oj;
    }
}

__device__ __forceinline__ float softplus_a(float x, float beta) {
    float bx = beta * x;
    float r = bx > 0.0f ? bx + log1pf(expf(-bx)) : log1pf(expf(bx));
    return r / beta;
}

// g(v, c) = |v| c - (v.c) v/|v| and the products J_g^T F, J_gc^T F.
__device__ __forceinline__ void cf_dir(const float v[3], const float c[3], float g[3]) {
    const float vv = fmaf(v[2], v[2], fmaf(v[1], v[1], v[0] * v[0]));
    g[0] = g[1] = g[2] = 0.0f;
    if (vv >= 1e-30f) {
        const float inv = 1.0f / sqrtf(vv);
        const float vc = fmaf(v[2], c[2], fmaf(v[1], c[1], v[0] * c[0]));
#pragma unroll
        for (int d = 0; d < 3; ++d) g[d] = (vv * c[d] - v[d] * vc) * inv;
    }
}

template <int AG, int NT>
__global__ void __launch_bounds__(NT, 1) k_adjoint(const AdjArgs A) {
    constexpr int NW = NT / 32;
    extern __shared__ __align__(128) float smem[];
    __shared__ float red[NW][AG][6];
    __shared__ __align__(16) float recv[2][kAdjMaxCluster][AG][6];
    __shared__ float4 pos[AG];
    __shared__ __align__(8) uint64_t bar;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t rank = cluster_rank();
    uint32_t C;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(C));
    int a0, na;
    adj_group_range(static_cast<int>(cluster_id_x()), A.n_agents, A.n_groups, a0, na);
    const int32_t n_obs = *A.n_obs;
    const int32_t shard_len = ((n_obs + (int32_t)C - 1) / (int32_t)C + 3) & ~3;
    if (n_obs < 0 || n_obs > A.cap || shard_len > A.shard_cap || na > AG || na <= 0) {
        if (tid == 0 && rank == 0) raise_error(A.err, GMAPP_DEVERR_CAPACITY);
        return;
    }
    const int32_t start = static_cast<int32_t>(rank) * shard_len;
    int32_t cnt = min(shard_len, max(0, n_obs - start));
    float *sx = smem, *sy = smem + A.shard_cap, *sz = smem + 2 * A.shard_cap;
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (cnt > 0 && tid == 0) {
        const uint32_t bytes = static_cast<uint32_t>((cnt + 3) & ~3) * 4u;
        mbar_arrive_expect_tx(&bar, 3 * bytes);
        bulk_g2s(sx, A.ox + start, bytes, &bar);
        bulk_g2s(sy, A.oy + start, bytes, &bar);
        bulk_g2s(sz, A.oz + start, bytes, &bar);
    }
    // per-agent constants, in the agent's thread (tid < na) and, for the
    // pair loop, in every thread (gR, gD)
    const int n = A.n_agents;
    const int i = a0 + tid;
    float cc[3] = {0, 0, 0}, k_r = 0, k_a = 0, R = 0;
    __shared__ float2 gate[AG];
    if (tid < AG) {
        float rd = -1.0f;
        if (tid < na) {
#pragma unroll
            for (int d = 0; d < 3; ++d) cc[d] = A.c[d * n + i];
            k_r = A.k_r[i];
            k_a = A.k_a[i];
            R = A.r_a[i] + A.r_O;
            rd = A.r_d[i];
        }
        gate[tid] = make_float2(R, rd);
    }
    if (cnt > 0 && !mbar_wait(&bar, 0)) {
        if (tid == 0) raise_error(A.err, GMAPP_DEVERR_TIMEOUT);
        cnt = 0;
    }
    __syncthreads();
    float gR[AG], gD[AG];
#pragma unroll
    for (int a = 0; a < AG; ++a) {
        gR[a] = gate[a].x;
        gD[a] = gate[a].y;
    }
    cluster_sync_all();

    const float eps = A.eps, h = A.vel_half * A.dt * A.inv_mass;
    const int K = A.K, N = A.n_steps;
    const int nseg = (N + K - 1) / K;
    float ap[3] = {0, 0, 0}, av[3] = {0, 0, 0}, dc[3] = {0, 0, 0};
    float dkr = 0.0f, dka = 0.0f, L = 0.0f, pen = 0.0f, dgoal = 0.0f;
    int t = 0;
    for (int seg = nseg - 1; seg >= 0; --seg) {
        const int k0 = seg * K, k1 = min(N, k0 + K);
        float p[3] = {0, 0, 0}, v[3] = {0, 0, 0};
        if (tid < AG) {
            if (tid < na) {
                const float *ck = A.ckpt + (size_t)seg * 6 * n + i;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    p[d] = ck[d * n];
                    v[d] = ck[(3 + d) * n];
                }
            }
            pos[tid] = make_float4(p[0], p[1], p[2], 0.0f);
        }
        __syncthreads();
        // ---- recompute the segment, storing one record per step ----------
        for (int k = k0; k < k1; ++k, ++t) {
            float px[AG], py[AG], pz[AG], W[AG], gx[AG], gy[AG], gz[AG], bd[AG];
            int bj[AG];
#pragma unroll
            for (int a = 0; a < AG; ++a) {
                const float4 q = pos[a];
                px[a] = q.x;
                py[a] = q.y;
                pz[a] = q.z;
                W[a] = gx[a] = gy[a] = gz[a] = 0.0f;
                bd[a] = INFINITY;
                bj[a] = INT_MAX;
            }
            for (int j = tid; j < cnt; j += NT) {
                const float ox = sx[j], oy = sy[j], oz = sz[j];
                const int jg = start + j;
#pragma unroll
                for (int a = 0; a < AG; ++a) {
                    const float dx = px[a] - ox, dy = py[a] - oy, dz = pz[a] - oz;
                    const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                    const float r = rsqrt_approx(d2);
                    const float s = fmaf(d2, r, -gR[a]);  // NaN when d = 0
                    const bool unclamped = s > eps;
                    const float sc = fmaxf(s, eps);
                    if (sc <= gD[a]) {
                        const float u = rcp_approx(sc);
                        W[a] += u;
                        if (unclamped) {
                            const float q = -u * u * r;
                            gx[a] = fmaf(q, dx, gx[a]);
                            gy[a] = fmaf(q, dy, gy[a]);
                            gz[a] = fmaf(q, dz, gz[a]);
                        }
                    }
                    if (d2 < bd[a]) {  // j ascends per thread: strict < keeps the lowest index
                        bd[a] = d2;
                        bj[a] = jg;
                    }
                }
            }
#pragma unroll
            for (int a = 0; a < AG; ++a) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    W[a] += __shfl_xor_sync(0xffffffffu, W[a], o);
                    gx[a] += __shfl_xor_sync(0xffffffffu, gx[a], o);
                    gy[a] += __shfl_xor_sync(0xffffffffu, gy[a], o);
                    gz[a] += __shfl_xor_sync(0xffffffffu, gz[a], o);
                    const float od = __shfl_xor_sync(0xffffffffu, bd[a], o);
                    const int oj = __shfl_xor_sync(0xffffffffu, bj[a], o);
                    argmin_merge(bd[a], bj[a], od, oj);
                }
            }
            if (lane == 0) {
#pragma unroll
                for (int a = 0; a < AG; ++a) {
                    red[warp][a][0] = W[a];
                    red[warp][a][1] = gx[a];
                    red[warp][a][2] = gy[a];
                    red[warp][a][3] = gz[a];
                    red[warp][a][4] = bd[a];
                    red[warp][a][5] = __int_as_float(bj[a]);
                }
            }
            __syncthreads();
            const int par = t & 1;
            if (tid < AG) {
                float s4[4] = {0, 0, 0, 0}, d = INFINITY;
                int jj = INT_MAX;
                for (int ww = 0; ww < NW; ++ww) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) s4[q] += red[ww][tid][q];
                    argmin_merge(d, jj, red[ww][tid][4], __float_as_int(red[ww][tid][5]));
                }
                const uint32_t base = smem_u32(&recv[par][rank][tid][0]);
                for (uint32_t r = 0; r < C; ++r) {
                    const uint32_t a = map_smem(base, r);
                    st_cluster_v2f32(a, s4[0], s4[1]);
                    st_cluster_v2f32(a + 8, s4[2], s4[3]);
                    st_cluster_v2f32(a + 16, d, __int_as_float(jj));
                }
            }
            cluster_sync_all();
            if (tid < na) {
                float Wt = 0.0f, g3[3] = {0, 0, 0}, d = INFINITY;
                int jj = INT_MAX;
                for (uint32_t r = 0; r < C; ++r) {
                    Wt += recv[par][r][tid][0];
#pragma unroll
                    for (int q = 0; q < 3; ++q) g3[q] += recv[par][r][tid][1 + q];
                    argmin_merge(d, jj, recv[par][r][tid][4], __float_as_int(recv[par][r][tid][5]));
                }
                const float dist = sqrtf(d);
                const float m = dist - R;
                float gm[3] = {0, 0, 0};
                if (jj != INT_MAX && dist > 0.0f) {
                    const float inv = 1.0f / dist;
                    gm[0] = (p[0] - A.ox[jj]) * inv;
                    gm[1] = (p[1] - A.oy[jj]) * inv;
                    gm[2] = (p[2] - A.oz[jj]) * inv;
                }
                if (rank == 0) {
                    float *rc = A.rec + ((size_t)i * K + (k - k0)) * kRec;
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        rc[q] = p[q];
                        rc[3 + q] = v[q];
                        rc[7 + q] = g3[q];
                        rc[11 + q] = gm[q];
                    }
                    rc[6] = Wt;
                    rc[10] = m;
                }
                float g[3];
                cf_dir(v, cc, g);
                const float kf = A.rho * k_r * Wt;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const float F = k_a * (A.goal[q] - p[q]) - A.damping * v[q] + kf * g[q];
                    v[q] = fmaf(h, F, v[q]);
                }
                L = fmaf(A.dt, sqrtf(fmaf(v[2], v[2], fmaf(v[1], v[1], v[0] * v[0]))), L);
#pragma unroll
                for (int q = 0; q < 3; ++q) p[q] = fmaf(A.dt, v[q], p[q]);
                pen += softplus_a(A.clear_margin - m, A.clear_beta);
                pos[tid] = make_float4(p[0], p[1], p[2], 0.0f);
            }
            __syncthreads();
        }
        // ---- reverse sweep over the segment (rank 0, agent threads) -------
        if (rank == 0 && tid < na) {
            if (seg == nseg - 1) {
                const float e0 = p[0] - A.goal[0], e1 = p[1] - A.goal[1], e2 = p[2] - A.goal[2];
                dgoal = sqrtf(fmaf(e2, e2, fmaf(e1, e1, e0 * e0)));
                if (dgoal > 0.0f) {
                    ap[0] = A.w_goal * e0 / dgoal;
                    ap[1] = A.w_goal * e1 / dgoal;
                    ap[2] = A.w_goal * e2 / dgoal;
                }
            }
            float vn[3] = {v[0], v[1], v[2]};  // v_k, the velocity after step k
            for (int k = k1 - 1; k >= k0; --k) {
                const float *rc = A.rec + ((size_t)i * K + (k - k0)) * kRec;
                const float pk[3] = {rc[0], rc[1], rc[2]};
                const float vk[3] = {rc[3], rc[4], rc[5]};  // v_{k-1}
                const float Wk = rc[6], mk = rc[10];
                const float gW[3] = {rc[7], rc[8], rc[9]};
                const float gm[3] = {rc[11], rc[12], rc[13]};
                const float ln = sqrtf(fmaf(vn[2], vn[2], fmaf(vn[1], vn[1], vn[0] * vn[0])));
                float avk[3], Fb[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    const float eq = ln > 0.0f ? vn[q] / ln : 0.0f;
                    avk[q] = av[q] + A.dt * (ap[q] + A.w_path * eq);
                    Fb[q] = h * avk[q];
                }
                float g[3];
                cf_dir(vk, cc, g);
                const float gF = g[0] * Fb[0] + g[1] * Fb[1] + g[2] * Fb[2];
                float JgF[3] = {0, 0, 0}, JcF[3] = {0, 0, 0};
                const float vv = fmaf(vk[2], vk[2], fmaf(vk[1], vk[1], vk[0] * vk[0]));
                if (vv >= 1e-30f) {
                    const float nrm = sqrtf(vv);
                    const float u[3] = {vk[0] / nrm, vk[1] / nrm, vk[2] / nrm};
                    const float cF = cc[0] * Fb[0] + cc[1] * Fb[1] + cc[2] * Fb[2];
                    const float uF = u[0] * Fb[0] + u[1] * Fb[1] + u[2] * Fb[2];
                    const float vc = vk[0] * cc[0] + vk[1] * cc[1] + vk[2] * cc[2];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        JgF[q] = u[q] * cF - cc[q] * uF - (vc / nrm) * (Fb[q] - u[q] * uF);
                        JcF[q] = nrm * Fb[q] - vk[q] * uF;
                    }
                }
                const float sg = 1.0f / (1.0f + expf(-A.clear_beta * (A.clear_margin - mk)));
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    av[q] = avk[q] - A.damping * Fb[q] + A.rho * k_r * Wk * JgF[q];
                    ap[q] += -k_a * Fb[q] + A.rho * k_r * gF * gW[q] - A.w_clear * sg * gm[q];
                    dka += Fb[q] * (A.goal[q] - pk[q]);
                    dc[q] += A.rho * k_r * Wk * JcF[q];
                    vn[q] = vk[q];
                }
                dkr += A.rho * Wk * gF;
            }
        }
    }
    if (rank == 0 && tid < na) {
        const float sc = A.grad_cost ? A.grad_cost[i] : 1.0f;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            A.g_v0[q * n + i] = sc * av[q];
            A.g_c[q * n + i] = sc * dc[q];
        }
        A.g_kr[i] = sc * dkr;
        A.g_ka[i] = sc * dka;
        if (A.cost) A.cost[i] = A.w_path * L + A.w_goal * dgoal + A.w_clear * pen;
    }
}

using AdjKernel = void (*)(const AdjArgs);

AdjKernel adj_kernel(int ag) {
    switch (ag) {
        case 1: return k_adjoint<1, 256>;
        case 2: return k_adjoint<2, 256>;
        case 4: return k_adjoint<4, 256>;
        case 8: return k_adjoint<8, 256>;
        case 16: return k_adjoint<16, 256>;
        default: return nullptr;
    }
}

}  // namespace
}  // namespace gmapp

using namespace gmapp;

extern "C" size_t gmapp_adjoint_workspace_bytes(int32_t n_agents, const gmapp_rollout_params *prm) {
    if (n_agents < 1 || !prm || prm->ckpt_every < 1) return 0;
    return align_up(static_cast<size_t>(n_agents) * prm->ckpt_every * kRec * sizeof(float), 256);
}

extern "C" gmapp_status rollout_adjoint(gmapp_ctx *ctx, const gmapp_obstacles *obs,
                                        const gmapp_agents *ag, const gmapp_rollout_params *prm,
                                        const gmapp_cost_weights *w, const float *ckpt,
                                        const float *grad_cost, gmapp_adjoint_out *out,
                                        void *workspace, size_t workspace_bytes,
                                        gmapp_stream stream) {
    if (!ctx || !obs || !ag || !prm || !w || !ckpt || !out || !workspace) {
        set_error("rollout_adjoint: NULL argument");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (!obs->x || !obs->y || !obs->z || !obs->n || obs->cap < 0 || obs->cap % 4 ||
        ((reinterpret_cast<uintptr_t>(obs->x) | reinterpret_cast<uintptr_t>(obs->y) |
          reinterpret_cast<uintptr_t>(obs->z)) % 16)) {
        set_error("rollout_adjoint: obstacle arrays must be set and 16-byte aligned, cap a "
                  "multiple of 4");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (ag->n < 1 || !ag->c || !ag->k_r || !ag->k_a || !ag->r_d || !ag->r_a) {
        set_error("rollout_adjoint: agent arrays must be set");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (prm->n_steps < 1 || prm->ckpt_every < 1 || !(prm->dt > 0.0f) || !(prm->eps > 0.0f) ||
        !(prm->clear_beta > 0.0f)) {
        set_error("rollout_adjoint: need n_steps >= 1, ckpt_every >= 1, dt, eps, clear_beta > 0");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (!out->g_v0 || !out->g_kr || !out->g_ka || !out->g_c) {
        set_error("rollout_adjoint: gradient outputs are required");
        return GMAPP_ERR_INVALID_ARG;
    }
    const size_t need = gmapp_adjoint_workspace_bytes(ag->n, prm);
    if (workspace_bytes < need) {
        set_error("rollout_adjoint: workspace of %zu bytes, %zu needed", workspace_bytes, need);
        return GMAPP_ERR_CAPACITY;
    }
    // launch shape: smallest cluster whose shard fits shared memory, then as
    // many agents per cluster as co-residency requires (more waves otherwise)
    AdjKernel fn = nullptr;
    int cluster = 0, agp = 1;
    size_t dyn = 0;
    for (int C = 1; C <= kAdjMaxCluster && !fn; ++C) {
        const int64_t shard = ((obs->cap + C - 1) / C + 3) & ~int64_t(3);
        const size_t bytes = static_cast<size_t>(shard) * 3 * sizeof(float);
        cudaFuncAttributes fa;
        GMAPP_CHECK_CUDA(cudaFuncGetAttributes(&fa, reinterpret_cast<const void *>(adj_kernel(16))));
        if (bytes + fa.sharedSizeBytes > static_cast<size_t>(ctx->max_smem_optin)) continue;
        cluster = C;
        dyn = bytes;
        const int slots = std::max(1, ctx->sm_count / C);
        int want = (ag->n + slots - 1) / slots;
        agp = want <= 1 ? 1 : want <= 2 ? 2 : want <= 4 ? 4 : want <= 8 ? 8 : 16;
        fn = adj_kernel(agp);
    }
    if (!fn) {
        set_error("rollout_adjoint: an obstacle capacity of %lld does not fit any cluster",
                  (long long)obs->cap);
        return GMAPP_ERR_CAPACITY;
    }
    GMAPP_CHECK_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          static_cast<int>(dyn)));
    if (cluster > 8)
        GMAPP_CHECK_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                              cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    AdjArgs A;
    A.ox = obs->x;
    A.oy = obs->y;
    A.oz = obs->z;
    A.n_obs = obs->n;
    A.cap = obs->cap;
    A.r_O = obs->r_O;
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
    A.K = prm->ckpt_every;
    A.w_path = w->w_path;
    A.w_goal = w->w_goal;
    A.w_clear = w->w_clear;
    A.ckpt = ckpt;
    A.grad_cost = grad_cost;
    A.g_v0 = out->g_v0;
    A.g_kr = out->g_kr;
    A.g_ka = out->g_ka;
    A.g_c = out->g_c;
    A.cost = out->cost;
    A.rec = static_cast<float *>(workspace);
    A.shard_cap = static_cast<int32_t>(((obs->cap + cluster - 1) / cluster + 3) & ~int64_t(3));
    A.n_groups = (ag->n + agp - 1) / agp;
    A.err = ctx->d_err;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(A.n_groups * cluster, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = stream;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = cluster;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    GMAPP_CHECK_CUDA(cudaLaunchKernelEx(&cfg, fn, A));
    return GMAPP_OK;
}
