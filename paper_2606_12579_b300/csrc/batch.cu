// Batched uneven planning queries (many scenes per launch sequence) for the
// hot path of Sec. IV-B (perception) and Sec. IV-A/IV-C (rollout, cost,
// selection); the paper runs one query per kernel launch per agent per step
// (Alg. 1), this module runs a whole batch of queries in a fixed sequence of
// seven launches that can be captured once in a CUDA graph:
//
//   kb_keys, kb_bitmap_sums, kb_emit, kb_count
//        the filter stages of every query in one launch each (a block ->
//        query table maps blocks to queries; same binary32 sequence as
//        filter_cloud, from filter_device.cuh; the scratch is zeroed at
//        creation and kb_emit leaves it clear, so no clearing launch)
//   kb_plan   one CTA: publishes each query's N_O and orders the work items
//        (query, agent group) by their cost N_a,item x N_O x N_k, largest
//        first (longest-processing-time order), into a device queue
//   kb_rollout  persistent: every CTA pops items from the queue (one atomic
//        per item), loads the item's obstacle set into shared memory with
//        the TMA bulk-copy engine and rolls the item's agents through all
//        N_k steps of its query (one CTA per item, so no cluster exchange)
//   kb_score   one CTA per query: costs and selected agent
//
// The batch object holds the device descriptor table, the queue and the
// filter scratch; all of it is allocated once at creation.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "filter_device.cuh"
#include "rollout_kernel.cuh"
#include "score_device.cuh"

namespace gmapp {
namespace {

constexpr int kMaxItems = 8192;
constexpr int kMaxPointBlocksPerQuery = 128;

struct QueryDev {
    // perception
    const float *xyz;
    int64_t n_raw;
    FilterArgs fa;
    uint32_t *bitmap, *chunk, *sums, *offsets, *counters, *keys;
    uint2 *pw;
    int32_t pt_blk0, pt_nblk, bm_blk0, bm_nblk, sb_blk0, sb_nblk;
    // obstacle set S_W of the query
    float *ox, *oy, *oz;
    uint32_t *okeys, *ocounts, *orep;
    int32_t *n_obs;
    int64_t cap;
    float r_O;
    // agents and rollout constants
    const float *p0, *v0, *c, *k_r, *k_a, *r_d, *r_a;
    int32_t n_agents, n_groups;
    float goal[3];
    float dt;
    int32_t n_steps;
    float damping, inv_mass, rho, eps, vel_half, clear_margin, clear_beta;
    // outputs
    float *traj, *p_final, *v_final, *path_len, *clear_pen, *min_clear;
    float w_path, w_goal, w_clear;
    float *costs;
    int32_t *best;
    float *best_traj;
    // four-term cost (out.cost_terms set): the sums [5][n], its radius,
    // weights, hysteresis and the plan's C_best
    float *cost_terms;
    float cost_radius;
    float w4[4], smooth_scale, alpha;
    float *c_best;
};

// Four-term cost accumulators per agent (as k_rollout's cost columns):
// 0 sum min(|p - goal|, r_c), 1 sum max(r_c - m, 0), 2 the path length before
// the last segment, 3 the jerk sum, 4 |p_0 - goal|, 5-7 F_{k-1}, 8-10 f_r at k-1.
constexpr int kCostRows = 11;

struct BatchDev {
    const QueryDev *q;
    int32_t n_q;
    const int32_t *pt_map, *bm_map, *sb_map;
    const int32_t *items_static;  // item -> (query << 16) | group, in query order
    int32_t *items;               // the planned queue
    int32_t n_items;
    uint32_t *head;
    int32_t shard_cap;
    uint32_t *err;
};

__global__ void __launch_bounds__(kThreads) kb_keys(const BatchDev B) {
    const QueryDev &Q = B.q[B.pt_map[blockIdx.x]];
    const FilterArgs fa = Q.fa;
    keys_range(Q.xyz, Q.n_raw, fa, Q.keys, Q.bitmap, blockIdx.x - Q.pt_blk0, Q.pt_nblk);
}

__global__ void __launch_bounds__(kBmThreads) kb_bitmap_sums(const BatchDev B) {
    const QueryDev &Q = B.q[B.sb_map[blockIdx.x]];
    bitmap_sums_block(Q.bitmap, Q.chunk, Q.sums, Q.offsets, Q.counters, Q.counters + 1,
                      blockIdx.x - Q.sb_blk0, Q.sb_nblk);
}

__global__ void __launch_bounds__(kBmThreads) kb_emit(const BatchDev B) {
    const QueryDev &Q = B.q[B.bm_map[blockIdx.x]];
    const FilterArgs fa = Q.fa;
    EmitOut o{Q.okeys, Q.ocounts, Q.orep, Q.ox, Q.oy, Q.oz, Q.cap};
    emit_block<kChunksPerWarp>(Q.bitmap, Q.offsets, Q.chunk, Q.pw, fa, o, blockIdx.x - Q.bm_blk0, true);
}

__global__ void __launch_bounds__(kThreads) kb_count(const BatchDev B) {
    const QueryDev &Q = B.q[B.pt_map[blockIdx.x]];
    count_range(Q.keys, Q.n_raw, Q.pw, Q.ocounts, Q.orep, Q.cap,
                blockIdx.x - Q.pt_blk0, Q.pt_nblk);
}

// Publish every query's N_O and order the work items by cost, largest first
// (ties by item index); resets the queue head.
__global__ void __launch_bounds__(1024) kb_plan(const BatchDev B, int32_t agents_per_item) {
    extern __shared__ float cost[];  // [n_items]
    const int tid = threadIdx.x;
    for (int q = tid; q < B.n_q; q += 1024) {
        const QueryDev &Q = B.q[q];
        const uint32_t t = Q.counters[1];
        *Q.n_obs = static_cast<int32_t>(t);
        if (t > Q.cap) raise_error(B.err, GMAPP_DEVERR_CAPACITY);
    }
    for (int i = tid; i < B.n_items; i += 1024) {
        const int packed = B.items_static[i];
        const QueryDev &Q = B.q[packed >> 16];
        const int g = packed & 0xffff;
        const int na = Q.n_agents / Q.n_groups + (g < Q.n_agents % Q.n_groups ? 1 : 0);
        const int64_t occ = Q.counters[1];
        const float n_obs = static_cast<float>(occ < Q.cap ? occ : Q.cap);
        cost[i] = static_cast<float>(na) * fmaxf(n_obs, 1.0f) * static_cast<float>(Q.n_steps);
    }
    __syncthreads();
    for (int i = tid; i < B.n_items; i += 1024) {
        const float ci = cost[i];
        int rank = 0;
        for (int j = 0; j < B.n_items; ++j) {
            const float cj = cost[j];
            rank += (cj > ci) || (cj == ci && j < i);
        }
        B.items[rank] = B.items_static[i];
    }
    if (tid == 0) *B.head = 0;
    (void)agents_per_item;
}

// BOX (gmapp_batch_set_culling): the pair loop visits only the resident
// blocks of 128 obstacles whose bounding box meets a gate of the item's
// agents, in the voting loop's order (results equal the unculled batch's bit
// for bit); the obstacles beyond the resident part are evaluated pair by pair.
template <int AG, int NT, bool CLEAR, bool BOX>
__global__ void __launch_bounds__(NT, 1) kb_rollout(const BatchDev B) {
    constexpr int NW = NT / 32;
    constexpr int NM = sfu_agents(AG);
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_item;
    __shared__ int s_om;  // bits of max |o|^2 of the resident obstacles
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *sx = smem, *sy = smem + B.shard_cap, *sz = smem + 2 * B.shard_cap;
    float *recv = smem + 3 * B.shard_cap;  // [2][NW][AG] x (W, min |d|^2)
    float *boxes = recv + 2 * NW * AG * 2;  // [shard_cap / 128][6] (BOX)
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    for (;;) {
        if (tid == 0) {
            s_item = static_cast<int>(atomicAdd(B.head, 1u));
            s_om = 0;
        }
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= B.n_items) break;
        const int packed = B.items[it];
        const QueryDev &Q = B.q[packed >> 16];
        int a0, na;
        group_range(packed & 0xffff, Q.n_agents, Q.n_groups, a0, na);
        const int32_t n_obs = *Q.n_obs;
        if (n_obs < 0 || n_obs > Q.cap || na > AG || (B.shard_cap & 127)) {
            if (tid == 0) raise_error(B.err, GMAPP_DEVERR_CAPACITY);
            continue;  // uniform across the CTA
        }
        // the first shard_cap obstacles stay in shared memory, the rest is
        // read from global memory (L2) every step
        int32_t cnt = min(n_obs, B.shard_cap);
        const GlobalTail tail{Q.ox, Q.oy, Q.oz, cnt, n_obs};
        if (cnt > 0 && tid == 0) {
            const uint32_t bytes = static_cast<uint32_t>((cnt + 3) & ~3) * 4u;
            mbar_arrive_expect_tx(&bar, 3 * bytes);
            bulk_g2s(sx, Q.ox, bytes, &bar);
            bulk_g2s(sy, Q.oy, bytes, &bar);
            bulk_g2s(sz, Q.oz, bytes, &bar);
        }
        const int n = Q.n_agents, N = Q.n_steps;
        float p[3] = {0, 0, 0}, v[3] = {0, 0, 0}, cc[3] = {0, 0, 0};
        float k_r = 0, k_a = 0, R = 0, G2 = -1.0f, L = 0, pen = 0, minc = INFINITY;
        if (lane < na) {
            const int i = a0 + lane;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                p[d] = Q.p0[d * n + i];
                v[d] = Q.v0[d * n + i];
                cc[d] = Q.c[d * n + i];
            }
            k_r = Q.k_r[i];
            k_a = Q.k_a[i];
            R = Q.r_a[i] + Q.r_O;
            const float rd = Q.r_d[i];
            G2 = rd >= Q.eps ? (rd + R) * (rd + R) : -1.0f;
            if (warp == 0 && Q.traj) {
                float *t = Q.traj + (size_t)i * (N + 1) * 3;
                t[0] = p[0];
                t[1] = p[1];
                t[2] = p[2];
            }
        }
        f2 nR2[AG];
        float G2a[AG];
#pragma unroll
        for (int a = 0; a < AG; ++a) {
            const float r = __shfl_sync(0xffffffffu, R, a);
            nR2[a] = pk(-r, -r);
            G2a[a] = __shfl_sync(0xffffffffu, G2, a);
        }
        if (cnt > 0) {
            if (!mbar_wait(&bar, phase)) {
                if (tid == 0) raise_error(B.err, GMAPP_DEVERR_TIMEOUT);
                cnt = 0;
            }
            phase ^= 1u;
        }
        // pad the resident part to whole blocks of 128 (shard_cap is a
        // multiple of 128) with NaN, which contributes nothing: the pair
        // loop tests a block per warp; omax2 = max |o|^2 of the resident part
        const int32_t cnt_pad = (cnt + 127) & ~127;
        for (int32_t i = cnt + tid; i < cnt_pad; i += NT) {
            sx[i] = __int_as_float(0x7fc00000);
            sy[i] = __int_as_float(0x7fc00000);
            sz[i] = __int_as_float(0x7fc00000);
        }
        {
            float m = 0.0f;
            for (int32_t i = tid; i < cnt; i += NT)
                m = fmaxf(m, fmaf(sx[i], sx[i], fmaf(sy[i], sy[i], sz[i] * sz[i])));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0) atomicMax(&s_om, __float_as_int(m));  // m >= 0: ordered as ints
        }
        __syncthreads();
        if constexpr (BOX) {
            // bounding box of every resident block (NaN pads ignored), one warp per block
            for (int b = warp; b < cnt_pad / 128; b += NW) {
                float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int i = b * 128 + 4 * lane + q;
                    lo[0] = fminf(lo[0], sx[i]);
                    lo[1] = fminf(lo[1], sy[i]);
                    lo[2] = fminf(lo[2], sz[i]);
                    hi[0] = fmaxf(hi[0], sx[i]);
                    hi[1] = fmaxf(hi[1], sy[i]);
                    hi[2] = fmaxf(hi[2], sz[i]);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
                        hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
                    }
                }
                if (lane < 6) boxes[6 * b + lane] = lane < 3 ? lo[lane] : hi[lane - 3];
            }
            __syncthreads();
        }
        const float omax2 = __int_as_float(s_om);
        const float h = Q.vel_half * Q.dt * Q.inv_mass;
        const float goal[3] = {Q.goal[0], Q.goal[1], Q.goal[2]};
        // four-term cost sums (the arithmetic of k_rollout's exchange warps)
        const bool four = CLEAR && Q.cost_terms != nullptr;  // uniform per item
        float cv[kCostRows];
#pragma unroll
        for (int r = 0; r < kCostRows; ++r) cv[r] = 0.0f;
        for (int k = 0; k < N; ++k) {
            float *rp = recv + (k & 1) * (NW * AG * 2);
            half_step<AG, AG, 0, NM, NT, CLEAR, true, true, false, true, BOX>(
                sx, sy, sz, cnt_pad, Q.eps, nR2, G2a, p, rp + 2 * (warp * AG), 1u, lane, tail,
                nullptr, nullptr, omax2, boxes);
            __syncthreads();
            float W = 0.0f, md2 = INFINITY;
            half_combine<AG, AG, 0, CLEAR>(rp, NW, lane, W, md2);
            if (lane < na) {
                float g[3], kf, m, F[3];
                const float vprev[3] = {v[0], v[1], v[2]};
                if (four) {
                    const float gx = p[0] - goal[0], gy = p[1] - goal[1], gz = p[2] - goal[2];
                    const float dg = sqrtf(fmaf(gz, gz, fmaf(gy, gy, gx * gx)));
                    cv[0] += fminf(dg, Q.cost_radius);
                    if (k == 0) cv[4] = dg;
                    if (k == N - 1) cv[2] = L;  // before the last segment
                }
                agent_step<CLEAR>(p, v, cc, k_r, k_a, R, goal, h, Q.dt, Q.rho, Q.damping,
                                  Q.clear_margin, Q.clear_beta, W, md2, L, pen, minc, m, g, kf, F);
                if (four) {
                    float fr[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) fr[d] = kf * g[d];
                    cv[1] += fmaxf(Q.cost_radius - m, 0.0f);
                    if (k >= 2 && k <= N - 2) {
                        float sj = 0.0f;
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            const float dF = fmaf(-k_a * Q.dt, vprev[d],
                                                  fmaf(-Q.damping * h, cv[5 + d], fr[d] - cv[8 + d]));
                            sj = fmaf(dF, dF, sj);
                        }
                        cv[3] += sj;
                    }
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        cv[5 + d] = F[d];
                        cv[8 + d] = fr[d];
                    }
                }
                if (warp == 0 && Q.traj) {
                    float *t = Q.traj + ((size_t)(a0 + lane) * (N + 1) + k + 1) * 3;
                    t[0] = p[0];
                    t[1] = p[1];
                    t[2] = p[2];
                }
            }
        }
        if (warp == 0 && lane < na) {
            const int i = a0 + lane;
            for (int d = 0; d < 3; ++d) {
                Q.p_final[d * n + i] = p[d];
                Q.v_final[d * n + i] = v[d];
            }
            Q.path_len[i] = L;
            if (Q.clear_pen) Q.clear_pen[i] = pen;
            if (Q.min_clear) Q.min_clear[i] = minc;
            if (four) {
                const float rc = Q.cost_radius, dh = Q.dt * h;
                Q.cost_terms[i] = cv[0] / rc;
                Q.cost_terms[n + i] = cv[1] / rc;
                Q.cost_terms[2 * n + i] = cv[2];
                Q.cost_terms[3 * n + i] = dh * dh * cv[3];
                Q.cost_terms[4 * n + i] = cv[4];
            }
        }
        __syncthreads();  // the next item's bulk copy overwrites the shard
    }
}

__global__ void __launch_bounds__(kScoreThreads) kb_score(const BatchDev B) {
    const QueryDev &Q = B.q[blockIdx.x];
    ScoreArgs S;
    S.p_final = Q.p_final;
    S.path_len = Q.path_len;
    S.clear_pen = Q.clear_pen;
    S.traj = Q.traj;
    S.n = Q.n_agents;
    S.n_steps = Q.n_steps;
    for (int d = 0; d < 3; ++d) S.goal[d] = Q.goal[d];
    S.w_path = Q.w_path;
    S.w_goal = Q.w_goal;
    S.w_clear = Q.w_clear;
    S.prev_best = __int_as_float(0x7fc00000);
    S.alpha = 1.0f;
    S.costs = Q.costs;
    S.best = Q.best;
    S.best_traj = Q.best_traj;
    if (Q.cost_terms) {  // the paper's four-term cost and selection against C_best
        S.terms = Q.cost_terms;
        for (int j = 0; j < 4; ++j) S.w4[j] = Q.w4[j];
        S.smooth_scale = Q.smooth_scale;
        S.alpha = Q.alpha;
        S.c_best = Q.c_best;
    }
    score_select_block(S);
}

using BatchKernel = void (*)(const BatchDev);

template <bool CLEAR, bool BOX>
BatchKernel batch_kernel_for(int ag, int nt) {
#define GMAPP_BK(AGV)                                                  \
    case AGV:                                                          \
        switch (nt) {                                                  \
            case 256: return kb_rollout<AGV, 256, CLEAR, BOX>;         \
            case 384: return kb_rollout<AGV, 384, CLEAR, BOX>;         \
            case 512:                                                  \
                if constexpr (AGV <= 8) return kb_rollout<AGV, 512, CLEAR, BOX>; \
                return nullptr;                                        \
            default: return nullptr;                                   \
        }
    switch (ag) {
        GMAPP_BK(2)
        GMAPP_BK(4)
        GMAPP_BK(6)
        GMAPP_BK(8)
        GMAPP_BK(12)
        GMAPP_BK(16)
        default: return nullptr;
    }
#undef GMAPP_BK
}

BatchKernel batch_kernel(int ag, int nt, bool clear, bool box) {
    if (box) return clear ? batch_kernel_for<true, true>(ag, nt) : batch_kernel_for<false, true>(ag, nt);
    return clear ? batch_kernel_for<true, false>(ag, nt) : batch_kernel_for<false, false>(ag, nt);
}

}  // namespace
}  // namespace gmapp

using namespace gmapp;

struct gmapp_batch {
    gmapp_ctx *ctx = nullptr;
    int32_t n_q = 0;
    std::vector<QueryDev> hq;
    QueryDev *d_q = nullptr;
    int32_t *d_pt_map = nullptr, *d_bm_map = nullptr, *d_sb_map = nullptr;
    int32_t *d_items_static = nullptr, *d_items = nullptr;
    uint32_t *d_head = nullptr;
    void *d_ws = nullptr;
    int32_t pt_blocks = 0, bm_blocks = 0, sb_blocks = 0, n_items = 0, shard_cap = 0;
    int64_t max_cap = 4;  // largest obstacle capacity over the queries
    bool clear = false;
    bool cull = false;  // block culling in the rollout kernel (gmapp_batch_set_culling)
    int32_t agents_per_item = 8, threads = 256;
    BatchKernel fn = nullptr;
    size_t smem = 0;
    int grid = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

void release(gmapp_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->d_q);
    cudaFree(b->d_pt_map);
    cudaFree(b->d_bm_map);
    cudaFree(b->d_sb_map);
    cudaFree(b->d_items_static);
    cudaFree(b->d_items);
    cudaFree(b->d_head);
    cudaFree(b->d_ws);
    b->exec = nullptr;
    b->graph = nullptr;
}

// (Re)build the item list and the kernel choice for a tuning.
gmapp_status apply_tuning(gmapp_batch *b, int32_t agents_per_item, int32_t threads) {
    BatchKernel fn = batch_kernel(agents_per_item, threads, b->clear, b->cull);
    if (!fn) {
        set_error("gmapp_batch: no kernel for %d agents per item and %d threads", agents_per_item,
                  threads);
        return GMAPP_ERR_INVALID_ARG;
    }
    // resident part of each obstacle set: as much as shared memory holds
    // after the receive slots (larger sets stream their remainder from L2).
    // The room for the culling boxes (6 floats per 128 obstacles) is kept
    // whether or not culling is on, so both modes hold the same obstacles in
    // shared memory and give bit-identical sums.
    cudaFuncAttributes fa;
    GMAPP_CHECK_CUDA(cudaFuncGetAttributes(&fa, reinterpret_cast<const void *>(fn)));
    const size_t recv_bytes =
        static_cast<size_t>(2) * (threads / 32) * agents_per_item * 2 * sizeof(float);
    const int64_t room = (static_cast<int64_t>(b->ctx->max_smem_optin) -
                          static_cast<int64_t>(fa.sharedSizeBytes + recv_bytes)) * 128 /
                         (12 * 128 + 24);
    // a multiple of 128: the pair loop tests whole blocks of 128 obstacles
    const int32_t shard_cap = static_cast<int32_t>(std::min<int64_t>(
        (b->max_cap + 127) & ~int64_t(127), room & ~int64_t(127)));
    if (shard_cap < 128) {
        set_error("gmapp_batch: no shared memory left for obstacles");
        return GMAPP_ERR_CAPACITY;
    }
    const size_t smem = static_cast<size_t>(shard_cap) * 3 * sizeof(float) + recv_bytes +
                        (b->cull ? static_cast<size_t>(shard_cap / 128) * 24 : 0);
    // every check runs before the batch changes: a rejected tuning leaves
    // the kernel, its shard size and the device item list as they were
    std::vector<QueryDev> hq = b->hq;
    std::vector<int32_t> items;
    for (int q = 0; q < b->n_q; ++q) {
        const int groups = (hq[q].n_agents + agents_per_item - 1) / agents_per_item;
        hq[q].n_groups = groups;
        if (q > 0xffff || groups > 0xffff) {
            set_error("gmapp_batch: too many queries or agent groups");
            return GMAPP_ERR_CAPACITY;
        }
        for (int g = 0; g < groups; ++g) items.push_back((q << 16) | g);
    }
    if (items.size() > static_cast<size_t>(kMaxItems)) {
        set_error("gmapp_batch: %zu work items, at most %d (use more agents per item)",
                  items.size(), kMaxItems);
        return GMAPP_ERR_CAPACITY;
    }
    GMAPP_CHECK_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          static_cast<int>(smem)));
    GMAPP_CHECK_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void *>(kb_plan),
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          kMaxItems * static_cast<int>(sizeof(float))));
    int per_sm = 0;
    GMAPP_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, reinterpret_cast<const void *>(fn), threads, smem));
    if (per_sm < 1) {
        set_error("gmapp_batch: rollout kernel cannot be resident");
        return GMAPP_ERR_CAPACITY;
    }
    // commit: device tables first; if a copy fails the batch refuses to run
    cudaError_t e = cudaMemcpy(b->d_q, hq.data(), sizeof(QueryDev) * b->n_q,
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_items_static, items.data(), sizeof(int32_t) * items.size(),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        b->fn = nullptr;
        return cuda_fail(e, "gmapp_batch: tuning tables");
    }
    b->hq = std::move(hq);
    b->shard_cap = shard_cap;
    b->n_items = static_cast<int32_t>(items.size());
    b->grid = std::max(1, std::min(b->n_items, per_sm * b->ctx->sm_count));
    b->fn = fn;
    b->smem = smem;
    b->agents_per_item = agents_per_item;
    b->threads = threads;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (b->graph) {
        cudaGraphDestroy(b->graph);
        b->graph = nullptr;
    }
    return GMAPP_OK;
}

BatchDev dev_view(const gmapp_batch *b) {
    BatchDev B;
    B.q = b->d_q;
    B.n_q = b->n_q;
    B.pt_map = b->d_pt_map;
    B.bm_map = b->d_bm_map;
    B.sb_map = b->d_sb_map;
    B.items_static = b->d_items_static;
    B.items = b->d_items;
    B.n_items = b->n_items;
    B.head = b->d_head;
    B.shard_cap = b->shard_cap;
    B.err = b->ctx->d_err;
    return B;
}

}  // namespace

extern "C" gmapp_status gmapp_batch_create(gmapp_ctx *ctx, const gmapp_query *queries,
                                           int32_t n_q, gmapp_batch **out) {
    if (!ctx || !queries || n_q < 1 || !out) {
        set_error("gmapp_batch_create: invalid argument");
        return GMAPP_ERR_INVALID_ARG;
    }
    *out = nullptr;
    gmapp_batch *b = new gmapp_batch();
    b->ctx = ctx;
    b->n_q = n_q;
    b->hq.resize(n_q);
    std::vector<int32_t> pt_map, bm_map, sb_map;
    std::vector<size_t> ws_off(n_q);
    size_t ws_total = 0;
    int64_t max_cap = 4;
    for (int q = 0; q < n_q; ++q) {
        const gmapp_query &Qh = queries[q];
        if (!valid_workspace(&Qh.ws) || Qh.ws.min_pts != 1 || Qh.n_raw < 0 ||
            Qh.n_raw >= 0xFFFFFFFFll || (Qh.n_raw > 0 && !Qh.xyz) ||
            reinterpret_cast<uintptr_t>(Qh.xyz) % 16) {
            set_error("gmapp_batch_create: query %d: invalid cloud or workspace (batched queries "
                      "need min_pts == 1 and 16-byte aligned clouds)", q);
            delete b;
            return GMAPP_ERR_INVALID_ARG;
        }
        const gmapp_obstacles &o = Qh.obs;
        if (!o.x || !o.y || !o.z || !o.keys || !o.counts || !o.rep_idx || !o.n || o.cap < 4 ||
            o.cap % 4 ||
            ((reinterpret_cast<uintptr_t>(o.x) | reinterpret_cast<uintptr_t>(o.y) |
              reinterpret_cast<uintptr_t>(o.z)) % 16)) {
            set_error("gmapp_batch_create: query %d: obstacle buffers must be set, 16-byte "
                      "aligned, cap a multiple of 4", q);
            delete b;
            return GMAPP_ERR_INVALID_ARG;
        }
        const gmapp_agents &a = Qh.agents;
        const gmapp_rollout_params &p = Qh.prm;
        if (a.n < 1 || !a.p0 || !a.v0 || !a.c || !a.k_r || !a.k_a || !a.r_d || !a.r_a ||
            p.n_steps < 1 || !(p.dt > 0.0f) || !(p.eps > 0.0f) || !(p.clear_beta > 0.0f) ||
            !Qh.out.p_final || !Qh.out.v_final || !Qh.out.path_len || !Qh.costs || !Qh.best ||
            (Qh.best_traj && !Qh.out.traj) || (Qh.w.w_clear != 0.0f && !Qh.out.clear_pen) ||
            (Qh.out.cost_terms &&
             (!(Qh.prm.cost_radius > 0.0f) || !(Qh.w4.a_max > 0.0f) || !isfinite(Qh.alpha) ||
              !isfinite(Qh.w4.w_goal) || !isfinite(Qh.w4.w_obs) || !isfinite(Qh.w4.w_path) ||
              !isfinite(Qh.w4.w_smooth)))) {
            set_error("gmapp_batch_create: query %d: invalid agents, parameters or outputs", q);
            delete b;
            return GMAPP_ERR_INVALID_ARG;
        }
        for (int i = 0; i < 12; ++i)
            if (!isfinite(Qh.T[i])) {
                set_error("gmapp_batch_create: query %d: transform not finite", q);
                delete b;
                return GMAPP_ERR_INVALID_ARG;
            }
        const Layout L = layout(Qh.n_raw, &Qh.ws);
        ws_off[q] = ws_total;
        ws_total = align_up(ws_total + L.total, 256);
        QueryDev &D = b->hq[q];
        memset(&D, 0, sizeof(D));
        D.xyz = Qh.xyz;
        D.n_raw = Qh.n_raw;
        for (int i = 0; i < 12; ++i) D.fa.T[i] = Qh.T[i];
        for (int d = 0; d < 3; ++d) {
            D.fa.lo[d] = Qh.ws.lo[d];
            D.fa.dimf[d] = static_cast<float>(Qh.ws.dims[d]);
        }
        D.fa.voxel = Qh.ws.voxel;
        D.fa.nx = Qh.ws.dims[0];
        D.fa.ny = Qh.ws.dims[1];
        D.fa.nz = Qh.ws.dims[2];
        D.fa.err = ctx->d_err;
        D.pt_blk0 = static_cast<int32_t>(pt_map.size());
        D.pt_nblk = static_cast<int32_t>(std::max<int64_t>(
            1, std::min<int64_t>((Qh.n_raw / 4 + kThreads - 1) / kThreads, kMaxPointBlocksPerQuery)));
        for (int i = 0; i < D.pt_nblk; ++i) pt_map.push_back(q);
        D.bm_blk0 = static_cast<int32_t>(bm_map.size());
        D.bm_nblk = static_cast<int32_t>(L.n_blocks);
        for (int i = 0; i < D.bm_nblk; ++i) bm_map.push_back(q);
        D.sb_blk0 = static_cast<int32_t>(sb_map.size());
        D.sb_nblk = static_cast<int32_t>(L.n_sblocks);
        for (int i = 0; i < D.sb_nblk; ++i) sb_map.push_back(q);
        D.ox = o.x;
        D.oy = o.y;
        D.oz = o.z;
        D.okeys = o.keys;
        D.ocounts = o.counts;
        D.orep = o.rep_idx;
        D.n_obs = o.n;
        D.cap = o.cap;
        D.r_O = 0.5f * Qh.ws.voxel;
        max_cap = std::max(max_cap, o.cap);
        D.p0 = a.p0;
        D.v0 = a.v0;
        D.c = a.c;
        D.k_r = a.k_r;
        D.k_a = a.k_a;
        D.r_d = a.r_d;
        D.r_a = a.r_a;
        D.n_agents = a.n;
        for (int d = 0; d < 3; ++d) D.goal[d] = p.goal[d];
        D.dt = p.dt;
        D.n_steps = p.n_steps;
        D.damping = p.damping;
        D.inv_mass = p.inv_mass;
        D.rho = p.rho;
        D.eps = p.eps;
        D.vel_half = p.vel_half;
        D.clear_margin = p.clear_margin;
        D.clear_beta = p.clear_beta;
        D.traj = Qh.out.traj;
        D.p_final = Qh.out.p_final;
        D.v_final = Qh.out.v_final;
        D.path_len = Qh.out.path_len;
        D.clear_pen = Qh.out.clear_pen;
        D.min_clear = Qh.out.min_clear;
        D.w_path = Qh.w.w_path;
        D.w_goal = Qh.w.w_goal;
        D.w_clear = Qh.w.w_clear;
        D.costs = Qh.costs;
        D.best = Qh.best;
        D.best_traj = Qh.best_traj;
        D.cost_terms = Qh.out.cost_terms;
        D.cost_radius = p.cost_radius;
        D.w4[0] = Qh.w4.w_goal;
        D.w4[1] = Qh.w4.w_obs;
        D.w4[2] = Qh.w4.w_path;
        D.w4[3] = Qh.w4.w_smooth;
        {
            const double dt = p.dt, am = Qh.w4.a_max;
            D.smooth_scale = Qh.out.cost_terms
                                 ? static_cast<float>(1.0 / (p.n_steps * dt * dt * dt * dt * am * am))
                                 : 0.0f;
        }
        D.alpha = Qh.alpha;
        D.c_best = Qh.c_best;
        b->clear = b->clear || Qh.out.clear_pen || Qh.out.min_clear || Qh.out.cost_terms;
    }
    b->pt_blocks = static_cast<int32_t>(pt_map.size());
    b->bm_blocks = static_cast<int32_t>(bm_map.size());
    b->sb_blocks = static_cast<int32_t>(sb_map.size());
    b->max_cap = max_cap;
    cudaError_t e = cudaMalloc(&b->d_ws, std::max<size_t>(ws_total, 256));
    // zero filter scratch: bitmaps and counters start clear, and each run
    // leaves them clear again (kb_emit clears the bitmap behind it)
    if (e == cudaSuccess) e = cudaMemset(b->d_ws, 0, std::max<size_t>(ws_total, 256));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_q, sizeof(QueryDev) * n_q);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_pt_map, sizeof(int32_t) * pt_map.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_bm_map, sizeof(int32_t) * bm_map.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_sb_map, sizeof(int32_t) * sb_map.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_items_static, sizeof(int32_t) * kMaxItems);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_items, sizeof(int32_t) * kMaxItems);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_head, sizeof(uint32_t));
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_pt_map, pt_map.data(), sizeof(int32_t) * pt_map.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_bm_map, bm_map.data(), sizeof(int32_t) * bm_map.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_sb_map, sb_map.data(), sizeof(int32_t) * sb_map.size(),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        gmapp_status st = cuda_fail(e, "gmapp_batch_create");
        release(b);
        delete b;
        return st;
    }
    char *ws = static_cast<char *>(b->d_ws);
    for (int q = 0; q < n_q; ++q) {
        const Layout L = layout(queries[q].n_raw, &queries[q].ws);
        char *base = ws + ws_off[q];
        QueryDev &D = b->hq[q];
        D.bitmap = reinterpret_cast<uint32_t *>(base + L.off_bitmap);
        D.pw = reinterpret_cast<uint2 *>(base + L.off_pw);
        D.chunk = reinterpret_cast<uint32_t *>(base + L.off_chunk);
        D.sums = reinterpret_cast<uint32_t *>(base + L.off_sums);
        D.offsets = reinterpret_cast<uint32_t *>(base + L.off_offsets);
        D.counters = reinterpret_cast<uint32_t *>(base + L.off_counters);
        D.keys = reinterpret_cast<uint32_t *>(base + L.off_keys);
    }
    gmapp_status st = apply_tuning(b, 8, 256);
    if (st != GMAPP_OK) {
        release(b);
        delete b;
        return st;
    }
    *out = b;
    return GMAPP_OK;
}

extern "C" void gmapp_batch_destroy(gmapp_batch *b) {
    if (!b) return;
    release(b);
    delete b;
}

extern "C" gmapp_status gmapp_batch_set_tuning(gmapp_batch *b, int32_t agents_per_item,
                                               int32_t threads) {
    if (!b) {
        set_error("gmapp_batch_set_tuning: NULL batch");
        return GMAPP_ERR_INVALID_ARG;
    }
    return apply_tuning(b, agents_per_item, threads);
}

extern "C" gmapp_status gmapp_batch_set_culling(gmapp_batch *b, int32_t on) {
    if (!b) {
        set_error("gmapp_batch_set_culling: NULL batch");
        return GMAPP_ERR_INVALID_ARG;
    }
    const bool prev = b->cull;
    b->cull = on != 0;
    const gmapp_status st = apply_tuning(b, b->agents_per_item, b->threads);
    if (st != GMAPP_OK) b->cull = prev;
    return st;
}

extern "C" gmapp_status rollout_batch(gmapp_batch *b, gmapp_stream stream) {
    if (!b) {
        set_error("rollout_batch: NULL batch");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (!b->fn) {
        set_error("rollout_batch: the batch has no usable tuning (a tuning copy failed)");
        return GMAPP_ERR_INVALID_ARG;
    }
    const BatchDev B = dev_view(b);
    kb_keys<<<b->pt_blocks, kThreads, 0, stream>>>(B);
    kb_bitmap_sums<<<b->sb_blocks, kBmThreads, 0, stream>>>(B);
    kb_emit<<<b->bm_blocks, kBmThreads, 0, stream>>>(B);
    kb_count<<<b->pt_blocks, kThreads, 0, stream>>>(B);
    kb_plan<<<1, 1024, b->n_items * sizeof(float), stream>>>(B, b->agents_per_item);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->grid, 1, 1);
    cfg.blockDim = dim3(b->threads, 1, 1);
    cfg.dynamicSmemBytes = b->smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;  // a cluster of one CTA
    attr.val.clusterDim.x = 1;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    GMAPP_CHECK_CUDA(cudaLaunchKernelEx(&cfg, b->fn, B));
    kb_score<<<b->n_q, kScoreThreads, 0, stream>>>(B);
    GMAPP_CHECK_CUDA(cudaGetLastError());
    return GMAPP_OK;
}

extern "C" gmapp_status gmapp_batch_launch_graph(gmapp_batch *b, gmapp_stream stream) {
    if (!b || !stream) {
        set_error("gmapp_batch_launch_graph: needs a batch and a non-default stream");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (!b->exec) {
        GMAPP_CHECK_CUDA(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
        gmapp_status st = rollout_batch(b, stream);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(stream, &g);
        if (st != GMAPP_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(e, "gmapp_batch_launch_graph: capture");
        b->graph = g;
        GMAPP_CHECK_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
    }
    GMAPP_CHECK_CUDA(cudaGraphLaunch(b->exec, stream));
    return GMAPP_OK;
}

extern "C" gmapp_status gmapp_batch_autotune(gmapp_batch *b, gmapp_stream stream,
                                             gmapp_tuning *best, float *best_ms) {
    if (!b) {
        set_error("gmapp_batch_autotune: NULL batch");
        return GMAPP_ERR_INVALID_ARG;
    }
    const int ags[] = {2, 4, 6, 8, 12, 16};
    const int nts[] = {256, 384, 512};
    cudaEvent_t e0, e1;
    GMAPP_CHECK_CUDA(cudaEventCreate(&e0));
    GMAPP_CHECK_CUDA(cudaEventCreate(&e1));
    float best_t = 1e30f;
    int best_ag = 8, best_nt = 256;
    for (int ag : ags)
        for (int nt : nts) {
            if (apply_tuning(b, ag, nt) != GMAPP_OK) continue;
            if (rollout_batch(b, stream) != GMAPP_OK) continue;
            cudaEventRecord(e0, stream);
            if (rollout_batch(b, stream) != GMAPP_OK) continue;
            cudaEventRecord(e1, stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return cuda_fail(cudaGetLastError(), "gmapp_batch_autotune");
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_t) {
                best_t = ms;
                best_ag = ag;
                best_nt = nt;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    gmapp_status st = apply_tuning(b, best_ag, best_nt);
    if (st != GMAPP_OK) return st;
    if (best) *best = gmapp_tuning{1, best_ag, best_nt};
    if (best_ms) *best_ms = best_t;
    return GMAPP_OK;
}
