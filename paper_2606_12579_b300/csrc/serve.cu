// Served control loop with continuous batching (the paper's planning thread
// answers one query per control cycle, Sec. V-B; here many requests are in
// flight at once).
//
// A gmapp_server owns a device arena.  Requests arrive from the host with
// host-resident clouds and agents; a request is admitted as soon as its
// bytes fit in the arena (first fit), its inputs are copied on a copy stream
// and filtered on the compute stream.  Every tick advances EVERY active
// request by up to M steps in ONE persistent launch over (request, agent
// group) work items -- requests that arrived while others run join at the
// next tick -- and requests that reach their horizon are scored, their plan
// copied to pinned host memory, and their memory released.  A work item's
// arithmetic depends only on its own request and the agent state is kept
// exactly between chunks, so each result is bit-identical whether the
// request runs alone or in any mix.
//
// With cfg.culled the server visits, for every agent, only the obstacles
// within its reach (the voxel grid as a neighbour grid, culled_device.cuh):
// each request gets its grid index after its filter, and the chunk kernel
// takes one agent per work item (ks_chunk_culled).
#include <math.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <vector>

#include "culled_device.cuh"

namespace gmapp {
namespace {

struct SlotDev {
    const float *ox, *oy, *oz;
    const int32_t *n_obs;
    int64_t cap;
    float r_O;
    const float *p0, *v0, *c, *k_r, *k_a, *r_d, *r_a;
    int32_t n_agents, n_groups;
    float goal[3];
    float dt;
    int32_t n_steps;
    float damping, inv_mass, rho, eps, vel_half, clear_margin, clear_beta;
    float *sp, *sv, *sL;       // saved state between chunks: p [3][n], v [3][n], L [n]
    float *traj, *p_final, *v_final, *path_len;
    NeighbourGrid grid;        // culled server: the request's neighbour index
    // four-term cost (cost_mode 1; CLEAR chunk kernels): outputs [5][n] and the
    // sums carried between chunks [kCostRows][n]
    float *cost_terms, *cacc;
    float cost_radius;
};

// Four-term cost accumulators per agent (the rows of k_rollout's cost
// columns): 0 sum min(|p - goal|, r_c), 1 sum max(r_c - m, 0), 2 the path
// length before the last segment, 3 the jerk sum, 4 |p_0 - goal|, 5-7
// F_{k-1}, 8-10 f_r at k-1.
constexpr int kCostRows = 11;

struct ChunkItem {
    int32_t slot, group, k0, k1;
};

struct ChunkArgs {
    const SlotDev *slots;
    const ChunkItem *items;
    int32_t n_items;
    uint32_t *head;
    int32_t shard_cap;
    uint32_t *err;
};

// BOX (cfg.culled == 2): the pair loop visits only the resident blocks of 128
// obstacles whose bounding box meets a gate of the item's agents (in the
// order and lane layout of the voting loop, so the sums equal the all-pairs
// server's bit for bit); the obstacles beyond the resident part are still
// evaluated pair by pair.
template <int AG, int NT, bool BOX, bool CLEAR>
__global__ void __launch_bounds__(NT, 1) ks_chunk(const ChunkArgs A) {
    constexpr int NW = NT / 32;
    constexpr int NM = sfu_agents(AG);
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_item;
    __shared__ int s_om;  // bits of max |o|^2 of the resident obstacles
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *sx = smem, *sy = smem + A.shard_cap, *sz = smem + 2 * A.shard_cap;
    float *recv = smem + 3 * A.shard_cap;
    float *boxes = recv + 2 * NW * AG * 2;  // [shard_cap / 128][6] (BOX)
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    for (;;) {
        if (tid == 0) {
            s_item = static_cast<int>(atomicAdd(A.head, 1u));
            s_om = 0;
        }
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= A.n_items) break;
        const ChunkItem item = A.items[it];
        const SlotDev &S = A.slots[item.slot];
        int a0, na;
        group_range(item.group, S.n_agents, S.n_groups, a0, na);
        const int32_t n_obs = *S.n_obs;
        if (n_obs < 0 || n_obs > S.cap || na > AG || (A.shard_cap & 127)) {
            if (tid == 0) raise_error(A.err, GMAPP_DEVERR_CAPACITY);
            continue;
        }
        int32_t cnt = min(n_obs, A.shard_cap);
        const GlobalTail tail{S.ox, S.oy, S.oz, cnt, n_obs};
        if (cnt > 0 && tid == 0) {
            const uint32_t bytes = static_cast<uint32_t>((cnt + 3) & ~3) * 4u;
            mbar_arrive_expect_tx(&bar, 3 * bytes);
            bulk_g2s(sx, S.ox, bytes, &bar);
            bulk_g2s(sy, S.oy, bytes, &bar);
            bulk_g2s(sz, S.oz, bytes, &bar);
        }
        const int n = S.n_agents, N = S.n_steps;
        float p[3] = {0, 0, 0}, v[3] = {0, 0, 0}, cc[3] = {0, 0, 0};
        float k_r = 0, k_a = 0, R = 0, G2 = -1.0f, L = 0, pen = 0, minc = INFINITY;
        if (lane < na) {
            const int i = a0 + lane;
            const bool first = item.k0 == 0;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                p[d] = first ? S.p0[d * n + i] : S.sp[d * n + i];
                v[d] = first ? S.v0[d * n + i] : S.sv[d * n + i];
                cc[d] = S.c[d * n + i];
            }
            L = first ? 0.0f : S.sL[i];
            k_r = S.k_r[i];
            k_a = S.k_a[i];
            R = S.r_a[i] + S.r_O;
            const float rd = S.r_d[i];
            G2 = rd >= S.eps ? (rd + R) * (rd + R) : -1.0f;
            if (first && warp == 0 && S.traj) {
                float *t = S.traj + (size_t)i * (N + 1) * 3;
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
                if (tid == 0) raise_error(A.err, GMAPP_DEVERR_TIMEOUT);
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
        const float h = S.vel_half * S.dt * S.inv_mass;
        const float goal[3] = {S.goal[0], S.goal[1], S.goal[2]};
        // four-term cost sums (the arithmetic of k_rollout's exchange warps),
        // carried between chunks in S.cacc
        const bool four = CLEAR && S.cost_terms != nullptr;  // uniform per item
        float cv[kCostRows];
#pragma unroll
        for (int r = 0; r < kCostRows; ++r)
            cv[r] = four && lane < na && item.k0 > 0 ? S.cacc[r * n + a0 + lane] : 0.0f;
        for (int k = item.k0; k < item.k1; ++k) {
            float *rp = recv + (k & 1) * (NW * AG * 2);
            half_step<AG, AG, 0, NM, NT, CLEAR, true, true, false, true, BOX>(
                sx, sy, sz, cnt_pad, S.eps, nR2, G2a, p, rp + 2 * (warp * AG), 1u, lane, tail,
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
                    cv[0] += fminf(dg, S.cost_radius);
                    if (k == 0) cv[4] = dg;
                    if (k == N - 1) cv[2] = L;  // before the last segment
                }
                agent_step<CLEAR>(p, v, cc, k_r, k_a, R, goal, h, S.dt, S.rho, S.damping,
                                  S.clear_margin, S.clear_beta, W, md2, L, pen, minc, m, g, kf,
                                  F);
                if (four) {
                    float fr[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) fr[d] = kf * g[d];
                    cv[1] += fmaxf(S.cost_radius - m, 0.0f);
                    if (k >= 2 && k <= N - 2) {
                        float sj = 0.0f;
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            const float dF = fmaf(-k_a * S.dt, vprev[d],
                                                  fmaf(-S.damping * h, cv[5 + d], fr[d] - cv[8 + d]));
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
                if (warp == 0 && S.traj) {
                    float *t = S.traj + ((size_t)(a0 + lane) * (N + 1) + k + 1) * 3;
                    t[0] = p[0];
                    t[1] = p[1];
                    t[2] = p[2];
                }
            }
        }
        if (warp == 0 && lane < na) {
            const int i = a0 + lane;
            for (int d = 0; d < 3; ++d) {
                S.sp[d * n + i] = p[d];
                S.sv[d * n + i] = v[d];
            }
            S.sL[i] = L;
            if (four) {
#pragma unroll
                for (int r = 0; r < kCostRows; ++r) S.cacc[r * n + i] = cv[r];
            }
            if (item.k1 == N) {
                for (int d = 0; d < 3; ++d) {
                    S.p_final[d * n + i] = p[d];
                    S.v_final[d * n + i] = v[d];
                }
                S.path_len[i] = L;
                if (four) {
                    const float rc = S.cost_radius, dh = S.dt * h;
                    S.cost_terms[i] = cv[0] / rc;
                    S.cost_terms[n + i] = cv[1] / rc;
                    S.cost_terms[2 * n + i] = cv[2];
                    S.cost_terms[3 * n + i] = dh * dh * cv[3];
                    S.cost_terms[4 * n + i] = cv[4];
                }
            }
        }
        __syncthreads();
    }
}

// Culled chunks (cfg.culled): one agent of one request per work item
// (ChunkItem.group is the agent index), its CTA deals the agent's grid rows
// to its threads every step (culled_terms), reduces in a fixed order and
// thread 0 integrates; the state is saved exactly between chunks as in
// ks_chunk.
constexpr int kServeCullThreads = 128;

__global__ void __launch_bounds__(kServeCullThreads) ks_chunk_culled(const ChunkArgs A) {
    constexpr int NT = kServeCullThreads, NW = NT / 32;
    __shared__ float s_w[NW], s_m[NW], s_p[3];
    __shared__ int s_item;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_item = static_cast<int>(atomicAdd(A.head, 1u));
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= A.n_items) break;
        const ChunkItem item = A.items[it];
        const SlotDev &S = A.slots[item.slot];
        const int i = item.group, n = S.n_agents, N = S.n_steps;
        const int32_t n_obs = *S.n_obs;
        if (n_obs < 0 || n_obs > S.cap) {
            if (tid == 0) raise_error(A.err, GMAPP_DEVERR_CAPACITY);
            continue;  // uniform across the CTA
        }
        const float R = S.r_a[i] + S.r_O, rd = S.r_d[i];
        if (!isfinite(rd)) {  // no gate: nothing to cull by
            if (tid == 0) raise_error(A.err, GMAPP_DEVERR_BOUNDS);
            continue;
        }
        const float G2 = rd >= S.eps ? (rd + R) * (rd + R) : -1.0f;
        const float reach = culled_reach(rd, R, S.eps, S.grid.voxel);
        const bool first = item.k0 == 0;
        float p[3], v[3], cc[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            p[d] = first ? S.p0[d * n + i] : S.sp[d * n + i];
            v[d] = first ? S.v0[d * n + i] : S.sv[d * n + i];
            cc[d] = S.c[d * n + i];
        }
        float L = first ? 0.0f : S.sL[i], pen = 0.0f, minc = INFINITY;
        const float k_r = S.k_r[i], k_a = S.k_a[i];
        const float h = S.vel_half * S.dt * S.inv_mass;
        const float goal[3] = {S.goal[0], S.goal[1], S.goal[2]};
        if (first && tid == 0 && S.traj) {
            float *t = S.traj + static_cast<size_t>(i) * (N + 1) * 3;
            t[0] = p[0];
            t[1] = p[1];
            t[2] = p[2];
        }
        // four-term cost sums (cost_mode 1), kept by thread 0 and carried
        // between chunks in S.cacc; the clearance is the culled one (the
        // nearest obstacle within the agent's reach)
        const bool four = S.cost_terms != nullptr;  // uniform per item
        float cv[kCostRows];
#pragma unroll
        for (int r = 0; r < kCostRows; ++r)
            cv[r] = four && tid == 0 && item.k0 > 0 ? S.cacc[r * n + i] : 0.0f;
        for (int k = item.k0; k < item.k1; ++k) {
            float W, md2;
            if (four) {
                culled_terms<NT, true>(p, reach, G2, R, S.eps, S.grid, S.ox, S.oy, S.oz, tid, W,
                                       md2);
                culled_reduce<NT, true>(W, md2, s_w, s_m);
            } else {
                culled_terms<NT, false>(p, reach, G2, R, S.eps, S.grid, S.ox, S.oy, S.oz, tid, W,
                                        md2);
                culled_reduce<NT, false>(W, md2, s_w, s_m);
            }
            if (tid == 0) {
                float g[3], kf, m, F[3];
                if (four) {
                    const float vprev[3] = {v[0], v[1], v[2]};
                    const float gx = p[0] - goal[0], gy = p[1] - goal[1], gz = p[2] - goal[2];
                    const float dg = sqrtf(fmaf(gz, gz, fmaf(gy, gy, gx * gx)));
                    cv[0] += fminf(dg, S.cost_radius);
                    if (k == 0) cv[4] = dg;
                    if (k == N - 1) cv[2] = L;  // before the last segment
                    agent_step<true>(p, v, cc, k_r, k_a, R, goal, h, S.dt, S.rho, S.damping,
                                     S.clear_margin, S.clear_beta, W, md2, L, pen, minc, m, g, kf,
                                     F);
                    float fr[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) fr[d] = kf * g[d];
                    cv[1] += fmaxf(S.cost_radius - m, 0.0f);
                    if (k >= 2 && k <= N - 2) {
                        float sj = 0.0f;
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            const float dF = fmaf(-k_a * S.dt, vprev[d],
                                                  fmaf(-S.damping * h, cv[5 + d], fr[d] - cv[8 + d]));
                            sj = fmaf(dF, dF, sj);
                        }
                        cv[3] += sj;
                    }
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        cv[5 + d] = F[d];
                        cv[8 + d] = fr[d];
                    }
                } else {
                    agent_step<false>(p, v, cc, k_r, k_a, R, goal, h, S.dt, S.rho, S.damping,
                                      S.clear_margin, S.clear_beta, W, md2, L, pen, minc, m, g,
                                      kf);
                }
                s_p[0] = p[0];
                s_p[1] = p[1];
                s_p[2] = p[2];
                if (S.traj) {
                    float *t = S.traj + (static_cast<size_t>(i) * (N + 1) + k + 1) * 3;
                    t[0] = p[0];
                    t[1] = p[1];
                    t[2] = p[2];
                }
            }
            __syncthreads();
            p[0] = s_p[0];
            p[1] = s_p[1];
            p[2] = s_p[2];
        }
        if (tid == 0) {
            for (int d = 0; d < 3; ++d) {
                S.sp[d * n + i] = p[d];
                S.sv[d * n + i] = v[d];
            }
            S.sL[i] = L;
            if (four) {
#pragma unroll
                for (int r = 0; r < kCostRows; ++r) S.cacc[r * n + i] = cv[r];
            }
            if (item.k1 == N) {
                for (int d = 0; d < 3; ++d) {
                    S.p_final[d * n + i] = p[d];
                    S.v_final[d * n + i] = v[d];
                }
                S.path_len[i] = L;
                if (four) {
                    const float rc = S.cost_radius, dh = S.dt * h;
                    S.cost_terms[i] = cv[0] / rc;
                    S.cost_terms[n + i] = cv[1] / rc;
                    S.cost_terms[2 * n + i] = cv[2];
                    S.cost_terms[3 * n + i] = dh * dh * cv[3];
                    S.cost_terms[4 * n + i] = cv[4];
                }
            }
        }
    }
}


using ChunkKernel = void (*)(const ChunkArgs);

template <bool BOX, bool CLEAR>
ChunkKernel chunk_kernel_t(int ag, int nt) {
#define GMAPP_CK(AGV)                                                  \
    case AGV:                                                          \
        switch (nt) {                                                  \
            case 256: return ks_chunk<AGV, 256, BOX, CLEAR>;           \
            case 384: return ks_chunk<AGV, 384, BOX, CLEAR>;           \
            case 512:                                                  \
                if constexpr (AGV <= 8) return ks_chunk<AGV, 512, BOX, CLEAR>; \
                return nullptr;                                        \
            default: return nullptr;                                   \
        }
    switch (ag) {
        GMAPP_CK(4)
        GMAPP_CK(8)
        GMAPP_CK(16)
        default: return nullptr;
    }
#undef GMAPP_CK
}

ChunkKernel chunk_kernel(int ag, int nt, bool box, bool clear) {
    if (clear) return box ? chunk_kernel_t<true, true>(ag, nt) : chunk_kernel_t<false, true>(ag, nt);
    return box ? chunk_kernel_t<true, false>(ag, nt) : chunk_kernel_t<false, false>(ag, nt);
}

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit byte allocator over the device arena (offsets, 256-aligned).
class Arena {
   public:
    void init(size_t bytes) { free_.assign(1, {0, bytes}); }
    bool alloc(size_t bytes, size_t *off) {
        bytes = align_up(bytes, 256);
        for (size_t i = 0; i < free_.size(); ++i)
            if (free_[i].second >= bytes) {
                *off = free_[i].first;
                free_[i].first += bytes;
                free_[i].second -= bytes;
                if (free_[i].second == 0) free_.erase(free_.begin() + i);
                return true;
            }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = align_up(bytes, 256);
        free_.push_back({off, bytes});
        std::sort(free_.begin(), free_.end());
        std::vector<std::pair<size_t, size_t>> merged;
        for (auto &r : free_) {
            if (!merged.empty() && merged.back().first + merged.back().second == r.first)
                merged.back().second += r.second;
            else
                merged.push_back(r);
        }
        free_.swap(merged);
    }
    size_t free_bytes() const {
        size_t s = 0;
        for (auto &r : free_) s += r.second;
        return s;
    }

   private:
    std::vector<std::pair<size_t, size_t>> free_;
};

}  // namespace
}  // namespace gmapp

using namespace gmapp;

struct ServerReq {
    gmapp_request req;
    int64_t ticket;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int slot = -1;
    size_t off = 0, bytes = 0;
    int32_t k = 0;  // steps done
    int64_t seq = 0;       // position in its plan stream (cost_mode 1, plan_stream >= 0)
    int32_t bypassed = 0;  // later requests admitted while this one waited
    enum { PENDING, ACTIVE, SCORING, DONE } state = PENDING;
    // results, copied out of the slot's pinned staging when the request retires
    int32_t best = -1, n_obs = 0;
    std::vector<float> costs, traj;
    // device buffers inside the arena
    float *d_xyz = nullptr;
    void *d_fws = nullptr;
    size_t fws_bytes = 0;
    gmapp_obstacles obs{};
    float *d_costs = nullptr, *d_best_traj = nullptr;
    int32_t *d_best = nullptr;
    gmapp_rollout_out out{};
    float *d_cacc = nullptr;  // four-term sums carried between chunks
};

struct gmapp_server {
    gmapp_ctx *ctx = nullptr;
    gmapp_server_config cfg{};
    cudaStream_t compute = nullptr, copy = nullptr;
    char *arena_base = nullptr;
    Arena arena;
    SlotDev *d_slots = nullptr;
    SlotDev *h_slots = nullptr;   // pinned mirror
    ChunkItem *d_items = nullptr;
    ChunkItem *h_items = nullptr;  // pinned
    uint32_t *d_head = nullptr;
    int max_items = 0;
    std::vector<int> free_slots;
    std::deque<int64_t> pending;
    std::map<int64_t, ServerReq *> reqs;
    int64_t next_ticket = 1;
    cudaEvent_t tick_ev = nullptr;
    bool tick_in_flight = false;
    // per slot: pinned result staging and events (created once)
    int32_t *h_best = nullptr, *h_nobs = nullptr;
    float *h_costs = nullptr, *h_traj = nullptr;
    std::vector<cudaEvent_t> slot_done, slot_h2d;
    ChunkKernel fn = nullptr;
    size_t smem = 0;
    int shard_cap = 0, resident = 0;
    int64_t completed = 0;
    // per plan stream: the current plan's cost C_best on the device (NaN =
    // none yet), the next sequence number to hand out and to score
    float *d_cbest = nullptr;
    std::vector<int64_t> next_seq, next_score;
};

namespace {

size_t request_bytes(const gmapp_server_config &c, const gmapp_request &r, size_t fws) {
    const size_t na = r.n_agents, nk = r.prm.n_steps;
    size_t b = 0;
    auto add = [&](size_t x) { b += align_up(x, 256); };
    add(static_cast<size_t>(r.n_raw) * 12);           // cloud
    add(fws);                                          // filter scratch
    add(static_cast<size_t>(c.obs_cap) * 24 + 16);     // obstacle set (x,y,z,keys,counts,rep) + n
    add(na * 13 * 4);                                  // agent arrays
    add(na * 7 * 4);                                   // saved state p, v, L
    add(na * 6 * 4 + na * 4);                          // p_final, v_final, path_len
    add(na * (nk + 1) * 12);                           // trajectories
    add(na * 4 + 4 + (nk + 1) * 12);                   // costs, best, best trajectory
    if (c.culled == 1) add(gmapp_grid_index_bytes(&r.ws));  // neighbour index
    if (r.cost_mode == 1) add(na * (5 + kCostRows) * 4);    // four-term sums and carry
    return b;
}

gmapp_status admit(gmapp_server *s, ServerReq *q) {
    const gmapp_request &r = q->req;
    const size_t na = r.n_agents, nk = r.prm.n_steps;
    char *base = s->arena_base + q->off;
    size_t o = 0;
    auto take = [&](size_t x) {
        char *p = base + o;
        o = align_up(o + x, 256);
        return p;
    };
    q->d_xyz = reinterpret_cast<float *>(take(static_cast<size_t>(r.n_raw) * 12));
    q->d_fws = take(q->fws_bytes);
    const int64_t cap = s->cfg.obs_cap;
    char *ob = take(static_cast<size_t>(cap) * 24 + 16);
    q->obs.x = reinterpret_cast<float *>(ob);
    q->obs.y = q->obs.x + cap;
    q->obs.z = q->obs.y + cap;
    q->obs.keys = reinterpret_cast<uint32_t *>(q->obs.z + cap);
    q->obs.counts = q->obs.keys + cap;
    q->obs.rep_idx = q->obs.counts + cap;
    q->obs.n = reinterpret_cast<int32_t *>(q->obs.rep_idx + cap);
    q->obs.cap = cap;
    float *ag = reinterpret_cast<float *>(take(na * 13 * 4));
    float *st = reinterpret_cast<float *>(take(na * 7 * 4));
    float *fin = reinterpret_cast<float *>(take(na * 6 * 4 + na * 4));
    q->out.traj = reinterpret_cast<float *>(take(na * (nk + 1) * 12));
    float *sel = reinterpret_cast<float *>(take(na * 4 + 4 + (nk + 1) * 12));
    const size_t index_bytes = s->cfg.culled == 1 ? gmapp_grid_index_bytes(&r.ws) : 0;
    uint32_t *index = s->cfg.culled == 1 ? reinterpret_cast<uint32_t *>(take(index_bytes)) : nullptr;
    q->out.cost_terms = nullptr;
    q->d_cacc = nullptr;
    if (r.cost_mode == 1) {
        float *ct = reinterpret_cast<float *>(take(na * (5 + kCostRows) * 4));
        q->out.cost_terms = ct;
        q->d_cacc = ct + 5 * na;
    }
    q->out.p_final = fin;
    q->out.v_final = fin + 3 * na;
    q->out.path_len = fin + 6 * na;
    q->d_costs = sel;
    q->d_best = reinterpret_cast<int32_t *>(sel + na);
    q->d_best_traj = sel + na + 1;
    // inputs: host -> device on the copy stream
    GMAPP_CHECK_CUDA(cudaMemcpyAsync(q->d_xyz, r.xyz, static_cast<size_t>(r.n_raw) * 12,
                                     cudaMemcpyHostToDevice, s->copy));
    const float *src[7] = {r.p0, r.v0, r.c, r.k_r, r.k_a, r.r_d, r.r_a};
    const size_t cnt[7] = {3 * na, 3 * na, 3 * na, na, na, na, na};
    size_t at = 0;
    for (int i = 0; i < 7; ++i) {
        GMAPP_CHECK_CUDA(cudaMemcpyAsync(ag + at, src[i], cnt[i] * 4, cudaMemcpyHostToDevice,
                                         s->copy));
        at += cnt[i];
    }
    cudaEvent_t ev = s->slot_h2d[q->slot];
    GMAPP_CHECK_CUDA(cudaEventRecord(ev, s->copy));
    GMAPP_CHECK_CUDA(cudaStreamWaitEvent(s->compute, ev, 0));
    gmapp_status st2 = filter_cloud(s->ctx, q->d_xyz, r.n_raw, r.T, &r.ws, &q->obs, q->d_fws,
                                    q->fws_bytes, s->compute);
    if (st2 != GMAPP_OK) return st2;
    if (index) {
        st2 = gmapp_grid_index(s->ctx, &q->obs, &r.ws, index, index_bytes, s->compute);
        if (st2 != GMAPP_OK) return st2;
    }
    // device descriptor of the slot
    SlotDev &D = s->h_slots[q->slot];
    memset(&D, 0, sizeof(D));
    D.ox = q->obs.x;
    D.oy = q->obs.y;
    D.oz = q->obs.z;
    D.n_obs = q->obs.n;
    D.cap = cap;
    D.r_O = q->obs.r_O;
    D.p0 = ag;
    D.v0 = ag + 3 * na;
    D.c = ag + 6 * na;
    D.k_r = ag + 9 * na;
    D.k_a = ag + 10 * na;
    D.r_d = ag + 11 * na;
    D.r_a = ag + 12 * na;
    D.n_agents = static_cast<int32_t>(na);
    D.n_groups = static_cast<int32_t>((na + s->cfg.agents_per_item - 1) / s->cfg.agents_per_item);
    for (int d = 0; d < 3; ++d) D.goal[d] = r.prm.goal[d];
    D.dt = r.prm.dt;
    D.n_steps = r.prm.n_steps;
    D.damping = r.prm.damping;
    D.inv_mass = r.prm.inv_mass;
    D.rho = r.prm.rho;
    D.eps = r.prm.eps;
    D.vel_half = r.prm.vel_half;
    D.clear_margin = r.prm.clear_margin;
    D.clear_beta = r.prm.clear_beta;
    D.sp = st;
    D.sv = st + 3 * na;
    D.sL = st + 6 * na;
    D.traj = q->out.traj;
    D.p_final = q->out.p_final;
    D.v_final = q->out.v_final;
    D.path_len = q->out.path_len;
    D.cost_terms = q->out.cost_terms;
    D.cacc = q->d_cacc;
    D.cost_radius = r.prm.cost_radius;
    if (index) {
        D.grid.wr = index;
        for (int a = 0; a < 3; ++a) D.grid.lo[a] = r.ws.lo[a];
        D.grid.voxel = r.ws.voxel;
        D.grid.nx = r.ws.dims[0];
        D.grid.ny = r.ws.dims[1];
        D.grid.nz = r.ws.dims[2];
    }
    GMAPP_CHECK_CUDA(cudaMemcpyAsync(s->d_slots + q->slot, &D, sizeof(SlotDev),
                                     cudaMemcpyHostToDevice, s->compute));
    return GMAPP_OK;
}

// The request's plan landed in its slot's pinned staging: keep a copy,
// free the slot and its arena bytes.
void retire(gmapp_server *s, ServerReq *q) {
    const int sl = q->slot;
    const size_t nk = q->req.prm.n_steps;
    q->best = s->h_best[sl];
    q->n_obs = s->h_nobs[sl];
    const float *c = s->h_costs + (size_t)sl * s->cfg.max_agents;
    q->costs.assign(c, c + q->req.n_agents);
    const float *t = s->h_traj + (size_t)sl * (s->cfg.max_steps + 1) * 3;
    q->traj.assign(t, t + (nk + 1) * 3);
    q->t_done = now_s();
    q->state = ServerReq::DONE;
    s->arena.release(q->off, q->bytes);
    s->free_slots.push_back(sl);
    ++s->completed;
}

}  // namespace

extern "C" gmapp_status gmapp_server_create(gmapp_ctx *ctx, const gmapp_server_config *cfg,
                                            gmapp_server **out) {
    if (!ctx || !cfg || !out || cfg->max_slots < 1 || cfg->arena_bytes < (1 << 20) ||
        cfg->chunk_steps < 1 || cfg->obs_cap < 4 || cfg->obs_cap % 4 ||
        cfg->max_agents < 1 || cfg->max_steps < 1 || cfg->culled < 0 || cfg->culled > 2 ||
        cfg->admit_bypass < 0 || cfg->four_term < 0 || cfg->four_term > 1 ||
        cfg->max_plan_streams < 0 ||
        (cfg->max_plan_streams > 0 && !cfg->four_term)) {
        set_error("gmapp_server_create: invalid configuration");
        return GMAPP_ERR_INVALID_ARG;
    }
    *out = nullptr;
    const bool grid_cull = cfg->culled == 1;  // 2: block culling in the chunk kernel
    ChunkKernel fn = grid_cull ? ks_chunk_culled
                               : chunk_kernel(cfg->agents_per_item, cfg->threads, cfg->culled == 2,
                                              cfg->four_term == 1);
    if (!fn) {
        set_error("gmapp_server_create: no chunk kernel for %d agents per item, %d threads",
                  cfg->agents_per_item, cfg->threads);
        return GMAPP_ERR_INVALID_ARG;
    }
    gmapp_server *s = new gmapp_server();
    s->ctx = ctx;
    s->cfg = *cfg;
    s->fn = fn;
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void *>(fn));
    const size_t recv_bytes =
        static_cast<size_t>(2) * (cfg->threads / 32) * cfg->agents_per_item * 2 * sizeof(float);
    const int64_t room =
        (static_cast<int64_t>(ctx->max_smem_optin) - static_cast<int64_t>(fa.sharedSizeBytes + recv_bytes)) / 12;
    // the culled kernel reads obstacles through the neighbour index (no shard)
    // a multiple of 128: the pair loop tests whole blocks of 128 obstacles.
    // Room for block culling's boxes (6 floats per 128 resident obstacles) is
    // kept in both chunk-kernel modes, so the all-pairs and the block-culled
    // server hold the same obstacles in shared memory and agree bit for bit.
    const int64_t room_b = room * 128 / (128 + 2);
    s->shard_cap = grid_cull ? 0
                             : static_cast<int>(std::min<int64_t>(
                                   (static_cast<int64_t>(cfg->obs_cap) + 127) & ~int64_t(127),
                                   room_b & ~int64_t(127)));
    s->smem = grid_cull ? 0
                        : static_cast<size_t>(s->shard_cap) * 12 + recv_bytes +
                              (cfg->culled == 2 ? static_cast<size_t>(s->shard_cap / 128) * 24 : 0);
    const int threads = grid_cull ? kServeCullThreads : cfg->threads;
    const int max_groups =
        grid_cull ? cfg->max_agents : (cfg->max_agents + cfg->agents_per_item - 1) / cfg->agents_per_item;
    s->max_items = cfg->max_slots * max_groups;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(s->smem));
    int per_sm = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void *>(fn),
                                                           threads, s->smem);
    s->resident = std::max(1, per_sm) * ctx->sm_count;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&s->arena_base, cfg->arena_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_slots, sizeof(SlotDev) * cfg->max_slots);
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_slots, sizeof(SlotDev) * cfg->max_slots);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_items, sizeof(ChunkItem) * s->max_items);
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_items, sizeof(ChunkItem) * s->max_items);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_head, sizeof(uint32_t));
    if (e == cudaSuccess && cfg->max_plan_streams > 0) {
        // C_best of every plan stream starts as NaN (all bits set): no plan yet
        e = cudaMalloc(&s->d_cbest, sizeof(float) * cfg->max_plan_streams);
        if (e == cudaSuccess) e = cudaMemset(s->d_cbest, 0xFF, sizeof(float) * cfg->max_plan_streams);
        s->next_seq.assign(cfg->max_plan_streams, 0);
        s->next_score.assign(cfg->max_plan_streams, 0);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->tick_ev, cudaEventDisableTiming);
    const size_t ms = cfg->max_slots;
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_best, sizeof(int32_t) * ms);
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_nobs, sizeof(int32_t) * ms);
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_costs, sizeof(float) * ms * cfg->max_agents);
    if (e == cudaSuccess)
        e = cudaMallocHost(&s->h_traj, sizeof(float) * ms * (cfg->max_steps + 1) * 3);
    for (size_t i = 0; i < ms && e == cudaSuccess; ++i) {
        cudaEvent_t a, b;
        e = cudaEventCreateWithFlags(&a, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b, cudaEventDisableTiming);
        if (e == cudaSuccess) {
            s->slot_done.push_back(a);
            s->slot_h2d.push_back(b);
        }
    }
    if (e != cudaSuccess) {
        gmapp_status st = cuda_fail(e, "gmapp_server_create");
        gmapp_server_destroy(s);
        return st;
    }
    s->arena.init(cfg->arena_bytes);
    for (int i = cfg->max_slots - 1; i >= 0; --i) s->free_slots.push_back(i);
    *out = s;
    return GMAPP_OK;
}

extern "C" void gmapp_server_destroy(gmapp_server *s) {
    if (!s) return;
    if (s->compute) cudaStreamSynchronize(s->compute);
    if (s->copy) cudaStreamSynchronize(s->copy);
    for (auto &kv : s->reqs) delete kv.second;
    for (cudaEvent_t e : s->slot_done) cudaEventDestroy(e);
    for (cudaEvent_t e : s->slot_h2d) cudaEventDestroy(e);
    cudaFreeHost(s->h_best);
    cudaFreeHost(s->h_nobs);
    cudaFreeHost(s->h_costs);
    cudaFreeHost(s->h_traj);
    if (s->tick_ev) cudaEventDestroy(s->tick_ev);
    cudaFree(s->arena_base);
    cudaFree(s->d_slots);
    cudaFreeHost(s->h_slots);
    cudaFree(s->d_items);
    cudaFreeHost(s->h_items);
    cudaFree(s->d_head);
    cudaFree(s->d_cbest);
    if (s->compute) cudaStreamDestroy(s->compute);
    if (s->copy) cudaStreamDestroy(s->copy);
    delete s;
}

extern "C" gmapp_status gmapp_server_submit(gmapp_server *s, const gmapp_request *r,
                                            int64_t *ticket) {
    if (!s || !r || !ticket) {
        set_error("gmapp_server_submit: NULL argument");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (!r->xyz || r->n_raw < 1 || r->n_agents < 1 || r->n_agents > s->cfg.max_agents ||
        r->prm.n_steps < 1 || r->prm.n_steps > s->cfg.max_steps || !(r->prm.dt > 0.0f) || !(r->prm.eps > 0.0f) || !r->p0 || !r->v0 ||
        !r->c || !r->k_r || !r->k_a || !r->r_d || !r->r_a || r->ws.min_pts < 1) {
        set_error("gmapp_server_submit: invalid request (agents and steps within the server's "
                  "maxima)");
        return GMAPP_ERR_INVALID_ARG;
    }
    const size_t fws = gmapp_filter_workspace_bytes(r->n_raw, &r->ws);
    if (fws == 0) {
        set_error("gmapp_server_submit: invalid voxel grid");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (r->cost_mode < 0 || r->cost_mode > 1) {
        set_error("gmapp_server_submit: cost_mode must be 0 or 1");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (r->cost_mode == 1) {
        const gmapp_cost4 &w = r->w4;
        if (!s->cfg.four_term || !(r->prm.cost_radius > 0.0f) || !isfinite(w.w_goal) ||
            !isfinite(w.w_obs) || !isfinite(w.w_path) || !isfinite(w.w_smooth) ||
            !(w.a_max > 0.0f) || !isfinite(r->alpha) || r->plan_stream < -1 ||
            r->plan_stream >= s->cfg.max_plan_streams) {
            set_error("gmapp_server_submit: the four-term cost needs a four_term server, "
                      "cost_radius > 0, finite weights and alpha, a_max > 0 and -1 <= "
                      "plan_stream < max_plan_streams");
            return GMAPP_ERR_INVALID_ARG;
        }
    }
    ServerReq *q = new ServerReq();
    q->req = *r;
    q->ticket = s->next_ticket++;
    q->t_submit = now_s();
    q->fws_bytes = fws;
    q->bytes = request_bytes(s->cfg, *r, fws);
    if (q->bytes > static_cast<size_t>(s->cfg.arena_bytes)) {
        delete q;
        set_error("gmapp_server_submit: request needs more than the whole arena");
        return GMAPP_ERR_CAPACITY;
    }
    if (r->cost_mode == 1 && r->plan_stream >= 0) q->seq = s->next_seq[r->plan_stream]++;
    s->reqs[q->ticket] = q;
    s->pending.push_back(q->ticket);
    *ticket = q->ticket;
    return GMAPP_OK;
}

extern "C" gmapp_status gmapp_server_tick(gmapp_server *s, int32_t *n_active) {
    if (!s) {
        set_error("gmapp_server_tick: NULL server");
        return GMAPP_ERR_INVALID_ARG;
    }
    // 1. the previous tick's chunk is done: its finished requests were
    //    scored with their results copied; retire those whose copy landed
    if (s->tick_in_flight) {
        GMAPP_CHECK_CUDA(cudaEventSynchronize(s->tick_ev));
        s->tick_in_flight = false;
    }
    for (auto &kv : s->reqs) {
        ServerReq *q = kv.second;
        if (q->state != ServerReq::SCORING) continue;
        if (cudaEventQuery(s->slot_done[q->slot]) != cudaSuccess) continue;
        retire(s, q);
    }
    // 2. admission: pending requests whose bytes fit, in arrival order; with
    //    admit_bypass > 0 a request that does not fit is passed over (first
    //    fit), until it has been overtaken admit_bypass times
    //    (requests of one plan stream keep their order among themselves, so a
    //    finished request never waits for the score of one still queued)
    {
        std::vector<ServerReq *> skipped;
        std::vector<char> held(s->next_seq.size(), 0);
        for (auto it = s->pending.begin(); it != s->pending.end() && !s->free_slots.empty();) {
            ServerReq *q = s->reqs[*it];
            const int ps = q->req.cost_mode == 1 ? q->req.plan_stream : -1;
            size_t off;
            if ((ps >= 0 && held[ps]) || !s->arena.alloc(q->bytes, &off)) {
                if (s->cfg.admit_bypass == 0 || q->bypassed >= s->cfg.admit_bypass) break;
                if (ps >= 0) held[ps] = 1;
                skipped.push_back(q);
                ++it;
                continue;
            }
            it = s->pending.erase(it);
            q->off = off;
            q->slot = s->free_slots.back();
            s->free_slots.pop_back();
            q->t_admit = now_s();
            gmapp_status st = admit(s, q);
            if (st != GMAPP_OK) return st;
            q->state = ServerReq::ACTIVE;
            q->k = 0;
            bool aged = false;
            for (ServerReq *o : skipped) aged |= ++o->bypassed >= s->cfg.admit_bypass;
            if (aged) break;
        }
    }
    // 3. one chunk of up to M steps for every active request, one launch
    std::vector<std::pair<int64_t, ChunkItem>> items;
    int active = 0;
    for (auto &kv : s->reqs) {
        ServerReq *q = kv.second;
        if (q->state != ServerReq::ACTIVE) continue;
        ++active;
        const int N = q->req.prm.n_steps;
        if (q->k >= N) continue;  // done, waiting for its turn to be scored
        const int k1 = std::min(N, q->k + s->cfg.chunk_steps);
        // culled: one agent per item (group = agent index)
        const int groups = s->cfg.culled == 1
                               ? q->req.n_agents
                               : (q->req.n_agents + s->cfg.agents_per_item - 1) / s->cfg.agents_per_item;
        for (int g = 0; g < groups; ++g) {
            const int na = q->req.n_agents / groups + (g < q->req.n_agents % groups ? 1 : 0);
            const int64_t cost = static_cast<int64_t>(na) * (k1 - q->k);
            items.push_back({cost, ChunkItem{q->slot, g, q->k, k1}});
        }
        q->k = k1;
    }
    if (n_active) *n_active = active;
    if (!items.empty()) {
        // longest chunks first
        std::stable_sort(items.begin(), items.end(),
                         [](const auto &a, const auto &b) { return a.first > b.first; });
        const int n_items = static_cast<int>(items.size());
        for (int i = 0; i < n_items; ++i) s->h_items[i] = items[i].second;
        GMAPP_CHECK_CUDA(cudaMemcpyAsync(s->d_items, s->h_items, sizeof(ChunkItem) * n_items,
                                         cudaMemcpyHostToDevice, s->compute));
        GMAPP_CHECK_CUDA(cudaMemsetAsync(s->d_head, 0, sizeof(uint32_t), s->compute));
        ChunkArgs A{s->d_slots, s->d_items, n_items, s->d_head, s->shard_cap, s->ctx->d_err};
        const int grid = std::max(1, std::min(n_items, s->resident));
        s->fn<<<grid, s->cfg.culled == 1 ? kServeCullThreads : s->cfg.threads, s->smem, s->compute>>>(A);
        GMAPP_CHECK_CUDA(cudaGetLastError());
    }
    // 4. requests that reached their horizon: score, copy the plan out
    for (auto &kv : s->reqs) {
        ServerReq *q = kv.second;
        if (q->state != ServerReq::ACTIVE || q->k < q->req.prm.n_steps) continue;
        gmapp_status st;
        if (q->req.cost_mode == 1) {
            // requests of one plan stream are scored in submission order, so
            // each compares against the plan its predecessor left in C_best
            const int ps = q->req.plan_stream;
            if (ps >= 0 && q->seq != s->next_score[ps]) continue;
            st = score_and_select4(s->ctx, &q->out, q->req.n_agents, &q->req.prm, &q->req.w4,
                                   ps >= 0 ? s->d_cbest + ps : nullptr, q->req.alpha,
                                   q->d_costs, q->d_best, q->d_best_traj, s->compute);
            if (ps >= 0) ++s->next_score[ps];
        } else {
            st = score_and_select(s->ctx, &q->out, q->req.n_agents, &q->req.prm, &q->req.w, NAN,
                                  1.0f, q->d_costs, q->d_best, q->d_best_traj, s->compute);
        }
        if (st != GMAPP_OK) return st;
        const size_t nk = q->req.prm.n_steps;
        const int sl = q->slot;
        GMAPP_CHECK_CUDA(cudaMemcpyAsync(s->h_best + sl, q->d_best, 4, cudaMemcpyDeviceToHost,
                                         s->compute));
        GMAPP_CHECK_CUDA(cudaMemcpyAsync(s->h_costs + (size_t)sl * s->cfg.max_agents, q->d_costs,
                                         4 * q->req.n_agents, cudaMemcpyDeviceToHost, s->compute));
        GMAPP_CHECK_CUDA(cudaMemcpyAsync(s->h_traj + (size_t)sl * (s->cfg.max_steps + 1) * 3,
                                         q->d_best_traj, 12 * (nk + 1), cudaMemcpyDeviceToHost,
                                         s->compute));
        GMAPP_CHECK_CUDA(cudaMemcpyAsync(s->h_nobs + sl, q->obs.n, 4, cudaMemcpyDeviceToHost,
                                         s->compute));
        GMAPP_CHECK_CUDA(cudaEventRecord(s->slot_done[sl], s->compute));
        q->state = ServerReq::SCORING;
    }
    GMAPP_CHECK_CUDA(cudaEventRecord(s->tick_ev, s->compute));
    s->tick_in_flight = true;
    return GMAPP_OK;
}

extern "C" gmapp_status gmapp_server_poll(gmapp_server *s, int64_t ticket, gmapp_result *res) {
    if (!s || !res) {
        set_error("gmapp_server_poll: NULL argument");
        return GMAPP_ERR_INVALID_ARG;
    }
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        set_error("gmapp_server_poll: unknown ticket %lld", (long long)ticket);
        return GMAPP_ERR_INVALID_ARG;
    }
    ServerReq *q = it->second;
    if (q->state == ServerReq::SCORING && cudaEventQuery(s->slot_done[q->slot]) == cudaSuccess)
        retire(s, q);  // landed between ticks
    res->done = q->state == ServerReq::DONE;
    res->t_submit = q->t_submit;
    res->t_admit = q->t_admit;
    res->t_done = q->t_done;
    if (!res->done) return GMAPP_ERR_NOT_READY;
    res->best = q->best;
    res->best_cost = q->best >= 0 ? q->costs[q->best] : NAN;
    res->n_obs = q->n_obs;
    res->best_traj = q->traj.data();
    res->costs = q->costs.data();
    return GMAPP_OK;
}

extern "C" gmapp_status gmapp_server_release(gmapp_server *s, int64_t ticket) {
    if (!s) {
        set_error("gmapp_server_release: NULL server");
        return GMAPP_ERR_INVALID_ARG;
    }
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end() || it->second->state != ServerReq::DONE) {
        set_error("gmapp_server_release: ticket %lld is unknown or not done", (long long)ticket);
        return GMAPP_ERR_INVALID_ARG;
    }
    delete it->second;
    s->reqs.erase(it);
    return GMAPP_OK;
}

extern "C" gmapp_status gmapp_server_stats(gmapp_server *s, gmapp_server_stats_t *out) {
    if (!s || !out) {
        set_error("gmapp_server_stats: NULL argument");
        return GMAPP_ERR_INVALID_ARG;
    }
    int active = 0, pending = static_cast<int>(s->pending.size());
    for (auto &kv : s->reqs) active += kv.second->state == ServerReq::ACTIVE;
    out->active = active;
    out->pending = pending;
    out->completed = s->completed;
    out->arena_free_bytes = static_cast<int64_t>(s->arena.free_bytes());
    out->shard_cap = s->shard_cap;
    return GMAPP_OK;
}
