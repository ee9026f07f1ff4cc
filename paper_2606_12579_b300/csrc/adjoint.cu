// rollout_adjoint: gradient of each agent's plan cost with respect to its
// initial velocity v0, field gain k_r, attractive gain k_a and current
// vector c, by the discrete adjoint of the rollout (Sec. IV-A step map with
// the Alg. 1 obstacle sum, Eq. (mfi) force and the cost sums).
//
// Design (B300): the layout of the forward kernel (rollout_kernel.cuh) --
// groups of C CTAs, CTA r of a group keeps obstacle shard r resident in
// shared memory (TMA bulk copy), a group owns AG agents; NT compute warps
// evaluate obstacle pairs with packed f32x2 arithmetic and one exchange
// warp owns the agents.  The forward rollout stored the state (p_k, v_{k-1})
// every K steps.  Segments are processed from the last to the first: the
// group recomputes the segment's steps -- per pair the Alg. 1 term 1/s, its
// gradient -(1/s^2)(p - o)/|p - o| (gated-in, unclamped pairs) and the
// nearest obstacle -- with the two agent halves one phase apart, exactly as
// the forward kernel, so the per-step exchange of (W, grad W, min |d|^2,
// argmin) between the group's CTAs hides behind the other half's pair loop.
// Rank 0's exchange warp stores one record per agent and step in a global
// scratch buffer (L2-resident: N_a x K x 64 B) and, at the end of the
// segment, runs the reverse sweep over it while the compute warps already
// recompute the next segment.  Memory grows with K, not with N_k.
//
// The groups exchange through tagged words in global memory inside a
// cooperative grid (every CTA co-resident), and each group of CTAs works
// through agent groups q, q + G, q + 2G, ... so any N_a runs in one launch.
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "rollout_kernel.cuh"

namespace gmapp {
namespace {

constexpr int kAdjMaxAgents = 12;
constexpr int kRec = 16;   // floats per step record: p(3) v(3) W gW(3) m gm(3) pad(2)
constexpr int kAdjVals = 6;  // exchanged per agent: W, grad W (3), min |d|^2, argmin index
constexpr int kAdjThreads = 256;

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
    int32_t shard_cap;
    int32_t n_agent_groups;  // agent groups of AG (or fewer) agents
    int32_t group_ctas;      // C
    uint64_t *xbuf;
    uint32_t *xctl;
    uint32_t *err;
};

// (d, j) <- lexicographic minimum of (d, j) and (od, oj): the nearest
// obstacle, lowest index on ties.
__device__ __forceinline__ void argmin_merge(float &d, int &j, float od, int oj) {
    if (od < d || (od == d && oj < j)) {
        d = od;
        j = oj;
    }
}

// Transposed butterfly (see transposed_reduce) for (distance, index) pairs.
template <int P>
__device__ __forceinline__ void transposed_argmin(float (&d)[P], int (&j)[P], int lane) {
    constexpr int LG = log2i(P);
#pragma unroll
    for (int i = 0; i < LG; ++i) {
        const int L = 16 >> i;
        const int half = P >> (i + 1);
        const bool up = lane & L;
#pragma unroll
        for (int k = 0; k < half; ++k) {
            const float sd = up ? d[k] : d[k + half];
            const int sj = up ? j[k] : j[k + half];
            float kd = up ? d[k + half] : d[k];
            int kj = up ? j[k + half] : j[k];
            const float gd = __shfl_xor_sync(0xffffffffu, sd, L);
            const int gj = __shfl_xor_sync(0xffffffffu, sj, L);
            argmin_merge(kd, kj, gd, gj);
            d[k] = kd;
            j[k] = kj;
        }
    }
#pragma unroll
    for (int L = 16 >> LG; L >= 1; L >>= 1) {
        const float gd = __shfl_xor_sync(0xffffffffu, d[0], L);
        const int gj = __shfl_xor_sync(0xffffffffu, j[0], L);
        argmin_merge(d[0], j[0], gd, gj);
    }
}

// 0xFFFFFFFF when a <= b (resp. a > b), else 0 (0 for NaN): bit masks that
// select a value without multiplying it (a masked-out inf or NaN gives 0).
__device__ __forceinline__ uint32_t le_bits(float a, float b) {
    uint32_t r;
    asm("set.le.u32.f32 %0, %1, %2;" : "=r"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ uint32_t gt_bits(float a, float b) {
    uint32_t r;
    asm("set.gt.u32.f32 %0, %1, %2;" : "=r"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float and_bits(float v, uint32_t m) {
    return __uint_as_float(__float_as_uint(v) & m);
}

// The recompute terms of one obstacle pair (two f32x2 lanes, global indices
// jg, jg + 1) for NA agents: W += [gate] u, grad += [gate, unclamped]
// u^2/|d| (p - o) (negated later), nearest obstacle.  TAIL: the pair holds
// the shard's odd last obstacle twice and its hi lane counts for nothing.
// OPEN: every agent of the half is without a gate (r_d = inf) and the pair
// is a real obstacle, so every gate test passes and is not evaluated.
template <int NA, int NM, bool TAIL, bool ARGMIN = true, bool MASKD = false, bool OPEN = false>
__device__ __forceinline__ void adj_pair(f2 ox, f2 oy, f2 oz, int jg, const f2 (&X)[NA],
                                         const f2 (&Y)[NA], const f2 (&Z)[NA],
                                         const f2 (&nR2)[NA], const float (&G2)[NA], float eps,
                                         f2 one2, f2 (&W)[NA], f2 (&GX)[NA], f2 (&GY)[NA],
                                         f2 (&GZ)[NA], float (&bd)[NA], int (&bj)[NA]) {
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const f2 dx = sub2(X[a], ox), dy = sub2(Y[a], oy), dz = sub2(Z[a], oz);
        const f2 d2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
        const float d2l = lo_of(d2), d2h = hi_of(d2);
        const f2 r = pk(rsqrt_approx(d2l), rsqrt_approx(d2h));
        const f2 s = fma2(d2, r, nR2[a]);  // |d| - R (NaN when d = 0)
        const float s0l = lo_of(s), s0h = hi_of(s);
        const float sl = fmaxf(s0l, eps), sh = fmaxf(s0h, eps);
        // gate (s <= r_d, as |d|^2 <= (r_d + R)^2); gradient: gate AND unclamped
        const uint32_t gl = OPEN ? ~0u : le_bits(d2l, G2[a]);
        const uint32_t gh = TAIL ? 0u : OPEN ? ~0u : le_bits(d2h, G2[a]);
        const uint32_t ql = gl & gt_bits(s0l, eps), qh = gh & gt_bits(s0h, eps);
        f2 u;  // 1/s (SFU agents) or -1/s (Newton-Raphson agents)
        if (sfu_agent(a, NM, NA)) {
            u = pk(rcp_approx(sl), rcp_approx(sh));
        } else {
            u = neg_rcp2(pk(sl, sh), sl, sh, one2);
        }
        if (OPEN && !TAIL)
            W[a] = add2(W[a], u);
        else
            W[a] = add2(W[a], pk(and_bits(lo_of(u), gl), and_bits(hi_of(u), gh)));
        const f2 t = mul2(mul2(u, u), r);  // u^2 / |d|
        const f2 q = pk(and_bits(lo_of(t), ql), and_bits(hi_of(t), qh));
        if (MASKD) {
            // d masked like q: a NaN pad obstacle has a NaN direction, and a
            // zero weight times NaN would still be NaN
            GX[a] = fma2(q, pk(and_bits(lo_of(dx), ql), and_bits(hi_of(dx), qh)), GX[a]);
            GY[a] = fma2(q, pk(and_bits(lo_of(dy), ql), and_bits(hi_of(dy), qh)), GY[a]);
            GZ[a] = fma2(q, pk(and_bits(lo_of(dz), ql), and_bits(hi_of(dz), qh)), GZ[a]);
        } else {
            GX[a] = fma2(q, dx, GX[a]);
            GY[a] = fma2(q, dy, GY[a]);
            GZ[a] = fma2(q, dz, GZ[a]);
        }
        if (ARGMIN) {
            // ascending index per thread: strict < keeps the lowest (and the
            // lo lane on a tie within the pair)
            if (TAIL) {
                if (d2l < bd[a]) {
                    bd[a] = d2l;
                    bj[a] = jg;
                }
            } else {
                const float m = fminf(d2l, d2h);  // NaN lanes never win
                if (m < bd[a]) {
                    bj[a] = d2h < d2l ? jg + 1 : jg;
                    bd[a] = m;
                }
            }
        }
    }
}

// Block gate test of one packed pair (Alg. 1's branch, taken per warp for a
// block of 128 obstacles): the exact |d|^2 of each pair (as adj_pair forms
// it), the nearest obstacle, and whether a pair passes an agent's gate.
// Outside the gate adj_pair adds masked zeros (W, gradient), so evaluating
// it only for blocks with a pair inside leaves the sums unchanged.
template <int NA>
__device__ __forceinline__ bool adj_test(f2 ox, f2 oy, f2 oz, int jg, const f2 (&X)[NA],
                                         const f2 (&Y)[NA], const f2 (&Z)[NA],
                                         const float (&G2)[NA], float (&bd)[NA], int (&bj)[NA]) {
    bool hit = false;
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const f2 dx = sub2(X[a], ox), dy = sub2(Y[a], oy), dz = sub2(Z[a], oz);
        const f2 d2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
        const float d2l = lo_of(d2), d2h = hi_of(d2);
        const float m = fminf(d2l, d2h);  // NaN lanes never win
        hit |= m <= G2[a];
        if (m < bd[a]) {  // ascending index: strict < keeps the lowest (lo lane on a tie)
            bj[a] = d2h < d2l ? jg + 1 : jg;
            bd[a] = m;
        }
    }
    return hit;
}

// One half step of the recompute for NA agents (OFF .. OFF+NA-1 of the
// group), NM of them on the SFU reciprocal: this thread's obstacle pairs,
// then the warp's partials part[warp][OFF + a][8] = (W, gx, gy, gz, min d^2,
// argmin) stored by the representative lanes.
template <int AG, int NA, int OFF, int NM, int NT>
__device__ __forceinline__ void adj_half(const float *sx, const float *sy, const float *sz,
                                         int cnt, int32_t j0, float eps, const float *pos,
                                         const float *sR, const float *sG2, float *part_warp,
                                         int lane) {
    if constexpr (NA > 0) {
        constexpr int P = pow2ceil(NA);
        const int tid = threadIdx.x;
        f2 X[NA], Y[NA], Z[NA], nR2[NA], W[NA], GX[NA], GY[NA], GZ[NA];
        float G2[NA], bd[NA];
        int bj[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            const float x = pos[OFF + a], y = pos[AG + OFF + a], z = pos[2 * AG + OFF + a];
            X[a] = pk(x, x);
            Y[a] = pk(y, y);
            Z[a] = pk(z, z);
            const float r = sR[OFF + a];
            nR2[a] = pk(-r, -r);
            G2[a] = sG2[OFF + a];
            W[a] = GX[a] = GY[a] = GZ[a] = 0ull;
            bd[a] = INFINITY;
            bj[a] = INT_MAX;
        }
        const f2 one2 = pk(1.0f, 1.0f);
        // the shard is padded with NaN to whole blocks of 128 (a lane takes 4
        // consecutive obstacles, a warp a block); NaN pairs add nothing and
        // never become the nearest obstacle
        const int cnt_pad = (cnt + 127) & ~127;
        // an agent without a gate (r_d = inf) passes every block: then every
        // block's terms run without the test (and when no agent of the half
        // has a gate, without the gate masks)
        bool every = false, open = true;
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            every |= G2[a] == INFINITY;
            open &= G2[a] == INFINITY;
        }
        if (every) {
            // the real obstacles only (no NaN pads): pairs, then an odd last one
            const int cnt_even = cnt & ~1;
            if (open) {
#pragma unroll 2
                for (int j = 2 * tid; j < cnt_even; j += 2 * NT) {
                    const f2 ox = *reinterpret_cast<const f2 *>(sx + j);
                    const f2 oy = *reinterpret_cast<const f2 *>(sy + j);
                    const f2 oz = *reinterpret_cast<const f2 *>(sz + j);
                    adj_pair<NA, NM, false, true, false, true>(ox, oy, oz, j0 + j, X, Y, Z, nR2,
                                                               G2, eps, one2, W, GX, GY, GZ, bd,
                                                               bj);
                }
            } else {
#pragma unroll 2
                for (int j = 2 * tid; j < cnt_even; j += 2 * NT) {
                    const f2 ox = *reinterpret_cast<const f2 *>(sx + j);
                    const f2 oy = *reinterpret_cast<const f2 *>(sy + j);
                    const f2 oz = *reinterpret_cast<const f2 *>(sz + j);
                    adj_pair<NA, NM, false>(ox, oy, oz, j0 + j, X, Y, Z, nR2, G2, eps, one2, W,
                                            GX, GY, GZ, bd, bj);
                }
            }
            if ((cnt & 1) && tid == (cnt_even / 2) % NT) {
                const float x = sx[cnt_even], y = sy[cnt_even], z = sz[cnt_even];
                adj_pair<NA, NM, true>(pk(x, x), pk(y, y), pk(z, z), j0 + cnt_even, X, Y, Z, nR2,
                                       G2, eps, one2, W, GX, GY, GZ, bd, bj);
            }
        }
#pragma unroll 1
        for (int j = every ? cnt_pad : 4 * tid; j < cnt_pad; j += 4 * NT) {
            const float4 x4 = *reinterpret_cast<const float4 *>(sx + j);
            const float4 y4 = *reinterpret_cast<const float4 *>(sy + j);
            const float4 z4 = *reinterpret_cast<const float4 *>(sz + j);
            const f2 ox0 = pk(x4.x, x4.y), oy0 = pk(y4.x, y4.y), oz0 = pk(z4.x, z4.y);
            const f2 ox1 = pk(x4.z, x4.w), oy1 = pk(y4.z, y4.w), oz1 = pk(z4.z, z4.w);
            bool hit = adj_test<NA>(ox0, oy0, oz0, j0 + j, X, Y, Z, G2, bd, bj);
            hit |= adj_test<NA>(ox1, oy1, oz1, j0 + j + 2, X, Y, Z, G2, bd, bj);
            if (__any_sync(0xffffffffu, hit)) {
                // reloaded from shared memory: keeps the block's coordinates
                // out of registers across the test
                const float4 u4 = *reinterpret_cast<const float4 *>(sx + j);
                const float4 v4 = *reinterpret_cast<const float4 *>(sy + j);
                const float4 w4 = *reinterpret_cast<const float4 *>(sz + j);
                adj_pair<NA, NM, false, false, true>(pk(u4.x, u4.y), pk(v4.x, v4.y),
                                                     pk(w4.x, w4.y), j0 + j, X, Y, Z, nR2, G2,
                                                     eps, one2, W, GX, GY, GZ, bd, bj);
                adj_pair<NA, NM, false, false, true>(pk(u4.z, u4.w), pk(v4.z, v4.w),
                                                     pk(w4.z, w4.w), j0 + j + 2, X, Y, Z, nR2,
                                                     G2, eps, one2, W, GX, GY, GZ, bd, bj);
            }
        }
        float vw[P], vx[P], vy[P], vz[P], vd[P];
        int vj[P];
#pragma unroll
        for (int a = 0; a < P; ++a) {
            if (a < NA) {
                const float w = lo_of(W[a]) + hi_of(W[a]);
                vw[a] = sfu_agent(a, NM, NA) ? w : -w;
                // gradient of sum 1/s is -sum u^2 (p - o)/|p - o|
                vx[a] = -(lo_of(GX[a]) + hi_of(GX[a]));
                vy[a] = -(lo_of(GY[a]) + hi_of(GY[a]));
                vz[a] = -(lo_of(GZ[a]) + hi_of(GZ[a]));
                vd[a] = bd[a];
                vj[a] = bj[a];
            } else {
                vw[a] = vx[a] = vy[a] = vz[a] = 0.0f;
                vd[a] = INFINITY;
                vj[a] = INT_MAX;
            }
        }
        const float w = transposed_reduce<P, false>(vw, lane);
        const float gx = transposed_reduce<P, false>(vx, lane);
        const float gy = transposed_reduce<P, false>(vy, lane);
        const float gz = transposed_reduce<P, false>(vz, lane);
        transposed_argmin<P>(vd, vj, lane);
        constexpr int REP = (32 >> log2i(P)) - 1;
        const int idx = transposed_index<P>(lane);
        if ((lane & REP) == 0 && idx < NA) {
            float *dst = part_warp + 8 * (OFF + idx);
            *reinterpret_cast<float4 *>(dst) = make_float4(w, gx, gy, gz);
            *reinterpret_cast<float2 *>(dst + 4) = make_float2(vd[0], __int_as_float(vj[0]));
        }
    }
}

// Exchange of one half between the C CTAs of the group (exchange warp): sum
// the NW warp partials in warp order, post the CTA's six values per agent
// as tagged words, poll the C x NA x 6 words of the half (bounded; spread
// over the lanes), stage them in shared memory and combine in rank order.
// Lane OFF + a receives agent a's totals.
template <int AG, int NA, int OFF, int NW>
__device__ __forceinline__ bool adj_exchange(const float *part, uint64_t *xs, float *slot,
                                             uint32_t C, uint32_t rank, int lane, uint32_t tag,
                                             bool ok, float (&tot)[kAdjVals]) {
    if (lane < NA) {
        float v[4] = {0, 0, 0, 0}, d = INFINITY;
        int jj = INT_MAX;
        for (int q = 0; q < NW; ++q) {
            const float *src = part + 8 * (q * AG + OFF + lane);
            const float4 t = *reinterpret_cast<const float4 *>(src);
            const float2 u = *reinterpret_cast<const float2 *>(src + 4);
            v[0] += t.x;
            v[1] += t.y;
            v[2] += t.z;
            v[3] += t.w;
            argmin_merge(d, jj, u.x, __float_as_int(u.y));
        }
        uint64_t *dst = xs + kAdjVals * (rank * AG + OFF + lane);
        st_relaxed_u64(dst + 0, xword(tag, v[0]));
        st_relaxed_u64(dst + 1, xword(tag, v[1]));
        st_relaxed_u64(dst + 2, xword(tag, v[2]));
        st_relaxed_u64(dst + 3, xword(tag, v[3]));
        st_relaxed_u64(dst + 4, xword(tag, d));
        st_relaxed_u64(dst + 5, xword(tag, __int_as_float(jj)));
    }
    const int nwords = static_cast<int>(C) * NA * kAdjVals;
    constexpr int kPer = NA > 0 ? NA * kAdjVals : 1;
    for (int p = lane; p < nwords; p += 32) {
        const int r = p / kPer, rem = p % kPer;
        const int a = OFF + rem / kAdjVals, e = rem % kAdjVals;
        const uint64_t *src = xs + kAdjVals * (r * AG + a) + e;
        uint64_t v = ld_relaxed_u64(src);
        for (uint32_t it = 0; ok && static_cast<uint32_t>(v >> 32) != tag; ++it) {
            if (it == kPollLimit) ok = false;
            else v = ld_relaxed_u64(src);
        }
        slot[kAdjVals * (r * AG + a) + e] = __uint_as_float(static_cast<uint32_t>(v));
    }
    __syncwarp();
    if (lane >= OFF && lane < OFF + NA) {
        float v[4] = {0, 0, 0, 0}, d = INFINITY;
        int jj = INT_MAX;
        for (uint32_t r = 0; r < C; ++r) {
            const float *src = slot + kAdjVals * (r * AG + lane);
#pragma unroll
            for (int e = 0; e < 4; ++e) v[e] += src[e];
            argmin_merge(d, jj, src[4], __float_as_int(src[5]));
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) tot[e] = v[e];
        tot[4] = d;
        tot[5] = __int_as_float(jj);
    }
    __syncwarp();
    return ok;
}

// g(v, c) = |v| c - (v.c) v/|v| (0 when |v|^2 < 1e-30).
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
__global__ void __launch_bounds__(NT + 32, 1) k_adjoint(const AdjArgs A) {
    constexpr int NW = NT / 32;
    constexpr int H0 = (AG + 1) / 2, H1 = AG - H0;
    // every agent on the SFU reciprocal: the gradient terms add FMA-pipe
    // work to each pair while the SFU has room (dense 50k x 512 x 1000:
    // 23.5 ms against 24.7 ms with the forward kernel's split)
    constexpr int NM = AG;
    constexpr int NM0 = (NM + 1) / 2 < H0 ? (NM + 1) / 2 : H0;
    constexpr int NM1 = NM - NM0 < H1 ? NM - NM0 : H1;
    constexpr int kPart = 1, kPos = 3, kBoth = NT + 32;
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bar_tma;
    __shared__ __align__(16) float part[2][NW][AG][8];
    __shared__ __align__(16) float slot[2][kMaxCluster * AG * kAdjVals];
    __shared__ __align__(16) float pos[3 * AG];
    __shared__ float sR[AG], sG2[AG];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool exch = warp == NW;
    const uint32_t C = static_cast<uint32_t>(A.group_ctas);
    const uint32_t rank = blockIdx.x % C, group = blockIdx.x / C;
    const uint32_t G = gridDim.x / C;
    const int32_t n_obs = *A.n_obs;
    const int32_t shard_len = ((n_obs + (int32_t)C - 1) / (int32_t)C + 3) & ~3;
    auto finish_grid = [&](uint32_t epoch) {
        if (atomicAdd(A.xctl + 1, 1u) == gridDim.x - 1) {
            A.xctl[1] = 0;
            const uint32_t next = (epoch + 1) & 0x3fffffffu;
            A.xctl[0] = next ? next : 1u;
        }
    };
    if (n_obs < 0 || n_obs > A.cap || shard_len > A.shard_cap || (A.shard_cap & 127)) {
        if (tid == 0 && rank == 0 && group == 0) raise_error(A.err, GMAPP_DEVERR_CAPACITY);
        if (tid == NT) finish_grid(ld_relaxed_u32(A.xctl));
        return;
    }
    const int32_t start = static_cast<int32_t>(rank) * shard_len;
    int32_t cnt = min(shard_len, max(0, n_obs - start));
    float *sx = smem, *sy = smem + A.shard_cap, *sz = smem + 2 * A.shard_cap;
    if (tid == 0) {
        mbar_init(&bar_tma, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (cnt > 0 && tid == 0) {
        const uint32_t bytes = static_cast<uint32_t>((cnt + 3) & ~3) * 4u;
        mbar_arrive_expect_tx(&bar_tma, 3 * bytes);
        bulk_g2s(sx, A.ox + start, bytes, &bar_tma);
        bulk_g2s(sy, A.oy + start, bytes, &bar_tma);
        bulk_g2s(sz, A.oz + start, bytes, &bar_tma);
    }
    if (cnt > 0 && !mbar_wait(&bar_tma, 0)) {
        if (tid == 0) raise_error(A.err, GMAPP_DEVERR_TIMEOUT);
        cnt = 0;
    }
    // pad the shard to whole blocks of 128 with NaN (shard_cap is a multiple
    // of 128)
    for (int32_t i = cnt + tid; i < ((cnt + 127) & ~127); i += blockDim.x) {
        sx[i] = __int_as_float(0x7fc00000);
        sy[i] = __int_as_float(0x7fc00000);
        sz[i] = __int_as_float(0x7fc00000);
    }
    __syncthreads();
    const float eps = A.eps;
    const int N = A.n_steps, K = A.K, nseg = (N + K - 1) / K;
    const int n = A.n_agents;
    const uint32_t epoch = ld_relaxed_u32(A.xctl);
    uint64_t *xg = A.xbuf + static_cast<size_t>(group) * 4 * kAdjVals * C * AG;
    auto xslot = [&](int h, int par) { return xg + (h * 2 + par) * kAdjVals * C * AG; };
    const float h = A.vel_half * A.dt * A.inv_mass;
    bool ok = true;
    int tglob = 0;  // steps taken by this group in this launch (for the tags)

    for (int q = static_cast<int>(group); q < A.n_agent_groups; q += static_cast<int>(G)) {
        int a0, na;
        group_range(q, n, A.n_agent_groups, a0, na);
        const int i = a0 + lane;
        // agent constants and the first segment's checkpoint (exchange warp)
        float cc[3] = {0, 0, 0}, p[3] = {0, 0, 0}, v[3] = {0, 0, 0};
        float k_r = 0, k_a = 0, R = 0;
        float L = 0, pen = 0, minc = INFINITY, dgoal = 0;
        float ap[3] = {0, 0, 0}, av[3] = {0, 0, 0}, dc[3] = {0, 0, 0}, dkr = 0, dka = 0;
        float pe[3] = {0, 0, 0}, ve[3] = {0, 0, 0};  // state at the end of the segment
        auto load_ckpt = [&](int seg) {
            if (lane < na) {
                const float *ck = A.ckpt + (size_t)seg * 6 * n + i;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    p[d] = ck[d * n];
                    v[d] = ck[(3 + d) * n];
                }
            } else {
                p[0] = p[1] = p[2] = v[0] = v[1] = v[2] = 0.0f;
            }
        };
        if (exch) {
            if (lane < na) {
#pragma unroll
                for (int d = 0; d < 3; ++d) cc[d] = A.c[d * n + i];
                k_r = A.k_r[i];
                k_a = A.k_a[i];
                R = A.r_a[i] + A.r_O;
            }
            if (lane < AG) {
                const float rd = lane < na ? A.r_d[i] : -1.0f;
                sR[lane] = R;
                // s = max(d - R, eps) <= r_d  <=>  d^2 <= (r_d + R)^2 when r_d >= eps
                sG2[lane] = (lane < na && rd >= eps) ? (rd + R) * (rd + R) : -1.0f;
            }
            load_ckpt(nseg - 1);
            if (lane < AG) {
                pos[lane] = p[0];
                pos[AG + lane] = p[1];
                pos[2 * AG + lane] = p[2];
            }
        }
        __syncthreads();

        if (!exch) {
            for (int t = 0; t < N; ++t) {
                if (t > 0) named_sync(kPos + 0, kBoth);
                adj_half<AG, H0, 0, NM0, NT>(sx, sy, sz, cnt, start, eps, pos, sR, sG2,
                                             &part[0][warp][0][0], lane);
                named_arrive(kPart + 0, kBoth);
                if (t > 0) named_sync(kPos + 1, kBoth);
                adj_half<AG, H1, H0, NM1, NT>(sx, sy, sz, cnt, start, eps, pos, sR, sG2,
                                              &part[1][warp][0][0], lane);
                named_arrive(kPart + 1, kBoth);
            }
        } else {
            // one exchange + integration of one half at recompute step k of
            // segment seg; returns after publishing the half's next positions
            auto half_step_x = [&](auto hc, int seg, int k, int t) {
                constexpr int HH = decltype(hc)::value;
                constexpr int OFF = HH == 0 ? 0 : H0, NA = HH == 0 ? H0 : H1;
                const int par = (tglob + t) & 1;
                float tot[kAdjVals] = {0, 0, 0, 0, INFINITY, 0};
                named_sync(kPart + HH, kBoth);
                ok = adj_exchange<AG, NA, OFF, NW>(&part[HH][0][0][0], xslot(HH, par), slot[HH],
                                                   C, rank, lane, xtag(epoch, tglob + t), ok, tot);
                if (lane >= OFF && lane < OFF + NA && lane < na) {
                    const int k0 = seg * K;
                    const float md2 = tot[4];
                    const int jj = __float_as_int(tot[5]);
                    float gm[3] = {0, 0, 0};
                    const float dist = sqrtf(md2);
                    if (jj != INT_MAX && dist > 0.0f) {
                        const float inv = 1.0f / dist;
                        gm[0] = (p[0] - A.ox[jj]) * inv;
                        gm[1] = (p[1] - A.oy[jj]) * inv;
                        gm[2] = (p[2] - A.oz[jj]) * inv;
                    }
                    if (rank == 0) {
                        float *rc = A.rec + ((size_t)i * K + (k - k0)) * kRec;
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            rc[d] = p[d];
                            rc[3 + d] = v[d];
                            rc[7 + d] = tot[1 + d];
                            rc[11 + d] = gm[d];
                        }
                        rc[6] = tot[0];
                    }
                    float g[3], kf, m;
                    agent_step<true>(p, v, cc, k_r, k_a, R, A.goal, h, A.dt, A.rho, A.damping,
                                     A.clear_margin, A.clear_beta, tot[0], md2, L, pen, minc, m,
                                     g, kf);
                    if (rank == 0) A.rec[((size_t)i * K + (k - k0)) * kRec + 10] = m;
                }
                const bool seg_end = k == min(N, (seg + 1) * K) - 1;
                if (seg_end && lane >= OFF && lane < OFF + NA) {
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        pe[d] = p[d];
                        ve[d] = v[d];
                    }
                    if (seg > 0) load_ckpt(seg - 1);
                }
                if (lane >= OFF && lane < OFF + NA) {
                    pos[lane] = p[0];
                    pos[AG + lane] = p[1];
                    pos[2 * AG + lane] = p[2];
                }
                __syncwarp();
                if (t + 1 < N) named_arrive(kPos + HH, kBoth);
            };
            int t = 0;
            for (int seg = nseg - 1; seg >= 0; --seg) {
                const int k0 = seg * K, k1 = min(N, k0 + K);
                for (int k = k0; k < k1; ++k, ++t) {
                    half_step_x(std::integral_constant<int, 0>{}, seg, k, t);
                    half_step_x(std::integral_constant<int, 1>{}, seg, k, t);
                }
                // ---- reverse sweep over the segment (rank 0) ----------------
                if (rank == 0 && lane < na) {
                    if (seg == nseg - 1) {
                        const float e0 = pe[0] - A.goal[0], e1 = pe[1] - A.goal[1],
                                    e2 = pe[2] - A.goal[2];
                        dgoal = sqrtf(fmaf(e2, e2, fmaf(e1, e1, e0 * e0)));
                        if (dgoal > 0.0f) {
                            ap[0] = A.w_goal * e0 / dgoal;
                            ap[1] = A.w_goal * e1 / dgoal;
                            ap[2] = A.w_goal * e2 / dgoal;
                        }
                    }
                    float vn[3] = {ve[0], ve[1], ve[2]};  // v_k, the velocity after step k
                    for (int k = k1 - 1; k >= k0; --k) {
                        const float *rc = A.rec + ((size_t)i * K + (k - k0)) * kRec;
                        const float pk_[3] = {rc[0], rc[1], rc[2]};
                        const float vk[3] = {rc[3], rc[4], rc[5]};  // v_{k-1}
                        const float Wk = rc[6], mk = rc[10];
                        const float gW[3] = {rc[7], rc[8], rc[9]};
                        const float gm[3] = {rc[11], rc[12], rc[13]};
                        const float ln =
                            sqrtf(fmaf(vn[2], vn[2], fmaf(vn[1], vn[1], vn[0] * vn[0])));
                        float avk[3], Fb[3];
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            const float eq = ln > 0.0f ? vn[d] / ln : 0.0f;
                            avk[d] = av[d] + A.dt * (ap[d] + A.w_path * eq);
                            Fb[d] = h * avk[d];
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
                            for (int d = 0; d < 3; ++d) {
                                JgF[d] = u[d] * cF - cc[d] * uF - (vc / nrm) * (Fb[d] - u[d] * uF);
                                JcF[d] = nrm * Fb[d] - vk[d] * uF;
                            }
                        }
                        const float sg =
                            1.0f / (1.0f + expf(-A.clear_beta * (A.clear_margin - mk)));
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            av[d] = avk[d] - A.damping * Fb[d] + A.rho * k_r * Wk * JgF[d];
                            ap[d] += -k_a * Fb[d] + A.rho * k_r * gF * gW[d] - A.w_clear * sg * gm[d];
                            dka += Fb[d] * (A.goal[d] - pk_[d]);
                            dc[d] += A.rho * k_r * Wk * JcF[d];
                            vn[d] = vk[d];
                        }
                        dkr += A.rho * Wk * gF;
                    }
                }
                __syncwarp();
            }
            if (rank == 0 && lane < na) {
                const float sc = A.grad_cost ? A.grad_cost[i] : 1.0f;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    A.g_v0[d * n + i] = sc * av[d];
                    A.g_c[d * n + i] = sc * dc[d];
                }
                A.g_kr[i] = sc * dkr;
                A.g_ka[i] = sc * dka;
                if (A.cost) A.cost[i] = A.w_path * L + A.w_goal * dgoal + A.w_clear * pen;
            }
        }
        tglob += N;
        __syncthreads();  // pos, sR, sG2 of the next agent group
    }
    if (exch) {
        if (!ok) raise_error(A.err, GMAPP_DEVERR_TIMEOUT);
        if (lane == 0) finish_grid(epoch);
    }
}

using AdjKernel = void (*)(const AdjArgs);

AdjKernel adj_kernel(int ag) {
    switch (ag) {
        case 1: return k_adjoint<1, kAdjThreads>;
        case 2: return k_adjoint<2, kAdjThreads>;
        case 3: return k_adjoint<3, kAdjThreads>;
        case 4: return k_adjoint<4, kAdjThreads>;
        case 5: return k_adjoint<5, kAdjThreads>;
        case 6: return k_adjoint<6, kAdjThreads>;
        case 7: return k_adjoint<7, kAdjThreads>;
        case 8: return k_adjoint<8, kAdjThreads>;
        case 9: return k_adjoint<9, kAdjThreads>;
        case 10: return k_adjoint<10, kAdjThreads>;
        case 11: return k_adjoint<11, kAdjThreads>;
        case 12: return k_adjoint<12, kAdjThreads>;
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
    // launch shape: the smallest group of CTAs whose shards fit shared
    // memory; as many groups as fit on the SMs (one CTA per SM); the agents
    // per group that spread N_a evenly over them (groups loop when N_a needs
    // more than kAdjMaxAgents per group)
    AdjKernel fn = nullptr;
    int C = 0, agp = 1, G = 0;
    size_t dyn = 0;
    for (int c = 1; c <= kMaxCluster && !fn; ++c) {
        const int64_t shard = ((obs->cap + c - 1) / c + 127) & ~int64_t(127);
        const size_t bytes = static_cast<size_t>(shard) * 3 * sizeof(float);
        cudaFuncAttributes fa;
        GMAPP_CHECK_CUDA(cudaFuncGetAttributes(
            &fa, reinterpret_cast<const void *>(adj_kernel(kAdjMaxAgents))));
        if (bytes + fa.sharedSizeBytes > static_cast<size_t>(ctx->max_smem_optin)) continue;
        const int groups = ctx->sm_count / c;
        if (groups < 1) break;
        C = c;
        dyn = bytes;
        G = groups;
        agp = std::min(kAdjMaxAgents, (ag->n + G - 1) / G);
        fn = adj_kernel(agp);
    }
    if (!fn) {
        set_error("rollout_adjoint: an obstacle capacity of %lld does not fit any group of CTAs",
                  (long long)obs->cap);
        return GMAPP_ERR_CAPACITY;
    }
    const int n_agent_groups = (ag->n + agp - 1) / agp;
    G = std::min(G, n_agent_groups);
    GMAPP_CHECK_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void *>(fn),
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          static_cast<int>(dyn)));
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
    // a multiple of 128: the recompute loop tests whole blocks of 128 obstacles
    A.shard_cap = static_cast<int32_t>(((obs->cap + C - 1) / C + 127) & ~int64_t(127));
    A.n_agent_groups = n_agent_groups;
    A.group_ctas = C;
    A.xbuf = ctx->d_xbuf;
    A.xctl = ctx->d_xctl;
    A.err = ctx->d_err;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G * C, 1, 1);
    cfg.blockDim = dim3(kAdjThreads + 32, 1, 1);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = stream;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeCooperative;
    attr.val.cooperative = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    bool capturing = false;
    gmapp_status st = grid_exchange_begin(ctx, stream, &capturing);
    if (st != GMAPP_OK) return st;
    GMAPP_CHECK_CUDA(cudaLaunchKernelEx(&cfg, fn, A));
    return grid_exchange_end(ctx, stream, capturing);
}
