// The rollout kernel template (Sec. IV-A agent dynamics, Eq. (mfi)
// circular-field force, Alg. 1 clamp, gate and obstacle sum).
//
// Layout of the work: a thread-block cluster of C CTAs owns a group of up to
// AG agents for the whole rollout; CTA r keeps obstacle shard r of S_W in
// shared memory (SoA float32, loaded once by the TMA bulk-copy engine, padded
// with NaN, which contributes exactly nothing).  Each thread walks pairs of
// obstacles of its shard against all AG agents of the group:
//
//   packed f32x2 arithmetic over the obstacle pair (one instruction, two
//   lanes of work): differences, |d|^2, s = |d| - R;
//   |d|^-1/2 on the SFU (rsqrt), clamp max(s, eps), detection gate as a
//   0/1 mask from |d|^2 <= (r_d + R)^2 folded into the accumulation FMA;
//   1/s on the SFU for the first NM agents and by a magic-constant seed plus
//   three Newton-Raphson steps on the FMA pipe for the others (Blinn,
//   "Floating-point tricks", IEEE CG&A 1997; the iteration runs on -1/s so it
//   needs no negation), which balances the SFU against the FMA pipe.
//
// The agents of a group are split into two halves that are kept one phase
// apart: each warp reduces a half's partial sums with a transposed shuffle
// butterfly and stores them, over DSMEM, into the double-buffered receive
// slots of every CTA of the cluster, then arrives on the cluster barrier and
// computes the other half while the first is in flight; after the wait,
// every warp sums the C x NW partials of the half in a fixed order (lanes
// in parallel) and integrates those agents itself (lane a = agent a), so
// results are bit-identical in every warp and CTA and no other barrier is
// needed.  Nothing inside the N_k loop touches global memory except the
// optional trajectory/trace stores.
#pragma once

#include <math.h>

#include "gmapp_internal.cuh"

namespace gmapp {

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
    int32_t shard_cap;   // obstacles one CTA can hold (multiple of 4)
    int32_t n_groups;    // clusters in the grid
    int32_t recv_floats; // size of one parity of the receive buffer
    uint32_t *err;
};

// ---- packed f32x2 helpers (two FP32 lanes in one 64-bit register) ----------
using f2 = unsigned long long;

__device__ __forceinline__ f2 pk(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float lo_of(f2 v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return a;
}
__device__ __forceinline__ float hi_of(f2 v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return b;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
// 1.0f when a <= b, else 0.0f (0.0f for NaN).
__device__ __forceinline__ float le_mask(float a, float b) {
    float r;
    asm("set.le.f32.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
// Seed of -1/s for s > 0 (bit pattern of -(0x7EF311C3 - bits(s)) = y0 with
// the sign bit set); relative error <= 5.1%.
__device__ __forceinline__ float neg_rcp_seed(float s) {
    return __int_as_float(static_cast<int>(0xFEF311C3u - static_cast<uint32_t>(__float_as_int(s))));
}

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
__device__ __forceinline__ float softplus_f(float x, float beta) {
    float bx = beta * x;
    float r = bx > 0.0f ? bx + log1pf(expf(-bx)) : log1pf(expf(bx));
    return r / beta;
}

// One step of Sec. IV-A for one agent, given the Alg. 1 sum W and the
// smallest squared obstacle distance md2:
//   g  = (|v|^2 c - v (v.c)) / |v|   (0 when |v|^2 < 1e-30), v = v_{k-1}
//   F  = k_a (goal - p) - D v + rho k_r W g;  v += h F (h = 1/2 dt inv_mass)
//   p += dt v;  L += dt |v|;  with CLEAR: m = sqrt(md2) - R,
//   pen += softplus_beta(margin - m), minc = min(minc, m).
// Returns g, the field strength kf = rho k_r W and m (inf without CLEAR).
template <bool CLEAR>
__device__ __forceinline__ void agent_step(float (&p)[3], float (&v)[3], const float (&cc)[3],
                                           float k_r, float k_a, float R, const float (&goal)[3],
                                           float h, float dt, float rho, float damping,
                                           float clear_margin, float clear_beta, float W,
                                           float md2, float &L, float &pen, float &minc,
                                           float &m, float (&g)[3], float &kf) {
    g[0] = g[1] = g[2] = 0.0f;
    const float vv = fmaf(v[2], v[2], fmaf(v[1], v[1], v[0] * v[0]));
    if (vv >= 1e-30f) {
        const float inv = rsqrt_approx(vv);  // SFU; ~2^-22 relative error
        const float vc = fmaf(v[2], cc[2], fmaf(v[1], cc[1], v[0] * cc[0]));
#pragma unroll
        for (int d = 0; d < 3; ++d) g[d] = (vv * cc[d] - v[d] * vc) * inv;
    }
    kf = rho * k_r * W;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float F = k_a * (goal[d] - p[d]) - damping * v[d] + kf * g[d];
        v[d] = fmaf(h, F, v[d]);
    }
    const float vn = fmaf(v[2], v[2], fmaf(v[1], v[1], v[0] * v[0]));
    L = fmaf(dt, vn > 0.0f ? vn * rsqrt_approx(vn) : 0.0f, L);  // dt |v_k|
#pragma unroll
    for (int d = 0; d < 3; ++d) p[d] = fmaf(dt, v[d], p[d]);
    m = INFINITY;
    if (CLEAR) {
        m = sqrtf(md2) - R;
        pen += softplus_f(clear_margin - m, clear_beta);
        minc = fminf(minc, m);
    }
}

// Agent range of cluster q: groups get floor or ceil of N_a / G agents.
__device__ __forceinline__ void group_range(int q, int n_agents, int n_groups, int &a0, int &na) {
    const int base = n_agents / n_groups, rem = n_agents % n_groups;
    a0 = q * base + min(q, rem);
    na = base + (q < rem ? 1 : 0);
}

constexpr int pow2ceil(int x) { return x <= 1 ? 1 : 2 * pow2ceil((x + 1) / 2); }
constexpr int log2i(int x) { return x <= 1 ? 0 : 1 + log2i(x / 2); }

// Transposed butterfly over the warp: P values per lane in, one value per
// lane out -- the sum (or min) over all 32 lanes of value index idx(lane),
// idx taken from lane bits 4, 3, ... (P - 1 + 5 - log2 P shuffles instead
// of 5 P).  Lanes whose low 5 - log2 P bits are zero are the representatives.
template <int P, bool MIN>
__device__ __forceinline__ float transposed_reduce(float (&v)[P], int lane) {
    constexpr int LG = log2i(P);
#pragma unroll
    for (int i = 0; i < LG; ++i) {
        const int L = 16 >> i;
        const int half = P >> (i + 1);
        const bool up = lane & L;
#pragma unroll
        for (int j = 0; j < half; ++j) {
            const float send = up ? v[j] : v[j + half];
            const float keep = up ? v[j + half] : v[j];
            const float got = __shfl_xor_sync(0xffffffffu, send, L);
            v[j] = MIN ? fminf(keep, got) : keep + got;
        }
    }
#pragma unroll
    for (int L = 16 >> LG; L >= 1; L >>= 1) {
        const float got = __shfl_xor_sync(0xffffffffu, v[0], L);
        v[0] = MIN ? fminf(v[0], got) : v[0] + got;
    }
    return v[0];
}

template <int P>
__device__ __forceinline__ int transposed_index(int lane) {
    constexpr int LG = log2i(P);
    int idx = 0;
#pragma unroll
    for (int i = 0; i < LG; ++i) idx |= ((lane >> (4 - i)) & 1) << (LG - 1 - i);
    return idx;
}

// Partial Alg. 1 sums of this thread's obstacle pairs for NA agents
// (agent indices OFF .. OFF+NA-1 of the group), reduced over the warp and
// stored into every cluster CTA's receive slots recv[h][par][rank][warp][a].
// The Alg. 1 terms of one obstacle pair (two f32x2 lanes) for NA agents,
// accumulated into acc (and the squared-distance minimum mn with CLEAR).
template <int AG, int NA, int OFF, int NM, bool CLEAR>
__device__ __forceinline__ void pair_terms(f2 ox, f2 oy, f2 oz, const f2 (&X)[NA],
                                           const f2 (&Y)[NA], const f2 (&Z)[NA], f2 (&acc)[NA],
                                           float (&mn)[NA], const f2 (&nR2)[AG],
                                           const float (&G2a)[AG], float eps, f2 one2) {
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const f2 dx = sub2(X[a], ox), dy = sub2(Y[a], oy), dz = sub2(Z[a], oz);
        const f2 d2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
        const float d2l = lo_of(d2), d2h = hi_of(d2);
        const f2 mask = pk(le_mask(d2l, G2a[OFF + a]), le_mask(d2h, G2a[OFF + a]));
        const f2 r = pk(rsqrt_approx(d2l), rsqrt_approx(d2h));
        const f2 s = fma2(d2, r, nR2[OFF + a]);  // |d| - R (NaN when d = 0)
        const float sl = fmaxf(lo_of(s), eps), sh = fmaxf(hi_of(s), eps);
        if (a < NM) {
            acc[a] = fma2(mask, pk(rcp_approx(sl), rcp_approx(sh)), acc[a]);
        } else {
            const f2 s2 = pk(sl, sh);
            f2 y = pk(neg_rcp_seed(sl), neg_rcp_seed(sh));
#pragma unroll
            for (int it = 0; it < 3; ++it) y = fma2(y, fma2(s2, y, one2), y);
            acc[a] = fma2(mask, y, acc[a]);
        }
        if (CLEAR) mn[a] = fminf(mn[a], fminf(d2l, d2h));
    }
}

// Obstacles beyond what shared memory holds, read from global memory
// (L2-resident): indices [begin, end) of the obstacle arrays.
struct GlobalTail {
    const float *x, *y, *z;
    int begin, end;
};

template <int AG, int NA, int OFF, int NM, int NT, bool CLEAR, bool TAIL = false,
          bool SHIP = true>
__device__ __forceinline__ void half_step(const float *sx, const float *sy, const float *sz,
                                          int cnt_pad, float eps, const f2 (&nR2)[AG],
                                          const float (&G2a)[AG], const float (&p)[3],
                                          float *recv_slot0, uint32_t C, int lane,
                                          GlobalTail tail = GlobalTail{}) {
    if constexpr (NA > 0) {
        constexpr int P = pow2ceil(NA);
        const int tid = threadIdx.x;
        f2 X[NA], Y[NA], Z[NA], acc[NA];
        float mn[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            const float x = __shfl_sync(0xffffffffu, p[0], OFF + a);
            const float y = __shfl_sync(0xffffffffu, p[1], OFF + a);
            const float z = __shfl_sync(0xffffffffu, p[2], OFF + a);
            X[a] = pk(x, x);
            Y[a] = pk(y, y);
            Z[a] = pk(z, z);
            acc[a] = 0ull;
            mn[a] = INFINITY;
        }
        const f2 one2 = pk(1.0f, 1.0f);
#pragma unroll 2
        for (int j = 2 * tid; j < cnt_pad; j += 2 * NT) {
            const f2 ox = *reinterpret_cast<const f2 *>(sx + j);
            const f2 oy = *reinterpret_cast<const f2 *>(sy + j);
            const f2 oz = *reinterpret_cast<const f2 *>(sz + j);
            pair_terms<AG, NA, OFF, NM, CLEAR>(ox, oy, oz, X, Y, Z, acc, mn, nR2, G2a, eps, one2);
        }
        if constexpr (TAIL) {
            // tail.begin is even; an odd last obstacle is paired with NaN
            for (int j = tail.begin + 2 * tid; j < tail.end; j += 2 * NT) {
                f2 ox = __ldg(reinterpret_cast<const f2 *>(tail.x + j));
                f2 oy = __ldg(reinterpret_cast<const f2 *>(tail.y + j));
                f2 oz = __ldg(reinterpret_cast<const f2 *>(tail.z + j));
                if (j + 1 >= tail.end) {
                    const float nan = __int_as_float(0x7fc00000);
                    ox = pk(lo_of(ox), nan);
                    oy = pk(lo_of(oy), nan);
                    oz = pk(lo_of(oz), nan);
                }
                pair_terms<AG, NA, OFF, NM, CLEAR>(ox, oy, oz, X, Y, Z, acc, mn, nR2, G2a, eps,
                                                   one2);
            }
        }
        float vw[P], vm[P];
#pragma unroll
        for (int a = 0; a < P; ++a) {
            if (a < NA) {
                const float w = lo_of(acc[a]) + hi_of(acc[a]);
                vw[a] = a < NM ? w : -w;
                vm[a] = mn[a];
            } else {
                vw[a] = 0.0f;
                vm[a] = INFINITY;
            }
        }
        const float w = transposed_reduce<P, false>(vw, lane);
        const float m = CLEAR ? transposed_reduce<P, true>(vm, lane) : INFINITY;
        constexpr int REP = (32 >> log2i(P)) - 1;
        const int idx = transposed_index<P>(lane);
        if ((lane & REP) == 0 && idx < NA) {
            if constexpr (SHIP) {
                const uint32_t local = smem_u32(recv_slot0 + 2 * (OFF + idx));
                for (uint32_t r = 0; r < C; ++r) st_cluster_v2f32(map_smem(local, r), w, m);
            } else {
                *reinterpret_cast<float2 *>(recv_slot0 + 2 * (OFF + idx)) = make_float2(w, m);
            }
        }
    }
}

__device__ __forceinline__ void named_barrier(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// CTA-level reduction of a half's per-warp partials part[NW][AG] (float2),
// one warp per agent (lane l loads warp l's partial, fixed shuffle tree),
// then lane 0 stores the CTA's partial into slot[rank][a] of every CTA of
// the cluster.  Call after a barrier that covers all partial stores.
template <int AG, int NA, int OFF, int NW, bool CLEAR>
__device__ __forceinline__ void cta_ship(const float *part, float *slot, uint32_t C,
                                         uint32_t rank, int warp, int lane) {
    for (int a = warp; a < NA; a += NW) {
        float w = 0.0f, m = INFINITY;
        if (lane < NW) {
            const float2 t = *reinterpret_cast<const float2 *>(part + 2 * (lane * AG + OFF + a));
            w = t.x;
            m = t.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            w += __shfl_xor_sync(0xffffffffu, w, o);
            if (CLEAR) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
        }
        if (lane == 0) {
            const uint32_t local = smem_u32(slot + 2 * (rank * AG + OFF + a));
            for (uint32_t r = 0; r < C; ++r) st_cluster_v2f32(map_smem(local, r), w, m);
        }
    }
}

// Sum (min) of the C per-CTA partials of agent `lane` in rank order.
template <int AG, bool CLEAR>
__device__ __forceinline__ void cluster_combine(const float *slot, uint32_t C, int lane, float &W,
                                                float &md2) {
    float w = 0.0f, m = INFINITY;
    for (uint32_t r = 0; r < C; ++r) {
        const float2 t = *reinterpret_cast<const float2 *>(slot + 2 * (r * AG + lane));
        w += t.x;
        if (CLEAR) m = fminf(m, t.y);
    }
    W = w;
    md2 = m;
}

// Sum of the C x NW partials of each agent of a half, in a fixed order;
// lanes OFF .. OFF+NA-1 receive the totals of their own agent.
template <int AG, int NA, int OFF, bool CLEAR>
__device__ __forceinline__ void half_combine(const float *recv_par, int nq, int lane, float &W,
                                             float &md2) {
    if constexpr (NA > 0) {
        constexpr int P = pow2ceil(NA);
        constexpr int G = 32 / P;
        const int a = lane & (P - 1), g = lane >> log2i(P);
        float w0 = 0.0f, w1 = 0.0f, m0 = INFINITY, m1 = INFINITY;
        if (a < NA) {
            int q = g;
            for (; q + G < nq; q += 2 * G) {
                const float2 t0 = *reinterpret_cast<const float2 *>(recv_par + 2 * (q * AG + OFF + a));
                const float2 t1 =
                    *reinterpret_cast<const float2 *>(recv_par + 2 * ((q + G) * AG + OFF + a));
                w0 += t0.x;
                w1 += t1.x;
                m0 = fminf(m0, t0.y);
                m1 = fminf(m1, t1.y);
            }
            if (q < nq) {
                const float2 t0 = *reinterpret_cast<const float2 *>(recv_par + 2 * (q * AG + OFF + a));
                w0 += t0.x;
                m0 = fminf(m0, t0.y);
            }
        }
        float w = w0 + w1, m = fminf(m0, m1);
#pragma unroll
        for (int L = P; L < 32; L <<= 1) {
            w += __shfl_xor_sync(0xffffffffu, w, L);
            if (CLEAR) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, L));
        }
        const int src = (lane - OFF) & 31;
        const float wt = __shfl_sync(0xffffffffu, w, src);
        const float mt = CLEAR ? __shfl_sync(0xffffffffu, m, src) : INFINITY;
        if (lane >= OFF && lane < OFF + NA) {
            W = wt;
            md2 = mt;
        }
    }
}

template <int AG, int NM, int NT, bool CLEAR>
__global__ void __launch_bounds__(NT, 1) k_rollout(const RolloutArgs A) {
    constexpr int NW = NT / 32;
    constexpr int H0 = (AG + 1) / 2;  // agents [0, H0) form half 0, [H0, AG) half 1
    constexpr int H1 = AG - H0;
    // SFU agents split evenly over the halves (each half's pair loop then
    // keeps the same SFU/FMA balance)
    constexpr int NM0 = (NM + 1) / 2 < H0 ? (NM + 1) / 2 : H0;
    constexpr int NM1 = NM - NM0 < H1 ? NM - NM0 : H1;
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bar;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t rank = cluster_rank();
    uint32_t C;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(C));
    int a0, na;
    group_range(static_cast<int>(cluster_id_x()), A.n_agents, A.n_groups, a0, na);

    // N_O is read on the device; all CTAs of the cluster see the same value,
    // so an early exit is taken by the whole cluster before any DSMEM access.
    const int32_t n_obs = *A.n_obs;
    const int32_t shard_len = ((n_obs + (int32_t)C - 1) / (int32_t)C + 3) & ~3;
    if (n_obs < 0 || n_obs > A.cap || shard_len > A.shard_cap || na > AG || na <= 0) {
        if (tid == 0 && rank == 0) raise_error(A.err, GMAPP_DEVERR_CAPACITY);
        return;
    }
    const int32_t start = static_cast<int32_t>(rank) * shard_len;
    int32_t cnt = min(shard_len, max(0, n_obs - start));
    float *sx = smem, *sy = smem + A.shard_cap, *sz = smem + 2 * A.shard_cap;
    // per-warp partials of this CTA: [half][NW][AG] x (W, min |d|^2)
    float *partbuf = smem + 3 * A.shard_cap;
    // per-CTA partials received from the cluster: [half][parity][rank][AG]
    float *recv = partbuf + 4 * NW * AG;
    auto part = [&](int h) { return partbuf + h * (2 * NW * AG); };
    auto slot = [&](int h, int par) {
        return recv + (h * 2 + par) * (2 * static_cast<int>(C) * AG);
    };

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

    // Agent state: lane a < na of EVERY warp holds agent a0 + a.
    float p[3] = {0, 0, 0}, v[3] = {0, 0, 0}, cc[3] = {0, 0, 0};
    float k_r = 0, k_a = 0, R = 0, G2 = -1.0f, L = 0, pen = 0, minc = INFINITY;
    if (lane < na) {
        const int i = a0 + lane, n = A.n_agents;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            p[d] = A.p0[d * n + i];
            v[d] = A.v0[d * n + i];
            cc[d] = A.c[d * n + i];
        }
        k_r = A.k_r[i];
        k_a = A.k_a[i];
        R = A.r_a[i] + A.r_O;
        const float rd = A.r_d[i];
        // s = max(d - R, eps) <= r_d  <=>  d^2 <= (r_d + R)^2  when r_d >= eps
        G2 = rd >= A.eps ? (rd + R) * (rd + R) : -1.0f;
        if (rank == 0 && warp == 0 && A.traj) {
            float *t = A.traj + (size_t)i * (A.n_steps + 1) * 3;
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
        if (!mbar_wait(&bar, 0)) {
            if (tid == 0) raise_error(A.err, GMAPP_DEVERR_TIMEOUT);
            cnt = 0;  // keep the barrier sequence; results are flagged invalid
        }
    }
    // pad the shard to an even length with NaN (contributes nothing)
    const int32_t cnt_pad = (cnt + 1) & ~1;
    if (tid == 0 && cnt_pad > cnt) {
        sx[cnt] = __int_as_float(0x7fc00000);
        sy[cnt] = __int_as_float(0x7fc00000);
        sz[cnt] = __int_as_float(0x7fc00000);
    }
    const float eps = A.eps;
    // every CTA of the cluster is running (and the padding is visible)
    // before anyone stores into its shared memory
    cluster_sync_all();

    const float h = A.vel_half * A.dt * A.inv_mass;
    auto integrate = [&](int k, float W, float md2) {
        if (A.ckpt && rank == 0 && warp == 0 && k % A.ckpt_every == 0) {
            // adjoint checkpoint: the state (p_k, v_{k-1}) entering step k
            const int n = A.n_agents, i = a0 + lane;
            float *ck = A.ckpt + (size_t)(k / A.ckpt_every) * 6 * n + i;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                ck[d * n] = p[d];
                ck[(3 + d) * n] = v[d];
            }
        }
        float g[3], kf, m;
        agent_step<CLEAR>(p, v, cc, k_r, k_a, R, A.goal, h, A.dt, A.rho, A.damping,
                          A.clear_margin, A.clear_beta, W, md2, L, pen, minc, m, g, kf);
        if (rank == 0 && warp == 0) {
            const int i = a0 + lane;
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
    };

    // Two agent halves in flight: while the partial sums of one half cross
    // the cluster (split barrier), the other half is being computed.
    //   prologue: half0(0) -> arrive
    //   step k:   half1(k) -> wait -> integrate half0(k) -> arrive
    //             half0(k+1) -> wait -> integrate half1(k) -> arrive
    //   each half: per-warp partials -> CTA barrier -> one warp per agent
    //   reduces the CTA's partial and stores it into every cluster CTA
    auto compute_half0 = [&](int par) {
        half_step<AG, H0, 0, NM0, NT, CLEAR, false, false>(sx, sy, sz, cnt_pad, eps, nR2, G2a, p,
                                                           part(0) + 2 * (warp * AG), C, lane);
        named_barrier(1, NT);
        cta_ship<AG, H0, 0, NW, CLEAR>(part(0), slot(0, par), C, rank, warp, lane);
    };
    auto compute_half1 = [&](int par) {
        half_step<AG, H1, H0, NM1, NT, CLEAR, false, false>(sx, sy, sz, cnt_pad, eps, nR2, G2a,
                                                            p, part(1) + 2 * (warp * AG), C, lane);
        named_barrier(2, NT);
        cta_ship<AG, H1, H0, NW, CLEAR>(part(1), slot(1, par), C, rank, warp, lane);
    };
    compute_half0(0);
    cluster_arrive();
    for (int k = 0; k < A.n_steps; ++k) {
        const int par = k & 1;
        compute_half1(par);
        cluster_wait();
        if (lane < H0 && lane < na) {
            float W, md2;
            cluster_combine<AG, CLEAR>(slot(0, par), C, lane, W, md2);
            integrate(k, W, md2);
        }
        cluster_arrive();
        if (k + 1 < A.n_steps) compute_half0(par ^ 1);
        cluster_wait();
        if (lane >= H0 && lane < na) {
            float W, md2;
            cluster_combine<AG, CLEAR>(slot(1, par), C, lane, W, md2);
            integrate(k, W, md2);
        }
        if (k + 1 < A.n_steps) cluster_arrive();
    }
    if (rank == 0 && warp == 0 && lane < na) {
        const int i = a0 + lane, n = A.n_agents;
        for (int d = 0; d < 3; ++d) {
            A.p_final[d * n + i] = p[d];
            A.v_final[d * n + i] = v[d];
        }
        A.path_len[i] = L;
        if (A.clear_pen) A.clear_pen[i] = pen;
        if (A.min_clear) A.min_clear[i] = minc;
    }
}

using RolloutKernel = void (*)(const RolloutArgs);

// Instantiation tables (rollout_inst_*.cu).
RolloutKernel rollout_kernel_noclear(int ag, int nt);
RolloutKernel rollout_kernel_clear(int ag, int nt);

// SFU share of the reciprocals: NM of AG agents use rcp.approx, the rest the
// Newton-Raphson path (NM/AG ~ 3/7 balances 16 SFU ops/clk against 128 FMA
// lanes/clk per SM); tiny groups stay on the SFU, where latency matters more.
constexpr int sfu_agents(int ag) { return ag <= 2 ? ag : (3 * ag + 3) / 7; }

}  // namespace gmapp
