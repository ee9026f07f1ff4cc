// The rollout kernel template (Sec. IV-A agent dynamics, Eq. (mfi)
// circular-field force, Alg. 1 clamp, gate and obstacle sum).
//
// Layout of the work: a thread-block cluster of C CTAs owns a group of up to
// AG agents for the whole rollout; CTA r keeps obstacle shard r of S_W (the
// blocks r, r + C, ... of 128 obstacles) in shared memory (SoA float32,
// loaded once by the TMA bulk-copy engine, padded with NaN, which
// contributes exactly nothing).  Each thread walks pairs of
// obstacles of its shard against all AG agents of the group:
//
//   packed f32x2 arithmetic over the obstacle pair (one instruction, two
//   lanes of work): differences, |d|^2, s = |d| - R;
//   |d|^-1/2 on the SFU (rsqrt), clamp max(s, eps), detection gate as a
//   0/1 mask from |d|^2 <= (r_d + R)^2 folded into the accumulation FMA;
//   1/s on the SFU for NM of the agents and by a magic-constant seed, one
//   third-order step and one Newton-Raphson step on the FMA pipe for the
//   others (Blinn, "Floating-point tricks", IEEE CG&A 1997; the iteration
//   runs on -1/s so it needs no negation), which balances the SFU against
//   the FMA pipe.
//
// Warp specialisation: the CTA's NT compute warps only evaluate pairs; two
// more warps (the exchange warps, one per agent half) own the agents' state.
// The agents of a group are split into two halves kept one phase apart.
// After a half, each compute warp reduces its partial sums with a transposed
// shuffle butterfly, stores them to shared memory and arrives on a named
// barrier, then goes on with the other half.  Meanwhile the half's exchange
// warp sums the NW warp partials in warp order, sends the CTA partial into
// the double-buffered receive slots of every CTA of the cluster with st.async
// (each store completes bytes on the receiver's mbarrier), waits for the C
// partials, sums them in rank order, integrates the half's agents (lane a =
// agent a) and publishes their positions to shared memory behind a second
// named barrier.  The exchange of one half is thus hidden behind the other
// half's pair loop (and the two halves' exchanges overlap); every CTA
// integrates the same sums in the same order, so all copies of an agent's
// state are bit-identical.  Nothing inside the N_k loop touches global
// memory except the optional trajectory/trace stores.
#pragma once

#include <math.h>

#include <type_traits>

#include "gmapp_internal.cuh"

namespace gmapp {

constexpr int kMaxCluster = 16;
constexpr int kMaxAgents = 16;
// agents per group of the heterogeneous-ensemble kernel
constexpr int kMaxEnsembleAgents = 12;
// heuristic kinds of an agent group
constexpr int kMfi = 0, kApf = 1, kProj = 2;
// rows of the per-agent four-term cost sums kept in shared memory
constexpr int kCostAcc = 11;
// exchange warps of a rollout CTA: one per agent half
constexpr int kExchWarps = 2;

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
    float *cost_terms;  // [5][N_a] sums of the four-term cost, or NULL
    unsigned long long *heur_pairs;  // pairs whose heuristic terms ran (added), or NULL
    int32_t box_cull;    // groups visit only the blocks whose bounding box meets a gate
    float cost_radius;  // r_c of its goal and obstacle terms
    int32_t shard_cap;   // obstacles one CTA can hold (multiple of 128)
    int32_t n_groups;    // agent groups (clusters, or CTA groups with the grid exchange)
    int32_t n_apf;       // ensemble kernel: the last n_apf agents use APF (Eq. (apf))
    int32_t n_groups_apf;  // ensemble kernel: ... and form the last n_groups_apf groups
    int32_t n_proj;      // ensemble kernel: the n_proj agents before them use the
    int32_t n_groups_proj;  // projected current, in n_groups_proj groups
    int32_t group_ctas;  // grid exchange: CTAs per group (C)
    uint64_t *xbuf;      // grid exchange: tagged slots [G][2][2][C][AG][2]
    uint32_t *xctl;      // grid exchange: launch epoch, finished-CTA counter
    int64_t xbuf_words;   // grid exchange: 64-bit words of xbuf
    uint32_t spin_limit;  // polls of an mbarrier wait before it gives up
    uint32_t poll_limit;  // polls of a grid-exchange word before it gives up
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
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
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

// -1/s for a pair s > 0 on the FMA pipe: the magic-constant seed y0 (5.1%
// worst relative error), one third-order step y1 = y0 (1 + e + e^2) with
// e = 1 + s y0 (error e^3 <= 1.4e-4), then one Newton-Raphson step
// y2 = y1 (1 + e1) (error e1^2 <= 2e-8): five f32x2 FMAs.
__device__ __forceinline__ f2 neg_rcp2(f2 s2, float sl, float sh, f2 one2) {
    const f2 y0 = pk(neg_rcp_seed(sl), neg_rcp_seed(sh));
    const f2 e = fma2(s2, y0, one2);
    const f2 y1 = fma2(y0, fma2(e, e, e), y0);
    return fma2(y1, fma2(s2, y1, one2), y1);
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
// Returns g, the field strength kf = rho k_r W and m (inf without CLEAR);
// with Fo, also the total force F.
template <bool CLEAR>
__device__ __forceinline__ void agent_step(float (&p)[3], float (&v)[3], const float (&cc)[3],
                                           float k_r, float k_a, float R, const float (&goal)[3],
                                           float h, float dt, float rho, float damping,
                                           float clear_margin, float clear_beta, float W,
                                           float md2, float &L, float &pen, float &minc,
                                           float &m, float (&g)[3], float &kf,
                                           float *Fo = nullptr) {
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
        if (Fo) Fo[d] = F;
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
// Agent a of NA uses the SFU reciprocal when it is one of NM agents spread
// evenly over the NA (Bresenham pattern), so SFU and FMA work interleave in
// the unrolled pair loop.
constexpr bool sfu_agent(int a, int NM, int NA) { return ((a + 1) * NM) / NA > (a * NM) / NA; }

//
// The terms are split in two parts: pair_dist forms |d|^2 of every pair (and
// the clearance minimum) and tells whether one of the thread's pairs passes
// the gate of one of the NA agents; pair_heur evaluates the gated heuristic
// terms (Alg. 1's branch) from |d|^2.  A pair outside the gate adds its
// mask 0 times a finite term, i.e. a signed zero, which leaves a sum that is
// never -0 unchanged; evaluating pair_heur only for blocks where some pair
// passes the gate therefore gives bit-identical sums.
template <int AG, int NA, int OFF, bool CLEAR>
__device__ __forceinline__ bool pair_dist(f2 ox, f2 oy, f2 oz, const f2 (&X)[NA],
                                          const f2 (&Y)[NA], const f2 (&Z)[NA], f2 (&d2)[NA],
                                          float (&mn)[NA], const float (&G2a)[AG]) {
    bool hit = false;
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const f2 dx = sub2(X[a], ox), dy = sub2(Y[a], oy), dz = sub2(Z[a], oz);
        d2[a] = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
        // min ignores a NaN lane, so m <= G2 iff one of the two lanes passes
        const float m = fminf(lo_of(d2[a]), hi_of(d2[a]));
        hit |= m <= G2a[OFF + a];
        if (CLEAR) mn[a] = fminf(mn[a], m);
    }
    return hit;
}

// OPEN: no agent of the half has a gate (r_d = inf) and both obstacles of
// the pair are real, so every gate mask is 1 and is not formed.
template <int AG, int NA, int OFF, int NM, bool OPEN = false>
__device__ __forceinline__ void pair_heur(const f2 (&d2)[NA], f2 (&acc)[NA], const f2 (&nR2)[AG],
                                          const float (&G2a)[AG], float eps, f2 one2) {
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const float d2l = lo_of(d2[a]), d2h = hi_of(d2[a]);
        const f2 r = pk(rsqrt_approx(d2l), rsqrt_approx(d2h));
        const f2 s = fma2(d2[a], r, nR2[OFF + a]);  // |d| - R (NaN when d = 0)
        const float sl = fmaxf(lo_of(s), eps), sh = fmaxf(hi_of(s), eps);
        const f2 y = sfu_agent(a, NM, NA) ? pk(rcp_approx(sl), rcp_approx(sh))
                                          : neg_rcp2(pk(sl, sh), sl, sh, one2);
        if constexpr (OPEN) {
            acc[a] = add2(y, acc[a]);
        } else {
            const f2 mask = pk(le_mask(d2l, G2a[OFF + a]), le_mask(d2h, G2a[OFF + a]));
            acc[a] = fma2(mask, y, acc[a]);
        }
    }
}

template <int AG, int NA, int OFF, int NM, bool CLEAR, bool OPEN = false>
__device__ __forceinline__ void pair_terms(f2 ox, f2 oy, f2 oz, const f2 (&X)[NA],
                                           const f2 (&Y)[NA], const f2 (&Z)[NA], f2 (&acc)[NA],
                                           float (&mn)[NA], const f2 (&nR2)[AG],
                                           const float (&G2a)[AG], float eps, f2 one2) {
    f2 d2[NA];
    pair_dist<AG, NA, OFF, CLEAR>(ox, oy, oz, X, Y, Z, d2, mn, G2a);
    pair_heur<AG, NA, OFF, NM, OPEN>(d2, acc, nR2, G2a, eps, one2);
}

// Obstacles beyond what shared memory holds, read from global memory
// (L2-resident): indices [begin, end) of the obstacle arrays.
struct GlobalTail {
    const float *x, *y, *z;
    int begin, end;
};

// Agent positions come from lane OFF+a of the warp (p), or with POS from
// shared memory pos[3][AG] (SoA).  With VOTE the shard is padded to a
// multiple of 128 obstacles (cnt_pad), so every lane of a warp runs the same
// iterations; a lane takes 4 consecutive obstacles per iteration (two packed
// pairs), the warp a block of 128, and the warp evaluates the heuristic
// terms of the block only when one of its pairs passes an agent's gate
// (Alg. 1's branch, taken per warp).  *nheur counts those blocks in units of
// 64 pairs per agent.
//
// Without the clearance the test of a block uses the expanded distance
// |d|^2 - |p|^2 = |o|^2 - 2 p.o (|o|^2 once per obstacle, then three FMAs
// per pair instead of six) against G2 - |p|^2 + delta.  Its rounding
// error (a few ulp of |o|^2 + 2|p||o| + |p|^2 <= 2 (|p|^2 + omax2), plus
// those of the exact |d|^2 and of the threshold) stays below
// 32 u (G2 + |p|^2 + omax2) with u = 2^-24; delta is eight times that, so
// every pair the exact |d|^2 puts inside the gate passes the test (a few
// more blocks than needed may run the heuristic terms, which then add
// signed zeros).  omax2 bounds |o|^2 over the shard.
template <int AG, int NA, int OFF, int NM, int NT, bool CLEAR, bool TAIL = false,
          bool SHIP = true, bool POS = false, bool VOTE = false, bool BOX = false>
__device__ __forceinline__ void half_step(const float *sx, const float *sy, const float *sz,
                                          int cnt_pad, float eps, const f2 (&nR2)[AG],
                                          const float (&G2a)[AG], const float (&p)[3],
                                          float *recv_slot0, uint32_t C, int lane,
                                          GlobalTail tail = GlobalTail{},
                                          const float *pos = nullptr,
                                          uint32_t *nheur = nullptr, float omax2 = 0.0f,
                                          const float *boxes = nullptr, int cnt_real = -1) {
    if constexpr (NA > 0) {
        constexpr int P = pow2ceil(NA);
        const int tid = threadIdx.x;
        f2 X[NA], Y[NA], Z[NA], acc[NA];
        float mn[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            float x, y, z;
            if constexpr (POS) {
                x = pos[OFF + a];
                y = pos[AG + OFF + a];
                z = pos[2 * AG + OFF + a];
            } else {
                x = __shfl_sync(0xffffffffu, p[0], OFF + a);
                y = __shfl_sync(0xffffffffu, p[1], OFF + a);
                z = __shfl_sync(0xffffffffu, p[2], OFF + a);
            }
            X[a] = pk(x, x);
            Y[a] = pk(y, y);
            Z[a] = pk(z, z);
            acc[a] = 0ull;
            mn[a] = INFINITY;
        }
        const f2 one2 = pk(1.0f, 1.0f);
        if constexpr (VOTE && BOX) {
            // Culled: a lane tests one block's bounding box (boxes[6 b]: lo
            // xyz, hi xyz) against the gates of the half's agents, and the
            // warp visits only the blocks whose box meets a gate, in the same
            // order and lane layout as the voting loop (a skipped block could
            // only add signed zeros).  The gate radius is widened by 2^-12
            // (relative) against the rounding of the box and pair distances.
            float TB[NA];
#pragma unroll
            for (int a = 0; a < NA; ++a) TB[a] = fmaf(G2a[OFF + a], 1.0f + 0x1p-12f, 1e-12f);
            constexpr int NWc = NT / 32;
            const int w = tid >> 5;
            const int n_it = (cnt_pad / 128 - w + NWc - 1) / NWc;  // blocks w, w + NWc, ...
            uint32_t blocks = 0;
            for (int base = 0; base < n_it; base += 32) {
                const int i = base + lane;
                bool near = false;
                if (i < n_it) {
                    const float *bx = boxes + 6 * (w + i * NWc);
                    const float lx = bx[0], ly = bx[1], lz = bx[2], hx = bx[3], hy = bx[4],
                                hz = bx[5];
#pragma unroll
                    for (int a = 0; a < NA; ++a) {
                        const float px = lo_of(X[a]), py = lo_of(Y[a]), pz = lo_of(Z[a]);
                        const float dx = fmaxf(fmaxf(lx - px, px - hx), 0.0f);
                        const float dy = fmaxf(fmaxf(ly - py, py - hy), 0.0f);
                        const float dz = fmaxf(fmaxf(lz - pz, pz - hz), 0.0f);
                        near |= fmaf(dz, dz, fmaf(dy, dy, dx * dx)) <= TB[a];
                    }
                }
                uint32_t m = __ballot_sync(0xffffffffu, near);
                while (m) {
                    const int l = __ffs(m) - 1;
                    m &= m - 1;
                    const int j = (w + (base + l) * NWc) * 128 + 4 * lane;
                    const float4 x4 = *reinterpret_cast<const float4 *>(sx + j);
                    const float4 y4 = *reinterpret_cast<const float4 *>(sy + j);
                    const float4 z4 = *reinterpret_cast<const float4 *>(sz + j);
                    f2 d20[NA], d21[NA];
                    pair_dist<AG, NA, OFF, CLEAR>(pk(x4.x, x4.y), pk(y4.x, y4.y), pk(z4.x, z4.y),
                                                  X, Y, Z, d20, mn, G2a);
                    pair_dist<AG, NA, OFF, CLEAR>(pk(x4.z, x4.w), pk(y4.z, y4.w), pk(z4.z, z4.w),
                                                  X, Y, Z, d21, mn, G2a);
                    pair_heur<AG, NA, OFF, NM>(d20, acc, nR2, G2a, eps, one2);
                    pair_heur<AG, NA, OFF, NM>(d21, acc, nR2, G2a, eps, one2);
                    ++blocks;
                }
            }
            if (nheur) *nheur += 2 * blocks * NA;
        } else if constexpr (VOTE) {
            // block test of the expanded distance (no clearance): -2p and
            // the threshold G2 - |p|^2 + delta per agent
            f2 QX[NA], QY[NA], QZ[NA];
            float T[NA];
            if constexpr (!CLEAR) {
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    const float x = lo_of(X[a]), y = lo_of(Y[a]), z = lo_of(Z[a]);
                    QX[a] = pk(-2.0f * x, -2.0f * x);
                    QY[a] = pk(-2.0f * y, -2.0f * y);
                    QZ[a] = pk(-2.0f * z, -2.0f * z);
                    const float pp = fmaf(x, x, fmaf(y, y, z * z)), g = G2a[OFF + a];
                    T[a] = (g - pp) + 0x1p-16f * (fabsf(g) + pp + omax2);
                }
            }
            uint32_t blocks = 0;
#pragma unroll 2
            for (int j = 4 * tid; j < cnt_pad; j += 4 * NT) {
                const float4 x4 = *reinterpret_cast<const float4 *>(sx + j);
                const float4 y4 = *reinterpret_cast<const float4 *>(sy + j);
                const float4 z4 = *reinterpret_cast<const float4 *>(sz + j);
                const f2 ox0 = pk(x4.x, x4.y), oy0 = pk(y4.x, y4.y), oz0 = pk(z4.x, z4.y);
                const f2 ox1 = pk(x4.z, x4.w), oy1 = pk(y4.z, y4.w), oz1 = pk(z4.z, z4.w);
                f2 d20[NA], d21[NA];
                bool hit = false;
                if constexpr (CLEAR) {
                    hit = pair_dist<AG, NA, OFF, true>(ox0, oy0, oz0, X, Y, Z, d20, mn, G2a);
                    hit |= pair_dist<AG, NA, OFF, true>(ox1, oy1, oz1, X, Y, Z, d21, mn, G2a);
                } else {
                    const f2 oo0 = fma2(ox0, ox0, fma2(oy0, oy0, mul2(oz0, oz0)));
                    const f2 oo1 = fma2(ox1, ox1, fma2(oy1, oy1, mul2(oz1, oz1)));
#pragma unroll
                    for (int a = 0; a < NA; ++a) {
                        const f2 e0 = fma2(QX[a], ox0, fma2(QY[a], oy0, fma2(QZ[a], oz0, oo0)));
                        const f2 e1 = fma2(QX[a], ox1, fma2(QY[a], oy1, fma2(QZ[a], oz1, oo1)));
                        hit |= fminf(fminf(lo_of(e0), hi_of(e0)), fminf(lo_of(e1), hi_of(e1))) <=
                               T[a];
                    }
                }
                if (__any_sync(0xffffffffu, hit)) {
                    if constexpr (!CLEAR) {
                        pair_dist<AG, NA, OFF, false>(ox0, oy0, oz0, X, Y, Z, d20, mn, G2a);
                        pair_dist<AG, NA, OFF, false>(ox1, oy1, oz1, X, Y, Z, d21, mn, G2a);
                    }
                    pair_heur<AG, NA, OFF, NM>(d20, acc, nR2, G2a, eps, one2);
                    pair_heur<AG, NA, OFF, NM>(d21, acc, nR2, G2a, eps, one2);
                    ++blocks;
                }
            }
            if (nheur) *nheur += 2 * blocks * NA;  // blocks of 128 obstacles
        } else {
            uint32_t its = 0;
            // with no gate in the half, the real obstacles' pairs run without
            // the gate masks (a NaN pad needs its mask of 0): up to the last
            // whole pair of real obstacles, then the rest masked
            bool open = cnt_real >= 0;
#pragma unroll
            for (int a = 0; a < NA; ++a) open &= G2a[OFF + a] == INFINITY;
            int j = 2 * tid;
            if (open) {
                const int cnt_even = cnt_real & ~1;
#pragma unroll 3
                for (; j < cnt_even; j += 2 * NT) {
                    const f2 ox = *reinterpret_cast<const f2 *>(sx + j);
                    const f2 oy = *reinterpret_cast<const f2 *>(sy + j);
                    const f2 oz = *reinterpret_cast<const f2 *>(sz + j);
                    pair_terms<AG, NA, OFF, NM, CLEAR, true>(ox, oy, oz, X, Y, Z, acc, mn, nR2,
                                                             G2a, eps, one2);
                    ++its;
                }
            }
#pragma unroll 3
            for (; j < cnt_pad; j += 2 * NT) {
                const f2 ox = *reinterpret_cast<const f2 *>(sx + j);
                const f2 oy = *reinterpret_cast<const f2 *>(sy + j);
                const f2 oz = *reinterpret_cast<const f2 *>(sz + j);
                pair_terms<AG, NA, OFF, NM, CLEAR>(ox, oy, oz, X, Y, Z, acc, mn, nR2, G2a, eps,
                                                   one2);
                ++its;
            }
            if (nheur) *nheur += its * NA;  // every pair, 64 per iteration and agent
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
                vw[a] = sfu_agent(a, NM, NA) ? w : -w;
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

// Exchange of one agent half for step k, run by the exchange warp (lane a
// holds agent a of the group): sum the NW per-warp partials of the CTA in
// warp order, send the CTA partial to slot[rank] of every cluster CTA with
// st.async (completing on that CTA's receive barrier), wait for the C
// partials of this half, sum them in rank order and integrate.
template <int AG, int NA, int OFF, int NW, bool CLEAR>
__device__ __forceinline__ bool exchange_half(const float *part, float *slot, uint64_t *bar,
                                              uint32_t C, uint32_t rank, int lane, int k,
                                              bool ok, float &W, float &md2, uint32_t limit) {
    float w = 0.0f, m = INFINITY;
    if (lane < NA) {
#pragma unroll 4
        for (int q = 0; q < NW; ++q) {
            const float2 t = *reinterpret_cast<const float2 *>(part + 2 * (q * AG + OFF + lane));
            w += t.x;
            if (CLEAR) m = fminf(m, t.y);
        }
    }
    if (lane == 0) mbar_arrive_expect_tx(bar, C * NA * 8u);
    if (lane < NA) {
        const uint32_t local = smem_u32(slot + 2 * (rank * AG + OFF + lane));
        const uint32_t lbar = smem_u32(bar);
        for (uint32_t r = 0; r < C; ++r)
            st_async_v2f32(map_smem(local, r), w, m, map_smem(lbar, r));
    }
    // each (half, parity) barrier completes once every second step
    if (ok && !mbar_wait_cluster(bar, (k >> 1) & 1, limit)) ok = false;
    if (lane >= OFF && lane < OFF + NA) {
        float ws = 0.0f, ms = INFINITY;
        for (uint32_t r = 0; r < C; ++r) {
            const float2 t = *reinterpret_cast<const float2 *>(slot + 2 * (r * AG + lane));
            ws += t.x;
            if (CLEAR) ms = fminf(ms, t.y);
        }
        W = ws;
        md2 = ms;
    }
    return ok;
}

// Tag of a grid-exchange word: the launch epoch (30 bits) and the step
// modulo 4 -- a slot is rewritten every second step, so a reader sees either
// step k or step k - 2 of its own launch, or a word of an older launch.
__device__ __forceinline__ uint32_t xtag(uint32_t epoch, int k) {
    return (epoch << 2) | static_cast<uint32_t>(k & 3);
}
__device__ __forceinline__ uint64_t xword(uint32_t tag, float v) {
    return (static_cast<uint64_t>(tag) << 32) | __float_as_uint(v);
}

// The same exchange between the C CTAs of a group that are not a cluster
// (a cooperative grid, every CTA co-resident): the CTA partial goes to its
// slot xs[rank][a] in global memory as tagged 64-bit words; the lanes of the
// exchange warp poll the C x NA slots of the half between them (bounded)
// until the tags of step k appear, stage the payloads in the shared-memory
// slot[rank][a], and the agent's lane sums them in rank order.
template <int AG, int NA, int OFF, int NW, bool CLEAR>
__device__ __forceinline__ bool exchange_half_grid(const float *part, uint64_t *xs, float *slot,
                                                   uint32_t C, uint32_t rank, int lane,
                                                   uint32_t tag, bool ok, float &W, float &md2,
                                                   uint32_t limit) {
    if (lane < NA) {
        float w = 0.0f, m = INFINITY;
#pragma unroll 4
        for (int q = 0; q < NW; ++q) {
            const float2 t = *reinterpret_cast<const float2 *>(part + 2 * (q * AG + OFF + lane));
            w += t.x;
            if (CLEAR) m = fminf(m, t.y);
        }
        uint64_t *dst = xs + 2 * (rank * AG + OFF + lane);
        st_relaxed_u64(dst, xword(tag, w));
        if (CLEAR) st_relaxed_u64(dst + 1, xword(tag, m));
    }
    // pairs (r, a) = (p / NA, OFF + p % NA), p = lane + 32 j: all loads are
    // issued before the first tag check
    constexpr int J = NA > 0 ? (kMaxCluster * NA + 31) / 32 : 1;
    const int npairs = static_cast<int>(C) * NA;
    uint64_t vw[J], vm[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int p = lane + 32 * j;
        if (p < npairs) {
            const uint64_t *src = xs + 2 * ((p / NA) * AG + OFF + p % NA);
            vw[j] = ld_relaxed_u64(src);
            vm[j] = CLEAR ? ld_relaxed_u64(src + 1) : 0;
        }
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int p = lane + 32 * j;
        if (p < npairs) {
            const int r = p / NA, a = OFF + p % NA;
            const uint64_t *src = xs + 2 * (r * AG + a);
            // both words of the pair are reloaded together while either is
            // stale: one round trip per poll, not one per word
            for (uint32_t it = 0; ok; ++it) {
                const bool fw = static_cast<uint32_t>(vw[j] >> 32) == tag;
                const bool fm = !CLEAR || static_cast<uint32_t>(vm[j] >> 32) == tag;
                if (fw && fm) break;
                if (it == limit) {
                    ok = false;
                    break;
                }
                if (!fw) vw[j] = ld_relaxed_u64(src);
                if (!fm) vm[j] = ld_relaxed_u64(src + 1);
            }
            *reinterpret_cast<float2 *>(slot + 2 * (r * AG + a)) =
                make_float2(__uint_as_float(static_cast<uint32_t>(vw[j])),
                            CLEAR ? __uint_as_float(static_cast<uint32_t>(vm[j])) : INFINITY);
        }
    }
    __syncwarp();
    if (lane >= OFF && lane < OFF + NA) {
        float ws = 0.0f, ms = INFINITY;
        for (uint32_t r = 0; r < C; ++r) {
            const float2 t = *reinterpret_cast<const float2 *>(slot + 2 * (r * AG + lane));
            ws += t.x;
            if (CLEAR) ms = fminf(ms, t.y);
        }
        W = ws;
        md2 = ms;
    }
    return ok;
}

// ---- APF heuristic (Eq. (apf)) of a heterogeneous ensemble -----------------
//
// For every obstacle j, with d = p - p_Oj and r = 1/|d|:
//   gate   surface distance |d| - R < r_d, i.e. |d|^2 < (r_d + R)^2
//   clamp  1/rho = min(r, 1/(R + eps))   (rho = max(|d|, R + eps), Alg. 1's
//          clamp of the surface distance at eps)
//   term   (1/rho - 1/r_d) rho^-2 r d    ((1/|d| - 1/r_d)|d|^-3 d unclamped)
// A pair outside the gate takes 1/rho = 1/r_d, so its coefficient is exactly
// zero; |d|^2 carries an added 1e-30 (below the rounding of any |d| above
// 1e-11 m), so a pair at d = 0 has a finite coefficient times d = 0.  Shard
// padding for APF groups is a far finite point (kApfPad), never NaN (NaN
// times a zero coefficient is NaN).  Per pair: 13 FMA-pipe lane-ops (3 sub,
// 3 for |d|^2, 4 for the coefficient, 3 accumulating FMAs), one SFU rsqrt,
// and the clamp and gate select on the ALU.
constexpr float kApfPad = 1e18f;

template <int AG, int NA, int OFF, bool CLEAR>
__device__ __forceinline__ void apf_pair_terms(f2 ox, f2 oy, f2 oz, const f2 (&X)[NA],
                                               const f2 (&Y)[NA], const f2 (&Z)[NA],
                                               f2 (&fx)[NA], f2 (&fy)[NA], f2 (&fz)[NA],
                                               float (&mn)[NA], const float (&cRa)[AG],
                                               const f2 (&ird2)[AG], const float (&G2a)[AG],
                                               f2 tiny2) {
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const f2 dx = sub2(X[a], ox), dy = sub2(Y[a], oy), dz = sub2(Z[a], oz);
        const f2 d2 = fma2(dz, dz, fma2(dy, dy, fma2(dx, dx, tiny2)));
        const float d2l = lo_of(d2), d2h = hi_of(d2);
        const float rl = rsqrt_approx(d2l), rh = rsqrt_approx(d2h);
        const float ird = lo_of(ird2[OFF + a]);
        const float il = d2l < G2a[OFF + a] ? fminf(rl, cRa[OFF + a]) : ird;
        const float ih = d2h < G2a[OFF + a] ? fminf(rh, cRa[OFF + a]) : ird;
        const f2 ir = pk(il, ih);
        const f2 cf = mul2(mul2(sub2(ir, ird2[OFF + a]), mul2(ir, ir)), pk(rl, rh));
        fx[a] = fma2(cf, dx, fx[a]);
        fy[a] = fma2(cf, dy, fy[a]);
        fz[a] = fma2(cf, dz, fz[a]);
        if (CLEAR) mn[a] = fminf(mn[a], fminf(d2l, d2h));
    }
}

// Block gate test of the APF and projected-current pair loops (the MFI loop
// in half_step does the same): a lane takes 4 consecutive obstacles (two
// packed pairs), a warp a block of 128.  Without the clearance the block is
// tested on the expanded distance |o|^2 - 2 p.o against G2 - |p|^2 + delta
// (block_setup); with it, on the exact |d|^2 (+1e-30, as the terms compute
// it) of every pair, which also updates the clearance minimum.  The
// heuristic terms then run only for blocks with a pair inside a gate;
// outside the gate they add exact signed zeros, so the sums are unchanged.
template <int AG, int NA, int OFF>
__device__ __forceinline__ void block_setup(const f2 (&X)[NA], const f2 (&Y)[NA],
                                            const f2 (&Z)[NA], const float (&G2a)[AG],
                                            float omax2, f2 (&QX)[NA], f2 (&QY)[NA],
                                            f2 (&QZ)[NA], float (&T)[NA]) {
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const float x = lo_of(X[a]), y = lo_of(Y[a]), z = lo_of(Z[a]);
        QX[a] = pk(-2.0f * x, -2.0f * x);
        QY[a] = pk(-2.0f * y, -2.0f * y);
        QZ[a] = pk(-2.0f * z, -2.0f * z);
        const float pp = fmaf(x, x, fmaf(y, y, z * z)), g = G2a[OFF + a];
        T[a] = (g - pp) + 0x1p-16f * (fabsf(g) + pp + omax2);
    }
}

template <int NA>
__device__ __forceinline__ bool block_test_expanded(f2 ox0, f2 oy0, f2 oz0, f2 ox1, f2 oy1,
                                                    f2 oz1, const f2 (&QX)[NA],
                                                    const f2 (&QY)[NA], const f2 (&QZ)[NA],
                                                    const float (&T)[NA]) {
    const f2 oo0 = fma2(ox0, ox0, fma2(oy0, oy0, mul2(oz0, oz0)));
    const f2 oo1 = fma2(ox1, ox1, fma2(oy1, oy1, mul2(oz1, oz1)));
    bool hit = false;
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const f2 e0 = fma2(QX[a], ox0, fma2(QY[a], oy0, fma2(QZ[a], oz0, oo0)));
        const f2 e1 = fma2(QX[a], ox1, fma2(QY[a], oy1, fma2(QZ[a], oz1, oo1)));
        hit |= fminf(fminf(lo_of(e0), hi_of(e0)), fminf(lo_of(e1), hi_of(e1))) <= T[a];
    }
    return hit;
}

template <int AG, int NA, int OFF>
__device__ __forceinline__ bool block_test_exact(f2 ox, f2 oy, f2 oz, const f2 (&X)[NA],
                                                 const f2 (&Y)[NA], const f2 (&Z)[NA],
                                                 float (&mn)[NA], const float (&G2a)[AG],
                                                 f2 tiny2) {
    bool hit = false;
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const f2 dx = sub2(X[a], ox), dy = sub2(Y[a], oy), dz = sub2(Z[a], oz);
        const f2 d2 = fma2(dz, dz, fma2(dy, dy, fma2(dx, dx, tiny2)));
        const float m = fminf(lo_of(d2), hi_of(d2));
        hit |= m <= G2a[OFF + a];
        mn[a] = fminf(mn[a], m);
    }
    return hit;
}

// The voting pair loop over the shard (cnt_pad a multiple of 128): terms(ox,
// oy, oz) evaluates and accumulates the heuristic terms of one packed pair.
// Returns the number of blocks whose terms ran.  With BOX (culled rollouts)
// a lane tests one block's bounding box (boxes[6 b]) against the half's
// gates and the warp visits only the blocks whose box meets one, in the
// same order and lane layout (the clearance then comes from the visited
// blocks only).
template <int AG, int NA, int OFF, int NT, bool CLEAR, bool BOX, class Terms>
__device__ __forceinline__ uint32_t vote_loop(const float *sx, const float *sy, const float *sz,
                                          int cnt_pad, const f2 (&X)[NA], const f2 (&Y)[NA],
                                          const f2 (&Z)[NA], float (&mn)[NA],
                                          const float (&G2a)[AG], float omax2, f2 tiny2,
                                          const float *boxes, Terms &&terms) {
    if constexpr (BOX) {
        float TB[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) TB[a] = fmaf(G2a[OFF + a], 1.0f + 0x1p-12f, 1e-12f);
        constexpr int NWc = NT / 32;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        const int n_it = (cnt_pad / 128 - w + NWc - 1) / NWc;  // blocks w, w + NWc, ...
        uint32_t blocks = 0;
        for (int base = 0; base < n_it; base += 32) {
            const int i = base + lane;
            bool near = false;
            if (i < n_it) {
                const float *bx = boxes + 6 * (w + i * NWc);
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    const float px = lo_of(X[a]), py = lo_of(Y[a]), pz = lo_of(Z[a]);
                    const float dx = fmaxf(fmaxf(bx[0] - px, px - bx[3]), 0.0f);
                    const float dy = fmaxf(fmaxf(bx[1] - py, py - bx[4]), 0.0f);
                    const float dz = fmaxf(fmaxf(bx[2] - pz, pz - bx[5]), 0.0f);
                    near |= fmaf(dz, dz, fmaf(dy, dy, dx * dx)) <= TB[a];
                }
            }
            uint32_t m = __ballot_sync(0xffffffffu, near);
            while (m) {
                const int l = __ffs(m) - 1;
                m &= m - 1;
                const int j = (w + (base + l) * NWc) * 128 + 4 * lane;
                const float4 x4 = *reinterpret_cast<const float4 *>(sx + j);
                const float4 y4 = *reinterpret_cast<const float4 *>(sy + j);
                const float4 z4 = *reinterpret_cast<const float4 *>(sz + j);
                const f2 ox0 = pk(x4.x, x4.y), oy0 = pk(y4.x, y4.y), oz0 = pk(z4.x, z4.y);
                const f2 ox1 = pk(x4.z, x4.w), oy1 = pk(y4.z, y4.w), oz1 = pk(z4.z, z4.w);
                if constexpr (CLEAR) {
                    block_test_exact<AG, NA, OFF>(ox0, oy0, oz0, X, Y, Z, mn, G2a, tiny2);
                    block_test_exact<AG, NA, OFF>(ox1, oy1, oz1, X, Y, Z, mn, G2a, tiny2);
                }
                terms(ox0, oy0, oz0);
                terms(ox1, oy1, oz1);
                ++blocks;
            }
        }
        return blocks;
    }
    f2 QX[NA], QY[NA], QZ[NA];
    float T[NA];
    if constexpr (!CLEAR) block_setup<AG, NA, OFF>(X, Y, Z, G2a, omax2, QX, QY, QZ, T);
    uint32_t blocks = 0;
#pragma unroll 2
    for (int j = 4 * threadIdx.x; j < cnt_pad; j += 4 * NT) {
        const float4 x4 = *reinterpret_cast<const float4 *>(sx + j);
        const float4 y4 = *reinterpret_cast<const float4 *>(sy + j);
        const float4 z4 = *reinterpret_cast<const float4 *>(sz + j);
        const f2 ox0 = pk(x4.x, x4.y), oy0 = pk(y4.x, y4.y), oz0 = pk(z4.x, z4.y);
        const f2 ox1 = pk(x4.z, x4.w), oy1 = pk(y4.z, y4.w), oz1 = pk(z4.z, z4.w);
        bool hit;
        if constexpr (CLEAR) {
            hit = block_test_exact<AG, NA, OFF>(ox0, oy0, oz0, X, Y, Z, mn, G2a, tiny2);
            hit |= block_test_exact<AG, NA, OFF>(ox1, oy1, oz1, X, Y, Z, mn, G2a, tiny2);
        } else {
            hit = block_test_expanded<NA>(ox0, oy0, oz0, ox1, oy1, oz1, QX, QY, QZ, T);
        }
        if (__any_sync(0xffffffffu, hit)) {
            terms(ox0, oy0, oz0);
            terms(ox1, oy1, oz1);
            ++blocks;
        }
    }
    return blocks;
}

// APF counterpart of half_step (positions from shared memory pos[3][AG]):
// partial force sums of this thread's obstacle pairs, reduced over the warp
// (one transposed butterfly per component) and stored as one record
// (f_x, f_y, f_z, min |d|^2) per agent at part_slot0[4 (OFF + a)].
template <int AG, int NA, int OFF, int NT, bool CLEAR, bool VOTE = true, bool BOX = false>
__device__ __forceinline__ void half_step_apf(const float *sx, const float *sy, const float *sz,
                                              int cnt_pad, const float (&cRa)[AG],
                                              const f2 (&ird2)[AG], const float (&G2a)[AG],
                                              float *part_slot0, int lane, const float *pos,
                                              float omax2, uint32_t *nheur,
                                              const float *boxes = nullptr) {
    if constexpr (NA > 0) {
        constexpr int P = pow2ceil(NA);
        const int tid = threadIdx.x;
        f2 X[NA], Y[NA], Z[NA], fx[NA], fy[NA], fz[NA];
        float mn[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            const float x = pos[OFF + a], y = pos[AG + OFF + a], z = pos[2 * AG + OFF + a];
            X[a] = pk(x, x);
            Y[a] = pk(y, y);
            Z[a] = pk(z, z);
            fx[a] = fy[a] = fz[a] = 0ull;
            mn[a] = INFINITY;
        }
        const f2 tiny2 = pk(1e-30f, 1e-30f);
        (void)tid;
        if constexpr (VOTE) {
            *nheur += 2 * NA * vote_loop<AG, NA, OFF, NT, CLEAR, BOX>(
                sx, sy, sz, cnt_pad, X, Y, Z, mn, G2a, omax2, tiny2, boxes, [&](f2 ox, f2 oy, f2 oz) {
                    apf_pair_terms<AG, NA, OFF, false>(ox, oy, oz, X, Y, Z, fx, fy, fz, mn, cRa,
                                                       ird2, G2a, tiny2);
                });
        } else {  // a group with an agent without a gate: every pair, no test
            uint32_t its = 0;
#pragma unroll 2
            for (int j = 2 * tid; j < cnt_pad; j += 2 * NT, ++its)
                apf_pair_terms<AG, NA, OFF, CLEAR>(*reinterpret_cast<const f2 *>(sx + j),
                                                   *reinterpret_cast<const f2 *>(sy + j),
                                                   *reinterpret_cast<const f2 *>(sz + j), X, Y, Z,
                                                   fx, fy, fz, mn, cRa, ird2, G2a, tiny2);
            *nheur += its * NA;
        }
        float v0[P], v1[P], v2[P], vm[P];
#pragma unroll
        for (int a = 0; a < P; ++a) {
            if (a < NA) {
                v0[a] = lo_of(fx[a]) + hi_of(fx[a]);
                v1[a] = lo_of(fy[a]) + hi_of(fy[a]);
                v2[a] = lo_of(fz[a]) + hi_of(fz[a]);
                vm[a] = mn[a];
            } else {
                v0[a] = v1[a] = v2[a] = 0.0f;
                vm[a] = INFINITY;
            }
        }
        const float rx = transposed_reduce<P, false>(v0, lane);
        const float ry = transposed_reduce<P, false>(v1, lane);
        const float rz = transposed_reduce<P, false>(v2, lane);
        const float m = CLEAR ? transposed_reduce<P, true>(vm, lane) : INFINITY;
        constexpr int REP = (32 >> log2i(P)) - 1;
        const int idx = transposed_index<P>(lane);
        if ((lane & REP) == 0 && idx < NA)
            *reinterpret_cast<float4 *>(part_slot0 + 4 * (OFF + idx)) = make_float4(rx, ry, rz, m);
    }
}

// ---- per-agent records of the vector heuristics ---------------------------
// An APF or projected-current agent exchanges a record of RS floats per step:
// NF summed components, then (with CLEAR) the smallest |d|^2 at index NF.
//   APF (Eq. apf):               NF = 3 (f_x, f_y, f_z),       RS = 4
//   projected current (Eq. mfi): NF = 4 (S_x, S_y, S_z, B),    RS = 6
// RS is even: records move as float2 pieces (8-byte aligned).

// Sum of the NW per-warp records of agent OFF + lane in warp order.
template <int AG, int OFF, int NW, bool CLEAR, int NF, int RS>
__device__ __forceinline__ void sum_warp_rec(const float *part, int lane, float (&s)[RS]) {
#pragma unroll
    for (int c = 0; c < RS; ++c) s[c] = c < NF ? 0.0f : INFINITY;
#pragma unroll 4
    for (int q = 0; q < NW; ++q) {
        const float *src = part + RS * (q * AG + OFF + lane);
#pragma unroll
        for (int c = 0; c < RS; c += 2) {
            const float2 t = *reinterpret_cast<const float2 *>(src + c);
            if (c < NF) s[c] += t.x;
            if (c + 1 < NF) s[c + 1] += t.y;
            if (CLEAR && c == NF) s[c] = fminf(s[c], t.x);
            if (CLEAR && c + 1 == NF) s[c + 1] = fminf(s[c + 1], t.y);
        }
    }
}

// Sum of the C per-CTA records of agent `lane` in rank order.
template <int AG, bool CLEAR, int NF, int RS>
__device__ __forceinline__ void sum_rank_rec(const float *slot, uint32_t C, int lane,
                                             float (&F)[4], float &md2) {
    float acc[NF];
#pragma unroll
    for (int c = 0; c < NF; ++c) acc[c] = 0.0f;
    float ms = INFINITY;
    for (uint32_t r = 0; r < C; ++r) {
        const float *src = slot + RS * (r * AG + lane);
#pragma unroll
        for (int c = 0; c < NF; ++c) acc[c] += src[c];
        if (CLEAR) ms = fminf(ms, src[NF]);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) F[c] = c < NF ? acc[c] : 0.0f;
    md2 = ms;
}

// exchange_half for records: the CTA record goes to slot[rank][agent] of
// every cluster CTA with st.async (RS / 2 pieces of 8 bytes each).
template <int AG, int NA, int OFF, int NW, bool CLEAR, int NF, int RS>
__device__ __forceinline__ bool exchange_half_rec(const float *part, float *slot, uint64_t *bar,
                                                  uint32_t C, uint32_t rank, int lane, int k,
                                                  bool ok, float (&F)[4], float &md2,
                                                  uint32_t limit) {
    float s[RS];
    if (lane < NA) sum_warp_rec<AG, OFF, NW, CLEAR, NF, RS>(part, lane, s);
    if (lane == 0) mbar_arrive_expect_tx(bar, C * NA * RS * 4u);
    if (lane < NA) {
        const uint32_t local = smem_u32(slot + RS * (rank * AG + OFF + lane));
        const uint32_t lbar = smem_u32(bar);
        for (uint32_t r = 0; r < C; ++r) {
            const uint32_t dst = map_smem(local, r), rb = map_smem(lbar, r);
#pragma unroll
            for (int c = 0; c < RS; c += 2) st_async_v2f32(dst + 4u * c, s[c], s[c + 1], rb);
        }
    }
    if (ok && !mbar_wait_cluster(bar, (k >> 1) & 1, limit)) ok = false;
    if (lane >= OFF && lane < OFF + NA) sum_rank_rec<AG, CLEAR, NF, RS>(slot, C, lane, F, md2);
    return ok;
}

// exchange_half_grid for records: NF tagged words per agent and CTA, one
// more (min |d|^2) with CLEAR, at xs[RS (rank AG + agent) + c].
template <int AG, int NA, int OFF, int NW, bool CLEAR, int NF, int RS>
__device__ __forceinline__ bool exchange_half_grid_rec(const float *part, uint64_t *xs,
                                                       float *slot, uint32_t C, uint32_t rank,
                                                       int lane, uint32_t tag, bool ok,
                                                       float (&F)[4], float &md2, uint32_t limit) {
    constexpr int NV = CLEAR ? NF + 1 : NF;
    if (lane < NA) {
        float s[RS];
        sum_warp_rec<AG, OFF, NW, CLEAR, NF, RS>(part, lane, s);
        uint64_t *dst = xs + RS * (rank * AG + OFF + lane);
#pragma unroll
        for (int c = 0; c < NV; ++c) st_relaxed_u64(dst + c, xword(tag, s[c]));
    }
    constexpr int J = NA > 0 ? (kMaxCluster * NA + 31) / 32 : 1;
    const int npairs = static_cast<int>(C) * NA;
    uint64_t w[J][NV];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int p = lane + 32 * j;
        if (p < npairs) {
            const uint64_t *src = xs + RS * ((p / NA) * AG + OFF + p % NA);
#pragma unroll
            for (int c = 0; c < NV; ++c) w[j][c] = ld_relaxed_u64(src + c);
        }
    }
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int p = lane + 32 * j;
        if (p < npairs) {
            const int r = p / NA, a = OFF + p % NA;
            const uint64_t *src = xs + RS * (r * AG + a);
            float *dst = slot + RS * (r * AG + a);
            // the record's stale words are reloaded together: one round trip
            // per poll, not one per word
            for (uint32_t it = 0; ok; ++it) {
                bool fresh = true;
#pragma unroll
                for (int c = 0; c < NV; ++c)
                    fresh = fresh && static_cast<uint32_t>(w[j][c] >> 32) == tag;
                if (fresh) break;
                if (it == limit) {
                    ok = false;
                    break;
                }
#pragma unroll
                for (int c = 0; c < NV; ++c)
                    if (static_cast<uint32_t>(w[j][c] >> 32) != tag) w[j][c] = ld_relaxed_u64(src + c);
            }
#pragma unroll
            for (int c = 0; c < NV; ++c) dst[c] = __uint_as_float(static_cast<uint32_t>(w[j][c]));
        }
    }
    __syncwarp();
    if (lane >= OFF && lane < OFF + NA) sum_rank_rec<AG, CLEAR, NF, RS>(slot, C, lane, F, md2);
    return ok;
}

// ---- MFI with the per-obstacle projected current ---------------------------
//
// Eq. (mfi) with the current c_j = d' - n_j (n_j . d') of each obstacle
// (static obstacles, d' = -v, n_j = d_j / |d_j|, d_j = p - p_Oj) and Alg. 1's
// clamp and gate.  The cross products reduce to
//   (d'/|d'|) x (c_j x d') = (n_j . v) / |v| (|v|^2 n_j - (n_j . v) v),
// so with t_j = d_j . v, a_j = w_j t_j / |d_j|^2 and w_j = [s_j <= r_d] / s_j
//   f = (|v|^2 S - v B) / |v|,  S = sum_j a_j d_j,  B = sum_j a_j t_j;
// the pair loop accumulates S and B (one record per agent), the exchange warp
// forms f.  |d|^2 carries an added 1e-30, so a pair at d = 0 (no normal)
// adds a_j d_j = 0.  Per pair: 17 FMA-pipe lane-ops (3 sub, 3 for |d|^2, 1
// for s, 3 for t, 3 for a, 4 accumulating FMAs), rsqrt and rcp on the SFU,
// clamp and gate select on the ALU.  The FMA pipe bounds it (an NR
// reciprocal would only add FMA work), so every agent takes rcp.approx.
template <int AG, int NA, int OFF, bool CLEAR>
__device__ __forceinline__ void proj_pair_terms(f2 ox, f2 oy, f2 oz, const f2 (&X)[NA],
                                                const f2 (&Y)[NA], const f2 (&Z)[NA],
                                                const f2 (&VX)[NA], const f2 (&VY)[NA],
                                                const f2 (&VZ)[NA], f2 (&sx)[NA], f2 (&sy)[NA],
                                                f2 (&sz)[NA], f2 (&sb)[NA], float (&mn)[NA],
                                                const f2 (&nR2)[AG], const float (&G2a)[AG],
                                                float eps, f2 tiny2) {
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const f2 dx = sub2(X[a], ox), dy = sub2(Y[a], oy), dz = sub2(Z[a], oz);
        const f2 d2 = fma2(dz, dz, fma2(dy, dy, fma2(dx, dx, tiny2)));
        const float d2l = lo_of(d2), d2h = hi_of(d2);
        const float rl = rsqrt_approx(d2l), rh = rsqrt_approx(d2h);
        const f2 r = pk(rl, rh);
        const f2 s = fma2(d2, r, nR2[OFF + a]);  // |d| - R
        const float wl = d2l <= G2a[OFF + a] ? rcp_approx(fmaxf(lo_of(s), eps)) : 0.0f;
        const float wh = d2h <= G2a[OFF + a] ? rcp_approx(fmaxf(hi_of(s), eps)) : 0.0f;
        const f2 t = fma2(dz, VZ[a], fma2(dy, VY[a], mul2(dx, VX[a])));
        const f2 q = mul2(mul2(pk(wl, wh), mul2(r, r)), t);
        sx[a] = fma2(q, dx, sx[a]);
        sy[a] = fma2(q, dy, sy[a]);
        sz[a] = fma2(q, dz, sz[a]);
        sb[a] = fma2(q, t, sb[a]);
        if (CLEAR) mn[a] = fminf(mn[a], fminf(d2l, d2h));
    }
}

// Projected-current counterpart of half_step: positions and velocities of
// the half's agents from shared memory (pos, vel: [3][AG]); the record
// (S_x, S_y, S_z, B, min |d|^2, 0) of each agent goes to part_slot0[6 a'].
template <int AG, int NA, int OFF, int NT, bool CLEAR, bool VOTE = true, bool BOX = false>
__device__ __forceinline__ void half_step_proj(const float *sx, const float *sy, const float *sz,
                                               int cnt_pad, float eps, const f2 (&nR2)[AG],
                                               const float (&G2a)[AG], float *part_slot0,
                                               int lane, const float *pos, const float *vel,
                                               float omax2, uint32_t *nheur,
                                               const float *boxes = nullptr) {
    if constexpr (NA > 0) {
        constexpr int P = pow2ceil(NA);
        const int tid = threadIdx.x;
        f2 X[NA], Y[NA], Z[NA], VX[NA], VY[NA], VZ[NA], ax[NA], ay[NA], az[NA], ab[NA];
        float mn[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            const float x = pos[OFF + a], y = pos[AG + OFF + a], z = pos[2 * AG + OFF + a];
            const float u = vel[OFF + a], v = vel[AG + OFF + a], w = vel[2 * AG + OFF + a];
            X[a] = pk(x, x);
            Y[a] = pk(y, y);
            Z[a] = pk(z, z);
            VX[a] = pk(u, u);
            VY[a] = pk(v, v);
            VZ[a] = pk(w, w);
            ax[a] = ay[a] = az[a] = ab[a] = 0ull;
            mn[a] = INFINITY;
        }
        const f2 tiny2 = pk(1e-30f, 1e-30f);
        (void)tid;
        if constexpr (VOTE) {
            *nheur += 2 * NA * vote_loop<AG, NA, OFF, NT, CLEAR, BOX>(
                sx, sy, sz, cnt_pad, X, Y, Z, mn, G2a, omax2, tiny2, boxes, [&](f2 ox, f2 oy, f2 oz) {
                    proj_pair_terms<AG, NA, OFF, false>(ox, oy, oz, X, Y, Z, VX, VY, VZ, ax, ay,
                                                        az, ab, mn, nR2, G2a, eps, tiny2);
                });
        } else {  // a group with an agent without a gate: every pair, no test
            uint32_t its = 0;
#pragma unroll 2
            for (int j = 2 * tid; j < cnt_pad; j += 2 * NT, ++its)
                proj_pair_terms<AG, NA, OFF, CLEAR>(*reinterpret_cast<const f2 *>(sx + j),
                                                    *reinterpret_cast<const f2 *>(sy + j),
                                                    *reinterpret_cast<const f2 *>(sz + j), X, Y, Z,
                                                    VX, VY, VZ, ax, ay, az, ab, mn, nR2, G2a, eps,
                                                    tiny2);
            *nheur += its * NA;
        }
        float v0[P], v1[P], v2[P], v3[P], vm[P];
#pragma unroll
        for (int a = 0; a < P; ++a) {
            if (a < NA) {
                v0[a] = lo_of(ax[a]) + hi_of(ax[a]);
                v1[a] = lo_of(ay[a]) + hi_of(ay[a]);
                v2[a] = lo_of(az[a]) + hi_of(az[a]);
                v3[a] = lo_of(ab[a]) + hi_of(ab[a]);
                vm[a] = mn[a];
            } else {
                v0[a] = v1[a] = v2[a] = v3[a] = 0.0f;
                vm[a] = INFINITY;
            }
        }
        const float r0 = transposed_reduce<P, false>(v0, lane);
        const float r1 = transposed_reduce<P, false>(v1, lane);
        const float r2 = transposed_reduce<P, false>(v2, lane);
        const float r3 = transposed_reduce<P, false>(v3, lane);
        const float m = CLEAR ? transposed_reduce<P, true>(vm, lane) : INFINITY;
        constexpr int REP = (32 >> log2i(P)) - 1;
        const int idx = transposed_index<P>(lane);
        if ((lane & REP) == 0 && idx < NA) {
            float2 *dst = reinterpret_cast<float2 *>(part_slot0 + 6 * (OFF + idx));
            dst[0] = make_float2(r0, r1);
            dst[1] = make_float2(r2, r3);
            dst[2] = make_float2(m, 0.0f);
        }
    }
}

// One step of Sec. IV-A for an APF agent: F = k_a (goal - p) - D v + kf f
// with kf = rho k_r and f the Eq. (apf) sum; the rest as agent_step.
template <bool CLEAR>
__device__ __forceinline__ void agent_step_apf(float (&p)[3], float (&v)[3], float kf, float k_a,
                                               float R, const float (&goal)[3], float h, float dt,
                                               float damping, float clear_margin,
                                               float clear_beta, const float (&f)[3], float md2,
                                               float &L, float &pen, float &minc, float &m,
                                               float *Fo = nullptr) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float F = k_a * (goal[d] - p[d]) - damping * v[d] + kf * f[d];
        if (Fo) Fo[d] = F;
        v[d] = fmaf(h, F, v[d]);
    }
    const float vn = fmaf(v[2], v[2], fmaf(v[1], v[1], v[0] * v[0]));
    L = fmaf(dt, vn > 0.0f ? vn * rsqrt_approx(vn) : 0.0f, L);
#pragma unroll
    for (int d = 0; d < 3; ++d) p[d] = fmaf(dt, v[d], p[d]);
    m = INFINITY;
    if (CLEAR) {
        m = sqrtf(md2) - R;
        pen += softplus_f(clear_margin - m, clear_beta);
        minc = fminf(minc, m);
    }
}

// GRID selects the exchange: false -- the C CTAs of a group form a thread-
// block cluster and exchange over DSMEM; true -- groups of C consecutive
// CTAs of a cooperative (all co-resident) grid exchange through global
// memory, which lets groups fill every SM whatever the GPC layout.
// EK compiles the heterogeneous ensemble (Sec. IV-A agent set with the
// heuristics of Eq. (apf) and Eq. (mfi)): EK = 0 -- MFI only; EK = 1 -- the
// last n_apf agents form the last n_groups_apf groups and use APF; EK = 2 --
// in addition the n_proj agents before them form n_groups_proj groups of
// MFI with the per-obstacle projected current.  Every group is homogeneous,
// so the branch between the pair loops is uniform per CTA.
template <int AG, int NM, int NT, bool CLEAR, bool GRID, int EK = 0>
__global__ void __launch_bounds__(NT + 32 * kExchWarps, 1) k_rollout(const RolloutArgs A) {
    constexpr int NW = NT / 32;       // compute warps; warps NW + h exchange half h
    constexpr int H0 = (AG + 1) / 2;  // agents [0, H0) form half 0, [H0, AG) half 1
    constexpr int H1 = AG - H0;
    // SFU agents split evenly over the halves (each half's pair loop then
    // keeps the same SFU/FMA balance)
    constexpr int NM0 = (NM + 1) / 2 < H0 ? (NM + 1) / 2 : H0;
    constexpr int NM1 = NM - NM0 < H1 ? NM - NM0 : H1;
    // named barriers: partials of half h ready (compute -> exchange warp h),
    // and positions of half h ready (exchange warp h -> compute); the two
    // exchange warps join on kJoin before the grid's epoch is advanced
    constexpr int kPart = 1, kPos = 3, kJoin = 5, kBoth = NT + 32;
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bar_tma;
    __shared__ __align__(8) uint64_t bar_recv[2][2];  // [half][parity]
    __shared__ int s_omax2;  // bits of max |o|^2 over the shard

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool exch = warp >= NW;
    const int xh = warp - NW;  // exchange warps: the half they own
    uint32_t rank, C, group;
    if constexpr (GRID) {
        C = static_cast<uint32_t>(A.group_ctas);
        rank = blockIdx.x % C;
        group = blockIdx.x / C;
    } else {
        rank = cluster_rank();
        asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(C));
        group = cluster_id_x();
    }
    int a0, na;
    int kind = kMfi;  // heuristic of this CTA's group
    if constexpr (EK > 0) {
        const int gp = EK > 1 ? A.n_groups_proj : 0, np = EK > 1 ? A.n_proj : 0;
        const int gm = A.n_groups - A.n_groups_apf - gp, nm = A.n_agents - A.n_apf - np;
        const int g = static_cast<int>(group);
        if (g < gm) {
            group_range(g, nm, gm, a0, na);
        } else if (g < gm + gp) {
            kind = kProj;
            group_range(g - gm, np, gp, a0, na);
            a0 += nm;
        } else {
            kind = kApf;
            group_range(g - gm - gp, A.n_apf, A.n_groups_apf, a0, na);
            a0 += nm + np;
        }
    } else {
        group_range(static_cast<int>(group), A.n_agents, A.n_groups, a0, na);
    }
    // floats per agent record exchanged each step: (W, min |d|^2) for MFI,
    // (f_x, f_y, f_z, min |d|^2) for APF, (S_x, S_y, S_z, B, min |d|^2, -)
    // for the projected current
    const int SR = kind == kApf ? 4 : kind == kProj ? 6 : 2;

    // N_O is read on the device; all CTAs of the cluster see the same value,
    // so an early exit is taken by the whole cluster before any DSMEM access.
    const int32_t n_obs = *A.n_obs;
    // Shards interleave blocks of 128 obstacles: CTA r of a group holds the
    // blocks r, r + C, r + 2C, ... of S_W, consecutive in its shared memory.
    // S_W is sorted by voxel key, so the obstacles near a group's agents form
    // runs of consecutive blocks, which this spreads evenly over the C CTAs
    // (each CTA's share of the gated pairs, and so its time per step, is
    // then about the same).  Only the last block of S_W may be partial.
    const int32_t n_blk = (max(n_obs, 0) + 127) / 128;
    const int32_t shard_len = (n_blk + (int32_t)C - 1) / (int32_t)C * 128;
    // grid exchange: the last CTA to finish (every CTA has read the epoch by
    // then) advances the epoch for the next launch
    auto finish_grid = [&](uint32_t epoch) {
        if (atomicAdd(A.xctl + 1, 1u) == gridDim.x - 1) {
            A.xctl[1] = 0;
            const uint32_t next = (epoch + 1) & 0x3fffffffu;
            A.xctl[0] = next ? next : 1u;
        }
    };
    if (n_obs < 0 || n_obs > A.cap || shard_len > A.shard_cap || (A.shard_cap & 127) ||
        na > AG || na <= 0) {
        if (tid == 0 && rank == 0) raise_error(A.err, GMAPP_DEVERR_CAPACITY);
        if constexpr (GRID) {
            if (tid == NT) finish_grid(ld_relaxed_u32(A.xctl));
        }
        return;
    }
    const int32_t n_loc = static_cast<int32_t>(rank) < n_blk
                              ? (n_blk - 1 - static_cast<int32_t>(rank)) / (int32_t)C + 1
                              : 0;
    int32_t cnt = n_loc * 128;
    if (n_loc > 0 && static_cast<uint32_t>(n_blk - 1) % C == rank) cnt -= n_blk * 128 - n_obs;
    float *sx = smem, *sy = smem + A.shard_cap, *sz = smem + 2 * A.shard_cap;
    // per-warp partials of this CTA: [half][NW][AG] records
    float *partbuf = smem + 3 * A.shard_cap;
    // per-CTA partials received from the cluster: [half][parity][rank][AG] records
    float *recv = partbuf + 2 * SR * NW * AG;
    // agent positions and (projected current) velocities for the compute
    // warps: [3][AG] each, 4 AG floats apart
    float *pos = recv + 4 * SR * static_cast<int>(C) * AG;
    float *vel = pos + 4 * AG;
    // four-term cost sums of the exchange warp (lane = agent): [kCostAcc][AG]
    float *cacc = vel + 4 * AG;
    // per-block bounding boxes of the shard (culled rollouts): [blocks][6]
    float *boxes = cacc + kCostAcc * AG;
    auto part = [&](int h) { return partbuf + h * (SR * NW * AG); };
    auto slot = [&](int h, int par) {
        return recv + (h * 2 + par) * (SR * static_cast<int>(C) * AG);
    };
    {
        // bounds-checked build: the invariants the index arithmetic below
        // relies on (uniform over the group's CTAs, so they leave together)
        uint32_t dyn;
        asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
        constexpr int kGroupWords = 4 * (EK > 1 ? 6 : EK == 1 ? 4 : 2);
        const bool in = bc_ok(cnt > 0 ? ((cnt + 127) & ~127) - 1 : 0, A.shard_cap, A.err) &&
                        bc_ok(a0 + na - 1, A.n_agents, A.err) &&
                        bc_ok((boxes + 6 * (A.shard_cap / 128)) - smem - 1, dyn / 4, A.err) &&
                        (!GRID || bc_ok((static_cast<int64_t>(group) + 1) * kGroupWords * C * AG - 1,
                                        A.xbuf_words, A.err));
        if (!in) {
            if constexpr (GRID) {
                if (tid == NT) finish_grid(ld_relaxed_u32(A.xctl));
            }
            return;
        }
    }

    if (tid == 0) {
        s_omax2 = 0;
        mbar_init(&bar_tma, 1);
        for (int i = 0; i < 4; ++i) mbar_init(&bar_recv[i >> 1][i & 1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (cnt > 0 && tid < 32) {
        // one bulk copy per block and array, issued by the lanes of warp 0
        // after the expected byte count (whole blocks, the partial one
        // rounded up to 4 obstacles: within obs->cap, a multiple of 4)
        if (tid == 0) mbar_arrive_expect_tx(&bar_tma, 3u * 4u * static_cast<uint32_t>((cnt + 3) & ~3));
        __syncwarp();
        for (int32_t i = tid; i < n_loc; i += 32) {
            const int64_t g = static_cast<int64_t>(rank) + static_cast<int64_t>(i) * C;
            const int32_t valid = min(128, n_obs - static_cast<int32_t>(128 * g));
            const uint32_t bytes = static_cast<uint32_t>((valid + 3) & ~3) * 4u;
            if (!bc_ok(128 * g + bytes / 4 - 1, A.cap, A.err)) continue;  // (the wait then times out)
            bulk_g2s(sx + 128 * i, A.ox + 128 * g, bytes, &bar_tma);
            bulk_g2s(sy + 128 * i, A.oy + 128 * g, bytes, &bar_tma);
            bulk_g2s(sz + 128 * i, A.oz + 128 * g, bytes, &bar_tma);
        }
    }

    // Agent state: lane a < na of every warp reads agent a0 + a; only the
    // exchange warp integrates, the compute warps keep R and the gate.
    float p[3] = {0, 0, 0}, v[3] = {0, 0, 0}, cc[3] = {0, 0, 0};
    float k_r = 0, k_a = 0, R = 0, rd = 0, G2 = -1.0f, L = 0, pen = 0, minc = INFINITY;
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
        rd = A.r_d[i];
        // s = max(d - R, eps) <= r_d  <=>  d^2 <= (r_d + R)^2  when r_d >= eps
        G2 = rd >= A.eps ? (rd + R) * (rd + R) : -1.0f;
        if (rank == 0 && xh == 0 && A.traj) {
            float *t = A.traj + (size_t)i * (A.n_steps + 1) * 3;
            t[0] = p[0];
            t[1] = p[1];
            t[2] = p[2];
        }
    }
    if (xh == 0 && lane < AG) {
        pos[lane] = p[0];
        pos[AG + lane] = p[1];
        pos[2 * AG + lane] = p[2];
        if (EK > 1) {
            vel[lane] = v[0];
            vel[AG + lane] = v[1];
            vel[2 * AG + lane] = v[2];
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
        if (!mbar_wait(&bar_tma, 0, A.spin_limit)) {
            if (tid == 0) raise_error(A.err, GMAPP_DEVERR_TIMEOUT);
            cnt = 0;  // keep the barrier sequence; results are flagged invalid
        }
    }
    // pad the shard to a multiple of 128 (shard_cap is one) with NaN
    // (contributes nothing to the MFI sum), or a far point for APF and
    // projected-current groups: every warp of the MFI pair loop then runs
    // the same iterations over whole blocks of 128 obstacles
    const int32_t cnt_pad = (cnt + 127) & ~127;
    {
        const float pad = kind != kMfi ? kApfPad : __int_as_float(0x7fc00000);
        for (int32_t i = cnt + tid; i < cnt_pad; i += blockDim.x) {
            sx[i] = pad;
            sy[i] = pad;
            sz[i] = pad;
        }
        // omax2 = max |o|^2 over the shard (bounds the rounding of the
        // expanded distance of the pair loop's block test)
        float m = 0.0f;
        for (int32_t i = tid; i < cnt; i += blockDim.x)
            m = fmaxf(m, fmaf(sx[i], sx[i], fmaf(sy[i], sy[i], sz[i] * sz[i])));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) atomicMax(&s_omax2, __float_as_int(m));  // m >= 0: ordered as ints
        if (A.box_cull) {
            // bounding box of every block (NaN pads ignored; an all-pad
            // block gets an empty box), one warp per block
            const int nwt = static_cast<int>(blockDim.x) / 32;
            for (int b = warp; b < cnt_pad / 128; b += nwt) {
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
        }
    }
    const float eps = A.eps;
    // every CTA of the cluster is running (barriers initialised, padding and
    // positions visible) before anyone stores into its shared memory
    if constexpr (GRID) __syncthreads();
    else cluster_sync_all();

    // The step loops of one group kind (kMfi, kApf or kProj).
    auto run = [&](auto kind_tag) {
        constexpr int KIND = decltype(kind_tag)::value;
        constexpr bool APF = KIND == kApf, PROJ = KIND == kProj;
        // APF per-agent constants: 1/(R + eps), 1/r_d and the strict gate
        // |d|^2 < (r_d + R)^2 (never when r_d + R <= 0)
        float cRa[AG], G2s[AG];
        f2 ird2[AG];
        if constexpr (APF) {
            const float cR = __fdiv_rn(1.0f, R + eps);
            const float ird = lane < na ? __fdiv_rn(1.0f, rd) : 0.0f;
            const float G2l = rd + R > 0.0f ? (rd + R) * (rd + R) : -1.0f;
#pragma unroll
            for (int a = 0; a < AG; ++a) {
                cRa[a] = __shfl_sync(0xffffffffu, cR, a);
                const float t = __shfl_sync(0xffffffffu, ird, a);
                ird2[a] = pk(t, t);
                G2s[a] = __shfl_sync(0xffffffffu, lane < na ? G2l : -1.0f, a);
            }
        }
        if (!exch) {
            // Compute warps: the two halves back to back; a half's partials
            // are handed to the exchange warp while the other half is
            // computed, and its new positions are ready long before they are
            // needed.
            uint32_t nheur = 0;  // heuristic pairs of the pair loops, in units of 64
            const float omax2 = __int_as_float(s_omax2);
            auto steps = [&](auto vote_tag, auto box_tag) {
                constexpr bool VOTE = decltype(vote_tag)::value;
                constexpr bool BOX = decltype(box_tag)::value;
                for (int k = 0; k < A.n_steps; ++k) {
                    if (k > 0) named_sync(kPos + 0, kBoth);
                    if constexpr (APF)
                        half_step_apf<AG, H0, 0, NT, CLEAR, VOTE, BOX>(sx, sy, sz, cnt_pad, cRa, ird2, G2s,
                                                            part(0) + 4 * (warp * AG), lane, pos,
                                                            omax2, &nheur, boxes);
                    else if constexpr (PROJ)
                        half_step_proj<AG, H0, 0, NT, CLEAR, VOTE, BOX>(sx, sy, sz, cnt_pad, eps, nR2, G2a,
                                                             part(0) + 6 * (warp * AG), lane, pos,
                                                             vel, omax2, &nheur, boxes);
                    else
                        half_step<AG, H0, 0, NM0, NT, CLEAR, false, false, true, VOTE, BOX>(
                            sx, sy, sz, cnt_pad, eps, nR2, G2a, p, part(0) + 2 * (warp * AG), C,
                            lane, GlobalTail{}, pos, &nheur, omax2, boxes, cnt);
                    named_arrive(kPart + 0, kBoth);
                    if (k > 0) named_sync(kPos + 1, kBoth);
                    if constexpr (APF)
                        half_step_apf<AG, H1, H0, NT, CLEAR, VOTE, BOX>(sx, sy, sz, cnt_pad, cRa, ird2, G2s,
                                                             part(1) + 4 * (warp * AG), lane, pos,
                                                             omax2, &nheur, boxes);
                    else if constexpr (PROJ)
                        half_step_proj<AG, H1, H0, NT, CLEAR, VOTE, BOX>(sx, sy, sz, cnt_pad, eps, nR2, G2a,
                                                              part(1) + 6 * (warp * AG), lane, pos,
                                                              vel, omax2, &nheur, boxes);
                    else
                        half_step<AG, H1, H0, NM1, NT, CLEAR, false, false, true, VOTE, BOX>(
                            sx, sy, sz, cnt_pad, eps, nR2, G2a, p, part(1) + 2 * (warp * AG), C,
                            lane, GlobalTail{}, pos, &nheur, omax2, boxes, cnt);
                    named_arrive(kPart + 1, kBoth);
                }
            };
            // a group with an agent without a gate (r_d = inf) passes every
            // block: its pair loops run without the block test
            bool every = false;
#pragma unroll
            for (int a = 0; a < AG; ++a) every |= (APF ? G2s[a] : G2a[a]) == INFINITY;
            if (every) steps(std::false_type{}, std::false_type{});
            else if (A.box_cull) steps(std::true_type{}, std::true_type{});
            else steps(std::true_type{}, std::false_type{});
            if (A.heur_pairs && lane == 0 && nheur)
                atomicAdd(A.heur_pairs, 64ull * nheur);
            return;
        }
        const float h = A.vel_half * A.dt * A.inv_mass;
        // Sums of the four-term cost (Eq. cost_function) over the candidate
        // trajectory p_0 .. p_{N_k-1} (only with the clearance compiled in):
        // sum min(|p_k - goal|, r_c), sum max(r_c - m_k, 0), the path length
        // of its N_k - 1 segments, the jerk sum and |p_0 - goal|.  The third
        // difference p_k - 3 p_{k-1} + 3 p_{k-2} - p_{k-3} equals
        // dt h (F_{k-1} - F_{k-2}) by the step rule, and F_k - F_{k-1} =
        // -k_a dt v_{k-1} - D h F_{k-1} + (f_r,k - f_r,k-1): small terms only,
        // where differencing FP32 positions (or forces) would cancel.
        // The sums live in shared memory, column `lane` of cacc: rows 0-4 the
        // five outputs, 5-7 F_{k-1}, 8-10 f_r,k-1.
        float *cs = cacc + lane;
        auto cv = [&](int row) -> float & { return cs[row * AG]; };
        // this exchange warp's agents: lanes of its half
        const bool mine = xh == 0 ? lane < H0 : (lane >= H0 && lane < AG);
        if (CLEAR && A.cost_terms && mine) {
            for (int r = 0; r < kCostAcc; ++r) cv(r) = 0.0f;
        }
        // rec: W (MFI), the force sum f (APF), or S and B (projected
        // current) of this lane's agent
        auto integrate = [&](int k, const float (&rec)[4], float md2) {
            if (A.ckpt && rank == 0 && k % A.ckpt_every == 0) {
                // adjoint checkpoint: the state (p_k, v_{k-1}) entering step k
                const int n = A.n_agents, i = a0 + lane;
                float *ck = A.ckpt + (size_t)(k / A.ckpt_every) * 6 * n + i;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    ck[d * n] = p[d];
                    ck[(3 + d) * n] = v[d];
                }
            }
            float vprev[3] = {v[0], v[1], v[2]};
            if constexpr (CLEAR) {
                if (A.cost_terms) {
                    const float gx = p[0] - A.goal[0], gy = p[1] - A.goal[1], gz = p[2] - A.goal[2];
                    const float dg = sqrtf(fmaf(gz, gz, fmaf(gy, gy, gx * gx)));
                    cv(0) += fminf(dg, A.cost_radius);
                    if (k == 0) cv(4) = dg;
                    if (k == A.n_steps - 1) cv(2) = L;  // before the last segment
                }
            }
            float fr[3], w, m, F[3];
            float *Fo = CLEAR && A.cost_terms ? F : nullptr;
            if constexpr (APF || PROJ) {
                const float kf = A.rho * k_r;
                float f3[3] = {rec[0], rec[1], rec[2]};
                if constexpr (PROJ) {
                    // f = (|v|^2 S - v B) / |v| with v = v_{k-1}; 0 at rest
                    const float vv = fmaf(v[2], v[2], fmaf(v[1], v[1], v[0] * v[0]));
                    const float inv = vv >= 1e-30f ? rsqrt_approx(vv) : 0.0f;
#pragma unroll
                    for (int d = 0; d < 3; ++d) f3[d] = (vv * rec[d] - v[d] * rec[3]) * inv;
                }
                agent_step_apf<CLEAR>(p, v, kf, k_a, R, A.goal, h, A.dt, A.damping,
                                      A.clear_margin, A.clear_beta, f3, md2, L, pen, minc, m,
                                      Fo);
#pragma unroll
                for (int d = 0; d < 3; ++d) fr[d] = kf * f3[d];
                w = sqrtf(fmaf(f3[2], f3[2], fmaf(f3[1], f3[1], f3[0] * f3[0])));
            } else {
                float g[3], kf;
                w = rec[0];
                agent_step<CLEAR>(p, v, cc, k_r, k_a, R, A.goal, h, A.dt, A.rho, A.damping,
                                  A.clear_margin, A.clear_beta, w, md2, L, pen, minc, m, g, kf,
                                  Fo);
#pragma unroll
                for (int d = 0; d < 3; ++d) fr[d] = kf * g[d];
            }
            if constexpr (CLEAR) {
                if (A.cost_terms) {
                    cv(1) += fmaxf(A.cost_radius - m, 0.0f);
                    if (k >= 2 && k <= A.n_steps - 2) {
                        float s = 0.0f;
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            const float dF = fmaf(-k_a * A.dt, vprev[d],
                                                  fmaf(-A.damping * h, cv(5 + d), fr[d] - cv(8 + d)));
                            s = fmaf(dF, dF, s);
                        }
                        cv(3) += s;
                    }
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        cv(5 + d) = F[d];
                        cv(8 + d) = fr[d];
                    }
                }
            }
            pos[lane] = p[0];
            pos[AG + lane] = p[1];
            pos[2 * AG + lane] = p[2];
            if constexpr (PROJ) {
                vel[lane] = v[0];
                vel[AG + lane] = v[1];
                vel[2 * AG + lane] = v[2];
            }
            if (rank == 0) {
                const int i = a0 + lane;
                if (A.traj) {
                    float *t = A.traj + ((size_t)i * (A.n_steps + 1) + k + 1) * 3;
                    t[0] = p[0];
                    t[1] = p[1];
                    t[2] = p[2];
                }
                if (A.w_trace) A.w_trace[(size_t)i * A.n_steps + k] = w;
                if (A.m_trace) A.m_trace[(size_t)i * A.n_steps + k] = m;
                if (A.f_trace) {
                    float *f = A.f_trace + ((size_t)i * A.n_steps + k) * 3;
                    f[0] = fr[0];
                    f[1] = fr[1];
                    f[2] = fr[2];
                }
            }
        };
        // Exchange warp: half 0 of step k is exchanged while the compute
        // warps work on half 1, and half 1 while they start step k + 1.
        bool ok = true;
        uint32_t epoch = 0;
        uint64_t *xg = nullptr;
        // grid slots of a group: [half][parity][rank][AG] records of SR
        // words; the ensemble kernel spaces groups for the larger record
        constexpr int kGroupRec = EK > 1 ? 6 : EK == 1 ? 4 : 2;
        if constexpr (GRID) {
            epoch = ld_relaxed_u32(A.xctl);
            xg = A.xbuf + static_cast<size_t>(group) * 4 * kGroupRec * C * AG;
        }
        auto xslot = [&](int hh, int par) { return xg + (hh * 2 + par) * SR * C * AG; };
        auto exchange = [&](auto half, int k, int par, float (&rec)[4], float &md2) {
            constexpr int HH = decltype(half)::value;
            constexpr int NA = HH ? H1 : H0, OFF = HH ? H0 : 0;
            if constexpr (APF || PROJ) {
                constexpr int NF = APF ? 3 : 4, RS = APF ? 4 : 6;
                if constexpr (GRID)
                    ok = exchange_half_grid_rec<AG, NA, OFF, NW, CLEAR, NF, RS>(
                        part(HH), xslot(HH, par), slot(HH, par), C, rank, lane, xtag(epoch, k), ok,
                        rec, md2, A.poll_limit);
                else
                    ok = exchange_half_rec<AG, NA, OFF, NW, CLEAR, NF, RS>(
                        part(HH), slot(HH, par), &bar_recv[HH][par], C, rank, lane, k, ok, rec,
                        md2, A.spin_limit);
            } else {
                if constexpr (GRID)
                    ok = exchange_half_grid<AG, NA, OFF, NW, CLEAR>(part(HH), xslot(HH, par),
                                                                    slot(HH, par), C, rank, lane,
                                                                    xtag(epoch, k), ok, rec[0],
                                                                    md2, A.poll_limit);
                else
                    ok = exchange_half<AG, NA, OFF, NW, CLEAR>(part(HH), slot(HH, par),
                                                               &bar_recv[HH][par], C, rank, lane,
                                                               k, ok, rec[0], md2, A.spin_limit);
            }
        };
        // exchange warp h: half h of every step, one phase apart from the
        // other half's warp (the two halves' exchanges overlap)
        auto xloop = [&](auto half) {
            constexpr int HH = decltype(half)::value;
            for (int k = 0; k < A.n_steps; ++k) {
                const int par = k & 1;
                float rec[4] = {0.0f, 0.0f, 0.0f, 0.0f}, md2 = INFINITY;
                named_sync(kPart + HH, kBoth);
                exchange(half, k, par, rec, md2);
                if (mine && lane < na) integrate(k, rec, md2);
                __syncwarp();
                if (k + 1 < A.n_steps) named_arrive(kPos + HH, kBoth);
            }
        };
        if (xh == 0) xloop(std::integral_constant<int, 0>{});
        else xloop(std::integral_constant<int, 1>{});
        if (!ok) raise_error(A.err, GMAPP_DEVERR_TIMEOUT);
        named_sync(kJoin, 32 * kExchWarps);
        if constexpr (GRID) {
            if (xh == 0 && lane == 0) finish_grid(epoch);
        }
        if (rank == 0 && mine && lane < na) {
            const int i = a0 + lane, n = A.n_agents;
            for (int d = 0; d < 3; ++d) {
                A.p_final[d * n + i] = p[d];
                A.v_final[d * n + i] = v[d];
            }
            A.path_len[i] = L;
            if (A.clear_pen) A.clear_pen[i] = pen;
            if (A.min_clear) A.min_clear[i] = minc;
            if constexpr (CLEAR) {
                if (A.cost_terms) {
                    const float rc = A.cost_radius, dh = A.dt * h;
                    A.cost_terms[i] = cv(0) / rc;
                    A.cost_terms[n + i] = cv(1) / rc;
                    A.cost_terms[2 * n + i] = cv(2);
                    A.cost_terms[3 * n + i] = dh * dh * cv(3);
                    A.cost_terms[4 * n + i] = cv(4);
                }
            }
        }
    };
    if constexpr (EK == 0) {
        run(std::integral_constant<int, kMfi>{});
    } else if constexpr (EK == 1) {
        if (kind == kApf) run(std::integral_constant<int, kApf>{});
        else run(std::integral_constant<int, kMfi>{});
    } else {
        if (kind == kApf) run(std::integral_constant<int, kApf>{});
        else if (kind == kProj) run(std::integral_constant<int, kProj>{});
        else run(std::integral_constant<int, kMfi>{});
    }
    // no CTA leaves while another may still deliver into its shared memory
    if constexpr (!GRID) cluster_sync_all();
}

using RolloutKernel = void (*)(const RolloutArgs);

// Instantiation tables (rollout_inst_*.cu).
RolloutKernel rollout_kernel_noclear(int ag, int nt);
RolloutKernel rollout_kernel_clear(int ag, int nt);
RolloutKernel rollout_kernel_grid_noclear(int ag, int nt);
RolloutKernel rollout_kernel_grid_clear(int ag, int nt);
RolloutKernel rollout_kernel_ens_noclear(int ag, int nt);
RolloutKernel rollout_kernel_ens_clear(int ag, int nt);
RolloutKernel rollout_kernel_ens_grid_noclear(int ag, int nt);
RolloutKernel rollout_kernel_ens_grid_clear(int ag, int nt);
RolloutKernel rollout_kernel_ens3_noclear(int ag, int nt);
RolloutKernel rollout_kernel_ens3_clear(int ag, int nt);
RolloutKernel rollout_kernel_ens3_grid_noclear(int ag, int nt);
RolloutKernel rollout_kernel_ens3_grid_clear(int ag, int nt);

// SFU share of the reciprocals: NM of AG agents use rcp.approx, the rest the
// Newton-Raphson path.  Per obstacle pair an SFU agent costs 8 FMA-pipe
// lane-ops and 2 SFU ops, a Newton-Raphson agent 14 and 1; with 128 FMA
// lanes and 16 SFU lanes per SM clock the two pipes balance near NM/AG = 1/2.
// Measured on B300: one SFU agent more than half of an even group (dense
// 50k x 512 x 1000 forward at AG = 14: 11.9 ms with 8 SFU agents, 12.3 ms
// with 7 or 9); odd groups keep (AG + 1) / 2 (the tabletop query at AG = 9:
// 2.67 ms with 5, 2.73 ms with 4).  Tiny groups stay on the SFU, where
// latency matters more.
constexpr int sfu_agents(int ag) { return ag <= 2 ? ag : (ag + 2) / 2; }

}  // namespace gmapp
