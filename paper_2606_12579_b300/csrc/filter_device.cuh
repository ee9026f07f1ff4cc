// Device-side building blocks of the perception filter (Sec. IV-B, Sec. V-A),
// shared by the single-query entry points (filter.cu) and the batched
// queries (batch.cu), so both run the exact same binary32 sequence.
#pragma once

#include <math.h>

#include <algorithm>

#include "gmapp_internal.cuh"

namespace gmapp {
namespace {

constexpr uint32_t kInvalid = 0xFFFFFFFFu;
constexpr int kThreads = 256;
// Bitmap kernels.  A chunk is 32 words (one warp, one word per lane).
// k_bitmap_sums: 256 threads x 16 words = 4096 words (128 chunks) per
// block; per-chunk popcount offsets within the block and the block total.
// k_emit: 1024 words per block, 4 chunks per warp, warps independent (no
// block barrier), so empty stretches cost one load and a dense stretch (a
// table plane fills whole words) spreads over many warps.
constexpr int kBmThreads = 256;
constexpr int kChunkWords = 32;
constexpr int kChunksPerWarp = 4;  // batched paths; a single cloud uses 1 (more warps)
constexpr int kWordsPerBlock = kBmThreads * kChunksPerWarp;  // batched emit block: 1024 words
constexpr int kWordsPerSumBlock = 4096;
constexpr int kChunksPerSumBlock = kWordsPerSumBlock / kChunkWords;
static_assert(kWordsPerSumBlock % kWordsPerBlock == 0, "emit blocks tile the sum blocks");
// min_pts > 1 compaction: 4 temporary entries per thread.
constexpr int kKeepPerBlock = kThreads * 4;

struct FilterArgs {
    float T[12];
    float lo[3];
    float voxel;
    float dimf[3];
    uint32_t nx, ny, nz;
    uint32_t *err;  // device error word (index checks of the bounds-checked build)
};

// The correctly rounded quotient x / voxel from the correctly rounded
// reciprocal y = RN(1 / voxel) by Markstein's theorem (P. Markstein,
// "Computation of elementary functions on the IBM RISC System/6000
// processor", IBM J. Res. Dev. 34(1), 1990): when q is within one ulp of
// x / voxel, r = x - q voxel is exact (one FMA) and RN(q + r y) = RN(x /
// voxel).  q0 = RN(x y) may be up to 1.5 ulp off (the errors of y and of
// the product add), so one correction first makes it faithful (error
// below 1/2 ulp plus a few units of 2^-46) and a second one, now under the
// theorem, rounds correctly: one multiply and four FMAs.  Outside the
// normal range (a quotient that overflows becomes NaN, a subnormal one may
// differ in its last bit) the crop and floor decisions are those of the
// IEEE quotient: an overflowing quotient lies beyond the grid, a tiny one
// floors to 0 with its sign kept.
__device__ __forceinline__ float voxel_quotient(float x, float voxel, float y) {
    const float q0 = __fmul_rn(x, y);
    const float q1 = __fmaf_rn(__fmaf_rn(-q0, voxel, x), y, q0);
    return __fmaf_rn(__fmaf_rn(-q1, voxel, x), y, q1);
}

// One point -> its linear voxel key, or kInvalid.  Exact binary32 sequence,
// no contraction: w = ((T0 x + T1 y) + T2 z) + T3; q = RN((w - lo) / voxel);
// inv_voxel = RN(1 / voxel).
__device__ __forceinline__ uint32_t voxel_key(float x, float y, float z, const FilterArgs &A,
                                              float inv_voxel) {
    if (!(isfinite(x) && isfinite(y) && isfinite(z))) return kInvalid;
    uint32_t idx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float t0 = __fmul_rn(A.T[4 * a + 0], x);
        float t1 = __fmul_rn(A.T[4 * a + 1], y);
        float t2 = __fmul_rn(A.T[4 * a + 2], z);
        float w = __fadd_rn(__fadd_rn(__fadd_rn(t0, t1), t2), A.T[4 * a + 3]);
        float q = voxel_quotient(__fsub_rn(w, A.lo[a]), A.voxel, inv_voxel);
        if (!(q >= 0.0f && q < A.dimf[a])) return kInvalid;
        idx[a] = static_cast<uint32_t>(q);  // q >= 0: truncation is floor
    }
    return (idx[2] * A.ny + idx[1]) * A.nx + idx[0];
}

// Centre of cell (ix, iy, iz): lo + ((float)i + 0.5) voxel per axis, exact
// binary32 sequence.
__device__ __forceinline__ void cell_centre(uint32_t ix, uint32_t iy, uint32_t iz,
                                            const FilterArgs &A, float &cx, float &cy, float &cz) {
    cx = __fadd_rn(A.lo[0], __fmul_rn(__fadd_rn(static_cast<float>(ix), 0.5f), A.voxel));
    cy = __fadd_rn(A.lo[1], __fmul_rn(__fadd_rn(static_cast<float>(iy), 0.5f), A.voxel));
    cz = __fadd_rn(A.lo[2], __fmul_rn(__fadd_rn(static_cast<float>(iz), 0.5f), A.voxel));
}

__device__ __forceinline__ void voxel_centre(uint32_t key, const FilterArgs &A, float &cx,
                                             float &cy, float &cz) {
    const uint32_t r = key / A.nx;
    const uint32_t ix = key - r * A.nx;
    const uint32_t iz = r / A.ny;
    const uint32_t iy = r - iz * A.ny;
    cell_centre(ix, iy, iz, A, cx, cy, cz);
}

__global__ void k_zero(uint4 *words, int64_t n_vec, uint32_t *counters, int n_counters) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < n_vec; i += stride) words[i] = make_uint4(0, 0, 0, 0);
    if (blockIdx.x == 0 && threadIdx.x < n_counters) counters[threadIdx.x] = 0;
}

// OR a run of bits into the bitmap, merging consecutive points of one thread
// that fall into the same 32-cell word.
struct BitMerge {
    uint32_t word = kInvalid, bits = 0;
    __device__ __forceinline__ void add(uint32_t key, uint32_t *bitmap) {
        if (key == kInvalid) return;
        uint32_t w = key >> 5, b = 1u << (key & 31);
        if (w == word) {
            bits |= b;
            return;
        }
        flush(bitmap);
        word = w;
        bits = b;
    }
    __device__ __forceinline__ void flush(uint32_t *bitmap) {
        if (word != kInvalid) atomicOr(&bitmap[word], bits);
        word = kInvalid;
    }
};

// Points -> keys (4 points = 48 B per thread per iteration: three 16-byte loads).
__device__ __forceinline__ void keys_range(const float *__restrict__ xyz, int64_t n,
                                                    FilterArgs A, uint32_t *__restrict__ keys,
                                                    uint32_t *__restrict__ bitmap,
                                           int64_t blk, int64_t nblk) {
    const int64_t n4 = n / 4;
    const int64_t stride = nblk * (int64_t)kThreads;
    const float inv_voxel = __frcp_rn(A.voxel);
    // every later bitmap word, rank and output index derives from a key:
    // the bounds-checked build checks each key against the grid
    const int64_t cells = static_cast<int64_t>(A.nx) * A.ny * A.nz;
    auto chk = [&](uint32_t k) {
        return k == kInvalid || bc_ok(k, cells, A.err) ? k : kInvalid;
    };
#pragma unroll 2
    for (int64_t g = blk * (int64_t)kThreads + threadIdx.x; g < n4; g += stride) {
        const float4 *src = reinterpret_cast<const float4 *>(xyz) + 3 * g;
        float4 a0 = __ldcs(src), a1 = __ldcs(src + 1), a2 = __ldcs(src + 2);
        uint4 k;
        k.x = chk(voxel_key(a0.x, a0.y, a0.z, A, inv_voxel));
        k.y = chk(voxel_key(a0.w, a1.x, a1.y, A, inv_voxel));
        k.z = chk(voxel_key(a1.z, a1.w, a2.x, A, inv_voxel));
        k.w = chk(voxel_key(a2.y, a2.z, a2.w, A, inv_voxel));
        reinterpret_cast<uint4 *>(keys)[g] = k;
        BitMerge m;
        m.add(k.x, bitmap);
        m.add(k.y, bitmap);
        m.add(k.z, bitmap);
        m.add(k.w, bitmap);
        m.flush(bitmap);
    }
    // ragged tail (n % 4 points)
    int64_t t = 4 * n4 + blk * (int64_t)kThreads + threadIdx.x;
    if (t < n) {
        uint32_t k = chk(voxel_key(xyz[3 * t], xyz[3 * t + 1], xyz[3 * t + 2], A, inv_voxel));
        keys[t] = k;
        if (k != kInvalid) atomicOr(&bitmap[k >> 5], 1u << (k & 31));
    }
}

__global__ void __launch_bounds__(kThreads) k_keys(const float *__restrict__ xyz, int64_t n,
                                                    FilterArgs A, uint32_t *__restrict__ keys,
                                                    uint32_t *__restrict__ bitmap) {
    keys_range(xyz, n, A, keys, bitmap, blockIdx.x, gridDim.x);
}

// Block-wide exclusive scan of one uint32 per thread (NTH threads).
template <int NTH>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *warp_tot,
                                                         uint32_t &block_total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = lane < NTH / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < NTH / 32) warp_tot[lane] = t;  // inclusive
    }
    __syncthreads();
    uint32_t before = warp ? warp_tot[warp - 1] : 0;
    block_total = warp_tot[NTH / 32 - 1];
    __syncthreads();
    return before + x - v;
}

// Exclusive scan of `n` block sums by ONE block (the last one to finish);
// writes offsets[] and returns the grand total to thread 0.
template <int NTH>
__device__ uint32_t scan_block_sums(const uint32_t *sums, uint32_t *offsets, int64_t n,
                                    uint32_t *warp_tot) {
    const int64_t per = (n + NTH - 1) / NTH;
    const int64_t b0 = threadIdx.x * per;
    uint32_t local = 0;
    for (int64_t i = b0; i < b0 + per && i < n; ++i) local += __ldcg(&sums[i]);
    uint32_t total;
    uint32_t run = block_exclusive_scan<NTH>(local, warp_tot, total);
    for (int64_t i = b0; i < b0 + per && i < n; ++i) {
        uint32_t s = __ldcg(&sums[i]);
        offsets[i] = run;
        run += s;
    }
    return total;
}

// Per block of kWordsPerSumBlock bitmap words: each 32-word chunk's
// exclusive popcount prefix within the block (chunk_off) and the block
// total.  The last block to finish scans all block totals into offsets and
// publishes the total number of occupied voxels.
// With `list` (and its counter *n_list), the index of every occupied chunk
// is also appended to list (in no particular order), so a later pass can
// visit only those.
__device__ __forceinline__ void bitmap_sums_block(const uint32_t *__restrict__ bitmap,
                                                  uint32_t *chunk_off, uint32_t *sums,
                                                  uint32_t *offsets, uint32_t *counter,
                                                  uint32_t *n_occ, int64_t blk, int64_t nblk,
                                                  uint32_t *list = nullptr,
                                                  uint32_t *n_list = nullptr) {
    __shared__ uint32_t warp_tot[kBmThreads / 32];
    __shared__ bool is_last;
    const int t = threadIdx.x;
    const uint4 *src = reinterpret_cast<const uint4 *>(bitmap + blk * kWordsPerSumBlock + 16 * t);
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint4 w = src[k];
        c += __popc(w.x) + __popc(w.y) + __popc(w.z) + __popc(w.w);
    }
    // a chunk is two consecutive threads: the even one carries its sum
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    if (list) {
        const bool occ = !(t & 1) && c != 0u;
        const uint32_t m = __ballot_sync(0xffffffffu, occ);
        uint32_t at = 0;
        if ((t & 31) == 0 && m) at = atomicAdd(n_list, static_cast<uint32_t>(__popc(m)));
        at = __shfl_sync(0xffffffffu, at, 0);
        if (occ)
            list[at + __popc(m & ((1u << (t & 31)) - 1u))] =
                static_cast<uint32_t>(blk * kChunksPerSumBlock + (t >> 1));
    }
    uint32_t tot;
    const uint32_t excl = block_exclusive_scan<kBmThreads>((t & 1) ? 0u : c, warp_tot, tot);
    if (!(t & 1)) chunk_off[blk * kChunksPerSumBlock + (t >> 1)] = excl;
    if (t == 0) {
        sums[blk] = tot;
        __threadfence();
        is_last = atomicAdd(counter, 1u) == nblk - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    uint32_t total = scan_block_sums<kBmThreads>(sums, offsets, nblk, warp_tot);
    if (t == 0) {
        *n_occ = total;
        *counter = 0;
    }
}

__global__ void __launch_bounds__(kBmThreads) k_bitmap_sums(const uint32_t *__restrict__ bitmap,
                                                            uint32_t *chunk_off, uint32_t *sums,
                                                            uint32_t *offsets, uint32_t *counter,
                                                            uint32_t *n_occ) {
    bitmap_sums_block(bitmap, chunk_off, sums, offsets, counter, n_occ, blockIdx.x, gridDim.x);
}

struct EmitOut {
    uint32_t *keys, *counts, *rep;
    float *x, *y, *z;  // NULL when centres are computed later (min_pts > 1)
    int64_t cap;
};

// Per word: rank of its first set bit = sum-block offset + chunk offset +
// in-chunk prefix (a warp scan), stored with the word itself as
// pw[w] = (rank, bits) for k_count (occupied words only: no point maps to
// an empty one).  Every set bit becomes one output entry (key, centre,
// count = 0, rep = ~0).  With `zero`, the occupied words are
// cleared after use (library-owned scratch stays ready for the next run
// without a clearing launch).  CPW: 32-word chunks per warp (warps independent).
template <int CPW>
__device__ __forceinline__ void emit_block(uint32_t *__restrict__ bitmap,
                                           const uint32_t *__restrict__ offsets,
                                           const uint32_t *__restrict__ chunk_off,
                                           uint2 *__restrict__ pw, FilterArgs A, EmitOut o,
                                           int64_t blk, bool zero) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t c0 = (blk * (kBmThreads / 32) + warp) * CPW;
    uint32_t w[CPW];
#pragma unroll
    for (int j = 0; j < CPW; ++j) w[j] = bitmap[(c0 + j) * kChunkWords + lane];
#pragma unroll 1
    for (int j = 0; j < CPW; ++j) {
        if (!__ballot_sync(0xffffffffu, w[j] != 0u)) continue;
        const int64_t c = c0 + j;
        const uint32_t cnt = __popc(w[j]);
        uint32_t x = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        const uint32_t pre = offsets[c / kChunksPerSumBlock] + chunk_off[c] + x - cnt;
        const int64_t wv = c * kChunkWords + lane;
        if (w[j]) {
            pw[wv] = make_uint2(pre, w[j]);
            if (zero) bitmap[wv] = 0u;
        }
        // lane per bit: for each occupied word (warp-uniform loop), lane b
        // writes the entry of bit b, so the ranks of a word are consecutive
        // and its stores coalesce; each lane first finds the cell
        // coordinates of its own word's first cell (one division chain per
        // word), which the loop broadcasts
        uint32_t ix0 = 0, iy0 = 0, iz0 = 0;
        if (w[j]) {
            const uint32_t key0 = static_cast<uint32_t>(wv) * 32u;
            const uint32_t q = key0 / A.nx;
            ix0 = key0 - q * A.nx;
            iz0 = q / A.ny;
            iy0 = q - iz0 * A.ny;
        }
        const uint32_t below = (1u << lane) - 1u;
        uint32_t nz = __ballot_sync(0xffffffffu, w[j] != 0u);
        while (nz) {
            const int i = __ffs(nz) - 1;
            nz &= nz - 1;
            const uint32_t bits = __shfl_sync(0xffffffffu, w[j], i);
            const uint32_t p0 = __shfl_sync(0xffffffffu, pre, i);
            const uint32_t bx = __shfl_sync(0xffffffffu, ix0, i);
            const uint32_t by = __shfl_sync(0xffffffffu, iy0, i);
            const uint32_t bz = __shfl_sync(0xffffffffu, iz0, i);
            if ((bits >> lane) & 1u) {
                const uint32_t rank = p0 + __popc(bits & below);
                if (rank < o.cap) {
                    o.keys[rank] = static_cast<uint32_t>((c * kChunkWords + i) * 32 + lane);
                    o.counts[rank] = 0;
                    o.rep[rank] = kInvalid;
                    if (o.x) {
                        uint32_t ix = bx + lane, iy = by, iz = bz;
                        while (ix >= A.nx) {  // the word crosses a row (and plane) end
                            ix -= A.nx;
                            if (++iy == A.ny) {
                                iy = 0;
                                ++iz;
                            }
                        }
                        float cx, cy, cz;
                        cell_centre(ix, iy, iz, A, cx, cy, cz);
                        o.x[rank] = cx;
                        o.y[rank] = cy;
                        o.z[rank] = cz;
                    }
                }
            }
        }
    }
}

// With n_out set (min_pts == 1), block 0 also publishes N_O = the number of
// occupied voxels (and a capacity error when it exceeds o.cap), which the
// later kernels of the stream read on the device.
__global__ void __launch_bounds__(kBmThreads) k_emit(uint32_t *__restrict__ bitmap,
                                                     const uint32_t *__restrict__ offsets,
                                                     const uint32_t *__restrict__ chunk_off,
                                                     uint2 *__restrict__ pw, FilterArgs A,
                                                     EmitOut o, const uint32_t *n_occ,
                                                     int32_t *n_out, uint32_t *err) {
    if (n_out && blockIdx.x == 0 && threadIdx.x == 0) {
        const uint32_t t = *n_occ;
        *n_out = static_cast<int32_t>(t);
        if (t > o.cap) raise_error(err, GMAPP_DEVERR_CAPACITY);
    }
    emit_block<1>(bitmap, offsets, chunk_off, pw, A, o, blockIdx.x, false);
}

// Accumulate count and smallest index of consecutive points with one rank.
struct RankMerge {
    uint32_t rank = kInvalid, cnt = 0, first = 0;
    __device__ __forceinline__ void add(uint32_t r, uint32_t idx, uint32_t *counts, uint32_t *rep) {
        if (r == rank) {
            ++cnt;
            return;
        }
        flush(counts, rep);
        rank = r;
        cnt = 1;
        first = idx;
    }
    __device__ __forceinline__ void flush(uint32_t *counts, uint32_t *rep) {
        if (rank != kInvalid) {
            atomicAdd(&counts[rank], cnt);
            atomicMin(&rep[rank], first);
        }
        rank = kInvalid;
    }
};

__device__ __forceinline__ uint32_t rank_of(uint32_t key, const uint2 *pw, int64_t cap) {
    if (key == kInvalid) return kInvalid;
    const uint2 p = __ldg(&pw[key >> 5]);  // (rank of the word's first bit, bits)
    const uint32_t r = p.x + __popc(p.y & ((1u << (key & 31)) - 1u));
    return r < cap ? r : kInvalid;
}

// Point t of the range has the index idx0 + t (several sensors share one
// index space).
__device__ __forceinline__ void count_range(const uint32_t *__restrict__ keys, int64_t n,
                                            const uint2 *__restrict__ pw, uint32_t *counts,
                                            uint32_t *rep, int64_t cap, int64_t blk,
                                            int64_t nblk, uint32_t idx0 = 0) {
    const int64_t n4 = n / 4;
    const int64_t stride = nblk * (int64_t)kThreads;
#pragma unroll 2
    for (int64_t g = blk * (int64_t)kThreads + threadIdx.x; g < n4; g += stride) {
        uint4 k = __ldcs(reinterpret_cast<const uint4 *>(keys) + g);
        RankMerge m;
        uint32_t i0 = idx0 + static_cast<uint32_t>(4 * g);
        uint32_t r;
        if ((r = rank_of(k.x, pw, cap)) != kInvalid) m.add(r, i0, counts, rep);
        if ((r = rank_of(k.y, pw, cap)) != kInvalid) m.add(r, i0 + 1, counts, rep);
        if ((r = rank_of(k.z, pw, cap)) != kInvalid) m.add(r, i0 + 2, counts, rep);
        if ((r = rank_of(k.w, pw, cap)) != kInvalid) m.add(r, i0 + 3, counts, rep);
        m.flush(counts, rep);
    }
    int64_t t = 4 * n4 + blk * (int64_t)kThreads + threadIdx.x;
    if (t < n) {
        uint32_t r = rank_of(keys[t], pw, cap);
        if (r != kInvalid) {
            atomicAdd(&counts[r], 1u);
            atomicMin(&rep[r], idx0 + static_cast<uint32_t>(t));
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_count(const uint32_t *__restrict__ keys, int64_t n,
                                                    const uint2 *__restrict__ pw, uint32_t *counts,
                                                    uint32_t *rep, int64_t cap, uint32_t idx0) {
    count_range(keys, n, pw, counts, rep, cap, blockIdx.x, gridDim.x, idx0);
}

// min_pts > 1: per block of 1024 temporary entries, how many pass; last
// block scans and publishes the kept total.
__global__ void __launch_bounds__(kThreads) k_keep_sums(const uint32_t *__restrict__ counts,
                                                        const uint32_t *__restrict__ n_occ,
                                                        uint32_t min_pts, uint32_t *sums,
                                                        uint32_t *offsets, uint32_t *counter,
                                                        int32_t *n_out, int64_t cap,
                                                        uint32_t *err) {
    __shared__ uint32_t warp_tot[kThreads / 32];
    __shared__ bool is_last;
    const uint32_t n = *n_occ;
    uint32_t c = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t i = (blockIdx.x * kThreads + threadIdx.x) * 4 + j;  // kKeepPerBlock per block
        if (i < n && counts[i] >= min_pts) ++c;
    }
    uint32_t tot;
    block_exclusive_scan<kThreads>(c, warp_tot, tot);
    if (threadIdx.x == 0) {
        sums[blockIdx.x] = tot;
        __threadfence();
        is_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    uint32_t total = scan_block_sums<kThreads>(sums, offsets, gridDim.x, warp_tot);
    if (threadIdx.x == 0) {
        *n_out = static_cast<int32_t>(total);
        if (total > cap) raise_error(err, GMAPP_DEVERR_CAPACITY);
        *counter = 0;
    }
}

__global__ void __launch_bounds__(kThreads) k_keep_emit(const uint32_t *__restrict__ tkeys,
                                                        const uint32_t *__restrict__ tcounts,
                                                        const uint32_t *__restrict__ trep,
                                                        const uint32_t *__restrict__ n_occ,
                                                        const uint32_t *__restrict__ offsets,
                                                        uint32_t min_pts, FilterArgs A,
                                                        EmitOut o) {
    __shared__ uint32_t warp_tot[kThreads / 32];
    const uint32_t n = *n_occ;
    bool keep[4];
    uint32_t c = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t i = (blockIdx.x * kThreads + threadIdx.x) * 4 + j;
        keep[j] = i < n && tcounts[i] >= min_pts;
        c += keep[j];
    }
    uint32_t tot;
    uint32_t rank = offsets[blockIdx.x] + block_exclusive_scan<kThreads>(c, warp_tot, tot);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (!keep[j]) continue;
        uint32_t i = (blockIdx.x * kThreads + threadIdx.x) * 4 + j;
        if (rank < o.cap) {
            uint32_t key = tkeys[i];
            o.keys[rank] = key;
            o.counts[rank] = tcounts[i];
            o.rep[rank] = trep[i];
            float cx, cy, cz;
            voxel_centre(key, A, cx, cy, cz);
            o.x[rank] = cx;
            o.y[rank] = cy;
            o.z[rank] = cz;
        }
        ++rank;
    }
}

// Workspace layout (all sections 256-byte aligned).
struct Layout {
    int64_t n_words;   // bitmap words, padded to whole k_bitmap_sums blocks
    int64_t n_blocks;  // batched emit blocks (kWordsPerBlock words)
    int64_t n_sblocks; // k_bitmap_sums blocks (4096 words)
    int64_t n_tmp;     // temporary entries (min_pts > 1), padded to kKeepPerBlock
    int64_t n_tblocks; // k_keep_* blocks
    size_t off_bitmap, off_pw, off_chunk, off_sums, off_offsets, off_counters, off_keys;
    size_t off_tkeys, off_tcounts, off_trep, off_tsums, off_toffsets;
    size_t total;
};

bool valid_workspace(const gmapp_workspace *ws) {
    if (!ws) return false;
    if (!(ws->voxel > 0.0f) || !isfinite(ws->voxel) || ws->min_pts < 1) return false;
    uint64_t cells = 1;
    for (int a = 0; a < 3; ++a) {
        if (ws->dims[a] < 1 || ws->dims[a] > (1 << 24) || !isfinite(ws->lo[a])) return false;
        cells *= static_cast<uint64_t>(ws->dims[a]);
    }
    return cells < 0xFFFFFFFFull;
}

Layout layout(int64_t n_raw, const gmapp_workspace *ws) {
    Layout L{};
    uint64_t cells = (uint64_t)ws->dims[0] * ws->dims[1] * ws->dims[2];
    int64_t words = static_cast<int64_t>((cells + 31) / 32);
    L.n_sblocks = (words + kWordsPerSumBlock - 1) / kWordsPerSumBlock;
    L.n_words = L.n_sblocks * kWordsPerSumBlock;  // a multiple of kWordsPerBlock too
    L.n_blocks = L.n_words / kWordsPerBlock;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    L.off_bitmap = take(L.n_words * 4);
    L.off_pw = take(L.n_words * 8);
    L.off_chunk = take(L.n_words / kChunkWords * 4);
    L.off_sums = take(L.n_sblocks * 4);
    L.off_offsets = take(L.n_sblocks * 4);
    L.off_counters = take(64);
    L.off_keys = take(align_up(n_raw > 0 ? n_raw : 1, 4) * 4);
    if (ws->min_pts > 1) {
        int64_t nt = std::min<int64_t>(n_raw, static_cast<int64_t>(cells));
        L.n_tblocks = std::max<int64_t>(1, (nt + kKeepPerBlock - 1) / kKeepPerBlock);
        L.n_tmp = L.n_tblocks * kKeepPerBlock;
        L.off_tkeys = take(L.n_tmp * 4);
        L.off_tcounts = take(L.n_tmp * 4);
        L.off_trep = take(L.n_tmp * 4);
        L.off_tsums = take(L.n_tblocks * 4);
        L.off_toffsets = take(L.n_tblocks * 4);
    }
    L.total = off;
    return L;
}


}  // namespace
}  // namespace gmapp
