// filter_cloud_batch: the perception filter of Sec. IV-B / Sec. V-A for many
// clouds at once (a stream of depth frames, or several sensors).
//
// A single frame is a few MB, far less than a launch needs to approach HBM
// bandwidth, and a whole stream's scratch is far larger than L2.  So the
// jobs are filtered in WAVES whose touched scratch fits in L2 (at most 48 MB:
// about 15 tabletop frames), each wave through three launches, and
// consecutive waves go round-robin to three streams (the caller's and two
// of the batch's own), so the latency-bound passes of three waves overlap.
// Each stream owns one set of scratch slots, reused wave after wave.
//
// Each slot holds, besides the bitmap over the grid, one 8-byte record per
// grid cell (point count, complement of the smallest point index).  The
// records start at zero and the emit pass puts every record it reads back
// to zero, so no pass clears them and only occupied cells are ever touched.
//
//   kf_points 8 points per thread and iteration (a warp's 256 points come
//             in by coalesced streaming loads through shared memory): key
//             per point; per run of equal keys one reduction into the
//             cell's count and one into its smallest index; the bitmap bits
//             gathered per warp and word in shared memory, one reduction per
//             word and tile (reductions return nothing: the thread never
//             waits on them)
//   kf_sums   per-block (and per-chunk) popcounts; each job's last block
//             scans its block sums; the occupied 32-word chunks are appended
//             to the job's chunk list
//   kf_emit   persistent over the wave's occupied chunks (empty ones cost
//             nothing): ranks of a chunk's words (warp scan), its set bits
//             compacted in shared memory, then written 32 obstacles at a
//             time (coalesced: key, count, smallest index, centre, the
//             records read and cleared); publishes each job's N_O and
//             clears the bitmap words behind it
//
// Every job's S_W is bit-identical to filter_cloud on the same cloud (same
// key and centre arithmetic, same ranks; a count is a sum and the smallest
// index a minimum, whatever the order of the reductions).
#include <math.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "filter_device.cuh"

namespace gmapp {
namespace {

constexpr int kPointsPerThread = 8;      // kf_points: points per thread per iteration
constexpr size_t kWaveL2Bytes = size_t(48) << 20;  // L2-resident scratch per wave
constexpr int kWaveStreams = 3;  // waves in flight: streams (the caller's + side ones), slot sets

// Division by an invariant divisor d by multiplication (T. Granlund and P. L.
// Montgomery, "Division by invariant integers using multiplication", PLDI
// 1994, Sec. 4, unsigned case): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, t = mulhi(m, n) and
// q = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0) equals floor(n / d) for
// every 32-bit n.
struct DivMagic {
    uint32_t m, s1, s2;
};

DivMagic div_magic(uint32_t d) {
    int l = 0;
    while ((uint64_t(1) << l) < d) ++l;
    const uint64_t m = ((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1;
    return DivMagic{static_cast<uint32_t>(m), static_cast<uint32_t>(std::min(l, 1)),
                    static_cast<uint32_t>(std::max(l - 1, 0))};
}

__device__ __forceinline__ uint32_t div_by(uint32_t n, DivMagic g) {
    const uint32_t t = __umulhi(g.m, n);
    return (t + ((n - t) >> g.s1)) >> g.s2;
}

struct FilterJob {
    const float *xyz;
    int64_t n_raw;
    FilterArgs fa;
    DivMagic dx, dy;  // division by dims_x, dims_y (key -> cell coordinates)
    uint32_t *bitmap, *chunk, *sums, *offsets, *counters;
    uint32_t *chunk_list;  // occupied 32-word chunks (kf_sums appends, kf_emit visits);
                           // their number in counters[3]
    uint32_t n_chunks;     // chunks of the bitmap (the list's capacity)
    uint2 *rec;            // per grid cell: (points, ~smallest point index); zero when unused
    int32_t pt_blk0, pt_nblk, sb_blk0, sb_nblk;  // point-pass and sums blocks
    EmitOut o;
    int32_t *n_out;
};

// One point -> its linear voxel key, or kInvalid: the binary32 sequence of
// voxel_key without the explicit finiteness test.  A non-finite coordinate
// makes every transformed coordinate NaN or infinite (0 x inf is NaN, any
// other product is infinite or NaN), and a NaN or infinite quotient fails
// the range test 0 <= q < dims, so the same points are dropped.
__device__ __forceinline__ uint32_t key_of(float x, float y, float z, const FilterArgs &A,
                                           float inv_voxel) {
    uint32_t idx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float t0 = __fmul_rn(A.T[4 * a + 0], x);
        const float t1 = __fmul_rn(A.T[4 * a + 1], y);
        const float t2 = __fmul_rn(A.T[4 * a + 2], z);
        const float w = __fadd_rn(__fadd_rn(__fadd_rn(t0, t1), t2), A.T[4 * a + 3]);
        const float q = voxel_quotient(__fsub_rn(w, A.lo[a]), A.voxel, inv_voxel);
        if (!(q >= 0.0f && q < A.dimf[a])) return kInvalid;
        idx[a] = static_cast<uint32_t>(q);
    }
    return (idx[2] * A.ny + idx[1]) * A.nx + idx[0];
}

// Reductions into global memory that return nothing (the issuing thread
// never waits for them).
__device__ __forceinline__ void red_add(uint32_t *p, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_max(uint32_t *p, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.max.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_or(uint32_t *p, uint32_t v) {
    asm volatile("red.relaxed.gpu.global.or.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// A warp's words of the bitmap, gathered in shared memory while it keys
// its 256 points (64 slots, open addressing on the word index): each word
// then goes to the bitmap in one reduction per tile instead of one per run;
// a word that finds no slot within 8 probes goes to the bitmap at once.
constexpr int kWordSlots = 64;
struct WordTable {
    uint32_t *key, *bits;  // this warp's slots; key kInvalid = empty
    __device__ __forceinline__ void add(uint32_t word, uint32_t b, uint32_t *bitmap) {
        uint32_t h = (word * 2654435761u) >> 26;
        for (int probe = 0; probe < 8; ++probe) {
            const uint32_t old = atomicCAS(&key[h], kInvalid, word);
            if (old == kInvalid || old == word) {
                atomicOr(&bits[h], b);
                return;
            }
            h = (h + 1) & (kWordSlots - 1);
        }
        red_or(&bitmap[word], b);
    }
    // the whole warp: every gathered word to the bitmap, slots emptied
    __device__ __forceinline__ void flush(uint32_t *bitmap, int lane) {
        __syncwarp();
#pragma unroll
        for (int s = lane; s < kWordSlots; s += 32) {
            const uint32_t w = key[s];
            if (w != kInvalid) {
                red_or(&bitmap[w], bits[s]);
                key[s] = kInvalid;
                bits[s] = 0u;
            }
        }
        __syncwarp();
    }
};

// Bits of one thread's consecutive points merged while they share a word.
struct BitMerge8 {
    uint32_t word = kInvalid, bits = 0;
    __device__ __forceinline__ void add(uint32_t key, WordTable &t, uint32_t *bitmap) {
        if (key == kInvalid) return;
        const uint32_t w = key >> 5, b = 1u << (key & 31);
        if (w == word) {
            bits |= b;
            return;
        }
        flush(t, bitmap);
        word = w;
        bits = b;
    }
    __device__ __forceinline__ void flush(WordTable &t, uint32_t *bitmap) {
        if (word != kInvalid) t.add(word, bits, bitmap);
        word = kInvalid;
    }
};

// Runs of equal keys among one thread's consecutive points: one reduction
// into the cell's count (the run's length) and one into its smallest index
// (the run's first point: a thread visits its points in ascending order),
// the index stored complemented so that zero means "none" and the largest
// complement is the smallest index.
struct CellMerge {
    uint32_t key = kInvalid, n = 0, first = 0;
    __device__ __forceinline__ void add(uint32_t k, uint32_t idx, uint2 *rec) {
        if (k == kInvalid) return;
        if (k == key) {
            ++n;
            return;
        }
        flush(rec);
        key = k;
        n = 1;
        first = idx;
    }
    __device__ __forceinline__ void flush(uint2 *rec) {
        if (key == kInvalid) return;
        red_add(&rec[key].x, n);
        red_max(&rec[key].y, ~first);
        key = kInvalid;
    }
};

// Points -> keys -> bitmap bits and cell records: 8 consecutive points per
// thread and iteration, bits merged per thread by word and then per warp in
// its word table, records by run of equal keys.  A warp's 256 points (3 KB) come in as six coalesced 16-byte
// loads per lane (512 contiguous bytes per instruction) and are handed to
// their threads through the warp's tile in shared memory.
__global__ void __launch_bounds__(kThreads, 4) kf_points(const FilterJob *J, const int32_t *pt_map,
                                                      int32_t blk0) {
    __shared__ float4 tile[kThreads / 32][6 * 32];
    __shared__ uint32_t wkey[kThreads / 32][kWordSlots], wbits[kThreads / 32][kWordSlots];
    const int lane = threadIdx.x & 31;
    float4 *tw = tile[threadIdx.x >> 5];
    WordTable table{wkey[threadIdx.x >> 5], wbits[threadIdx.x >> 5]};
    for (int s = lane; s < kWordSlots; s += 32) {
        table.key[s] = kInvalid;
        table.bits[s] = 0u;
    }
    __syncwarp();
    const int32_t gb = blockIdx.x + blk0;
    const FilterJob &Q = J[pt_map[gb]];
    const FilterArgs A = Q.fa;
    const int64_t n = Q.n_raw, n8 = n / kPointsPerThread;
    const int64_t blk = gb - Q.pt_blk0, stride = static_cast<int64_t>(Q.pt_nblk) * kThreads;
    const float inv = __frcp_rn(A.voxel);
    // the job's pointers in registers: the reductions below are memory
    // clobbers, after which fields read through Q would be loaded again
    uint32_t *__restrict__ bitmap = Q.bitmap;
    uint2 *__restrict__ rec = Q.rec;
    const float *__restrict__ xyz = Q.xyz;
    const int64_t cells = static_cast<int64_t>(A.nx) * A.ny * A.nz;
    auto chk = [&](uint32_t k) { return k == kInvalid || bc_ok(k, cells, A.err) ? k : kInvalid; };
    if (blk == 0 && threadIdx.x == 0) Q.counters[3] = 0;  // kf_sums refills the chunk list
    for (int64_t gw = blk * kThreads + (threadIdx.x & ~31); gw < n8; gw += stride) {
        // the warp's groups gw .. gw + 31 (the last warp of a job may hold fewer)
        const float4 *src = reinterpret_cast<const float4 *>(xyz) + 6 * gw;
        const int64_t lim = 6 * (n8 - gw);
        float4 v[6];
#pragma unroll
        for (int j = 0; j < 6; ++j)
            if (32 * j + lane < lim) v[j] = __ldcs(src + 32 * j + lane);
#pragma unroll
        for (int j = 0; j < 6; ++j) tw[32 * j + lane] = v[j];
        __syncwarp();
        const float4 a0 = tw[6 * lane], a1 = tw[6 * lane + 1], a2 = tw[6 * lane + 2];
        const float4 a3 = tw[6 * lane + 3], a4 = tw[6 * lane + 4], a5 = tw[6 * lane + 5];
        __syncwarp();
        const int64_t g = gw + lane;
        if (g < n8) {
            uint32_t k[8];
            k[0] = chk(key_of(a0.x, a0.y, a0.z, A, inv));
            k[1] = chk(key_of(a0.w, a1.x, a1.y, A, inv));
            k[2] = chk(key_of(a1.z, a1.w, a2.x, A, inv));
            k[3] = chk(key_of(a2.y, a2.z, a2.w, A, inv));
            k[4] = chk(key_of(a3.x, a3.y, a3.z, A, inv));
            k[5] = chk(key_of(a3.w, a4.x, a4.y, A, inv));
            k[6] = chk(key_of(a4.z, a4.w, a5.x, A, inv));
            k[7] = chk(key_of(a5.y, a5.z, a5.w, A, inv));
            const uint32_t i0 = static_cast<uint32_t>(kPointsPerThread * g);
            BitMerge8 m;
            CellMerge c;
#pragma unroll
            for (int i = 0; i < kPointsPerThread; ++i) {
                m.add(k[i], table, bitmap);
                c.add(k[i], i0 + i, rec);
            }
            m.flush(table, bitmap);
            c.flush(rec);
        }
        table.flush(bitmap, lane);
    }
    // ragged tail (n % 8 points): the first threads of the job's first block
    const int64_t t = kPointsPerThread * n8 + blk * kThreads + threadIdx.x;
    if (t < n) {
        const uint32_t k = chk(key_of(xyz[3 * t], xyz[3 * t + 1], xyz[3 * t + 2], A, inv));
        if (k != kInvalid) {
            red_or(&bitmap[k >> 5], 1u << (k & 31));
            red_add(&rec[k].x, 1u);
            red_max(&rec[k].y, ~static_cast<uint32_t>(t));
        }
    }
}

__global__ void __launch_bounds__(kBmThreads) kf_sums(const FilterJob *J, const int32_t *sb_map,
                                                      int32_t blk0) {
    const int32_t gb = blockIdx.x + blk0;
    const FilterJob &Q = J[sb_map[gb]];
    bitmap_sums_block(Q.bitmap, Q.chunk, Q.sums, Q.offsets, Q.counters, Q.counters + 1,
                      gb - Q.sb_blk0, Q.sb_nblk, Q.chunk_list, Q.counters + 3);
}

// The occupied 32-word chunks of the wave's jobs, one per warp at a time
// (every warp of the grid strides over each job's chunk list): each lane
// ranks its word (warp scan of popcounts on top of the chunk's offset),
// clears the word, and writes the keys of its set bits to the warp's stage
// in shared memory at their ranks within the chunk; the warp then writes the
// chunk's obstacles 32 consecutive ranks at a time, each with its cell's
// record, which it puts back to zero (also beyond the output's capacity).
// Empty chunks cost nothing here.
constexpr int kEmitThreads = 64;  // 2 warps a CTA: 3.14 us per frame against 3.19 with 4, 3.25 with 8
constexpr int kEmitWarps = kEmitThreads / 32;
constexpr int kEmitLoads = 8;  // record loads a lane keeps in flight

__global__ void __launch_bounds__(kEmitThreads) kf_emit(const FilterJob *J, int32_t q0, int32_t q1,
                                                      uint32_t *err) {
    __shared__ uint32_t stage[kEmitWarps][kChunkWords * 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = q0 + static_cast<int>(blockIdx.x * blockDim.x + threadIdx.x); q < q1;
         q += static_cast<int>(gridDim.x * blockDim.x)) {
        const uint32_t t = J[q].counters[1];
        *J[q].n_out = static_cast<int32_t>(t);
        if (t > J[q].o.cap) raise_error(err, GMAPP_DEVERR_CAPACITY);
    }
    uint32_t *st = stage[warp];
    const uint32_t gw = blockIdx.x * kEmitWarps + warp, tw = gridDim.x * kEmitWarps;
    // the wave's chunk lists as one index space: lane l holds the number of
    // occupied chunks of jobs q0 .. q0 + l (inclusive scan), 32 jobs a round
    for (int qb = q0; qb < q1; qb += 32) {
        const int qn = min(32, q1 - qb);
        uint32_t incl = lane < qn ? J[qb + lane].counters[3] : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += y;
        }
        const uint32_t total_chunks = __shfl_sync(0xffffffffu, incl, 31);
        for (uint32_t gi = gw; gi < total_chunks; gi += tw) {
            // job of gi: the first lane whose inclusive count exceeds gi
            const uint32_t jl = __ffs(__ballot_sync(0xffffffffu, lane < qn && incl > gi)) - 1;
            const uint32_t prev = __shfl_sync(0xffffffffu, incl, (jl + 31) & 31);  // lane jl - 1
            const uint32_t li = gi - (jl ? prev : 0u);
            const FilterJob &Q = J[qb + jl];
            const EmitOut o = Q.o;
            const FilterArgs A = Q.fa;
            const DivMagic dx = Q.dx, dy = Q.dy;
            const uint32_t c = Q.chunk_list[li];
            // every rank, output slot and bitmap word below derives from c:
            // the bounds-checked build checks it (warp-uniform: c is)
            if (!bc_ok(c, Q.n_chunks, err)) continue;
            const uint32_t wv = c * kChunkWords + lane;
            const uint32_t w = Q.bitmap[wv];
            uint32_t base = 0;
            if (lane == 0) base = Q.offsets[c / kChunksPerSumBlock] + Q.chunk[c];
            const uint32_t cnt = __popc(w);
            uint32_t incl = cnt;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            const uint32_t excl = incl - cnt;
            base = __shfl_sync(0xffffffffu, base, 0);
            if (w) Q.bitmap[wv] = 0u;
            uint32_t bits = w, pos = excl;
            const uint32_t k0 = wv * 32u;
            while (bits) {
                const uint32_t b = __ffs(bits) - 1;
                bits &= bits - 1;
                st[pos++] = k0 + b;
            }
            __syncwarp();
            // kEmitLoads rounds of 32 at a time: their record loads are
            // issued together, then each entry is written
            for (uint32_t r0 = 0; r0 < total; r0 += 32 * kEmitLoads) {
                uint32_t key[kEmitLoads];
                uint2 rc[kEmitLoads];
#pragma unroll
                for (int j = 0; j < kEmitLoads; ++j) {
                    const uint32_t r = r0 + 32 * j + lane;
                    key[j] = r < total ? st[r] : kInvalid;
                    rc[j] = key[j] != kInvalid ? Q.rec[key[j]] : make_uint2(0u, 0u);
                }
#pragma unroll
                for (int j = 0; j < kEmitLoads; ++j) {
                    if (key[j] == kInvalid) continue;
                    Q.rec[key[j]] = make_uint2(0u, 0u);
                    const uint32_t rank = base + r0 + 32 * j + lane;
                    if (rank < o.cap) {
                        const uint32_t qy = div_by(key[j], dx);
                        const uint32_t ix = key[j] - qy * A.nx;
                        const uint32_t iz = div_by(qy, dy);
                        const uint32_t iy = qy - iz * A.ny;
                        float cx, cy, cz;
                        cell_centre(ix, iy, iz, A, cx, cy, cz);
                        o.keys[rank] = key[j];
                        o.counts[rank] = rc[j].x;
                        o.rep[rank] = ~rc[j].y;
                        o.x[rank] = cx;
                        o.y[rank] = cy;
                        o.z[rank] = cz;
                    }
                }
            }
            __syncwarp();
        }
    }
}

}  // namespace
}  // namespace gmapp

using namespace gmapp;

struct gmapp_filter_batch {
    gmapp_ctx *ctx = nullptr;
    FilterJob *d_jobs = nullptr;
    int32_t *d_pt_map = nullptr, *d_sb_map = nullptr;
    void *d_ws = nullptr;
    // per wave: first block and block count of each launch, first and last job
    std::vector<int32_t> pt0, ptn, sb0, sbn, q0, q1;
    int emit_grid = 0;
    // wave w runs on stream w mod kWaveStreams: 0 is the caller's, the
    // others are the batch's own side streams, forked from and joined back
    // into the caller's stream by events
    cudaStream_t side[kWaveStreams - 1] = {};
    cudaEvent_t fork = nullptr, join[kWaveStreams - 1] = {};
};

namespace {

void release(gmapp_filter_batch *fb) {
    cudaFree(fb->d_jobs);
    cudaFree(fb->d_pt_map);
    cudaFree(fb->d_sb_map);
    cudaFree(fb->d_ws);
    if (fb->fork) cudaEventDestroy(fb->fork);
    for (int i = 0; i < kWaveStreams - 1; ++i) {
        if (fb->join[i]) cudaEventDestroy(fb->join[i]);
        if (fb->side[i]) cudaStreamDestroy(fb->side[i]);
    }
}

// One slot's scratch: the bitmap over the grid (padded to whole kf_sums
// blocks), per-chunk and per-block popcount offsets, counters, the occupied
// chunk list and one record per (padded) cell.
struct SlotLayout {
    int64_t n_words, n_sblocks;
    size_t off_bitmap, off_chunk, off_sums, off_offsets, off_counters, off_list, off_rec;
    size_t total;
};

SlotLayout slot_layout(uint64_t cells) {
    SlotLayout L{};
    const int64_t words = static_cast<int64_t>((cells + 31) / 32);
    L.n_sblocks = (words + kWordsPerSumBlock - 1) / kWordsPerSumBlock;
    L.n_words = L.n_sblocks * kWordsPerSumBlock;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    L.off_bitmap = take(L.n_words * 4);
    L.off_chunk = take(L.n_words / kChunkWords * 4);
    L.off_sums = take(L.n_sblocks * 4);
    L.off_offsets = take(L.n_sblocks * 4);
    L.off_counters = take(64);
    L.off_list = take(L.n_words / kChunkWords * 4);
    L.off_rec = take(static_cast<size_t>(L.n_words) * 32 * sizeof(uint2));
    L.total = off;
    return L;
}

}  // namespace

extern "C" gmapp_status gmapp_filter_batch_create(gmapp_ctx *ctx, const gmapp_cloud_job *jobs,
                                                  int32_t n_jobs, gmapp_filter_batch **out) {
    if (!ctx || !jobs || n_jobs < 1 || !out) {
        set_error("gmapp_filter_batch_create: invalid argument");
        return GMAPP_ERR_INVALID_ARG;
    }
    *out = nullptr;
    size_t touched = 1;
    // one layout for every slot, sized by the largest grid of the batch: a
    // slot serves different jobs wave after wave, and each region (bitmap,
    // offsets, counters, records) must sit at the same place for all of them
    // -- the bitmap and the records stay zero beyond what a job sets and
    // clears
    uint64_t max_cells = 0;
    for (int q = 0; q < n_jobs; ++q) {
        const gmapp_cloud_job &J = jobs[q];
        if (!valid_workspace(&J.ws) || J.ws.min_pts != 1 || J.n_raw < 0 ||
            J.n_raw >= 0xFFFFFFFFll || (J.n_raw > 0 && !J.xyz) ||
            reinterpret_cast<uintptr_t>(J.xyz) % 16) {
            set_error("gmapp_filter_batch_create: job %d: invalid cloud or workspace (min_pts "
                      "must be 1, clouds 16-byte aligned)", q);
            return GMAPP_ERR_INVALID_ARG;
        }
        const gmapp_obstacles &o = J.out;
        if (!o.x || !o.y || !o.z || !o.keys || !o.counts || !o.rep_idx || !o.n || o.cap < 0) {
            set_error("gmapp_filter_batch_create: job %d: every output buffer must be set", q);
            return GMAPP_ERR_INVALID_ARG;
        }
        for (int i = 0; i < 12; ++i)
            if (!isfinite(J.T[i])) {
                set_error("gmapp_filter_batch_create: job %d: transform not finite", q);
                return GMAPP_ERR_INVALID_ARG;
            }
        const uint64_t cells = static_cast<uint64_t>(J.ws.dims[0]) * J.ws.dims[1] * J.ws.dims[2];
        max_cells = std::max(max_cells, cells);
        // scratch a wave keeps in L2: the bitmap and, at most, one record
        // per point (a point touches one cell)
        touched = std::max(touched, static_cast<size_t>((cells + 31) / 32) * 4 +
                                        static_cast<size_t>(std::min<uint64_t>(
                                            cells, static_cast<uint64_t>(J.n_raw))) * 8);
    }
    const SlotLayout SL = slot_layout(max_cells);
    const size_t slot_bytes = SL.total;
    int W_max = static_cast<int>(std::max<size_t>(
        1, std::min<size_t>(n_jobs, kWaveL2Bytes / touched)));
    // the slot sets take at most half of the device memory free now (a
    // large grid makes a slot large): fewer jobs per wave otherwise
    size_t free_bytes = 0, total_bytes = 0;
    if (cudaMemGetInfo(&free_bytes, &total_bytes) == cudaSuccess) {
        const size_t per_wave_job = static_cast<size_t>(kWaveStreams) * slot_bytes;
        const size_t fit = free_bytes / 2 / std::max<size_t>(1, per_wave_job);
        W_max = static_cast<int>(std::max<size_t>(1, std::min<size_t>(W_max, fit)));
    } else {
        cudaGetLastError();  // no memory figure: keep the L2-sized waves
    }
    const int n_waves = (n_jobs + W_max - 1) / W_max;
    const int W = (n_jobs + n_waves - 1) / n_waves;  // balanced waves
    const int n_slots = std::min(n_waves, kWaveStreams) * W;

    std::vector<FilterJob> hj(n_jobs);
    std::vector<int32_t> pt_map, sb_map;
    // point pass: per wave, about one full wave of resident CTAs (the SM
    // count times the CTAs an SM holds), shared by the wave's jobs
    int pts_per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pts_per_sm, kf_points, kThreads, 0);
    const int64_t pts_blocks = std::max(1, pts_per_sm) * static_cast<int64_t>(ctx->sm_count);
    auto blocks_for = [&](int64_t n8, int64_t wave_blocks) {
        const int64_t per_job = (wave_blocks + W - 1) / W;
        return static_cast<int32_t>(std::max<int64_t>(
            1, std::min<int64_t>(per_job, (n8 + kThreads - 1) / kThreads)));
    };
    gmapp_filter_batch *fb = new gmapp_filter_batch();
    fb->ctx = ctx;
    // emit: persistent over the wave's occupied chunks, one wave of resident CTAs
    int emit_per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&emit_per_sm, kf_emit, kEmitThreads, 0);
    fb->emit_grid = std::max(1, emit_per_sm) * ctx->sm_count;
    for (int q = 0; q < n_jobs; ++q) {
        const gmapp_cloud_job &J = jobs[q];
        FilterJob &D = hj[q];
        memset(&D, 0, sizeof(D));
        D.xyz = J.xyz;
        D.n_raw = J.n_raw;
        for (int i = 0; i < 12; ++i) D.fa.T[i] = J.T[i];
        for (int d = 0; d < 3; ++d) {
            D.fa.lo[d] = J.ws.lo[d];
            D.fa.dimf[d] = static_cast<float>(J.ws.dims[d]);
        }
        D.fa.voxel = J.ws.voxel;
        D.fa.nx = J.ws.dims[0];
        D.fa.ny = J.ws.dims[1];
        D.fa.nz = J.ws.dims[2];
        D.fa.err = ctx->d_err;
        D.dx = div_magic(D.fa.nx);
        D.dy = div_magic(D.fa.ny);
        const uint64_t cells = static_cast<uint64_t>(J.ws.dims[0]) * J.ws.dims[1] * J.ws.dims[2];
        const SlotLayout L = slot_layout(cells);
        const int64_t n8 = J.n_raw / kPointsPerThread;
        D.pt_blk0 = static_cast<int32_t>(pt_map.size());
        D.pt_nblk = blocks_for(n8, pts_blocks);
        for (int i = 0; i < D.pt_nblk; ++i) pt_map.push_back(q);
        D.sb_blk0 = static_cast<int32_t>(sb_map.size());
        D.sb_nblk = static_cast<int32_t>(L.n_sblocks);
        for (int i = 0; i < D.sb_nblk; ++i) sb_map.push_back(q);
        D.n_chunks = static_cast<uint32_t>(L.n_words / kChunkWords);
        D.o = EmitOut{J.out.keys, J.out.counts, J.out.rep_idx, J.out.x, J.out.y, J.out.z,
                      J.out.cap};
        D.n_out = J.out.n;
        if (pt_map.size() > 0x7fffffffu || sb_map.size() > 0x7fffffffu) {
            delete fb;
            set_error("gmapp_filter_batch_create: too many blocks");
            return GMAPP_ERR_CAPACITY;
        }
    }
    for (int w = 0; w < n_waves; ++w) {
        const int q0 = w * W, q1 = std::min(n_jobs, q0 + W) - 1;
        fb->pt0.push_back(hj[q0].pt_blk0);
        fb->ptn.push_back(hj[q1].pt_blk0 + hj[q1].pt_nblk - hj[q0].pt_blk0);
        fb->q0.push_back(q0);
        fb->q1.push_back(q1 + 1);
        fb->sb0.push_back(hj[q0].sb_blk0);
        fb->sbn.push_back(hj[q1].sb_blk0 + hj[q1].sb_nblk - hj[q0].sb_blk0);
    }
    const size_t ws_total = static_cast<size_t>(n_slots) * slot_bytes;
    cudaError_t e = cudaMalloc(&fb->d_ws, ws_total);
    // zero scratch: bitmaps, records and counters start clear, and each run
    // leaves them clear again
    if (e == cudaSuccess) e = cudaMemset(fb->d_ws, 0, ws_total);
    if (e == cudaSuccess) e = cudaMalloc(&fb->d_jobs, sizeof(FilterJob) * n_jobs);
    if (e == cudaSuccess) e = cudaMalloc(&fb->d_pt_map, sizeof(int32_t) * pt_map.size());
    if (e == cudaSuccess) e = cudaMalloc(&fb->d_sb_map, sizeof(int32_t) * sb_map.size());
    for (int i = 0; i < kWaveStreams - 1; ++i) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&fb->side[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fb->join[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fb->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) {
        char *ws = static_cast<char *>(fb->d_ws);
        for (int q = 0; q < n_jobs; ++q) {
            // wave w = q / W uses slot set w mod kWaveStreams (its stream's), slot q - w W
            const int w = q / W, slot = (w % kWaveStreams) * W + (q - w * W);
            char *base = ws + static_cast<size_t>(slot) * slot_bytes;
            FilterJob &D = hj[q];
            D.bitmap = reinterpret_cast<uint32_t *>(base + SL.off_bitmap);
            D.chunk = reinterpret_cast<uint32_t *>(base + SL.off_chunk);
            D.sums = reinterpret_cast<uint32_t *>(base + SL.off_sums);
            D.offsets = reinterpret_cast<uint32_t *>(base + SL.off_offsets);
            D.counters = reinterpret_cast<uint32_t *>(base + SL.off_counters);
            D.chunk_list = reinterpret_cast<uint32_t *>(base + SL.off_list);
            D.rec = reinterpret_cast<uint2 *>(base + SL.off_rec);
        }
        e = cudaMemcpy(fb->d_jobs, hj.data(), sizeof(FilterJob) * n_jobs,
                       cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(fb->d_pt_map, pt_map.data(), sizeof(int32_t) * pt_map.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(fb->d_sb_map, sb_map.data(), sizeof(int32_t) * sb_map.size(),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        gmapp_status st = cuda_fail(e, "gmapp_filter_batch_create");
        release(fb);
        delete fb;
        return st;
    }
    *out = fb;
    return GMAPP_OK;
}

extern "C" void gmapp_filter_batch_destroy(gmapp_filter_batch *fb) {
    if (!fb) return;
    for (int i = 0; i < kWaveStreams - 1; ++i)
        if (fb->side[i]) cudaStreamSynchronize(fb->side[i]);
    release(fb);
    delete fb;
}

extern "C" gmapp_status filter_cloud_batch(gmapp_filter_batch *fb, gmapp_stream stream) {
    if (!fb) {
        set_error("filter_cloud_batch: NULL batch");
        return GMAPP_ERR_INVALID_ARG;
    }
    const int n_waves = static_cast<int>(fb->pt0.size());
    const int n_side = std::min(n_waves, kWaveStreams) - 1;  // side streams in use
    if (n_side > 0) {
        GMAPP_CHECK_CUDA(cudaEventRecord(fb->fork, stream));
        for (int i = 0; i < n_side; ++i)
            GMAPP_CHECK_CUDA(cudaStreamWaitEvent(fb->side[i], fb->fork, 0));
    }
    for (int w = 0; w < n_waves; ++w) {
        const int l = w % kWaveStreams;
        cudaStream_t s = l == 0 ? stream : fb->side[l - 1];
        kf_points<<<fb->ptn[w], kThreads, 0, s>>>(fb->d_jobs, fb->d_pt_map, fb->pt0[w]);
        kf_sums<<<fb->sbn[w], kBmThreads, 0, s>>>(fb->d_jobs, fb->d_sb_map, fb->sb0[w]);
        kf_emit<<<fb->emit_grid, kEmitThreads, 0, s>>>(fb->d_jobs, fb->q0[w], fb->q1[w],
                                                   fb->ctx->d_err);
    }
    for (int i = 0; i < n_side; ++i) {
        GMAPP_CHECK_CUDA(cudaEventRecord(fb->join[i], fb->side[i]));
        GMAPP_CHECK_CUDA(cudaStreamWaitEvent(stream, fb->join[i], 0));
    }
    GMAPP_CHECK_CUDA(cudaGetLastError());
    return GMAPP_OK;
}
