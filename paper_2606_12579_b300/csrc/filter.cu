// filter_cloud: depth cloud -> sphere world S_W (Sec. IV-B, Sec. V-A).
//
// Design (B300): the occupied-voxel set is kept as a bitmap over the voxel
// grid (1 bit per cell: 0.8 MB for a 200x200x160 grid, L2-resident), not as
// a hash table.  The rank of a set bit in the bitmap is the obstacle's output
// slot, so the output comes out in ascending key order without any sort and
// is bit-identical from run to run (only commutative integer atomics).
//
//   k_zero          clear bitmap + the block counter              (bitmap bytes)
//   k_keys          points -> key per point + bitmap bits          (12 B/pt in, 4 B/pt out)
//   k_bitmap_sums   popcount per block of words; the last block to
//                   finish scans the block sums (no spin-wait)
//   k_emit          per word: prefix rank; per set bit (one lane per bit of a
//                   word, warp-cooperative): key, centre; publishes N_O
//   k_count         points -> rank -> count (atomicAdd), smallest index (atomicMin)
//   (several sensors: k_keys_fused / k_count_fused, one launch for up to 8
//   sensors, each sensor's blocks with its own transform and index base)
//   k_keep_sums / k_keep_emit   only when min_pts > 1: order-preserving compaction
#include <math.h>

#include <algorithm>
#include <vector>

#include "filter_device.cuh"


namespace gmapp {
namespace {

// Several sensors' key and count passes in one launch each: sensor q owns
// blocks [blk0, blk0 + nblk) of the grid (ascending blk0), its transform, its
// key slot and the index of its first point.
constexpr int kFuseMax = 8;
struct SensorRange {
    const float *xyz;
    int64_t n, slot;
    float T[12];
    uint32_t idx0;
    int32_t blk0, nblk;
};
struct SensorSet {
    SensorRange s[kFuseMax];
    int32_t n;
};

// The sensor of this block (the last one whose first block is at or before
// it), read with compile-time indices only.
__device__ __forceinline__ void sensor_of_block(const SensorSet &S, SensorRange &R) {
#pragma unroll
    for (int t = 0; t < kFuseMax; ++t)
        if (t < S.n && static_cast<int32_t>(blockIdx.x) >= S.s[t].blk0) R = S.s[t];
}

__global__ void __launch_bounds__(kThreads) k_keys_fused(const SensorSet S, FilterArgs A,
                                                         uint32_t *__restrict__ keys,
                                                         uint32_t *__restrict__ bitmap) {
    SensorRange R = S.s[0];
    sensor_of_block(S, R);
#pragma unroll
    for (int i = 0; i < 12; ++i) A.T[i] = R.T[i];
    keys_range(R.xyz, R.n, A, keys + R.slot, bitmap, blockIdx.x - R.blk0, R.nblk);
}

__global__ void __launch_bounds__(kThreads) k_count_fused(const SensorSet S,
                                                          const uint32_t *__restrict__ keys,
                                                          const uint2 *__restrict__ pw,
                                                          uint32_t *counts, uint32_t *rep,
                                                          int64_t cap) {
    SensorRange R = S.s[0];
    sensor_of_block(S, R);
    count_range(keys + R.slot, R.n, pw, counts, rep, cap, blockIdx.x - R.blk0, R.nblk, R.idx0);
}

}  // namespace
}  // namespace gmapp

using namespace gmapp;

extern "C" size_t gmapp_filter_workspace_bytes(int64_t n_raw, const gmapp_workspace *ws) {
    if (n_raw < 0 || !valid_workspace(ws)) return 0;
    return layout(n_raw, ws).total;
}

namespace {

// Key slots of the sensors in the workspace's key array: sensor s starts at
// the sum of the earlier clouds rounded up to 4 (16-byte aligned stores).
int64_t key_slots(const gmapp_sensor_cloud *clouds, int32_t n_sensors) {
    int64_t tot = 0;
    for (int32_t s = 0; s < n_sensors; ++s) tot += (clouds[s].n_raw + 3) & ~int64_t(3);
    return tot;
}

// filter_cloud / filter_clouds: every sensor's points set bits in one bitmap
// (k_keys with its own transform) and are counted with their global index
// (k_count with the sensor's index base); bitmap sums and emit run once.
gmapp_status filter_impl(const char *who, gmapp_ctx *ctx, const gmapp_sensor_cloud *clouds,
                         int32_t n_sensors, const gmapp_workspace *ws, gmapp_obstacles *out,
                         void *workspace, size_t workspace_bytes, gmapp_stream stream) {
    if (!ctx || !clouds || n_sensors < 1 || !out || !workspace) {
        set_error("%s: NULL ctx, clouds, out or workspace, or no sensor", who);
        return GMAPP_ERR_INVALID_ARG;
    }
    int64_t total = 0;
    for (int32_t s = 0; s < n_sensors; ++s) {
        const gmapp_sensor_cloud &c = clouds[s];
        if (c.n_raw < 0 || c.n_raw >= 0xFFFFFFFFll || (c.n_raw > 0 && !c.xyz)) {
            set_error("%s: n_raw %lld of sensor %d out of range or xyz NULL", who,
                      (long long)c.n_raw, s);
            return GMAPP_ERR_INVALID_ARG;
        }
        if (reinterpret_cast<uintptr_t>(c.xyz) % 16) {
            set_error("%s: xyz of sensor %d must be 16-byte aligned", who, s);
            return GMAPP_ERR_INVALID_ARG;
        }
        for (int i = 0; i < 12; ++i)
            if (!isfinite(c.T[i])) {
                set_error("%s: transform entry %d of sensor %d is not finite", who, i, s);
                return GMAPP_ERR_INVALID_ARG;
            }
        total += c.n_raw;
    }
    if (total >= 0xFFFFFFFFll) {
        set_error("%s: %lld points in all, at most 2^32 - 2", who, (long long)total);
        return GMAPP_ERR_INVALID_ARG;
    }
    if (!valid_workspace(ws)) {
        set_error("%s: invalid workspace grid (voxel > 0, 1 <= dims <= 2^24, "
                  "cells < 2^32-1, min_pts >= 1)", who);
        return GMAPP_ERR_INVALID_ARG;
    }
    if (reinterpret_cast<uintptr_t>(workspace) % 256) {
        set_error("%s: workspace must be 256-byte aligned", who);
        return GMAPP_ERR_INVALID_ARG;
    }
    if (!out->x || !out->y || !out->z || !out->keys || !out->counts || !out->rep_idx || !out->n ||
        out->cap < 0) {
        set_error("%s: output buffers must all be set and cap >= 0", who);
        return GMAPP_ERR_INVALID_ARG;
    }
    Layout L = layout(key_slots(clouds, n_sensors), ws);
    if (workspace_bytes < L.total) {
        set_error("%s: workspace of %zu bytes, %zu needed", who, workspace_bytes, L.total);
        return GMAPP_ERR_CAPACITY;
    }
    FilterArgs A;
    for (int a = 0; a < 3; ++a) {
        A.lo[a] = ws->lo[a];
        A.dimf[a] = static_cast<float>(ws->dims[a]);
    }
    A.voxel = ws->voxel;
    A.nx = ws->dims[0];
    A.ny = ws->dims[1];
    A.nz = ws->dims[2];
    A.err = ctx->d_err;
    out->r_O = 0.5f * ws->voxel;  // exact: scaling by a power of two

    char *base = static_cast<char *>(workspace);
    uint32_t *bitmap = reinterpret_cast<uint32_t *>(base + L.off_bitmap);
    uint2 *pw = reinterpret_cast<uint2 *>(base + L.off_pw);
    uint32_t *chunk = reinterpret_cast<uint32_t *>(base + L.off_chunk);
    uint32_t *sums = reinterpret_cast<uint32_t *>(base + L.off_sums);
    uint32_t *offsets = reinterpret_cast<uint32_t *>(base + L.off_offsets);
    uint32_t *counters = reinterpret_cast<uint32_t *>(base + L.off_counters);
    uint32_t *keys = reinterpret_cast<uint32_t *>(base + L.off_keys);
    uint32_t *n_occ = counters + 1;
    uint32_t *n_keep_counter = counters + 2;

    auto grid_for = [&](int64_t n) {
        return static_cast<int>(std::max<int64_t>(
            1, std::min<int64_t>((n / 4 + kThreads - 1) / kThreads, (int64_t)ctx->sm_count * 8)));
    };
    const int grid_zero = static_cast<int>(
        std::min<int64_t>((L.n_words / 4 + kThreads - 1) / kThreads, (int64_t)ctx->sm_count * 8));

    k_zero<<<grid_zero, kThreads, 0, stream>>>(reinterpret_cast<uint4 *>(bitmap), L.n_words / 4,
                                               counters, 16);
    // sensors in groups of up to kFuseMax, one key launch (and later one
    // count launch) per group; a single cloud launches the plain kernels
    std::vector<SensorSet> sets;
    std::vector<int32_t> set_blocks;  // blocks of each group's launch
    {
        int64_t slot = 0, idx0 = 0;
        for (int32_t s = 0; s < n_sensors; ++s) {
            if (s % kFuseMax == 0) {
                sets.push_back(SensorSet{});
                set_blocks.push_back(0);
            }
            SensorSet &S = sets.back();
            SensorRange &R = S.s[S.n++];
            R.xyz = clouds[s].xyz;
            R.n = clouds[s].n_raw;
            R.slot = slot;
            for (int i = 0; i < 12; ++i) R.T[i] = clouds[s].T[i];
            R.idx0 = static_cast<uint32_t>(idx0);
            R.nblk = grid_for(clouds[s].n_raw);
            R.blk0 = set_blocks.back();
            set_blocks.back() += R.nblk;
            slot += (clouds[s].n_raw + 3) & ~int64_t(3);
            idx0 += clouds[s].n_raw;
        }
    }
    if (n_sensors == 1) {
        for (int i = 0; i < 12; ++i) A.T[i] = clouds[0].T[i];
        k_keys<<<grid_for(clouds[0].n_raw), kThreads, 0, stream>>>(clouds[0].xyz, clouds[0].n_raw,
                                                                   A, keys, bitmap);
    } else {
        for (size_t g = 0; g < sets.size(); ++g)
            k_keys_fused<<<set_blocks[g], kThreads, 0, stream>>>(sets[g], A, keys, bitmap);
    }
    k_bitmap_sums<<<static_cast<int>(L.n_sblocks), kBmThreads, 0, stream>>>(bitmap, chunk, sums, offsets,
                                                                          counters, n_occ);
    // per-sensor counts: points of sensor s carry the indices idx0 + i
    auto count_all = [&](uint32_t *cnt, uint32_t *rep, int64_t cap) {
        if (n_sensors == 1) {
            k_count<<<grid_for(clouds[0].n_raw), kThreads, 0, stream>>>(keys, clouds[0].n_raw, pw,
                                                                        cnt, rep, cap, 0u);
            return;
        }
        for (size_t g = 0; g < sets.size(); ++g)
            k_count_fused<<<set_blocks[g], kThreads, 0, stream>>>(sets[g], keys, pw, cnt, rep, cap);
    };
    if (ws->min_pts == 1) {
        EmitOut o{out->keys, out->counts, out->rep_idx, out->x, out->y, out->z, out->cap};
        k_emit<<<static_cast<int>(L.n_words / kBmThreads), kBmThreads, 0, stream>>>(bitmap, offsets, chunk, pw, A, o,
                                                                      n_occ, out->n, ctx->d_err);
        count_all(out->counts, out->rep_idx, out->cap);
    } else {
        uint32_t *tkeys = reinterpret_cast<uint32_t *>(base + L.off_tkeys);
        uint32_t *tcounts = reinterpret_cast<uint32_t *>(base + L.off_tcounts);
        uint32_t *trep = reinterpret_cast<uint32_t *>(base + L.off_trep);
        uint32_t *tsums = reinterpret_cast<uint32_t *>(base + L.off_tsums);
        uint32_t *toffsets = reinterpret_cast<uint32_t *>(base + L.off_toffsets);
        EmitOut t{tkeys, tcounts, trep, nullptr, nullptr, nullptr, L.n_tmp};
        k_emit<<<static_cast<int>(L.n_words / kBmThreads), kBmThreads, 0, stream>>>(bitmap, offsets, chunk, pw, A, t,
                                                                      nullptr, nullptr, nullptr);
        count_all(tcounts, trep, L.n_tmp);
        k_keep_sums<<<static_cast<int>(L.n_tblocks), kThreads, 0, stream>>>(
            tcounts, n_occ, ws->min_pts, tsums, toffsets, n_keep_counter, out->n, out->cap,
            ctx->d_err);
        EmitOut o{out->keys, out->counts, out->rep_idx, out->x, out->y, out->z, out->cap};
        k_keep_emit<<<static_cast<int>(L.n_tblocks), kThreads, 0, stream>>>(
            tkeys, tcounts, trep, n_occ, toffsets, ws->min_pts, A, o);
    }
    GMAPP_CHECK_CUDA(cudaGetLastError());
    return GMAPP_OK;
}

}  // namespace

extern "C" gmapp_status filter_cloud(gmapp_ctx *ctx, const float *xyz, int64_t n_raw,
                                     const float T[12], const gmapp_workspace *ws,
                                     gmapp_obstacles *out, void *workspace,
                                     size_t workspace_bytes, gmapp_stream stream) {
    if (!T) {
        set_error("filter_cloud: NULL T");
        return GMAPP_ERR_INVALID_ARG;
    }
    gmapp_sensor_cloud c;
    c.xyz = xyz;
    c.n_raw = n_raw;
    for (int i = 0; i < 12; ++i) c.T[i] = T[i];
    return filter_impl("filter_cloud", ctx, &c, 1, ws, out, workspace, workspace_bytes, stream);
}

extern "C" size_t gmapp_filter_clouds_workspace_bytes(const gmapp_sensor_cloud *clouds,
                                                      int32_t n_sensors,
                                                      const gmapp_workspace *ws) {
    if (!clouds || n_sensors < 1 || !valid_workspace(ws)) return 0;
    for (int32_t s = 0; s < n_sensors; ++s)
        if (clouds[s].n_raw < 0) return 0;
    return layout(key_slots(clouds, n_sensors), ws).total;
}

extern "C" gmapp_status filter_clouds(gmapp_ctx *ctx, const gmapp_sensor_cloud *clouds,
                                      int32_t n_sensors, const gmapp_workspace *ws,
                                      gmapp_obstacles *out, void *workspace,
                                      size_t workspace_bytes, gmapp_stream stream) {
    return filter_impl("filter_clouds", ctx, clouds, n_sensors, ws, out, workspace,
                       workspace_bytes, stream);
}

// ---------------------------------------------------------------------------
// filter_cloud_noalloc: the same kernels with their scratch in a fixed,
// file-scope device array instead of a caller-provided workspace.
//
// For callers that may not allocate device memory once running: a real-time
// control loop whose memory is fixed at start-up, a process without the
// right to call cudaMalloc at that point, or code that must not grow the
// device footprint per call.  The array is part of this library's device
// image: every GPU that loads the library holds kNoAllocScratchBytes until
// the process exits.
// ---------------------------------------------------------------------------

namespace gmapp {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
// Capacity flag of the latest call (GMAPP_DEVERR_CAPACITY when more voxels
// qualified than out->cap); cleared at the start of every call and read by
// filter_cloud_noalloc_status.
static __device__ uint32_t g_noalloc_err;

// Device addresses of the two symbols on the current device (host code may
// not use the symbols' names as addresses).  Looked up on every call: the
// lookup allocates nothing, and a cached address would go stale after a
// device reset reloads the module.
struct NoAllocSymbols {
    void *scratch = nullptr;
    uint32_t *err = nullptr;
};

gmapp_status noalloc_symbols(NoAllocSymbols *out) {
    void *scratch = nullptr, *err = nullptr;
    GMAPP_CHECK_CUDA(cudaGetSymbolAddress(&scratch, g_noalloc_scratch));
    GMAPP_CHECK_CUDA(cudaGetSymbolAddress(&err, g_noalloc_err));
    out->scratch = scratch;
    out->err = static_cast<uint32_t *>(err);
    return GMAPP_OK;
}

}  // namespace
}  // namespace gmapp

extern "C" gmapp_status filter_cloud_noalloc(const float *xyz, int64_t n_raw, const float T[12],
                                             const gmapp_workspace *ws, gmapp_obstacles *out,
                                             gmapp_stream stream) {
    if (!T || !out) {
        set_error("filter_cloud_noalloc: NULL T or out");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (n_raw < 0 || n_raw >= 0xFFFFFFFFll || (n_raw > 0 && !xyz)) {
        set_error("filter_cloud_noalloc: n_raw %lld out of range or xyz NULL", (long long)n_raw);
        return GMAPP_ERR_INVALID_ARG;
    }
    if (!valid_workspace(ws)) {
        set_error("filter_cloud_noalloc: invalid workspace grid (voxel > 0, 1 <= dims <= 2^24, "
                  "cells < 2^32-1, min_pts >= 1)");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (reinterpret_cast<uintptr_t>(xyz) % 16) {
        set_error("filter_cloud_noalloc: xyz must be 16-byte aligned");
        return GMAPP_ERR_INVALID_ARG;
    }
    if (!out->x || !out->y || !out->z || !out->keys || !out->counts || !out->rep_idx || !out->n ||
        out->cap < 0) {
        set_error("filter_cloud_noalloc: output buffers must all be set and cap >= 0");
        return GMAPP_ERR_INVALID_ARG;
    }
    for (int i = 0; i < 12; ++i)
        if (!isfinite(T[i])) {
            set_error("filter_cloud_noalloc: transform entry %d is not finite", i);
            return GMAPP_ERR_INVALID_ARG;
        }
    Layout L = layout(n_raw, ws);
    if (L.total > kNoAllocScratchBytes) {
        set_error("filter_cloud_noalloc: this cloud and grid need %zu bytes of scratch, more than "
                  "the fixed %zu bytes (use filter_cloud with a workspace)",
                  L.total, kNoAllocScratchBytes);
        return GMAPP_ERR_CAPACITY;
    }
    NoAllocSymbols sym;
    gmapp_status st = noalloc_symbols(&sym);
    if (st != GMAPP_OK) return st;
    // the flag reports this call only (a device memset allocates nothing)
    GMAPP_CHECK_CUDA(cudaMemsetAsync(sym.err, 0, sizeof(uint32_t), stream));
    int dev = 0, sms = 0;
    GMAPP_CHECK_CUDA(cudaGetDevice(&dev));
    GMAPP_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

    FilterArgs A;
    for (int i = 0; i < 12; ++i) A.T[i] = T[i];
    for (int a = 0; a < 3; ++a) {
        A.lo[a] = ws->lo[a];
        A.dimf[a] = static_cast<float>(ws->dims[a]);
    }
    A.voxel = ws->voxel;
    A.nx = ws->dims[0];
    A.ny = ws->dims[1];
    A.nz = ws->dims[2];
    A.err = nullptr;  // no context: index checks of the bounds-checked build are silent here
    out->r_O = 0.5f * ws->voxel;

    char *base = static_cast<char *>(sym.scratch);
    uint32_t *bitmap = reinterpret_cast<uint32_t *>(base + L.off_bitmap);
    uint2 *pw = reinterpret_cast<uint2 *>(base + L.off_pw);
    uint32_t *chunk = reinterpret_cast<uint32_t *>(base + L.off_chunk);
    uint32_t *sums = reinterpret_cast<uint32_t *>(base + L.off_sums);
    uint32_t *offsets = reinterpret_cast<uint32_t *>(base + L.off_offsets);
    uint32_t *counters = reinterpret_cast<uint32_t *>(base + L.off_counters);
    uint32_t *keys = reinterpret_cast<uint32_t *>(base + L.off_keys);
    uint32_t *n_occ = counters + 1;
    uint32_t *n_keep_counter = counters + 2;

    const int grid_pts = static_cast<int>(std::max<int64_t>(
        1, std::min<int64_t>((n_raw / 4 + kThreads - 1) / kThreads, (int64_t)sms * 8)));
    const int grid_zero = static_cast<int>(
        std::min<int64_t>((L.n_words / 4 + kThreads - 1) / kThreads, (int64_t)sms * 8));

    // k_zero clears the bitmap and the counters: the array keeps whatever
    // the previous call left in it.
    k_zero<<<grid_zero, kThreads, 0, stream>>>(reinterpret_cast<uint4 *>(bitmap), L.n_words / 4,
                                               counters, 16);
    k_keys<<<grid_pts, kThreads, 0, stream>>>(xyz, n_raw, A, keys, bitmap);
    k_bitmap_sums<<<static_cast<int>(L.n_sblocks), kBmThreads, 0, stream>>>(bitmap, chunk, sums, offsets,
                                                                          counters, n_occ);
    if (ws->min_pts == 1) {
        EmitOut o{out->keys, out->counts, out->rep_idx, out->x, out->y, out->z, out->cap};
        k_emit<<<static_cast<int>(L.n_words / kBmThreads), kBmThreads, 0, stream>>>(bitmap, offsets, chunk, pw, A, o,
                                                                      n_occ, out->n, sym.err);
        k_count<<<grid_pts, kThreads, 0, stream>>>(keys, n_raw, pw, out->counts,
                                                   out->rep_idx, out->cap, 0u);
    } else {
        uint32_t *tkeys = reinterpret_cast<uint32_t *>(base + L.off_tkeys);
        uint32_t *tcounts = reinterpret_cast<uint32_t *>(base + L.off_tcounts);
        uint32_t *trep = reinterpret_cast<uint32_t *>(base + L.off_trep);
        uint32_t *tsums = reinterpret_cast<uint32_t *>(base + L.off_tsums);
        uint32_t *toffsets = reinterpret_cast<uint32_t *>(base + L.off_toffsets);
        EmitOut t{tkeys, tcounts, trep, nullptr, nullptr, nullptr, L.n_tmp};
        k_emit<<<static_cast<int>(L.n_words / kBmThreads), kBmThreads, 0, stream>>>(bitmap, offsets, chunk, pw, A, t,
                                                                      nullptr, nullptr, nullptr);
        k_count<<<grid_pts, kThreads, 0, stream>>>(keys, n_raw, pw, tcounts, trep,
                                                   L.n_tmp, 0u);
        k_keep_sums<<<static_cast<int>(L.n_tblocks), kThreads, 0, stream>>>(
            tcounts, n_occ, ws->min_pts, tsums, toffsets, n_keep_counter, out->n, out->cap,
            sym.err);
        EmitOut o{out->keys, out->counts, out->rep_idx, out->x, out->y, out->z, out->cap};
        k_keep_emit<<<static_cast<int>(L.n_tblocks), kThreads, 0, stream>>>(
            tkeys, tcounts, trep, n_occ, toffsets, ws->min_pts, A, o);
    }
    GMAPP_CHECK_CUDA(cudaGetLastError());
    return GMAPP_OK;
}

extern "C" gmapp_status filter_cloud_noalloc_status(gmapp_stream stream) {
    NoAllocSymbols sym;
    gmapp_status st = noalloc_symbols(&sym);
    if (st != GMAPP_OK) return st;
    uint32_t word = 0;
    GMAPP_CHECK_CUDA(cudaMemcpyAsync(&word, sym.err, sizeof(word), cudaMemcpyDeviceToHost, stream));
    GMAPP_CHECK_CUDA(cudaStreamSynchronize(stream));
    if (word & GMAPP_DEVERR_CAPACITY) {
        set_error("filter_cloud_noalloc: more voxels qualified than out->cap (*out->n holds "
                  "the number needed)");
        return GMAPP_ERR_CAPACITY;
    }
    return GMAPP_OK;
}
