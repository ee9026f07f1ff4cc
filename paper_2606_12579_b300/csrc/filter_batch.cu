// filter_cloud_batch: the perception filter of Sec. IV-B / Sec. V-A for many
// clouds at once.  A single frame is a few MB -- far less than one launch
// needs to approach HBM bandwidth -- so a stream of frames (or several
// sensors) goes through ONE sequence of four launches: every launch covers
// the blocks of all jobs, a block -> job table maps each block to its cloud,
// and the building blocks are those of filter_cloud (filter_device.cuh), so
// each job's S_W is bit-identical to filter_cloud on the same cloud.
//
//   kf_keys   points -> keys + bitmap bits
//   kf_sums   per-block (and per-chunk) popcounts; each job's last block
//             scans its block sums
//   kf_emit   ranks, keys, centres; publishes each job's N_O; clears the
//             bitmap behind it (the scratch is zeroed once at creation, so
//             no clearing launch is needed)
//   kf_count  per-voxel point counts and smallest indices
#include <math.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "filter_device.cuh"

namespace gmapp {
namespace {

constexpr int kMaxPointBlocksPerJob = 64;  // a few 4-point groups per thread

struct FilterJob {
    const float *xyz;
    int64_t n_raw;
    FilterArgs fa;
    uint32_t *bitmap, *chunk, *sums, *offsets, *counters, *keys;
    uint2 *pw;
    int32_t pt_blk0, pt_nblk, bm_blk0, bm_nblk, sb_blk0, sb_nblk;
    EmitOut o;
    int32_t *n_out;
};

__global__ void __launch_bounds__(kThreads) kf_keys(const FilterJob *J, const int32_t *pt_map) {
    const FilterJob &Q = J[pt_map[blockIdx.x]];
    const FilterArgs fa = Q.fa;
    keys_range(Q.xyz, Q.n_raw, fa, Q.keys, Q.bitmap, blockIdx.x - Q.pt_blk0, Q.pt_nblk);
}

__global__ void __launch_bounds__(kBmThreads) kf_sums(const FilterJob *J, const int32_t *sb_map) {
    const FilterJob &Q = J[sb_map[blockIdx.x]];
    bitmap_sums_block(Q.bitmap, Q.chunk, Q.sums, Q.offsets, Q.counters, Q.counters + 1,
                      blockIdx.x - Q.sb_blk0, Q.sb_nblk);
}

__global__ void __launch_bounds__(kBmThreads) kf_emit(const FilterJob *J, const int32_t *bm_map,
                                                      uint32_t *err) {
    const FilterJob &Q = J[bm_map[blockIdx.x]];
    const int64_t blk = blockIdx.x - Q.bm_blk0;
    const EmitOut o = Q.o;
    if (blk == 0 && threadIdx.x == 0) {
        const uint32_t t = Q.counters[1];
        *Q.n_out = static_cast<int32_t>(t);
        if (t > o.cap) raise_error(err, GMAPP_DEVERR_CAPACITY);
    }
    const FilterArgs fa = Q.fa;
    emit_block<kChunksPerWarp>(Q.bitmap, Q.offsets, Q.chunk, Q.pw, fa, o, blk, true);
}

__global__ void __launch_bounds__(kThreads) kf_count(const FilterJob *J, const int32_t *pt_map) {
    const FilterJob &Q = J[pt_map[blockIdx.x]];
    count_range(Q.keys, Q.n_raw, Q.pw, Q.o.counts, Q.o.rep, Q.o.cap,
                blockIdx.x - Q.pt_blk0, Q.pt_nblk);
}

}  // namespace
}  // namespace gmapp

using namespace gmapp;

struct gmapp_filter_batch {
    gmapp_ctx *ctx = nullptr;
    FilterJob *d_jobs = nullptr;
    int32_t *d_pt_map = nullptr, *d_bm_map = nullptr, *d_sb_map = nullptr;
    void *d_ws = nullptr;
    int32_t pt_blocks = 0, bm_blocks = 0, sb_blocks = 0;
};

namespace {

void release(gmapp_filter_batch *fb) {
    cudaFree(fb->d_jobs);
    cudaFree(fb->d_pt_map);
    cudaFree(fb->d_bm_map);
    cudaFree(fb->d_sb_map);
    cudaFree(fb->d_ws);
}

}  // namespace

extern "C" gmapp_status gmapp_filter_batch_create(gmapp_ctx *ctx, const gmapp_cloud_job *jobs,
                                                  int32_t n_jobs, gmapp_filter_batch **out) {
    if (!ctx || !jobs || n_jobs < 1 || !out) {
        set_error("gmapp_filter_batch_create: invalid argument");
        return GMAPP_ERR_INVALID_ARG;
    }
    *out = nullptr;
    std::vector<FilterJob> hj(n_jobs);
    std::vector<int32_t> pt_map, bm_map, sb_map;
    std::vector<size_t> ws_off(n_jobs);
    size_t ws_total = 0;
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
        const Layout L = layout(J.n_raw, &J.ws);
        ws_off[q] = ws_total;
        ws_total = align_up(ws_total + L.total, 256);
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
        D.pt_blk0 = static_cast<int32_t>(pt_map.size());
        D.pt_nblk = static_cast<int32_t>(std::max<int64_t>(
            1, std::min<int64_t>((J.n_raw / 4 + kThreads - 1) / kThreads, kMaxPointBlocksPerJob)));
        for (int i = 0; i < D.pt_nblk; ++i) pt_map.push_back(q);
        D.bm_blk0 = static_cast<int32_t>(bm_map.size());
        D.bm_nblk = static_cast<int32_t>(L.n_blocks);
        for (int i = 0; i < D.bm_nblk; ++i) bm_map.push_back(q);
        D.sb_blk0 = static_cast<int32_t>(sb_map.size());
        D.sb_nblk = static_cast<int32_t>(L.n_sblocks);
        for (int i = 0; i < D.sb_nblk; ++i) sb_map.push_back(q);
        D.o = EmitOut{o.keys, o.counts, o.rep_idx, o.x, o.y, o.z, o.cap};
        D.n_out = o.n;
        if (pt_map.size() > 0x7fffffffu || bm_map.size() > 0x7fffffffu) {
            set_error("gmapp_filter_batch_create: too many blocks");
            return GMAPP_ERR_CAPACITY;
        }
    }
    gmapp_filter_batch *fb = new gmapp_filter_batch();
    fb->ctx = ctx;
    fb->pt_blocks = static_cast<int32_t>(pt_map.size());
    fb->bm_blocks = static_cast<int32_t>(bm_map.size());
    fb->sb_blocks = static_cast<int32_t>(sb_map.size());
    cudaError_t e = cudaMalloc(&fb->d_ws, std::max<size_t>(ws_total, 256));
    // zero scratch: bitmaps and counters start clear, and each run leaves
    // them clear again
    if (e == cudaSuccess) e = cudaMemset(fb->d_ws, 0, std::max<size_t>(ws_total, 256));
    if (e == cudaSuccess) e = cudaMalloc(&fb->d_jobs, sizeof(FilterJob) * n_jobs);
    if (e == cudaSuccess) e = cudaMalloc(&fb->d_pt_map, sizeof(int32_t) * pt_map.size());
    if (e == cudaSuccess) e = cudaMalloc(&fb->d_bm_map, sizeof(int32_t) * bm_map.size());
    if (e == cudaSuccess) e = cudaMalloc(&fb->d_sb_map, sizeof(int32_t) * sb_map.size());
    if (e == cudaSuccess) {
        char *ws = static_cast<char *>(fb->d_ws);
        for (int q = 0; q < n_jobs; ++q) {
            const Layout L = layout(jobs[q].n_raw, &jobs[q].ws);
            char *base = ws + ws_off[q];
            FilterJob &D = hj[q];
            D.bitmap = reinterpret_cast<uint32_t *>(base + L.off_bitmap);
            D.pw = reinterpret_cast<uint2 *>(base + L.off_pw);
            D.chunk = reinterpret_cast<uint32_t *>(base + L.off_chunk);
            D.sums = reinterpret_cast<uint32_t *>(base + L.off_sums);
            D.offsets = reinterpret_cast<uint32_t *>(base + L.off_offsets);
            D.counters = reinterpret_cast<uint32_t *>(base + L.off_counters);
            D.keys = reinterpret_cast<uint32_t *>(base + L.off_keys);
        }
        e = cudaMemcpy(fb->d_jobs, hj.data(), sizeof(FilterJob) * n_jobs,
                       cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(fb->d_pt_map, pt_map.data(), sizeof(int32_t) * pt_map.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(fb->d_bm_map, bm_map.data(), sizeof(int32_t) * bm_map.size(),
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
    release(fb);
    delete fb;
}

extern "C" gmapp_status filter_cloud_batch(gmapp_filter_batch *fb, gmapp_stream stream) {
    if (!fb) {
        set_error("filter_cloud_batch: NULL batch");
        return GMAPP_ERR_INVALID_ARG;
    }
    kf_keys<<<fb->pt_blocks, kThreads, 0, stream>>>(fb->d_jobs, fb->d_pt_map);
    kf_sums<<<fb->sb_blocks, kBmThreads, 0, stream>>>(fb->d_jobs, fb->d_sb_map);
    kf_emit<<<fb->bm_blocks, kBmThreads, 0, stream>>>(fb->d_jobs, fb->d_bm_map, fb->ctx->d_err);
    kf_count<<<fb->pt_blocks, kThreads, 0, stream>>>(fb->d_jobs, fb->d_pt_map);
    GMAPP_CHECK_CUDA(cudaGetLastError());
    return GMAPP_OK;
}
