// Internal declarations shared by the CUDA sources of libgmapp.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/gmapp.h"

struct gmapp_ctx {
    int device;
    int sm_count;
    int max_smem_optin;   // bytes of dynamic shared memory one CTA may opt into
    uint32_t *d_err;      // device error word (GMAPP_DEVERR_* bits)
    // exchange slots of the grid-exchange rollout (one launch at a time):
    // [sm_count][2 halves][2 parities][kMaxAgents][2] tagged words, and the
    // launch epoch / finished-CTA counter
    uint64_t *d_xbuf;
    uint32_t *d_xctl;
    cudaEvent_t x_done;   // completion of the last grid-exchange launch
    bool x_pending;       // x_done has been recorded
    uint32_t wait_limit;  // cap on the polls of a bounded rollout wait (0 = defaults)
};

namespace gmapp {

// Thread-local last error text (declared in api.cu).
void set_error(const char *fmt, ...);
gmapp_status cuda_fail(cudaError_t e, const char *what);

#define GMAPP_CHECK_CUDA(call)                                  \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return gmapp::cuda_fail(e_, #call); \
    } while (0)

// Bounded-wait limit for every device-side spin (iterations of try_wait).
constexpr uint32_t kSpinLimit = 1u << 24;
// Bounded polls of a word in global memory (each an L2 round trip).
constexpr uint32_t kPollLimit = 1u << 22;

// ---------------------------------------------------------------------------
// Inline-PTX helpers: shared-memory addresses, mbarriers, 1-D bulk copies
// (TMA engine), thread-block-cluster rank/mapping/barrier.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Wait until the mbarrier phase with parity `parity` completes; gives up
// after kSpinLimit polls and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          uint32_t limit = kSpinLimit) {
    uint32_t addr = smem_u32(bar);
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// As mbar_wait, with acquire at cluster scope: data that other CTAs of the
// cluster delivered with st_async_v2f32 on this barrier is visible after it.
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t *bar, uint32_t parity,
                                                  uint32_t limit = kSpinLimit) {
    uint32_t addr = smem_u32(bar);
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Asynchronous 8-byte store into the shared memory of a cluster CTA; its
// byte count completes on that CTA's mbarrier `remote_bar` (both addresses
// from map_smem).
__device__ __forceinline__ void st_async_v2f32(uint32_t remote_addr, float a, float b,
                                               uint32_t remote_bar) {
    asm volatile(
        "st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(
            remote_addr),
        "f"(a), "f"(b), "r"(remote_bar)
        : "memory");
}

// 64-bit relaxed accesses at GPU scope (single-copy atomic, never served
// from a stale L1 line): the grid exchange packs a 32-bit tag and a 32-bit
// payload into one word, so no other ordering is needed.
__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Named CTA barriers for producer/consumer hand-offs between warps: the
// producers arrive (no wait), the consumers sync; n counts all threads of
// both sides (a multiple of 32, whole warps).
__device__ __forceinline__ void named_sync(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int n) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// 1-D bulk copy global -> this CTA's shared memory, completing on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t cluster_id_x() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}

// Address of the same shared-memory variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_smem(uint32_t local_addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local_addr), "r"(rank));
    return r;
}

__device__ __forceinline__ void st_cluster_f32(uint32_t addr, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

__device__ __forceinline__ void st_cluster_v2f32(uint32_t addr, float a, float b) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(a), "f"(b)
                 : "memory");
}

// Split cluster barrier: arrive (release: this thread's earlier stores,
// including DSMEM stores, become visible to the cluster) ... wait (acquire).
__device__ __forceinline__ void cluster_arrive() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
}

__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void raise_error(uint32_t *err, uint32_t bits) {
    if (err) atomicOr(err, bits);
}

// Index checks of the bounds-checked build (compiled with
// -DGMAPP_BOUNDS_CHECK): an index outside [0, n) sets GMAPP_DEVERR_BOUNDS
// in the device error word and the caller skips the access.  In the normal
// build the check is the constant true and compiles to nothing.
#ifdef GMAPP_BOUNDS_CHECK
__device__ __forceinline__ bool bc_ok(int64_t i, int64_t n, uint32_t *err) {
    if (i >= 0 && i < n) return true;
    raise_error(err, GMAPP_DEVERR_BOUNDS);
    return false;
}
#else
__device__ __forceinline__ constexpr bool bc_ok(int64_t, int64_t, uint32_t *) { return true; }
#endif

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bytes of the grid-exchange slots for up to `ctas` CTAs: per CTA
// [2 halves][2 parities][16 agents][6 words] -- the rollout uses 2 words
// per agent (W, min d^2), the adjoint 6 (W, grad W, min d^2, argmin).
inline size_t xbuf_bytes(int ctas) {
    return static_cast<size_t>(ctas) * 2 * 2 * 16 * 6 * sizeof(uint64_t);
}

// Launches that exchange through the context's grid slots use them one at
// a time: outside stream capture, each waits for the previous one (on any
// stream) and records its own completion; inside capture the caller's graph
// orders them.
inline gmapp_status grid_exchange_begin(gmapp_ctx *ctx, cudaStream_t stream, bool *capturing) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    GMAPP_CHECK_CUDA(cudaStreamIsCapturing(stream, &cs));
    *capturing = cs != cudaStreamCaptureStatusNone;
    if (!*capturing && ctx->x_pending) GMAPP_CHECK_CUDA(cudaStreamWaitEvent(stream, ctx->x_done, 0));
    return GMAPP_OK;
}
inline gmapp_status grid_exchange_end(gmapp_ctx *ctx, cudaStream_t stream, bool capturing) {
    if (!capturing) {
        GMAPP_CHECK_CUDA(cudaEventRecord(ctx->x_done, stream));
        ctx->x_pending = true;
    }
    return GMAPP_OK;
}

}  // namespace gmapp
