// Context management and error reporting of the C ABI (include/gmapp.h).
#include <stdarg.h>
#include <stdio.h>

#include "gmapp_internal.cuh"

namespace gmapp {

static thread_local char g_last_error[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}

gmapp_status cuda_fail(cudaError_t e, const char *what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return GMAPP_ERR_CUDA;
}

}  // namespace gmapp

using namespace gmapp;

extern "C" const char *gmapp_last_error(void) { return g_last_error; }

extern "C" gmapp_status gmapp_create(gmapp_ctx **out, int device) {
    if (!out) {
        set_error("gmapp_create: out is NULL");
        return GMAPP_ERR_INVALID_ARG;
    }
    *out = nullptr;
    int n = 0;
    GMAPP_CHECK_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) {
        set_error("gmapp_create: device %d out of range (%d devices)", device, n);
        return GMAPP_ERR_INVALID_ARG;
    }
    GMAPP_CHECK_CUDA(cudaSetDevice(device));
    gmapp_ctx *c = new gmapp_ctx();
    c->device = device;
    cudaError_t e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&c->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                   device);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_err, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(uint32_t));
    const size_t xbytes = xbuf_bytes(c->sm_count);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_xbuf, xbytes);
    if (e == cudaSuccess) e = cudaMemset(c->d_xbuf, 0, xbytes);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_xctl, 2 * sizeof(uint32_t));
    // epoch 1, counter 0: all-zero slots (epoch 0) never match a tag
    const uint32_t ctl0[2] = {1u, 0u};
    if (e == cudaSuccess) e = cudaMemcpy(c->d_xctl, ctl0, sizeof(ctl0), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->x_done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (c->d_err) cudaFree(c->d_err);
        if (c->d_xbuf) cudaFree(c->d_xbuf);
        if (c->d_xctl) cudaFree(c->d_xctl);
        delete c;
        return cuda_fail(e, "gmapp_create");
    }
    *out = c;
    return GMAPP_OK;
}

extern "C" void gmapp_destroy(gmapp_ctx *ctx) {
    if (!ctx) return;
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->d_xbuf) cudaFree(ctx->d_xbuf);
    if (ctx->d_xctl) cudaFree(ctx->d_xctl);
    if (ctx->x_done) cudaEventDestroy(ctx->x_done);
    delete ctx;
}

extern "C" gmapp_status gmapp_peek_device_error(gmapp_ctx *ctx, uint32_t *bits) {
    if (!ctx || !bits) {
        set_error("gmapp_peek_device_error: NULL argument");
        return GMAPP_ERR_INVALID_ARG;
    }
    GMAPP_CHECK_CUDA(cudaMemcpy(bits, ctx->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    return GMAPP_OK;
}

extern "C" gmapp_status gmapp_set_wait_limit(gmapp_ctx *ctx, uint32_t polls) {
    if (!ctx) {
        set_error("gmapp_set_wait_limit: ctx is NULL");
        return GMAPP_ERR_INVALID_ARG;
    }
    ctx->wait_limit = polls;
    return GMAPP_OK;
}

extern "C" gmapp_status gmapp_sync(gmapp_ctx *ctx, gmapp_stream stream) {
    if (!ctx) {
        set_error("gmapp_sync: ctx is NULL");
        return GMAPP_ERR_INVALID_ARG;
    }
    GMAPP_CHECK_CUDA(cudaStreamSynchronize(stream));
    uint32_t bits = 0;
    GMAPP_CHECK_CUDA(cudaMemcpy(&bits, ctx->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (bits) GMAPP_CHECK_CUDA(cudaMemset(ctx->d_err, 0, sizeof(uint32_t)));
    if (bits & GMAPP_DEVERR_TIMEOUT) {
        set_error("device: a bounded wait gave up (error bits 0x%x)", bits);
        return GMAPP_ERR_TIMEOUT;
    }
    if (bits & GMAPP_DEVERR_CAPACITY) {
        set_error("device: capacity exceeded (error bits 0x%x)", bits);
        return GMAPP_ERR_CAPACITY;
    }
    if (bits & GMAPP_DEVERR_BOUNDS) {
        set_error("device: an input read on the device is out of range (error bits 0x%x)", bits);
        return GMAPP_ERR_INVALID_ARG;
    }
    if (bits) {
        set_error("device: error bits 0x%x", bits);
        return GMAPP_ERR_CUDA;
    }
    return GMAPP_OK;
}
