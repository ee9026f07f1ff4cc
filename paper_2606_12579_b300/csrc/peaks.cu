// gmapp_measure_peaks: event-timed probes of the FP32 FMA pipe and the SFU
// (the two pipes the all-pairs force loop of Eq. (mfi) / Alg. 1 runs on),
// so the roofline divides by rates measured on the part, not by a nominal
// lane count.  See include/gmapp_peaks.h.
#include <algorithm>

#include "../../include/gmapp_peaks.h"
#include "gmapp_internal.cuh"

namespace gmapp {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeCtasPerSm = 4;

using u64 = unsigned long long;

struct ProbeClock {
    long long cycles;
    u64 ns;
};

__device__ __forceinline__ u64 global_ns() {
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ u64 pack2(float lo, float hi) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float sum2(u64 v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return a + b;
}
__device__ __forceinline__ u64 ffma2(u64 a, u64 b, u64 c) {
    u64 r;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ float mufu_rsqrt(float x) {
    float r;
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// CTA 0's thread 0 brackets its own run with the SM cycle counter and the
// global nanosecond timer: their ratio is the SM clock during the probe.
struct ClockMark {
    long long c0 = 0;
    u64 t0 = 0;
    __device__ __forceinline__ void start() {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            t0 = global_ns();
            c0 = clock64();
        }
    }
    __device__ __forceinline__ void stop(ProbeClock *out) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            const long long c1 = clock64();
            const u64 t1 = global_ns();
            out->cycles = c1 - c0;
            out->ns = t1 - t0;
        }
    }
};

// A result no chain can produce (a NaN payload): the store never happens,
// but the compiler must keep every chain.
__device__ __forceinline__ void keep(float s, uint32_t *sink) {
    if (__float_as_uint(s) == 0x7fc00001u) atomicOr(sink, 1u);
}

// Each chain is x <- x a + b with a just below 1: it settles near b/(1-a),
// never overflows and never goes subnormal.
__global__ void __launch_bounds__(kProbeThreads) k_probe_ffma2(int iters, uint32_t *sink,
                                                               ProbeClock *clk) {
    ClockMark m;
    m.start();
    const float s0 = 1.0f + 1e-3f * (threadIdx.x & 7);
    u64 acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = pack2(s0 + i, s0 - i);
    const u64 a = pack2(0.9999999f, 0.99999994f), b = pack2(1e-7f, 2e-7f);
#pragma unroll 2
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 12; ++i) acc[i] = ffma2(acc[i], a, b);
    }
    m.stop(clk);
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 12; ++i) s += sum2(acc[i]);
    keep(s, sink);
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_ffma(int iters, uint32_t *sink,
                                                              ProbeClock *clk) {
    ClockMark m;
    m.start();
    const float s0 = 1.0f + 1e-3f * (threadIdx.x & 7);
    float acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = s0 + i;
    const float a = 0.9999999f, b = 1e-7f;
#pragma unroll 4
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 16; ++i) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(acc[i]) : "f"(a), "f"(b));
    }
    m.stop(clk);
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 16; ++i) s += acc[i];
    keep(s, sink);
}

// rsqrt(rsqrt(x)) = x^(1/4): every chain converges to 1.
__global__ void __launch_bounds__(kProbeThreads) k_probe_mufu(int iters, uint32_t *sink,
                                                              ProbeClock *clk) {
    ClockMark m;
    m.start();
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = 1.5f + 0.25f * i + 1e-3f * (threadIdx.x & 7);
#pragma unroll 4
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = mufu_rsqrt(x[i]);
    }
    m.stop(clk);
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    keep(s, sink);
}

// The pair loop's mix: 8 packed FMAs (16 lane-FMAs) and 2 SFU results per
// thread and iteration, on independent chains.
__global__ void __launch_bounds__(kProbeThreads) k_probe_mix(int iters, uint32_t *sink,
                                                             ProbeClock *clk) {
    ClockMark m;
    m.start();
    const float s0 = 1.0f + 1e-3f * (threadIdx.x & 7);
    u64 acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = pack2(s0 + i, s0 - i);
    float x0 = 1.5f + s0, x1 = 2.5f + s0;
    const u64 a = pack2(0.9999999f, 0.99999994f), b = pack2(1e-7f, 2e-7f);
#pragma unroll 4
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] = ffma2(acc[i], a, b);
        x0 = mufu_rsqrt(x0);
        x1 = mufu_rsqrt(x1);
    }
    m.stop(clk);
    float s = x0 + x1;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += sum2(acc[i]);
    keep(s, sink);
}

using ProbeFn = void (*)(int, uint32_t *, ProbeClock *);

// Fastest of `reps` launches (seconds) and the SM clock (MHz) of that launch.
gmapp_status time_probe(ProbeFn fn, int grid, int iters, int reps, uint32_t *sink,
                        ProbeClock *d_clk, double *best_s, double *mhz) {
    cudaEvent_t e0, e1;
    GMAPP_CHECK_CUDA(cudaEventCreate(&e0));
    GMAPP_CHECK_CUDA(cudaEventCreate(&e1));
    fn<<<grid, kProbeThreads>>>(iters / 8, sink, d_clk);  // warm-up (clock ramp, module load)
    cudaError_t e = cudaGetLastError();
    double best = 1e30, best_mhz = 0.0;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        e = cudaEventRecord(e0);
        if (e == cudaSuccess) fn<<<grid, kProbeThreads>>>(iters, sink, d_clk);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(e1);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        ProbeClock h{};
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess) e = cudaMemcpy(&h, d_clk, sizeof(h), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && ms > 0.0f && ms * 1e-3 < best) {
            best = ms * 1e-3;
            best_mhz = h.ns ? static_cast<double>(h.cycles) / static_cast<double>(h.ns) * 1e3 : 0.0;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "gmapp_measure_peaks");
    *best_s = best;
    *mhz = best_mhz;
    return GMAPP_OK;
}

}  // namespace
}  // namespace gmapp

using namespace gmapp;

extern "C" int gmapp_measure_peaks(int32_t reps, gmapp_peaks *out) {
    if (!out || reps < 1) {
        set_error("gmapp_measure_peaks: NULL output or reps < 1");
        return GMAPP_ERR_INVALID_ARG;
    }
    int dev = 0, sms = 0;
    GMAPP_CHECK_CUDA(cudaGetDevice(&dev));
    GMAPP_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = sms * kProbeCtasPerSm;
    const double threads = static_cast<double>(grid) * kProbeThreads;
    void *buf = nullptr;
    GMAPP_CHECK_CUDA(cudaMalloc(&buf, 64));
    uint32_t *sink = static_cast<uint32_t *>(buf);
    ProbeClock *clk = reinterpret_cast<ProbeClock *>(static_cast<char *>(buf) + 16);
    cudaError_t e = cudaMemset(buf, 0, 64);
    if (e != cudaSuccess) {
        cudaFree(buf);
        return cuda_fail(e, "gmapp_measure_peaks");
    }
    // iteration counts: a few milliseconds per probe on a 148-SM part
    const int it_fma = 1 << 16, it_mufu = 1 << 13, it_mix = 1 << 14;
    double t2 = 0, t1 = 0, tm = 0, tx = 0, mhz2 = 0, mhz1 = 0, mhzm = 0, mhzx = 0;
    gmapp_status st = time_probe(k_probe_ffma2, grid, it_fma, reps, sink, clk, &t2, &mhz2);
    if (st == GMAPP_OK) st = time_probe(k_probe_ffma, grid, it_fma / 2, reps, sink, clk, &t1, &mhz1);
    if (st == GMAPP_OK) st = time_probe(k_probe_mufu, grid, it_mufu, reps, sink, clk, &tm, &mhzm);
    if (st == GMAPP_OK) st = time_probe(k_probe_mix, grid, it_mix, reps, sink, clk, &tx, &mhzx);
    cudaFree(buf);
    if (st != GMAPP_OK) return st;
    const double fma2_lanes = threads * it_fma * 24.0 / t2;        // lane-FMAs per second
    const double fma1_lanes = threads * (it_fma / 2) * 16.0 / t1;
    const double mufu = threads * it_mufu * 8.0 / tm;             // results per second
    const double mix_fma = threads * it_mix * 16.0 / tx, mix_mufu = threads * it_mix * 2.0 / tx;
    out->fp32_tflops = 2.0 * fma2_lanes / 1e12;
    out->fp32_tflops_scalar = 2.0 * fma1_lanes / 1e12;
    out->fma_lanes_per_clk_sm = mhz2 > 0 ? fma2_lanes / (mhz2 * 1e6) / sms : 0.0;
    out->fma_lanes_per_clk_sm_scalar = mhz1 > 0 ? fma1_lanes / (mhz1 * 1e6) / sms : 0.0;
    out->sfu_lanes_per_clk_sm = mhzm > 0 ? mufu / (mhzm * 1e6) / sms : 0.0;
    out->sfu_gops = mufu / 1e9;
    out->mix_fma_busy = mix_fma / fma2_lanes * (mhz2 > 0 && mhzx > 0 ? mhz2 / mhzx : 1.0);
    out->mix_sfu_busy = mix_mufu / mufu * (mhzm > 0 && mhzx > 0 ? mhzm / mhzx : 1.0);
    out->sm_mhz = mhz2;
    out->sm_count = sms;
    return GMAPP_OK;
}
