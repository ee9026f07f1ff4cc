/* Measured compute peaks of the GPU the library runs on.
 *
 * The force kernel's roofline (Eq. (mfi) summed over all obstacle pairs,
 * Alg. 1) is the FP32 FMA pipe plus the SFU, not the tensor cores, so its
 * fraction of peak needs the rate those pipes actually sustain on this
 * part.  gmapp_measure_peaks times short event-bracketed probe kernels:
 *
 *   - packed FMA:   fma.rn.f32x2 on 12 independent accumulators per thread
 *                   (the instruction the pair loop uses);
 *   - scalar FMA:   fma.rn.f32 on 16 independent accumulators per thread;
 *   - SFU:          rsqrt.approx.ftz.f32 on 8 independent chains per thread;
 *   - pair mix:     8 packed FMAs + 2 rsqrt.approx per iteration (the
 *                   pair loop's ratio of FMA-pipe to SFU work), reported as
 *                   the busy fraction of each pipe against the two rates
 *                   above.
 *
 * Every probe runs 4 CTAs of 256 threads per SM, takes the best of `reps`
 * launches, and reads the SM clock during the probe from clock64() and the
 * global nanosecond timer of CTA 0, so per-clock rates are independent of
 * the clock the GPU ran at.  The paper prints no hardware peak; this is
 * measurement infrastructure for the roofline, not part of the method. */
#ifndef GMAPP_PEAKS_H
#define GMAPP_PEAKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double fp32_tflops;            /* packed FMA: 2 flops per lane-FMA, whole GPU */
    double fp32_tflops_scalar;     /* scalar FMA, whole GPU */
    double fma_lanes_per_clk_sm;   /* packed FMA lane-operations per SM clock per SM */
    double fma_lanes_per_clk_sm_scalar;
    double sfu_lanes_per_clk_sm;   /* rsqrt.approx results per SM clock per SM */
    double sfu_gops;               /* rsqrt.approx results per second, whole GPU (1e9) */
    double mix_fma_busy;           /* pair mix: FMA-pipe rate / packed FMA rate */
    double mix_sfu_busy;           /* pair mix: SFU rate / rsqrt.approx rate */
    double sm_mhz;                 /* SM clock during the packed-FMA probe */
    int32_t sm_count;
} gmapp_peaks;

/* Runs the probes on the current device (synchronous; a few milliseconds
 * each).  `reps` >= 1 launches per probe, the fastest kept.  Allocates a
 * 64-byte device buffer for the clock readings and frees it before
 * returning.  Returns 0 on success, else a gmapp_status code with the
 * message in gmapp_last_error(). */
int gmapp_measure_peaks(int32_t reps, gmapp_peaks *out);

#ifdef __cplusplus
}
#endif

#endif /* GMAPP_PEAKS_H */
