/*
 * sph_probe.h -- measurement aid beside the solver: the FP32 arithmetic peak of the GPU.
 *
 * The density pass is bound by FP32 arithmetic, not by memory or tensor cores, so its roofline
 * fraction needs the FP32 rate the GPU actually reaches.  The paper has no counterpart (its
 * kernel ran on CPUs); this call only measures the hardware.  It lives in its own library,
 * libsph_probe.so, so the solver library carries no benchmark code.
 */
#ifndef SPH_PROBE_H
#define SPH_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Time a grid of independent chains of dependent FP32 fused multiply-adds on the current
 * device and stream (cuda_stream: a cudaStream_t, NULL = legacy default stream): `blocks_per_sm`
 * blocks of 256 threads per SM, each thread running 8 chains of `iters` FMAs (packed == 0:
 * scalar fma.rn.f32) or of `iters` two-wide FMAs (packed == 1: fma.rn.f32x2, 4 flop each).
 * Writes the rate in TFLOP/s (2 flop per FMA lane) and the kernel time measured with CUDA
 * events around the launch.  Synchronises the stream.  Returns 0 on success, 1 for a bad
 * argument (NULL outputs, blocks_per_sm outside 1..32, iters outside 1..2^24), 2 for a CUDA
 * error. */
int sph_probe_fp32_fma(void *cuda_stream, int32_t blocks_per_sm, int32_t iters, int32_t packed,
                       double *tflops_out, double *ms_out);

#ifdef __cplusplus
}
#endif

#endif /* SPH_PROBE_H */
