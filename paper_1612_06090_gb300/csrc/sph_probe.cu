// sph_probe.cu -- libsph_probe.so: the FP32 FMA rate of the GPU (include/sph_probe.h), the
// denominator of the density pass's arithmetic roofline.
#include <cuda_runtime.h>

#include "sph_probe.h"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

// Eight independent dependent chains per thread keep every FMA pipe busy; the result feeds a
// store that never happens (the chains cannot reach the sentinel), so nothing is optimised away.
__global__ void __launch_bounds__(kThreads) k_fma(float *out, int iters, float b, float c)
{
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += a[k];
    if (s == -1.0f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_fma2(float *out, int iters, float b, float c)
{
    float2 a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = make_float2((float)(threadIdx.x + k) * 1e-3f, (float)k);
    const float2 bb = make_float2(b, b), cc = make_float2(c, c);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) a[k] = __ffma2_rn(a[k], bb, cc);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += a[k].x + a[k].y;
    if (s == -1.0f) out[blockIdx.x] = s;
}

}  // namespace

extern "C" int sph_probe_fp32_fma(void *cuda_stream, int32_t blocks_per_sm, int32_t iters, int32_t packed,
                                  double *tflops_out, double *ms_out)
{
    if (!tflops_out || !ms_out || blocks_per_sm < 1 || blocks_per_sm > 32 || iters < 1 || iters > (1 << 24))
        return 1;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 2;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 2;
    const int blocks = sms * blocks_per_sm;
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = 2;
    if (cudaMalloc(&out, blocks * sizeof(float)) != cudaSuccess) goto done;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) goto done;
    // one untimed launch brings the clocks up, then the timed one
    for (int rep = 0; rep < 2; rep++) {
        if (rep == 1 && cudaEventRecord(e0, st) != cudaSuccess) goto done;
        if (packed) k_fma2<<<blocks, kThreads, 0, st>>>(out, iters, 0.9999999f, 1e-7f);
        else k_fma<<<blocks, kThreads, 0, st>>>(out, iters, 0.9999999f, 1e-7f);
        if (cudaGetLastError() != cudaSuccess) goto done;
    }
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) goto done;
    {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f) goto done;
        const double flop = (double)blocks * kThreads * kChains * (double)iters * (packed ? 4.0 : 2.0);
        *ms_out = ms;
        *tflops_out = flop / (ms * 1e-3) / 1e12;
        rc = 0;
    }
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    return rc;
}
