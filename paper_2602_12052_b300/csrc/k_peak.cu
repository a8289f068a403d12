// Measured FP32 FMA throughput of the device: the denominator of the convolution's
// roofline (its bound is the FP32 ALU, whose peak the measured copy and GEMM
// figures do not give).  A grid of 8 CTAs per SM, each thread running eight
// independent FMA chains, so every scheduler has enough independent FMAs in flight to
// issue one per cycle.  The paper has no counterpart: this is a measurement tool.
#include "tred_internal.cuh"

namespace tred {

constexpr int PEAK_THREADS = 256;
constexpr int PEAK_CTAS_PER_SM = 8;
constexpr int PEAK_CHAINS = 8;

__global__ void __launch_bounds__(PEAK_THREADS, PEAK_CTAS_PER_SM) k_fp32_peak(float *__restrict__ sink, int iters,
                                                                            float b, float c) {
    float a[PEAK_CHAINS];
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = fmaf(a[k], b, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) s += a[k];
    sink[blockIdx.x * PEAK_THREADS + threadIdx.x] = s;   // keeps the chains live
}

}  // namespace tred

extern "C" int32_t tred_fp32_peak(float *sink, int64_t sink_len, int32_t iters, void *stream, double *tflops,
                                  int32_t *sms_out) {
    using namespace tred;
    if (!sink || !tflops || iters < 1) return TRED_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms < 1)
        return TRED_ERR_CUDA;
    const int grid = sms * PEAK_CTAS_PER_SM;
    if (sink_len < (int64_t)grid * PEAK_THREADS) return TRED_ERR_CAPACITY;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return TRED_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return TRED_ERR_CUDA;
    }
    // b slightly below one and c small keep every chain finite and away from denormals
    k_fp32_peak<<<grid, PEAK_THREADS, 0, s>>>(sink, iters, 0.9999f, 1e-4f);   // warm-up (clocks, caches)
    cudaEventRecord(e0, s);
    k_fp32_peak<<<grid, PEAK_THREADS, 0, s>>>(sink, iters, 0.9999f, 1e-4f);
    cudaEventRecord(e1, s);
    int rc = TRED_OK;
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
        rc = TRED_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    const double flop = 2.0 * 16.0 * PEAK_CHAINS * (double)iters * grid * PEAK_THREADS;
    *tflops = flop / (ms * 1e-3) / 1e12;
    if (sms_out) *sms_out = sms;
    return TRED_OK;
}
