// Calibration: FP64 FMA throughput of the current GPU, the denominator of the
// Legendre stage's roofline (the stage is bound by the FP64 pipe).
#include "sht_internal.h"

namespace {

constexpr int DIAG_T = 256;
constexpr int DIAG_ITERS = 2048;
constexpr int DIAG_CHAINS = 8;

// Independent FMA chains per thread; one result per thread keeps the work live.
__global__ void __launch_bounds__(DIAG_T) dfma_kernel(double *out, double a, double b)
{
    double x[DIAG_CHAINS];
#pragma unroll
    for (int i = 0; i < DIAG_CHAINS; ++i) x[i] = threadIdx.x * 1e-3 + i;
    for (int it = 0; it < DIAG_ITERS; ++it) {
#pragma unroll
        for (int i = 0; i < DIAG_CHAINS; ++i) x[i] = fma(x[i], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < DIAG_CHAINS; ++i) s += x[i];
    out[blockIdx.x * DIAG_T + threadIdx.x] = s;
}

}  // namespace

extern "C" sht_status sht_fp64_fma_tflops(double *tflops)
{
    if (!tflops) return SHT_EINVAL;
    *tflops = 0.0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SHT_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SHT_ECUDA;
    const int blocks = sms * 8;
    double *out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks * DIAG_T) != cudaSuccess) return SHT_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    cudaError_t err = cudaSuccess;
    for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {
        cudaEventRecord(e0, 0);
        dfma_kernel<<<blocks, DIAG_T>>>(out, 0.999999, 1e-7);
        cudaEventRecord(e1, 0);
        err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms > 0.f && ms < best) best = ms;  // first launch is a warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return SHT_ECUDA;
    const double flops = 2.0 * (double)blocks * DIAG_T * DIAG_ITERS * DIAG_CHAINS;
    *tflops = flops / (best * 1e-3) / 1e12;
    return SHT_OK;
}
