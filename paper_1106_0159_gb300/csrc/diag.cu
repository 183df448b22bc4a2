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

// The failure path of the bounded waits: an mbarrier that expects one arrival nobody makes, polled
// `polls` times with a short sleep like the tensor-core kernels' waits; when the poll budget runs
// out the kernel records the timeout in the status word and returns (no trap, no hang).
__global__ void wait_timeout_probe(int *status, long long polls)
{
    __shared__ __align__(8) unsigned long long mbar;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(&mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t done = 0;
        for (long long it = 0; it < polls && !done; ++it) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                : "=r"(done)
                : "r"(a), "r"(0));
            if (!done) __nanosleep(32);
        }
        if (!done) atomicOr(status, 1);
    }
}

}  // namespace

// Exercise the timeout path of the device waits on the plan's status word (see the header).
extern "C" sht_status sht_plan_selftest_timeout(sht_plan_t plan, void *stream)
{
    if (!plan) return SHT_EINVAL;
    wait_timeout_probe<<<1, 32, 0, (cudaStream_t)stream>>>(plan->p.d_status, 1 << 12);
    return cudaGetLastError() == cudaSuccess ? SHT_OK : SHT_ECUDA;
}

extern "C" sht_status sht_fp64_fma_tflops(double *tflops)
{
    if (!tflops) return SHT_EINVAL;
    *tflops = 0.0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SHT_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return SHT_ECUDA;
    const int blocks = sms * 8;
    double *out = nullptr;
    if (sht::dev_malloc(&out, sizeof(double) * blocks * DIAG_T) != cudaSuccess) return SHT_ENOMEM;
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
