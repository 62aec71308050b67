// Self-test of the bounded device-side wait that the library's TMA and
// tensor-core kernels use: a wait on an mbarrier gives up after a budget of
// SM clock cycles, records that it did, and returns, and the host turns the
// record into HLBM_ERR_TIMEOUT.  The probe arms an mbarrier for one arrival
// and either makes that arrival or not, so both outcomes can be checked
// without stalling or faulting the device.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hlbm.h"

namespace {

__device__ int g_probe_status;

__global__ void wait_probe_kernel(long long budget, int arrive)
{
    __shared__ __align__(8) uint64_t bar;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
    const long long t0 = clock64();
    int status = 1;  // 1: the wait ran out, 0: the phase completed
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(0u)
            : "memory");
        if (ok) {
            status = 0;
            break;
        }
        if (clock64() - t0 > budget) break;
    }
    g_probe_status = status;
}

}  // namespace

extern "C" int hlbm_selftest_wait(void *stream, long long budget_cycles, int arrive)
{
    if (budget_cycles < 1 || budget_cycles > (1ll << 31)) return HLBM_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int unset = -1;
    if (cudaMemcpyToSymbolAsync(g_probe_status, &unset, sizeof(int), 0, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return HLBM_ERR_CUDA;
    wait_probe_kernel<<<1, 1, 0, s>>>(budget_cycles, arrive ? 1 : 0);
    if (cudaGetLastError() != cudaSuccess) return HLBM_ERR_CUDA;
    int status = unset;
    if (cudaMemcpyFromSymbolAsync(&status, g_probe_status, sizeof(int), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return HLBM_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return HLBM_ERR_CUDA;
    if (status == 1) return HLBM_ERR_TIMEOUT;
    return status == 0 ? HLBM_OK : HLBM_ERR_CUDA;
}

// ---- FP64 arithmetic rate ------------------------------------------------------
// The FP64 form of the step is bound by the GPU's FP64 pipe, whose rate on
// this part is far below the FP32 and tensor rates and is not in the
// measured peaks.  The probe measures it: every thread runs eight
// independent chains of fused multiply-adds x <- x a + b (a just below one,
// so the values stay normal), enough CTAs to fill every SM several times.
namespace {

constexpr int kRateChains = 8;
constexpr int kRateThreads = 256;

__device__ double g_rate_sink;

__global__ void __launch_bounds__(kRateThreads) fp64_rate_kernel(int iters, double a, double b)
{
    double x[kRateChains];
#pragma unroll
    for (int k = 0; k < kRateChains; k++) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < kRateChains; k++) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kRateChains; k++) s += x[k];
    if (s == -1.0) g_rate_sink = s;  // never true; keeps the chains live
}

}  // namespace

extern "C" int hlbm_selftest_fp64_rate(void *stream, int iters, double *fma_per_s)
{
    if (!fma_per_s || iters < 1 || iters > (1 << 24)) return HLBM_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return HLBM_ERR_CUDA;
    const int grid = 8 * sms;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return HLBM_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return HLBM_ERR_CUDA;
    }
    int rc = HLBM_OK;
    fp64_rate_kernel<<<grid, kRateThreads, 0, s>>>(iters / 8 > 0 ? iters / 8 : 1, 0.999999999, 1e-9);  // warm-up
    cudaEventRecord(e0, s);
    fp64_rate_kernel<<<grid, kRateThreads, 0, s>>>(iters, 0.999999999, 1e-9);
    cudaEventRecord(e1, s);
    float ms = 0.0f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.0f))
        rc = HLBM_ERR_CUDA;
    else
        *fma_per_s = (double)grid * kRateThreads * kRateChains * (double)iters / (ms * 1e-3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}
