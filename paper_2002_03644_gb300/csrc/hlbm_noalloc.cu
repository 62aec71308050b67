// hlbm_noalloc.cu -- diagnostics of a caller-owned state with no allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// runtime's memory budget (a host framework that hands out device buffers
// but forbids new allocations), or embedded callers that must not grow the
// device footprint after start-up.  hlbm_diagnostics_noalloc serves them: it
// runs the same FP64 reduction as hlbm_diagnostics, but its block partials
// live in a file-scope device array of fixed size instead of handle-owned
// memory.
//
// The array is a static __device__ symbol.  Host code must not pass its name
// to a kernel (on the host the name is only a stand-in, not a device
// address): every call looks up the real address with cudaGetSymbolAddress
// while the caller's device is current.  The lookup allocates nothing, and
// looking it up each time keeps the address right after a cudaDeviceReset
// (which unloads the module and places the array anew).  The first call on
// a device (and the first after a reset) loads the module: the array and all
// three kernels of this file.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>

#include "hlbm.h"

// The kernels of the shared header get internal linkage in this translation
// unit, so that its non-template kernels do not clash with hlbm_api.cu's.
namespace {
#include "hlbm_device.cuh"
}

using namespace hlbm;

namespace {

constexpr int NA_CHUNK = 16384;     // cells per block
constexpr int NA_MAX_BLOCKS = 1024; // partial slots in the static array
static_assert((long long)NA_CHUNK * NA_MAX_BLOCKS == HLBM_NOALLOC_MAX_CELLS, "capacity");

// [NA_MAX_BLOCKS][DIAG_NV] block partials followed by DIAG_NV results:
// (1024 * 8 + 8) doubles = 65.6 KB, held by every device that loads the
// library until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[NA_MAX_BLOCKS * DIAG_NV + DIAG_NV];

// Same reduction as diag_partial_kernel, but block b covers the fixed chunk
// [b * NA_CHUNK, (b + 1) * NA_CHUNK) so that the number of partials is
// bounded by the size of the static array.
template <typename T>
__global__ void __launch_bounds__(DIAG_NT)
diag_partial_chunk_kernel(const T *__restrict__ in, double *__restrict__ partial, const KParams kp)
{
    Consts<T> cs;
    cs.load(kp);
    const long long P = kp.plane;
    const long long ncell = (long long)kp.nx * kp.ny;
    const long long c0 = (long long)blockIdx.x * NA_CHUNK;
    const long long c1 = c0 + NA_CHUNK < ncell ? c0 + NA_CHUNK : ncell;
    double acc[DIAG_NV] = {0.0, 0.0, 0.0, 0.0, 1e300, 1e300, 0.0, 0.0};
    for (long long c = c0 + threadIdx.x; c < c1; c += DIAG_NT) {
        const int gy = (int)(c / kp.nx), gx = (int)(c - (long long)gy * kp.nx);
        const long long o = (long long)gy * kp.pitch + gx;
        T f[9];
#pragma unroll
        for (int i = 0; i < 9; i++) f[i] = in[i * P + o];
        T r, jx, jy;
        moments(f, r, jx, jy);
        const double rho = (double)r;
        const double u = (double)jx / rho, v = (double)jy / rho;
        const double th = (double)cs.theta(r, in[P_S * P + o]);
        const bool bad = !(rho > 0.0) || !(th > 0.0) || !isfinite(rho) || !isfinite(th) || !isfinite(u) || !isfinite(v);
        if (bad) { acc[7] += 1.0; continue; }
        acc[0] += rho; acc[1] += rho * u; acc[2] += rho * v;
        acc[3] += rho * kp.cv * th + 0.5 * rho * (u * u + v * v);
        acc[4] = fmin(acc[4], rho); acc[5] = fmin(acc[5], th);
        acc[6] = fmax(acc[6], sqrt(u * u + v * v) + sqrt(kp.gamma * th / 3.0));
    }
    __shared__ double red[DIAG_NV][DIAG_NT];
#pragma unroll
    for (int k = 0; k < DIAG_NV; k++) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = DIAG_NT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
#pragma unroll
            for (int k = 0; k < DIAG_NV; k++) {
                const double a = red[k][threadIdx.x], b = red[k][threadIdx.x + w];
                red[k][threadIdx.x] = (k == 4 || k == 5) ? fmin(a, b) : (k == 6 ? fmax(a, b) : a + b);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < DIAG_NV) partial[blockIdx.x * DIAG_NV + threadIdx.x] = red[threadIdx.x][0];
}

// Device address of the static array on the current device, looked up on
// every call.  The kernels are touched as well (cudaFuncGetAttributes), so
// that the first call loads everything a later call of either precision
// launches; neither step allocates device memory.
cudaError_t scratch_address(double **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, diag_partial_chunk_kernel<double>)) != cudaSuccess) return e;
    if ((e = cudaFuncGetAttributes(&fa, diag_partial_chunk_kernel<float>)) != cudaSuccess) return e;
    if ((e = cudaFuncGetAttributes(&fa, diag_final_kernel)) != cudaSuccess) return e;
    *out = static_cast<double *>(p);
    return cudaSuccess;
}

}  // namespace

extern "C" int hlbm_diagnostics_noalloc(const void *state, int precision, int nx, int ny, int pitch, double gamma,
                                        double out[8], void *stream)
{
    if (nx < 1 || ny < 1 || pitch < nx || !out) return HLBM_ERR_ARG;
    if ((long long)nx * ny > HLBM_NOALLOC_MAX_CELLS) return HLBM_ERR_ARG;  // beyond the static scratch
    if (precision != HLBM_FP64 && precision != HLBM_FP32) return HLBM_ERR_ARG;
    if (!(gamma > 1.0) || !state) return HLBM_ERR_ARG;
    // the legacy default stream synchronises with every blocking stream, and
    // work enqueued on it while another stream captures in global mode breaks
    // that capture: only an explicit stream is taken, and not one that is
    // being captured (the call ends with a synchronisation)
    if (!stream) return HLBM_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return HLBM_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) return HLBM_ERR_ARG;
    double *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return HLBM_ERR_CUDA;
    double *partial = scratch;
    double *result = scratch + NA_MAX_BLOCKS * DIAG_NV;

    KParams kp;
    memset(&kp, 0, sizeof(kp));
    kp.nx = nx; kp.ny = ny; kp.pitch = pitch; kp.plane = (long long)pitch * ny;
    kp.gamma = gamma;
    kp.gm1 = gamma - 1.0;
    kp.cv = (1.0 / 3.0) / (gamma - 1.0);
    kp.inv_cv = 1.0 / kp.cv;
    kp.two_minus_gamma = 2.0 - gamma;
    kp.f_gm1 = (float)kp.gm1;                     // FP32 copies read by FP32 kernels
    kp.f_s2exp = (float)(kp.inv_cv / 0.6931471805599453);

    const long long ncell = (long long)nx * ny;
    const int nblocks = (int)((ncell + NA_CHUNK - 1) / NA_CHUNK);
    // every call overwrites the nblocks partials and the result it reads, so
    // nothing has to start at zero
    if (precision == HLBM_FP64)
        diag_partial_chunk_kernel<double><<<nblocks, DIAG_NT, 0, st>>>(static_cast<const double *>(state), partial, kp);
    else
        diag_partial_chunk_kernel<float><<<nblocks, DIAG_NT, 0, st>>>(static_cast<const float *>(state), partial, kp);
    if (cudaGetLastError() != cudaSuccess) return HLBM_ERR_CUDA;
    diag_final_kernel<<<1, DIAG_NT, 0, st>>>(partial, nblocks, result);
    if (cudaGetLastError() != cudaSuccess) return HLBM_ERR_CUDA;
    if (cudaMemcpyAsync(out, result, DIAG_NV * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return HLBM_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return HLBM_ERR_CUDA;
    return HLBM_OK;
}
