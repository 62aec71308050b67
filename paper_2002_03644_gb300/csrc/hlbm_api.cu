// hlbm_api.cu -- the C ABI of include/hlbm.h: handle, device state, launches.
//
// The library owns two copies of the 13-plane state (ping-pong), one FP64
// staging area for caller fields on the host, and the diagnostics partials.
// hlbm_step only launches kernels on the handle's stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "hlbm.h"
#include "hlbm_device.cuh"

using namespace hlbm;

namespace {

constexpr int TX32 = 32, TY32 = 16, NT32 = 256;  // FP32 tile
constexpr int TX64 = 32, TY64 = 8, NT64 = 256;   // FP64 tile
constexpr int DIAG_BLOCKS = 2 * 152;
constexpr uint64_t STATE_MAGIC = 0x31305453424c4848ull;  // "HHLBST01"

struct StateHeader {
    uint64_t magic;
    int32_t abi, precision, nx, ny, pitch, nplane;
    int64_t step;
    int64_t payload_bytes;
};

}  // namespace

struct hlbm_handle {
    hlbm_params p;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    size_t esize = 0;         // bytes per state element
    int pitch = 0;
    size_t plane = 0;         // elements per plane
    void *state[2] = {nullptr, nullptr};
    int cur = 0;
    double *staging = nullptr;  // 9 FP64 planes of nx*ny
    double *diag_partial = nullptr;
    double *diag_out = nullptr;
    KParams kp;
    int64_t step = 0;
    bool initialized = false;
    char err[256] = {0};
};

static int fail(hlbm_handle *h, int code, const char *what)
{
    if (h) snprintf(h->err, sizeof(h->err), "%s", what);
    return code;
}

static int cuda_fail(hlbm_handle *h, cudaError_t e, const char *where)
{
    if (h) snprintf(h->err, sizeof(h->err), "%s: %s", where, cudaGetErrorString(e));
    return HLBM_ERR_CUDA;
}

#define CK(call, where)                                      \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
    } while (0)

template <typename T, int TX, int TY, int NT>
static cudaError_t launch_step(hlbm_handle *h, const void *in, void *out)
{
    using Geo = TileGeom<T, TX, TY>;
    static bool attr_done[64] = {false};
    if (!attr_done[h->device & 63]) {
        cudaError_t e = cudaFuncSetAttribute(fused_step_kernel<T, TX, TY, NT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Geo::smem_bytes);
        if (e != cudaSuccess) return e;
        attr_done[h->device & 63] = true;
    }
    dim3 grid((h->p.nx + TX - 1) / TX, (h->p.ny + TY - 1) / TY);
    fused_step_kernel<T, TX, TY, NT><<<grid, NT, Geo::smem_bytes, h->stream>>>(
        static_cast<const T *>(in), static_cast<T *>(out), h->kp);
    return cudaGetLastError();
}

static cudaError_t launch_one_step(hlbm_handle *h)
{
    const void *in = h->state[h->cur];
    void *out = h->state[h->cur ^ 1];
    if (h->p.precision == HLBM_FP64) return launch_step<double, TX64, TY64, NT64>(h, in, out);
    return launch_step<float, TX32, TY32, NT32>(h, in, out);
}

static dim3 cell_grid(const hlbm_handle *h, dim3 blk)
{
    return dim3((h->p.nx + blk.x - 1) / blk.x, (h->p.ny + blk.y - 1) / blk.y);
}

// Host-side FP64 equilibrium of a Dirichlet state, product of two D1Q3
// equilibria (used only for the constants of Dirichlet sides).
static void host_feq(double rho, double ux, double uy, double th, double f[9])
{
    static const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    static const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    auto g = [th](int c, double u) { return c == 0 ? 1.0 - u * u - th / 3.0 : 0.5 * (u * u + c * u + th / 3.0); };
    for (int i = 0; i < 9; i++) f[i] = rho * g(cx[i], ux) * g(cy[i], uy);
}

static int validate(const hlbm_params *p)
{
    if (!p) return HLBM_ERR_ARG;
    if (p->nx < 1 || p->ny < 1) return HLBM_ERR_ARG;
    if ((long long)p->nx * p->ny > (1ll << 28)) return HLBM_ERR_ARG;
    if (p->precision != HLBM_FP64 && p->precision != HLBM_FP32) return HLBM_ERR_UNSUPPORTED;
    if (p->phi_mode != 0 && p->phi_mode != 1) return HLBM_ERR_ARG;
    if (!(p->gamma > 1.0) || !(p->Pr > 0.0) || !(p->mu >= 0.0) || !(p->sigma >= 0.0 && p->sigma <= 1.0))
        return HLBM_ERR_ARG;
    if (!std::isfinite(p->gamma) || !std::isfinite(p->Pr) || !std::isfinite(p->mu)) return HLBM_ERR_ARG;
    for (int k = 0; k < 4; k++) {
        if (p->bc[k] < HLBM_BC_PERIODIC || p->bc[k] > HLBM_BC_DIRICHLET) return HLBM_ERR_UNSUPPORTED;
        if (p->bc[k] == HLBM_BC_DIRICHLET && (!(p->bc_state[k][0] > 0.0) || !(p->bc_state[k][3] > 0.0)))
            return HLBM_ERR_ARG;
    }
    // a periodic side needs a periodic partner
    if ((p->bc[0] == HLBM_BC_PERIODIC) != (p->bc[1] == HLBM_BC_PERIODIC)) return HLBM_ERR_ARG;
    if ((p->bc[2] == HLBM_BC_PERIODIC) != (p->bc[3] == HLBM_BC_PERIODIC)) return HLBM_ERR_ARG;
    if (p->diag_every < 0) return HLBM_ERR_ARG;
    for (int k = 0; k < 6; k++)
        if (p->reserved[k] != 0) return HLBM_ERR_ARG;
    return HLBM_OK;
}

static void fill_kparams(hlbm_handle *h)
{
    const hlbm_params &p = h->p;
    KParams &k = h->kp;
    memset(&k, 0, sizeof(k));
    k.nx = p.nx; k.ny = p.ny; k.pitch = h->pitch; k.plane = (long long)h->plane;
    for (int s = 0; s < 4; s++) k.bc[s] = p.bc[s];
    k.phi_mode = p.phi_mode;
    k.sigma_nonzero = p.sigma != 0.0;
    k.mu = p.mu; k.sigma = p.sigma;
    const double cs2 = 1.0 / 3.0;
    k.cv = cs2 / (p.gamma - 1.0);
    const double cp = p.gamma * cs2 / (p.gamma - 1.0);
    k.lambda = p.mu * cp / p.Pr;  // conductivity from the definition of Pr
    k.gm1 = p.gamma - 1.0;
    k.inv_cv = 1.0 / k.cv;
    k.two_minus_gamma = 2.0 - p.gamma;  // (D + 2) / D - gamma, D = 2
    k.gamma = p.gamma;
    for (int s = 0; s < 4; s++) {
        if (p.bc[s] != HLBM_BC_DIRICHLET) continue;
        const double r = p.bc_state[s][0], u = p.bc_state[s][1], v = p.bc_state[s][2], t = p.bc_state[s][3];
        k.d_rho[s] = r; k.d_ux[s] = u; k.d_uy[s] = v; k.d_th[s] = t;
        k.d_s[s] = k.cv * (std::log(t) - k.gm1 * std::log(r));
        k.d_gx[s] = r * u * (1.0 - t - u * u);
        k.d_gy[s] = r * v * (1.0 - t - v * v);
        host_feq(r, u, v, t, k.d_F[s]);
    }
}

extern "C" {

int hlbm_abi_version(void) { return HLBM_ABI_VERSION; }

const char *hlbm_strerror(int code)
{
    switch (code) {
    case HLBM_OK: return "ok";
    case HLBM_ERR_ARG: return "invalid argument";
    case HLBM_ERR_CFL: return "initial state violates CFL < 1";
    case HLBM_ERR_NONFINITE: return "non-finite or non-positive density or temperature";
    case HLBM_ERR_CUDA: return "CUDA runtime error";
    case HLBM_ERR_STATE: return "call out of order or state mismatch";
    case HLBM_ERR_NOMEM: return "out of memory";
    case HLBM_ERR_UNSUPPORTED: return "option not supported";
    default: return "unknown status";
    }
}

const char *hlbm_last_error(const hlbm_handle *h) { return h ? h->err : ""; }

int64_t hlbm_step_count(const hlbm_handle *h) { return h ? h->step : -1; }

void hlbm_destroy(hlbm_handle *h)
{
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    cudaFree(h->state[0]);
    cudaFree(h->state[1]);
    cudaFree(h->staging);
    cudaFree(h->diag_partial);
    cudaFree(h->diag_out);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

int hlbm_create(const hlbm_params *params, void *stream, hlbm_handle **out)
{
    if (!out) return HLBM_ERR_ARG;
    *out = nullptr;
    const int v = validate(params);
    if (v != HLBM_OK) return v;
    hlbm_handle *h = new (std::nothrow) hlbm_handle();
    if (!h) return HLBM_ERR_NOMEM;
    h->p = *params;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) { delete h; return HLBM_ERR_CUDA; }
    if (stream) {
        h->stream = static_cast<cudaStream_t>(stream);
    } else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { delete h; return HLBM_ERR_CUDA; }
        h->own_stream = true;
    }
    h->esize = params->precision == HLBM_FP64 ? sizeof(double) : sizeof(float);
    h->pitch = (params->nx + 31) / 32 * 32;
    h->plane = (size_t)h->pitch * params->ny;
    const size_t bytes = h->plane * NPLANE * h->esize;
    const size_t ncell = (size_t)params->nx * params->ny;
    if (cudaMalloc(&h->state[0], bytes) != cudaSuccess || cudaMalloc(&h->state[1], bytes) != cudaSuccess ||
        cudaMalloc(&h->staging, 9 * ncell * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&h->diag_partial, DIAG_BLOCKS * DIAG_NV * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&h->diag_out, DIAG_NV * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        hlbm_destroy(h);
        return HLBM_ERR_NOMEM;
    }
    // pad columns stay zero (never read as cells)
    if (cudaMemsetAsync(h->state[0], 0, bytes, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->state[1], 0, bytes, h->stream) != cudaSuccess) {
        hlbm_destroy(h);
        return HLBM_ERR_CUDA;
    }
    fill_kparams(h);
    *out = h;
    return HLBM_OK;
}

static int run_diagnostics(hlbm_handle *h, double out[8])
{
    const void *st = h->state[h->cur];
    if (h->p.precision == HLBM_FP64)
        diag_partial_kernel<double><<<DIAG_BLOCKS, DIAG_NT, 0, h->stream>>>(static_cast<const double *>(st), h->diag_partial, h->kp);
    else
        diag_partial_kernel<float><<<DIAG_BLOCKS, DIAG_NT, 0, h->stream>>>(static_cast<const float *>(st), h->diag_partial, h->kp);
    CK(cudaGetLastError(), "diag_partial_kernel");
    diag_final_kernel<<<1, DIAG_NT, 0, h->stream>>>(h->diag_partial, DIAG_BLOCKS, h->diag_out);
    CK(cudaGetLastError(), "diag_final_kernel");
    CK(cudaMemcpyAsync(out, h->diag_out, DIAG_NV * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "diag copy");
    CK(cudaStreamSynchronize(h->stream), "diag sync");
    return HLBM_OK;
}

int hlbm_init_fields(hlbm_handle *h, const double *rho, const double *ux, const double *uy, const double *theta,
                     const double *a1, int mem_kind)
{
    if (!h) return HLBM_ERR_ARG;
    if (!rho || !ux || !uy || !theta) return fail(h, HLBM_ERR_ARG, "rho, ux, uy and theta are required");
    if (mem_kind != HLBM_MEM_HOST && mem_kind != HLBM_MEM_DEVICE) return fail(h, HLBM_ERR_ARG, "mem_kind");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    const size_t n = (size_t)h->p.nx * h->p.ny;
    const double *src[5] = {rho, ux, uy, theta, a1};
    const double *dev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    if (mem_kind == HLBM_MEM_HOST) {
        for (int k = 0; k < 4; k++) {
            CK(cudaMemcpyAsync(h->staging + k * n, src[k], n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "init copy");
            dev[k] = h->staging + k * n;
        }
        if (a1) {
            CK(cudaMemcpyAsync(h->staging + 4 * n, a1, 3 * n * sizeof(double), cudaMemcpyHostToDevice, h->stream), "init copy a1");
            dev[4] = h->staging + 4 * n;
        }
    } else {
        for (int k = 0; k < 5; k++) dev[k] = src[k];
    }
    dim3 blk(32, 8);
    if (h->p.precision == HLBM_FP64)
        init_kernel<double><<<cell_grid(h, blk), blk, 0, h->stream>>>(dev[0], dev[1], dev[2], dev[3], dev[4],
                                                                        static_cast<double *>(h->state[0]), h->kp);
    else
        init_kernel<float><<<cell_grid(h, blk), blk, 0, h->stream>>>(dev[0], dev[1], dev[2], dev[3], dev[4],
                                                                       static_cast<float *>(h->state[0]), h->kp);
    CK(cudaGetLastError(), "init_kernel");
    h->cur = 0;
    h->step = 0;
    h->initialized = true;
    CK(cudaStreamSynchronize(h->stream), "init sync");
    if (h->p.check_cfl) {
        double d[8];
        const int r = run_diagnostics(h, d);
        if (r != HLBM_OK) return r;
        if (d[7] > 0) return fail(h, HLBM_ERR_NONFINITE, "initial fields hold non-finite or non-positive values");
        if (!(d[6] < 1.0)) return fail(h, HLBM_ERR_CFL, "max(|u| + c) >= 1");
    }
    h->err[0] = 0;
    return HLBM_OK;
}

int hlbm_step(hlbm_handle *h, int64_t n)
{
    if (!h) return HLBM_ERR_ARG;
    if (!h->initialized) return fail(h, HLBM_ERR_STATE, "hlbm_step before hlbm_init_fields");
    if (n < 0) return fail(h, HLBM_ERR_ARG, "n < 0");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    for (int64_t k = 0; k < n; k++) {
        CK(launch_one_step(h), "fused_step_kernel");
        h->cur ^= 1;
        h->step++;
        if (h->p.diag_every > 0 && h->step % h->p.diag_every == 0) {
            double d[8];
            const int r = run_diagnostics(h, d);
            if (r != HLBM_OK) return r;
            if (d[7] > 0) {
                char msg[96];
                snprintf(msg, sizeof(msg), "non-finite state at step %lld", (long long)h->step);
                return fail(h, HLBM_ERR_NONFINITE, msg);
            }
        }
    }
    return HLBM_OK;
}

static int extract(hlbm_handle *h, double *rho, double *ux, double *uy, double *theta, double *s, double *a1,
                   double *F, int mem_kind)
{
    if (!h) return HLBM_ERR_ARG;
    if (!h->initialized) return fail(h, HLBM_ERR_STATE, "no state yet");
    if (mem_kind != HLBM_MEM_HOST && mem_kind != HLBM_MEM_DEVICE) return fail(h, HLBM_ERR_ARG, "mem_kind");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    const size_t n = (size_t)h->p.nx * h->p.ny;
    double *dst[7] = {rho, ux, uy, theta, s, a1, F};
    double *dev[7];
    if (mem_kind == HLBM_MEM_HOST) {
        // staging holds 9 planes: fields use planes 0..7 (a1 = 3), F uses all 9
        if (F) {
            for (int k = 0; k < 6; k++) dev[k] = nullptr;
            dev[6] = h->staging;
        } else {
            const size_t off[6] = {0, 1, 2, 3, 4, 5};
            for (int k = 0; k < 6; k++) dev[k] = dst[k] ? h->staging + off[k] * n : nullptr;
            dev[6] = nullptr;
        }
    } else {
        for (int k = 0; k < 7; k++) dev[k] = dst[k];
    }
    dim3 blk(32, 8);
    const void *st = h->state[h->cur];
    if (h->p.precision == HLBM_FP64)
        macros_kernel<double><<<cell_grid(h, blk), blk, 0, h->stream>>>(static_cast<const double *>(st), dev[0], dev[1], dev[2],
                                                                          dev[3], dev[4], dev[5], dev[6], h->kp);
    else
        macros_kernel<float><<<cell_grid(h, blk), blk, 0, h->stream>>>(static_cast<const float *>(st), dev[0], dev[1], dev[2],
                                                                         dev[3], dev[4], dev[5], dev[6], h->kp);
    CK(cudaGetLastError(), "macros_kernel");
    if (mem_kind == HLBM_MEM_HOST) {
        for (int k = 0; k < 7; k++) {
            if (!dst[k] || !dev[k]) continue;
            const size_t cnt = (k == 5 ? 3 : (k == 6 ? 9 : 1)) * n;
            CK(cudaMemcpyAsync(dst[k], dev[k], cnt * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "get copy");
        }
    }
    CK(cudaStreamSynchronize(h->stream), "get sync");
    return HLBM_OK;
}

int hlbm_get_macros(hlbm_handle *h, double *rho, double *ux, double *uy, double *theta, double *s, double *a1,
                    int mem_kind)
{
    return extract(h, rho, ux, uy, theta, s, a1, nullptr, mem_kind);
}

int hlbm_get_populations(hlbm_handle *h, double *F, int mem_kind)
{
    if (!F) return fail(h, HLBM_ERR_ARG, "F is NULL");
    return extract(h, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, F, mem_kind);
}

int hlbm_diagnostics(hlbm_handle *h, double out[8])
{
    if (!h || !out) return HLBM_ERR_ARG;
    if (!h->initialized) return fail(h, HLBM_ERR_STATE, "no state yet");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    return run_diagnostics(h, out);
}

int hlbm_synchronize(hlbm_handle *h)
{
    if (!h) return HLBM_ERR_ARG;
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    CK(cudaStreamSynchronize(h->stream), "sync");
    return HLBM_OK;
}

int hlbm_state_bytes(const hlbm_handle *h, size_t *bytes)
{
    if (!h || !bytes) return HLBM_ERR_ARG;
    *bytes = sizeof(StateHeader) + h->plane * NPLANE * h->esize;
    return HLBM_OK;
}

int hlbm_get_state(hlbm_handle *h, void *buf, size_t bytes)
{
    if (!h || !buf) return HLBM_ERR_ARG;
    if (!h->initialized) return fail(h, HLBM_ERR_STATE, "no state yet");
    size_t need = 0;
    hlbm_state_bytes(h, &need);
    if (bytes < need) return fail(h, HLBM_ERR_ARG, "buffer too small");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    StateHeader hd;
    memset(&hd, 0, sizeof(hd));
    hd.magic = STATE_MAGIC; hd.abi = HLBM_ABI_VERSION; hd.precision = h->p.precision;
    hd.nx = h->p.nx; hd.ny = h->p.ny; hd.pitch = h->pitch; hd.nplane = NPLANE; hd.step = h->step;
    hd.payload_bytes = (int64_t)(need - sizeof(StateHeader));
    memcpy(buf, &hd, sizeof(hd));
    CK(cudaMemcpyAsync(static_cast<char *>(buf) + sizeof(hd), h->state[h->cur], (size_t)hd.payload_bytes,
                       cudaMemcpyDeviceToHost, h->stream), "state copy");
    CK(cudaStreamSynchronize(h->stream), "state sync");
    return HLBM_OK;
}

int hlbm_set_state(hlbm_handle *h, const void *buf, size_t bytes)
{
    if (!h || !buf) return HLBM_ERR_ARG;
    size_t need = 0;
    hlbm_state_bytes(h, &need);
    if (bytes != need) return fail(h, HLBM_ERR_STATE, "state size mismatch");
    StateHeader hd;
    memcpy(&hd, buf, sizeof(hd));
    if (hd.magic != STATE_MAGIC || hd.abi != HLBM_ABI_VERSION || hd.precision != h->p.precision || hd.nx != h->p.nx ||
        hd.ny != h->p.ny || hd.pitch != h->pitch || hd.nplane != NPLANE || hd.step < 0 ||
        hd.payload_bytes != (int64_t)(need - sizeof(StateHeader)))
        return fail(h, HLBM_ERR_STATE, "state header mismatch");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    CK(cudaMemcpyAsync(h->state[0], static_cast<const char *>(buf) + sizeof(hd), (size_t)hd.payload_bytes,
                       cudaMemcpyHostToDevice, h->stream), "state copy");
    CK(cudaStreamSynchronize(h->stream), "state sync");
    h->cur = 0;
    h->step = hd.step;
    h->initialized = true;
    return HLBM_OK;
}

}  // extern "C"
