// hlbm_api.cu -- the C ABI of include/hlbm.h: handle, device state, launches.
//
// The library owns two copies of the 13-plane state (ping-pong), one FP64
// staging area for caller fields on the host, and the diagnostics partials.
// hlbm_step only launches kernels on the handle's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include "hlbm.h"
#include "hlbm_device.cuh"
#include "hlbm_tma.cuh"
#include "hlbm_march.cuh"

using namespace hlbm;

namespace {

constexpr int TX64 = 32, TY64 = 8, NT64 = 256;   // FP64 tile
constexpr int DIAG_BLOCKS = 2 * 152;
constexpr uint64_t STATE_MAGIC = 0x31305453424c4848ull;  // "HHLBST01"

struct StateHeader {
    uint64_t magic;
    int32_t abi, precision, nx, ny, pitch, nplane;
    int64_t step;
    int64_t payload_bytes;
    float ref[9];  // reference populations of the 16-bit storage forms
    int32_t pad;
};

template <typename T, typename S>
struct Types {
    using t = T;
    using s = S;
};

}  // namespace

struct hlbm_handle {
    hlbm_params p;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    size_t fsize = 0;         // bytes per stored population
    size_t asize = 0;         // bytes per auxiliary element (s, a1)
    int pitch = 0;
    size_t plane = 0;         // elements per plane
    void *state[2] = {nullptr, nullptr};
    int cur = 0;
    double *staging = nullptr;  // 9 FP64 planes of nx*ny
    double *diag_partial = nullptr;
    double *diag_out = nullptr;
    KParams kp;
    TmaMaps maps[2];            // tensor maps of state[0] and state[1] (FP32)
    bool tma_ready = false;
    int tma_grid = 0;
    int tma_variant = 0;        // FP32 kernel choice, fixed at create
    int tile_variant = 0;
    int march_variant = -1;     // row-marching kernel variant, -1: tiled / TMA kernels
    bool moments = false;       // HLBM_FP32_MOMENTS: 7 FP32 planes, moment-state kernel
    bool walls = false;         // a wall side: tiled kernel plus wall_ghost_kernel each step
    bool periodic = false;      // all four sides periodic and ny >= 4 (specialised marching kernels)
    bool mcache = false;        // FP64 marching: level-n rho, u, theta planes behind the state (A_RHO .. A_TH)
    void *wall_g = nullptr;     // wall ghost rows (KParams::wall_g)
    int march_nseg = 1;         // row segments per strip
    int *d_err = nullptr;       // device-side timeout flag of the TMA kernel
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

// Population and auxiliary planes of state copy idx: 9 planes of S::raw,
// then 4 planes of T (s, a1_xx, a1_xy, a1_yy).
template <typename T, typename S>
static typename S::raw *pop_planes(const hlbm_handle *h, int idx)
{
    return static_cast<typename S::raw *>(h->state[idx]);
}

template <typename T, typename S>
static T *aux_planes(const hlbm_handle *h, int idx)
{
    return reinterpret_cast<T *>(static_cast<char *>(h->state[idx]) + 9 * h->plane * sizeof(typename S::raw));
}

// Bytes of one state copy (what a checkpoint holds).
static size_t payload_bytes(const hlbm_handle *h)
{
    return h->moments ? h->plane * MS_NPLANE * sizeof(float) : h->plane * (9 * h->fsize + 4 * h->asize);
}

// Bytes allocated per state copy: the payload, then the FP64 marching
// form's cache planes.
static size_t alloc_bytes(const hlbm_handle *h)
{
    return payload_bytes(h) + (h->mcache ? h->plane * A_NCACHE * sizeof(double) : 0);
}

// FP64 marching form: derive the cache planes of state copy cur from its
// F(n) and s(n), after init or a checkpoint set the state.
static cudaError_t fill_cache(hlbm_handle *h)
{
    if (!h->mcache) return cudaSuccess;
    const int blk = 256;
    const long long n = (long long)h->p.nx * h->p.ny;
    const int grid = (int)std::min<long long>((n + blk - 1) / blk, 65535);
    cache_macros_kernel<<<grid, blk, 0, h->stream>>>(pop_planes<double, FullStore<double>>(h, h->cur),
                                                     aux_planes<double, FullStore<double>>(h, h->cur), h->kp);
    return cudaGetLastError();
}

// Call fn(Types<T, S>{}) for the handle's precision.
template <typename Fn>
static cudaError_t with_types(const hlbm_handle *h, Fn &&fn)
{
    switch (h->p.precision) {
    case HLBM_FP64: return fn(Types<double, FullStore<double>>{});
    case HLBM_FP32_F16POP: return fn(Types<float, HalfStore>{});
    case HLBM_FP32_BF16POP: return fn(Types<float, BF16Store>{});
    default: return fn(Types<float, FullStore<float>>{});
    }
}

template <typename T, typename S, int TX, int TY, int NT>
static cudaError_t launch_step(hlbm_handle *h)
{
    using Geo = TileGeom<T, TX, TY>;
    static bool attr_done[64] = {false};
    if (!attr_done[h->device & 63]) {
        cudaError_t e = cudaFuncSetAttribute(fused_step_kernel<T, S, TX, TY, NT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Geo::smem_bytes);
        if (e != cudaSuccess) return e;
        attr_done[h->device & 63] = true;
    }
    dim3 grid((h->p.nx + TX - 1) / TX, (h->p.ny + TY - 1) / TY);
    const int a = h->cur, b = h->cur ^ 1;
    fused_step_kernel<T, S, TX, TY, NT><<<grid, NT, Geo::smem_bytes, h->stream>>>(
        pop_planes<T, S>(h, a), aux_planes<T, S>(h, a), pop_planes<T, S>(h, b), aux_planes<T, S>(h, b), h->kp);
    return cudaGetLastError();
}

// Tiled FP32 kernels (HLBM_MARCH=-1).  Grids of up to 2048^2 cells use the
// plain tiled kernel with 32x32 tiles and larger grids the persistent TMA
// kernel with 32x16 tiles.  HLBM_FP32_TMA=<k> forces TMA tile k,
// HLBM_FP32_TMA=-1 the plain kernel with HLBM_FP32_TILE=<k> (tuning sweeps).
constexpr int kNumFp32Tiles = 5;  // plain: 32x16x256, 64x16x256, 32x8x128, 64x32x512, 32x32x512
constexpr int kNumTma = 4;        // TMA: 32x16x512, 32x16x256, 64x16x512, 32x32x512

static int env_choice(const char *name, int dflt, int lo, int hi)
{
    const char *e = getenv(name);
    if (!e) return dflt;
    const int v = atoi(e);
    return (v >= lo && v < hi) ? v : dflt;
}

// A named NVTX range over one entry point's host work (what it enqueues and
// any wait), visible in a profiler's timeline; without a tool attached a
// range costs a function call.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};


template <int TX, int TY, int NT>
static cudaError_t tma_grid_size(hlbm_handle *h, int *grid)
{
    using G = TmaGeom<TX, TY>;
    cudaError_t e = cudaFuncSetAttribute(fused_step_tma_kernel<TX, TY, NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem_bytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_step_tma_kernel<TX, TY, NT>, NT, G::smem_bytes);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) return e;
    const int tiles = ((h->p.nx + TX - 1) / TX) * ((h->p.ny + TY - 1) / TY);
    const int g = (per_sm > 0 ? per_sm : 1) * sms;
    *grid = g < tiles ? g : tiles;
    return cudaSuccess;
}

template <int TX, int TY>
static bool encode_maps(hlbm_handle *h, void *state, TmaMaps *m)
{
    using G = TmaGeom<TX, TY>;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[3] = {(cuuint64_t)h->pitch, (cuuint64_t)h->p.ny, (cuuint64_t)NPLANE};
    const cuuint64_t strides[2] = {(cuuint64_t)h->pitch * 4, (cuuint64_t)h->plane * 4};
    const cuuint32_t estr[3] = {1, 1, 1};
    const cuuint32_t boxF[3] = {G::BX, G::F_ROWS, 9}, boxS[3] = {G::BX, G::S_ROWS, 1}, boxA[3] = {G::BX, G::A_ROWS, 3};
    const cuuint32_t *boxes[3] = {boxF, boxS, boxA};
    CUtensorMap *out[3] = {&m->f, &m->s, &m->a};
    for (int k = 0; k < 3; k++) {
        if (encode(out[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, state, dims, strides, boxes[k], estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}

// The TMA kernel serves grids that have interior tiles (away from every
// edge by the halo); smaller grids, or a tensor map the driver refuses,
// use the plain tiled kernel, which handles every tile itself.
template <int TX, int TY, int NT>
static cudaError_t prepare_tma(hlbm_handle *h)
{
    if (h->p.nx < TX + 8 + 2 * TX || h->p.ny < TY + 6 + 2 * TY) return cudaSuccess;
    if (!encode_maps<TX, TY>(h, h->state[0], &h->maps[0]) || !encode_maps<TX, TY>(h, h->state[1], &h->maps[1]))
        return cudaSuccess;
    const cudaError_t e = tma_grid_size<TX, TY, NT>(h, &h->tma_grid);
    if (e == cudaSuccess) h->tma_ready = true;
    return e;
}

static cudaError_t setup_fp32_kernel(hlbm_handle *h)
{
    const bool large = (long long)h->p.nx * h->p.ny > 2048ll * 2048ll;
    h->tma_variant = env_choice("HLBM_FP32_TMA", large ? 0 : -1, -1, kNumTma);
    h->tile_variant = env_choice("HLBM_FP32_TILE", 4, 0, kNumFp32Tiles);
    switch (h->tma_variant) {
    case -1: return cudaSuccess;
    case 1: return prepare_tma<32, 16, 256>(h);
    case 2: return prepare_tma<64, 16, 512>(h);
    case 3: return prepare_tma<32, 32, 512>(h);
    default: return prepare_tma<32, 16, 512>(h);
    }
}

template <int TX, int TY, int NT>
static cudaError_t launch_tma(hlbm_handle *h)
{
    using G = TmaGeom<TX, TY>;
    fused_step_tma_kernel<TX, TY, NT><<<h->tma_grid, NT, G::smem_bytes, h->stream>>>(
        h->maps[h->cur], static_cast<const float *>(h->state[h->cur]), static_cast<float *>(h->state[h->cur ^ 1]),
        h->kp, h->d_err);
    return cudaGetLastError();
}

// Row-marching kernel (paired columns, see hlbm_march.cuh); its row
// segments come from march_segments().
constexpr int kNumMarch = 4;
constexpr int kMarchMinRows = 8;
constexpr int kMarchMaxRows = 32;
constexpr long long kMarchMinCells = 768ll * 768ll;  // GB300 sweep: tiled faster up to 768^2, marching at 1024^2

// Row segments per strip: the fewest whole waves of resident CTAs (per_sm x
// SMs) whose segments are at most kMarchMaxRows high, cut as finely as that
// number of waves allows, so that no wave runs part-empty; at least
// kMarchMinRows rows per segment.  HLBM_MARCH_ROWS=<n> fixes the height.
static int march_segments(const hlbm_handle *h, long long strips, int per_sm, int sms)
{
    const long long cap = (long long)(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    const long long least = (h->p.ny + kMarchMaxRows - 1) / kMarchMaxRows;
    const long long waves = (strips * least + cap - 1) / cap;
    long long nseg = (waves > 0 ? waves : 1) * cap / strips;
    if (nseg < least) nseg = least;
    const long long most = h->p.ny / kMarchMinRows > 0 ? h->p.ny / kMarchMinRows : 1;
    if (nseg > most) nseg = most;
    const int rows = env_choice("HLBM_MARCH_ROWS", 0, 1, 1 << 20);
    if (rows > 0) nseg = (h->p.ny + rows - 1) / rows;
    if (nseg > 65535) nseg = 65535;
    return (int)(nseg > 0 ? nseg : 1);
}

// Paired-column marching kernel with NT threads (strips of 2 (NT - 4)
// columns), register budget set by MINB resident CTAs per SM; the
// instantiation matches the handle's sigma > 0 and Phi choice.
template <typename T, typename S, int NT, int MINB, bool PER = false>
static void *pair_kernel_ptr(const hlbm_handle *h)
{
    const bool sig = h->kp.sigma_nonzero != 0, phi0 = h->kp.phi_mode == 0;
    if (sig) return phi0 ? (void *)march_pair_kernel<T, S, NT, MINB, true, true, PER>
                         : (void *)march_pair_kernel<T, S, NT, MINB, true, false, PER>;
    return phi0 ? (void *)march_pair_kernel<T, S, NT, MINB, false, true, PER>
                : (void *)march_pair_kernel<T, S, NT, MINB, false, false, PER>;
}

template <typename T, typename S, int NT, int MINB, bool PER = false>
static cudaError_t pair_setup(hlbm_handle *h)
{
    using G = PairGeom<T, NT>;
    const void *fn = pair_kernel_ptr<T, S, NT, MINB, PER>(h);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem_bytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NT, G::smem_bytes);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) return e;
    h->march_nseg = march_segments(h, (h->p.nx + G::W - 1) / G::W, per_sm, sms);
    return cudaSuccess;
}

template <typename T, typename S, int NT, int MINB, bool PER = false>
static cudaError_t launch_pair(hlbm_handle *h)
{
    using G = PairGeom<T, NT>;
    dim3 grid((h->p.nx + G::W - 1) / G::W, h->march_nseg);
    const int a = h->cur, b = h->cur ^ 1;
    const typename S::raw *inF = pop_planes<T, S>(h, a);
    const T *inA = aux_planes<T, S>(h, a);
    typename S::raw *outF = pop_planes<T, S>(h, b);
    T *outA = aux_planes<T, S>(h, b);
    const bool sig = h->kp.sigma_nonzero != 0, phi0 = h->kp.phi_mode == 0;
    if (sig && phi0)
        march_pair_kernel<T, S, NT, MINB, true, true, PER><<<grid, NT, G::smem_bytes, h->stream>>>(inF, inA, outF, outA, h->kp, h->march_nseg);
    else if (sig)
        march_pair_kernel<T, S, NT, MINB, true, false, PER><<<grid, NT, G::smem_bytes, h->stream>>>(inF, inA, outF, outA, h->kp, h->march_nseg);
    else if (phi0)
        march_pair_kernel<T, S, NT, MINB, false, true, PER><<<grid, NT, G::smem_bytes, h->stream>>>(inF, inA, outF, outA, h->kp, h->march_nseg);
    else
        march_pair_kernel<T, S, NT, MINB, false, false, PER><<<grid, NT, G::smem_bytes, h->stream>>>(inF, inA, outF, outA, h->kp, h->march_nseg);
    return cudaGetLastError();
}

// Marching kernel variants: 0 = 64 threads at <= 128 registers (strips of
// 120 columns; the default), 1 = 96 threads at <= 136, 2 = 128 threads at
// <= 128, 3 = 64 threads without a register cap.  FP64 runs without a cap
// (its pair state does not fit 128 registers).
template <typename T, typename S, bool Launch>
static cudaError_t march_dispatch(hlbm_handle *h)
{
    constexpr bool f64 = sizeof(T) == 8;
    switch (h->march_variant) {
    case 1: return Launch ? launch_pair<T, S, 96, f64 ? 1 : 5>(h) : pair_setup<T, S, 96, f64 ? 1 : 5>(h);
    case 2: return Launch ? launch_pair<T, S, 128, f64 ? 1 : 4>(h) : pair_setup<T, S, 128, f64 ? 1 : 4>(h);
    case 3: return Launch ? launch_pair<T, S, 64, 1>(h) : pair_setup<T, S, 64, 1>(h);
    default:
        // the default FP32-arithmetic kernel (FP32 or 16-bit storage) has an
        // all-periodic instantiation
        if constexpr (!f64) {
            if (h->periodic) return Launch ? launch_pair<T, S, 64, 8, true>(h) : pair_setup<T, S, 64, 8, true>(h);
        }
        return Launch ? launch_pair<T, S, 64, f64 ? 1 : 8>(h) : pair_setup<T, S, 64, f64 ? 1 : 8>(h);
    }
}

static cudaError_t setup_march(hlbm_handle *h)
{
    // Every precision marches by default on grids of more than
    // kMarchMinCells cells (below that a grid has too few strips and
    // segments to fill the GPU, and the tiled kernel is faster).  In FP64 the
    // marching kernel is 2-8 % faster at 1024^2-2048^2: it recomputes less
    // halo on the FP64 pipe.  HLBM_MARCH=<k> picks a variant, -1 the tiled /
    // TMA kernels.
    const bool big = (long long)h->p.nx * h->p.ny > kMarchMinCells;
    h->march_variant = env_choice("HLBM_MARCH", big ? 0 : -1, -1, kNumMarch);
    if (h->march_variant < 0) return cudaSuccess;
    return with_types(h, [&](auto ty) {
        using T = typename decltype(ty)::t;
        using S = typename decltype(ty)::s;
        return march_dispatch<T, S, false>(h);
    });
}

// Moment-state kernel: 64 threads at <= 128 registers (strips of 116
// columns), row segments as for the marching kernel; the instantiation
// matches the handle's sigma > 0 and Phi choice.
constexpr int kMomNT = 64, kMomMinB = 8;

template <bool PER>
static const void *moment_kernel_ptr_t(const hlbm_handle *h)
{
    const bool sig = h->kp.sigma_nonzero != 0, phi0 = h->kp.phi_mode == 0;
    if (sig) return phi0 ? (const void *)march_moment_kernel<kMomNT, kMomMinB, true, true, PER>
                         : (const void *)march_moment_kernel<kMomNT, kMomMinB, true, false, PER>;
    return phi0 ? (const void *)march_moment_kernel<kMomNT, kMomMinB, false, true, PER>
                : (const void *)march_moment_kernel<kMomNT, kMomMinB, false, false, PER>;
}

// all-periodic grids take the instantiation without boundary selections
static const void *moment_kernel_ptr(const hlbm_handle *h)
{
    return h->periodic ? moment_kernel_ptr_t<true>(h) : moment_kernel_ptr_t<false>(h);
}

static cudaError_t setup_moments(hlbm_handle *h)
{
    using G = MomGeom<kMomNT>;
    const void *fn = moment_kernel_ptr(h);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem_bytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kMomNT, G::smem_bytes);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) return e;
    h->march_nseg = march_segments(h, (h->p.nx + G::W - 1) / G::W, per_sm, sms);
    return cudaSuccess;
}

static cudaError_t launch_moments(hlbm_handle *h)
{
    using G = MomGeom<kMomNT>;
    dim3 grid((h->p.nx + G::W - 1) / G::W, h->march_nseg);
    const float *in = static_cast<const float *>(h->state[h->cur]);
    float *out = static_cast<float *>(h->state[h->cur ^ 1]);
    // one launch through the selected instantiation's pointer
    void *args[] = {(void *)&in, (void *)&out, (void *)&h->kp, (void *)&h->march_nseg};
    return cudaLaunchKernel(moment_kernel_ptr(h), grid, dim3(kMomNT), args, G::smem_bytes, h->stream);
}

// Level-n ghost rows of the wall sides, from the current state.
static cudaError_t launch_wall_ghosts(hlbm_handle *h)
{
    return with_types(h, [&](auto ty) {
        using T = typename decltype(ty)::t;
        using S = typename decltype(ty)::s;
        dim3 grid((std::max(h->kp.wall_p, h->kp.wall_q) + 127) / 128, 8);
        wall_ghost_kernel<T, S><<<grid, 128, 0, h->stream>>>(pop_planes<T, S>(h, h->cur), aux_planes<T, S>(h, h->cur),
                                                             h->kp);
        return cudaGetLastError();
    });
}

static cudaError_t launch_one_step(hlbm_handle *h)
{
    if (h->moments) return launch_moments(h);
    if (h->walls) {
        const cudaError_t e = launch_wall_ghosts(h);
        if (e != cudaSuccess) return e;
    }
    using F32 = FullStore<float>;
    if (h->march_variant >= 0) {
        return with_types(h, [&](auto ty) {
            using T = typename decltype(ty)::t;
            using S = typename decltype(ty)::s;
            return march_dispatch<T, S, true>(h);
        });
    }
    if (h->p.precision == HLBM_FP64) return launch_step<double, FullStore<double>, TX64, TY64, NT64>(h);
    if (h->p.precision == HLBM_FP32_F16POP) return launch_step<float, HalfStore, 32, 32, 512>(h);
    if (h->p.precision == HLBM_FP32_BF16POP) return launch_step<float, BF16Store, 32, 32, 512>(h);
    if (h->tma_ready) {
        switch (h->tma_variant) {
        case 1: return launch_tma<32, 16, 256>(h);
        case 2: return launch_tma<64, 16, 512>(h);
        case 3: return launch_tma<32, 32, 512>(h);
        default: return launch_tma<32, 16, 512>(h);
        }
    }
    switch (h->tile_variant) {
    case 1: return launch_step<float, F32, 64, 16, 256>(h);
    case 2: return launch_step<float, F32, 32, 8, 128>(h);
    case 3: return launch_step<float, F32, 64, 32, 512>(h);
    case 4: return launch_step<float, F32, 32, 32, 512>(h);
    default: return launch_step<float, F32, 32, 16, 256>(h);
    }
}

// Device timeout flag -> HLBM_ERR_TIMEOUT (called after a stream sync).
static int check_timeout(hlbm_handle *h)
{
    if (!h->d_err) return HLBM_OK;
    int flag = 0;
    CK(cudaMemcpy(&flag, h->d_err, sizeof(int), cudaMemcpyDeviceToHost), "timeout flag");
    if (flag) return fail(h, HLBM_ERR_TIMEOUT, "a bulk copy into shared memory did not arrive within 1 s");
    return HLBM_OK;
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
    if (p->precision < HLBM_FP64 || p->precision > HLBM_FP32_MOMENTS) return HLBM_ERR_UNSUPPORTED;
    if (p->phi_mode != 0 && p->phi_mode != 1) return HLBM_ERR_ARG;
    if (!(p->gamma > 1.0) || !(p->Pr > 0.0) || !(p->mu >= 0.0) || !(p->sigma >= 0.0 && p->sigma <= 1.0))
        return HLBM_ERR_ARG;
    if (!std::isfinite(p->gamma) || !std::isfinite(p->Pr) || !std::isfinite(p->mu)) return HLBM_ERR_ARG;
    for (int k = 0; k < 4; k++) {
        if (p->bc[k] < HLBM_BC_PERIODIC || p->bc[k] > HLBM_BC_WALL) return HLBM_ERR_UNSUPPORTED;
        if (p->bc[k] == HLBM_BC_DIRICHLET && (!(p->bc_state[k][0] > 0.0) || !(p->bc_state[k][3] > 0.0)))
            return HLBM_ERR_ARG;
        if (p->bc[k] == HLBM_BC_WALL) {
            // two interior layers to mirror, a positive temperature
            if ((k < 2 ? p->nx : p->ny) < 2 || !(p->bc_state[k][3] > 0.0)) return HLBM_ERR_ARG;
            if (!std::isfinite(p->bc_state[k][1]) || !std::isfinite(p->bc_state[k][2])) return HLBM_ERR_ARG;
            if (p->precision == HLBM_FP32_MOMENTS) return HLBM_ERR_UNSUPPORTED;
        }
    }
    // a periodic side needs a periodic partner
    if ((p->bc[0] == HLBM_BC_PERIODIC) != (p->bc[1] == HLBM_BC_PERIODIC)) return HLBM_ERR_ARG;
    if ((p->bc[2] == HLBM_BC_PERIODIC) != (p->bc[3] == HLBM_BC_PERIODIC)) return HLBM_ERR_ARG;
    if (p->diag_every < 0) return HLBM_ERR_ARG;
    if (p->ablation < 0 || p->ablation > (HLBM_ABL_CENTRED_E1 | HLBM_ABL_NO_E2)) return HLBM_ERR_ARG;
    for (int k = 0; k < 5; k++)
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
    k.two_minus_gamma = (p.ablation & HLBM_ABL_NO_E2) ? 0.0 : 2.0 - p.gamma;  // (D + 2) / D - gamma, D = 2
    k.e1_centred = (p.ablation & HLBM_ABL_CENTRED_E1) ? 1 : 0;
    k.gamma = p.gamma;
    for (int s = 0; s < 4; s++) {
        if (p.bc[s] == HLBM_BC_WALL) {
            // wall velocity and temperature (the density is not imposed)
            k.d_ux[s] = p.bc_state[s][1]; k.d_uy[s] = p.bc_state[s][2]; k.d_th[s] = p.bc_state[s][3];
            continue;
        }
        if (p.bc[s] != HLBM_BC_DIRICHLET) continue;
        const double r = p.bc_state[s][0], u = p.bc_state[s][1], v = p.bc_state[s][2], t = p.bc_state[s][3];
        k.d_rho[s] = r; k.d_ux[s] = u; k.d_uy[s] = v; k.d_th[s] = t;
        k.d_s[s] = k.cv * (std::log(t) - k.gm1 * std::log(r));
        k.d_gx[s] = r * u * (1.0 - t - u * u);
        k.d_gy[s] = r * v * (1.0 - t - v * v);
        host_feq(r, u, v, t, k.d_F[s]);
    }
    k.f_gm1 = (float)k.gm1;
    k.f_s2exp = (float)(k.inv_cv / std::log(2.0));
    k.f_mu = (float)k.mu; k.f_lam = (float)k.lambda;
    k.f_sigma = (float)k.sigma; k.f_one_m_sigma = (float)(1.0 - k.sigma);
    k.f_two_m_gamma = (float)k.two_minus_gamma;
    for (int s = 0; s < 4; s++) {
        k.f_d_rho[s] = (float)k.d_rho[s]; k.f_d_ux[s] = (float)k.d_ux[s]; k.f_d_uy[s] = (float)k.d_uy[s];
        k.f_d_th[s] = (float)k.d_th[s]; k.f_d_s[s] = (float)k.d_s[s];
        for (int i = 0; i < 9; i++) k.f_d_F[s][i] = (float)k.d_F[s][i];
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
    case HLBM_ERR_TIMEOUT: return "device-side wait timed out";
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
    cudaFree(h->d_err);
    cudaFree(h->wall_g);
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
    h->moments = params->precision == HLBM_FP32_MOMENTS;
    h->asize = params->precision == HLBM_FP64 ? sizeof(double) : sizeof(float);
    h->fsize = (params->precision == HLBM_FP32_F16POP || params->precision == HLBM_FP32_BF16POP) ? 2 : h->asize;
    h->pitch = (params->nx + 31) / 32 * 32;
    h->plane = (size_t)h->pitch * params->ny;
    // FP64 without wall sides may take the marching kernel (decided below);
    // its cache planes are allocated up front and dropped from use if not
    bool wall_side = false;
    for (int k = 0; k < 4; k++) wall_side = wall_side || params->bc[k] == HLBM_BC_WALL;
    h->mcache = params->precision == HLBM_FP64 && !wall_side;
    const size_t bytes = alloc_bytes(h);
    const size_t ncell = (size_t)params->nx * params->ny;
    if (cudaMalloc(&h->state[0], bytes) != cudaSuccess || cudaMalloc(&h->state[1], bytes) != cudaSuccess ||
        cudaMalloc(&h->staging, 9 * ncell * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&h->diag_partial, DIAG_BLOCKS * DIAG_NV * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&h->diag_out, DIAG_NV * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&h->d_err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        hlbm_destroy(h);
        return HLBM_ERR_NOMEM;
    }
    // Every byte 0xFF: a NaN in each storage type (FP64, FP32, FP16, BF16).
    // The pad columns of each row (pitch > nx) keep it for good -- no kernel
    // writes them -- so a kernel that used a value it should never read
    // would carry a NaN into the fields, where every parity test sees it.
    if (cudaMemsetAsync(h->state[0], 0xFF, bytes, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->state[1], 0xFF, bytes, h->stream) != cudaSuccess) {
        hlbm_destroy(h);
        return HLBM_ERR_CUDA;
    }
    if (cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream) != cudaSuccess) {
        hlbm_destroy(h);
        return HLBM_ERR_CUDA;
    }
    fill_kparams(h);
    h->walls = false;
    h->periodic = true;
    for (int k = 0; k < 4; k++) {
        h->walls = h->walls || params->bc[k] == HLBM_BC_WALL;
        h->periodic = h->periodic && params->bc[k] == HLBM_BC_PERIODIC;
    }
    // HLBM_MARCH_GENERAL=1 keeps the general marching kernels on periodic
    // grids (tests compare the two)
    h->periodic = h->periodic && params->ny >= 4 && env_choice("HLBM_MARCH_GENERAL", 0, 0, 2) == 0;
    if (h->walls) {
        // ghost layers for the tiled kernel; walls never take the marching
        // or TMA kernels
        const size_t wb = (size_t)kWallPlanes * 4 * ((params->nx + 4) + (params->ny + 4)) * h->asize;
        if (cudaMalloc(&h->wall_g, wb) != cudaSuccess) {
            cudaGetLastError();
            hlbm_destroy(h);
            return HLBM_ERR_NOMEM;
        }
        h->kp.wall_g = h->wall_g;
        h->kp.wall_p = params->nx + 4;
        h->kp.wall_q = params->ny + 4;
        h->tile_variant = env_choice("HLBM_FP32_TILE", 4, 0, kNumFp32Tiles);
        *out = h;
        return HLBM_OK;
    }
    if (h->moments) {
        if (setup_moments(h) != cudaSuccess) {
            cudaGetLastError();
            hlbm_destroy(h);
            return HLBM_ERR_CUDA;
        }
        *out = h;
        return HLBM_OK;
    }
    if (setup_march(h) != cudaSuccess ||
        (h->march_variant < 0 && params->precision == HLBM_FP32 && setup_fp32_kernel(h) != cudaSuccess)) {
        cudaGetLastError();
        hlbm_destroy(h);
        return HLBM_ERR_CUDA;
    }
    h->mcache = h->mcache && h->march_variant >= 0;
    *out = h;
    return HLBM_OK;
}

static int run_diagnostics(hlbm_handle *h, double out[8])
{
    if (h->moments) {
        moments_diag_partial_kernel<<<DIAG_BLOCKS, DIAG_NT, 0, h->stream>>>(static_cast<const float *>(h->state[h->cur]),
                                                                            h->diag_partial, h->kp);
        CK(cudaGetLastError(), "moments_diag_partial_kernel");
    } else CK(with_types(h, [&](auto ty) {
           using T = typename decltype(ty)::t;
           using S = typename decltype(ty)::s;
           diag_partial_kernel<T, S><<<DIAG_BLOCKS, DIAG_NT, 0, h->stream>>>(
               pop_planes<T, S>(h, h->cur), aux_planes<T, S>(h, h->cur), h->diag_partial, h->kp);
           return cudaGetLastError();
       }), "diag_partial_kernel");
    diag_final_kernel<<<1, DIAG_NT, 0, h->stream>>>(h->diag_partial, DIAG_BLOCKS, h->diag_out);
    CK(cudaGetLastError(), "diag_final_kernel");
    CK(cudaMemcpyAsync(out, h->diag_out, DIAG_NV * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "diag copy");
    CK(cudaStreamSynchronize(h->stream), "diag sync");
    return check_timeout(h);
}

// The device address of a host buffer that kernels may read and write in
// place -- page-locked (pinned or registered) host memory, which this GPU
// reaches over its host link -- or nullptr for pageable memory, which goes
// through the staging buffer and a copy.  HLBM_ZERO_COPY=0 sends every host
// buffer through the staging buffer.
static double *host_view(const void *p)
{
    if (!p || env_choice("HLBM_ZERO_COPY", 1, 0, 2) == 0) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? static_cast<double *>(at.devicePointer) : nullptr;
}

int hlbm_init_fields(hlbm_handle *h, const double *rho, const double *ux, const double *uy, const double *theta,
                     const double *a1, int mem_kind)
{
    NvtxRange nvtx_range("hlbm_init_fields");
    if (!h) return HLBM_ERR_ARG;
    if (!rho || !ux || !uy || !theta) return fail(h, HLBM_ERR_ARG, "rho, ux, uy and theta are required");
    if (mem_kind != HLBM_MEM_HOST && mem_kind != HLBM_MEM_DEVICE) return fail(h, HLBM_ERR_ARG, "mem_kind");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    const size_t n = (size_t)h->p.nx * h->p.ny;
    const double *src[5] = {rho, ux, uy, theta, a1};
    const double *dev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    if (mem_kind == HLBM_MEM_HOST) {
        // pinned fields are read in place by the kernels; pageable ones are
        // copied to the staging buffer first
        for (int k = 0; k < 5; k++) {
            if (!src[k]) continue;
            if ((dev[k] = host_view(src[k]))) continue;
            const size_t cnt = (k == 4 ? 3 : 1) * n;
            CK(cudaMemcpyAsync(h->staging + k * n, src[k], cnt * sizeof(double), cudaMemcpyHostToDevice, h->stream),
               "init copy");
            dev[k] = h->staging + k * n;
        }
    } else {
        for (int k = 0; k < 5; k++) dev[k] = src[k];
    }
    if (h->p.precision == HLBM_FP32_F16POP || h->p.precision == HLBM_FP32_BF16POP) {
        // reference equilibrium of the mean state for the 16-bit forms
        field_sums_partial_kernel<<<DIAG_BLOCKS, DIAG_NT, 0, h->stream>>>(dev[0], dev[1], dev[2], dev[3],
                                                                          (long long)n, h->diag_partial);
        CK(cudaGetLastError(), "field_sums_partial_kernel");
        diag_final_kernel<<<1, DIAG_NT, 0, h->stream>>>(h->diag_partial, DIAG_BLOCKS, h->diag_out);
        CK(cudaGetLastError(), "diag_final_kernel");
        double sums[DIAG_NV];
        CK(cudaMemcpyAsync(sums, h->diag_out, sizeof(sums), cudaMemcpyDeviceToHost, h->stream), "sums copy");
        CK(cudaStreamSynchronize(h->stream), "sums sync");
        const double rm = sums[0] / (double)n;
        if (!(rm > 0.0) || !std::isfinite(sums[1]) || !std::isfinite(sums[2]) || !(sums[3] > 0.0))
            return fail(h, HLBM_ERR_NONFINITE, "initial fields hold non-finite or non-positive values");
        double fr[9];
        host_feq(rm, sums[1] / sums[0], sums[2] / sums[0], sums[3] / (double)n, fr);
        for (int i = 0; i < 9; i++) h->kp.f_ref[i] = (float)fr[i];
    }
    dim3 blk(32, 8);
    if (h->moments) {
        init_moments_kernel<<<cell_grid(h, blk), blk, 0, h->stream>>>(dev[0], dev[1], dev[2], dev[3], dev[4],
                                                                      static_cast<float *>(h->state[0]), h->kp);
        CK(cudaGetLastError(), "init_moments_kernel");
    } else CK(with_types(h, [&](auto ty) {
           using T = typename decltype(ty)::t;
           using S = typename decltype(ty)::s;
           init_kernel<T, S><<<cell_grid(h, blk), blk, 0, h->stream>>>(dev[0], dev[1], dev[2], dev[3], dev[4],
                                                                       pop_planes<T, S>(h, 0), aux_planes<T, S>(h, 0), h->kp);
           return cudaGetLastError();
       }), "init_kernel");
    h->cur = 0;
    CK(fill_cache(h), "cache_macros_kernel");
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

int hlbm_debug_check(long long *site, long long *a, long long *b)
{
#ifdef HLBM_DEBUG
    unsigned long long v = 0;
    const unsigned long long zero = 0;
    if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpyFromSymbol(&v, dbg_first, sizeof(v)) != cudaSuccess ||
        cudaMemcpyToSymbol(dbg_first, &zero, sizeof(zero)) != cudaSuccess)
        return HLBM_ERR_CUDA;
    if (site) *site = v ? (long long)((v >> 56) & 0x7F) : 0;
    if (a) *a = (long long)((v >> 28) & 0xFFFFFFF);
    if (b) *b = (long long)(v & 0xFFFFFFF);
    return HLBM_OK;
#else
    (void)site; (void)a; (void)b;
    return HLBM_ERR_UNSUPPORTED;
#endif
}

int hlbm_step(hlbm_handle *h, int64_t n)
{
    NvtxRange nvtx_range("hlbm_step");
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
    NvtxRange nvtx_range("hlbm_get_fields");
    if (!h) return HLBM_ERR_ARG;
    if (!h->initialized) return fail(h, HLBM_ERR_STATE, "no state yet");
    if (mem_kind != HLBM_MEM_HOST && mem_kind != HLBM_MEM_DEVICE) return fail(h, HLBM_ERR_ARG, "mem_kind");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    const size_t n = (size_t)h->p.nx * h->p.ny;
    double *dst[7] = {rho, ux, uy, theta, s, a1, F};
    double *dev[7];
    bool copy_back[7] = {false, false, false, false, false, false, false};
    if (mem_kind == HLBM_MEM_HOST) {
        // pinned destinations are written in place by the kernel; pageable
        // ones go through the staging buffer (9 planes: fields use planes
        // 0..7 (a1 = 3), F uses all 9) and a copy
        const size_t off[7] = {0, 1, 2, 3, 4, 5, 0};
        for (int k = 0; k < 7; k++) {
            dev[k] = nullptr;
            if (!dst[k] || (F && k < 6)) continue;  // populations are read alone
            if ((dev[k] = host_view(dst[k]))) continue;
            dev[k] = h->staging + off[k] * n;
            copy_back[k] = true;
        }
    } else {
        for (int k = 0; k < 7; k++) dev[k] = dst[k];
    }
    dim3 blk(32, 8);
    if (h->moments) {
        if (F) return fail(h, HLBM_ERR_UNSUPPORTED, "the moment state stores no populations");
        moments_macros_kernel<<<cell_grid(h, blk), blk, 0, h->stream>>>(static_cast<const float *>(h->state[h->cur]),
                                                                        dev[0], dev[1], dev[2], dev[3], dev[4], dev[5],
                                                                        h->kp);
        CK(cudaGetLastError(), "moments_macros_kernel");
    } else CK(with_types(h, [&](auto ty) {
           using T = typename decltype(ty)::t;
           using S = typename decltype(ty)::s;
           macros_kernel<T, S><<<cell_grid(h, blk), blk, 0, h->stream>>>(pop_planes<T, S>(h, h->cur),
                                                                        aux_planes<T, S>(h, h->cur), dev[0], dev[1],
                                                                        dev[2], dev[3], dev[4], dev[5], dev[6], h->kp);
           return cudaGetLastError();
       }), "macros_kernel");
    for (int k = 0; k < 7; k++) {
        if (!copy_back[k]) continue;
        const size_t cnt = (k == 5 ? 3 : (k == 6 ? 9 : 1)) * n;
        CK(cudaMemcpyAsync(dst[k], dev[k], cnt * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "get copy");
    }
    CK(cudaStreamSynchronize(h->stream), "get sync");
    return check_timeout(h);
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
    NvtxRange nvtx_range("hlbm_diagnostics");
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
    return check_timeout(h);
}

int hlbm_state_bytes(const hlbm_handle *h, size_t *bytes)
{
    if (!h || !bytes) return HLBM_ERR_ARG;
    *bytes = sizeof(StateHeader) + alloc_bytes(h);
    return HLBM_OK;
}

int hlbm_get_state(hlbm_handle *h, void *buf, size_t bytes)
{
    NvtxRange nvtx_range("hlbm_get_state");
    if (!h || !buf) return HLBM_ERR_ARG;
    if (!h->initialized) return fail(h, HLBM_ERR_STATE, "no state yet");
    size_t need = 0;
    hlbm_state_bytes(h, &need);
    if (bytes < need) return fail(h, HLBM_ERR_ARG, "buffer too small");
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    StateHeader hd;
    memset(&hd, 0, sizeof(hd));
    hd.magic = STATE_MAGIC; hd.abi = HLBM_ABI_VERSION; hd.precision = h->p.precision;
    hd.nx = h->p.nx; hd.ny = h->p.ny; hd.pitch = h->pitch;
    hd.nplane = h->moments ? MS_NPLANE : NPLANE + (h->mcache ? A_NCACHE : 0);
    hd.step = h->step;
    hd.payload_bytes = (int64_t)(need - sizeof(StateHeader));
    for (int i = 0; i < 9; i++) hd.ref[i] = h->kp.f_ref[i];
    memcpy(buf, &hd, sizeof(hd));
    CK(cudaMemcpyAsync(static_cast<char *>(buf) + sizeof(hd), h->state[h->cur], (size_t)hd.payload_bytes,
                       cudaMemcpyDeviceToHost, h->stream), "state copy");
    CK(cudaStreamSynchronize(h->stream), "state sync");
    return HLBM_OK;
}

int hlbm_set_state(hlbm_handle *h, const void *buf, size_t bytes)
{
    NvtxRange nvtx_range("hlbm_set_state");
    if (!h || !buf) return HLBM_ERR_ARG;
    if (bytes < sizeof(StateHeader)) return fail(h, HLBM_ERR_STATE, "state size mismatch");
    StateHeader hd;
    memcpy(&hd, buf, sizeof(hd));
    // The population forms accept 13 planes, and in FP64 also 17 (the 13
    // and the marching form's cache planes, which hlbm_get_state of such a
    // handle writes): the cache is copied when both sides have it, derived
    // from F(n) and s(n) when only the handle has it, and skipped when only
    // the blob has it.
    const size_t base = payload_bytes(h);
    const size_t cache = h->plane * A_NCACHE * sizeof(double);
    bool ok_planes;
    size_t blob_payload;
    if (h->moments) {
        ok_planes = hd.nplane == MS_NPLANE;
        blob_payload = base;
    } else if (hd.nplane == NPLANE + A_NCACHE) {
        ok_planes = h->p.precision == HLBM_FP64;
        blob_payload = base + cache;
    } else {
        ok_planes = hd.nplane == NPLANE;
        blob_payload = base;
    }
    if (hd.magic != STATE_MAGIC || hd.abi != HLBM_ABI_VERSION || hd.precision != h->p.precision || hd.nx != h->p.nx ||
        hd.ny != h->p.ny || hd.pitch != h->pitch || !ok_planes || hd.step < 0 ||
        hd.payload_bytes != (int64_t)blob_payload)
        return fail(h, HLBM_ERR_STATE, "state header mismatch");
    if (bytes != sizeof(hd) + blob_payload) return fail(h, HLBM_ERR_STATE, "state size mismatch");
    const bool copy_cache = h->mcache && blob_payload > base;
    CK(cudaSetDevice(h->device), "cudaSetDevice");
    CK(cudaMemcpyAsync(h->state[0], static_cast<const char *>(buf) + sizeof(hd), copy_cache ? base + cache : base,
                       cudaMemcpyHostToDevice, h->stream), "state copy");
    for (int i = 0; i < 9; i++) h->kp.f_ref[i] = hd.ref[i];
    h->cur = 0;
    if (!copy_cache) CK(fill_cache(h), "cache_macros_kernel");
    CK(cudaStreamSynchronize(h->stream), "state sync");
    h->step = hd.step;
    h->initialized = true;
    return HLBM_OK;
}

}  // extern "C"

// ---- batches --------------------------------------------------------------------------
namespace {

struct TileShape {
    int tx, ty, nt;
};
constexpr TileShape kBatchTiles[] = {{32, 16, 256}, {64, 16, 256}, {32, 8, 128}, {64, 32, 512}, {32, 32, 512}};
constexpr int kNumBatchTiles = 5;
// Kinds 5 to 10: the row-marching kernel (64 threads, strips of 120
// columns) with segments of 16, 32, 48, 64, 96 and 128 rows (longer
// segments repeat the four-row ring refill less often, shorter ones balance
// the persistent grid better).  They need one sigma > 0 / Phi choice for all
// cases (the kernel is specialised on both).
constexpr int kBatchMarchRows[] = {16, 32, 48, 64, 96, 128};
constexpr int kNumBatchKinds = kNumBatchTiles + (int)(sizeof(kBatchMarchRows) / sizeof(kBatchMarchRows[0]));
constexpr int kBatchMarchNT = 64, kBatchMarchMinB = 8;
constexpr int kGraphSteps = 16;  // steps per captured graph (even: parity returns)

}  // namespace

struct hlbm_batch {
    std::vector<hlbm_handle *> cases;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int tile = 0;
    // device tables for the current tile shape
    KParams *d_kps = nullptr;
    CasePlanes *d_planes = nullptr;
    int *d_tile_case = nullptr, *d_tile_first = nullptr;
    int ntiles = 0;
    MarchItem *d_items = nullptr;  // marching kinds: (case, strip, segment) list
    int nitems = 0;
    bool march_ok = false, sig = false, phi0 = true;
    bool periodic = false;  // every case periodic on all sides
    int grid = 0;
    size_t smem = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // starting parity 0 / 1
};

template <int TX, int TY, int NT>
static cudaError_t batch_launch(hlbm_batch *b, int parity)
{
    BatchTables tab;
    tab.kps = b->d_kps; tab.planes = b->d_planes; tab.tile_case = b->d_tile_case; tab.tile_first = b->d_tile_first;
    tab.ntiles = b->ntiles;
    batched_step_kernel<TX, TY, NT><<<b->grid, NT, b->smem, b->stream>>>(tab, parity);
    return cudaGetLastError();
}

template <bool SIG, bool PHI0, bool PER>
static cudaError_t batch_march_launch(hlbm_batch *b, int parity)
{
    MarchTables tab;
    tab.kps = b->d_kps; tab.planes = b->d_planes; tab.items = b->d_items; tab.nitems = b->nitems;
    batched_march_kernel<kBatchMarchNT, kBatchMarchMinB, SIG, PHI0, PER><<<b->grid, kBatchMarchNT, b->smem, b->stream>>>(
        tab, parity);
    return cudaGetLastError();
}

template <bool PER>
static const void *batch_march_fn_t(const hlbm_batch *b)
{
    if (b->sig) return b->phi0 ? (const void *)batched_march_kernel<kBatchMarchNT, kBatchMarchMinB, true, true, PER>
                               : (const void *)batched_march_kernel<kBatchMarchNT, kBatchMarchMinB, true, false, PER>;
    return b->phi0 ? (const void *)batched_march_kernel<kBatchMarchNT, kBatchMarchMinB, false, true, PER>
                   : (const void *)batched_march_kernel<kBatchMarchNT, kBatchMarchMinB, false, false, PER>;
}

// all cases periodic: the specialised kernel
static const void *batch_march_fn(const hlbm_batch *b)
{
    return b->periodic ? batch_march_fn_t<true>(b) : batch_march_fn_t<false>(b);
}

template <bool PER>
static cudaError_t batch_march_launch_any(hlbm_batch *b, int parity)
{
    if (b->sig) return b->phi0 ? batch_march_launch<true, true, PER>(b, parity) : batch_march_launch<true, false, PER>(b, parity);
    return b->phi0 ? batch_march_launch<false, true, PER>(b, parity) : batch_march_launch<false, false, PER>(b, parity);
}

static cudaError_t batch_launch_any(hlbm_batch *b, int parity)
{
    if (b->tile >= kNumBatchTiles)
        return b->periodic ? batch_march_launch_any<true>(b, parity) : batch_march_launch_any<false>(b, parity);
    switch (b->tile) {
    case 1: return batch_launch<64, 16, 256>(b, parity);
    case 2: return batch_launch<32, 8, 128>(b, parity);
    case 3: return batch_launch<64, 32, 512>(b, parity);
    case 4: return batch_launch<32, 32, 512>(b, parity);
    default: return batch_launch<32, 16, 256>(b, parity);
    }
}

template <int TX, int TY, int NT>
static cudaError_t batch_kernel_setup(hlbm_batch *b, int *per_sm)
{
    using Geo = TileGeom<float, TX, TY>;
    b->smem = (Geo::smem_bytes + 15) / 16 * 16 + sizeof(KParams);
    cudaError_t e = cudaFuncSetAttribute(batched_step_kernel<TX, TY, NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batched_step_kernel<TX, TY, NT>, NT, b->smem);
}

static void batch_drop_graphs(hlbm_batch *b)
{
    for (int q = 0; q < 2; q++) {
        if (b->graph[q]) cudaGraphExecDestroy(b->graph[q]);
        b->graph[q] = nullptr;
    }
}

// (Re)build the tile tables and the persistent grid for tile shape b->tile.
static int batch_tables(hlbm_batch *b)
{
    batch_drop_graphs(b);
    const bool march = b->tile >= kNumBatchTiles;
    const TileShape ts = kBatchTiles[march ? 0 : b->tile];
    const int nc = (int)b->cases.size();
    std::vector<int> tile_case, tile_first(nc);
    std::vector<MarchItem> items;
    std::vector<KParams> kps(nc);
    std::vector<CasePlanes> planes(nc);
    for (int c = 0; c < nc; c++) {
        hlbm_handle *h = b->cases[c];
        tile_first[c] = (int)tile_case.size();
        const int nt = ((h->p.nx + ts.tx - 1) / ts.tx) * ((h->p.ny + ts.ty - 1) / ts.ty);
        tile_case.insert(tile_case.end(), nt, c);
        if (march) {
            // the segmentation of the single-case kernel with HLBM_MARCH_ROWS = rows
            const int W = PairGeom<float, kBatchMarchNT>::W, rows = kBatchMarchRows[b->tile - kNumBatchTiles];
            const int nseg = (h->p.ny + rows - 1) / rows;
            for (int k = 0; k < nseg; k++)
                for (int x0 = 0; x0 < h->p.nx; x0 += W)
                    items.push_back({c, x0, (int)((long long)k * h->p.ny / nseg), (int)((long long)(k + 1) * h->p.ny / nseg)});
        }
        kps[c] = h->kp;
        for (int q = 0; q < 2; q++) {
            planes[c].inF[q] = pop_planes<float, FullStore<float>>(h, q);
            planes[c].inA[q] = aux_planes<float, FullStore<float>>(h, q);
            planes[c].outF[q] = pop_planes<float, FullStore<float>>(h, q ^ 1);
            planes[c].outA[q] = aux_planes<float, FullStore<float>>(h, q ^ 1);
        }
    }
    b->ntiles = (int)tile_case.size();
    b->nitems = (int)items.size();
    cudaFree(b->d_kps); cudaFree(b->d_planes); cudaFree(b->d_tile_case); cudaFree(b->d_tile_first); cudaFree(b->d_items);
    b->d_kps = nullptr; b->d_planes = nullptr; b->d_tile_case = nullptr; b->d_tile_first = nullptr; b->d_items = nullptr;
    if (march && (cudaMalloc(&b->d_items, b->nitems * sizeof(MarchItem)) != cudaSuccess ||
                  cudaMemcpy(b->d_items, items.data(), b->nitems * sizeof(MarchItem), cudaMemcpyHostToDevice) != cudaSuccess))
        return HLBM_ERR_NOMEM;
    if (cudaMalloc(&b->d_kps, nc * sizeof(KParams)) != cudaSuccess ||
        cudaMalloc(&b->d_planes, nc * sizeof(CasePlanes)) != cudaSuccess ||
        cudaMalloc(&b->d_tile_case, b->ntiles * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->d_tile_first, nc * sizeof(int)) != cudaSuccess)
        return HLBM_ERR_NOMEM;
    if (cudaMemcpy(b->d_kps, kps.data(), nc * sizeof(KParams), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_planes, planes.data(), nc * sizeof(CasePlanes), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_tile_case, tile_case.data(), b->ntiles * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_tile_first, tile_first.data(), nc * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
        return HLBM_ERR_CUDA;
    int per_sm = 0, sms = 0;
    cudaError_t e;
    if (march) {
        b->smem = (PairGeom<float, kBatchMarchNT>::smem_bytes + 15) / 16 * 16 + sizeof(KParams);
        const void *fn = batch_march_fn(b);
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBatchMarchNT, b->smem);
        if (e != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess)
            return HLBM_ERR_CUDA;
        const int g = (per_sm > 0 ? per_sm : 1) * sms;
        b->grid = g < b->nitems ? g : b->nitems;
        return HLBM_OK;
    }
    switch (b->tile) {
    case 1: e = batch_kernel_setup<64, 16, 256>(b, &per_sm); break;
    case 2: e = batch_kernel_setup<32, 8, 128>(b, &per_sm); break;
    case 3: e = batch_kernel_setup<64, 32, 512>(b, &per_sm); break;
    case 4: e = batch_kernel_setup<32, 32, 512>(b, &per_sm); break;
    default: e = batch_kernel_setup<32, 16, 256>(b, &per_sm); break;
    }
    if (e != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess)
        return HLBM_ERR_CUDA;
    const int g = (per_sm > 0 ? per_sm : 1) * sms;
    b->grid = g < b->ntiles ? g : b->ntiles;
    return HLBM_OK;
}

// All cases initialised and at one parity; returns that parity or -1.
static int batch_parity(const hlbm_batch *b)
{
    int par = -1;
    for (hlbm_handle *h : b->cases) {
        if (!h->initialized) return -1;
        if (par < 0) par = h->cur;
        else if (par != h->cur) return -1;
    }
    return par;
}

static int batch_advance(hlbm_batch *b, int64_t n)
{
    int par = batch_parity(b);
    if (par < 0) return HLBM_ERR_STATE;
    int64_t done = 0;
    while (n - done >= kGraphSteps) {
        if (!b->graph[par]) {
            cudaGraph_t g;
            if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return HLBM_ERR_CUDA;
            cudaError_t e = cudaSuccess;
            for (int k = 0; k < kGraphSteps && e == cudaSuccess; k++) e = batch_launch_any(b, par ^ (k & 1));
            const cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
            if (e != cudaSuccess || e2 != cudaSuccess) return HLBM_ERR_CUDA;
            e = cudaGraphInstantiate(&b->graph[par], g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return HLBM_ERR_CUDA;
        }
        if (cudaGraphLaunch(b->graph[par], b->stream) != cudaSuccess) return HLBM_ERR_CUDA;
        done += kGraphSteps;
    }
    for (; done < n; done++) {
        if (batch_launch_any(b, par) != cudaSuccess) return HLBM_ERR_CUDA;
        par ^= 1;
    }
    for (hlbm_handle *h : b->cases) {
        h->cur = (int)((h->cur + n) & 1);
        h->step += n;
    }
    return HLBM_OK;
}

extern "C" {

void hlbm_batch_destroy(hlbm_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_drop_graphs(b);
    cudaFree(b->d_kps); cudaFree(b->d_planes); cudaFree(b->d_tile_case); cudaFree(b->d_tile_first); cudaFree(b->d_items);
    for (hlbm_handle *h : b->cases) hlbm_destroy(h);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

int hlbm_batch_create(const hlbm_params *params, int ncase, void *stream, hlbm_batch **out)
{
    if (!out || !params || ncase < 1) return HLBM_ERR_ARG;
    *out = nullptr;
    for (int c = 0; c < ncase; c++) {
        if (params[c].precision != HLBM_FP32) return HLBM_ERR_UNSUPPORTED;
        for (int k = 0; k < 4; k++)
            if (params[c].bc[k] == HLBM_BC_WALL) return HLBM_ERR_UNSUPPORTED;
    }
    hlbm_batch *b = new (std::nothrow) hlbm_batch();
    if (!b) return HLBM_ERR_NOMEM;
    if (cudaGetDevice(&b->device) != cudaSuccess) { delete b; return HLBM_ERR_CUDA; }
    if (stream) {
        b->stream = static_cast<cudaStream_t>(stream);
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) { delete b; return HLBM_ERR_CUDA; }
        b->own_stream = true;
    }
    for (int c = 0; c < ncase; c++) {
        hlbm_handle *h = nullptr;
        const int r = hlbm_create(&params[c], b->stream, &h);
        if (r != HLBM_OK) { hlbm_batch_destroy(b); return r; }
        b->cases.push_back(h);
    }
    b->sig = b->cases[0]->kp.sigma_nonzero != 0;
    b->phi0 = b->cases[0]->kp.phi_mode == 0;
    b->march_ok = true;
    b->periodic = true;
    for (hlbm_handle *h : b->cases) {
        if ((h->kp.sigma_nonzero != 0) != b->sig || (h->kp.phi_mode == 0) != b->phi0) b->march_ok = false;
        b->periodic = b->periodic && h->periodic;
    }
    // starting shape (HLBM_BATCH_TILE=<k> for tests and sweeps; autotune may change it)
    b->tile = env_choice("HLBM_BATCH_TILE", 0, 0, kNumBatchKinds);
    if (b->tile >= kNumBatchTiles && !b->march_ok) b->tile = 0;
    const int r = batch_tables(b);
    if (r != HLBM_OK) { hlbm_batch_destroy(b); return r; }
    *out = b;
    return HLBM_OK;
}

int hlbm_batch_case(hlbm_batch *b, int index, hlbm_handle **h)
{
    if (!b || !h || index < 0 || index >= (int)b->cases.size()) return HLBM_ERR_ARG;
    *h = b->cases[index];
    return HLBM_OK;
}

int hlbm_batch_step(hlbm_batch *b, int64_t n)
{
    NvtxRange nvtx_range("hlbm_batch_step");
    if (!b || n < 0) return HLBM_ERR_ARG;
    if (cudaSetDevice(b->device) != cudaSuccess) return HLBM_ERR_CUDA;
    return batch_advance(b, n);
}

int hlbm_batch_tile(const hlbm_batch *b, int *index, int *tx, int *ty, int *threads)
{
    if (!b) return HLBM_ERR_ARG;
    const bool march = b->tile >= kNumBatchTiles;
    if (index) *index = b->tile;
    if (tx) *tx = march ? PairGeom<float, kBatchMarchNT>::W : kBatchTiles[b->tile].tx;
    if (ty) *ty = march ? kBatchMarchRows[b->tile - kNumBatchTiles] : kBatchTiles[b->tile].ty;
    if (threads) *threads = march ? kBatchMarchNT : kBatchTiles[b->tile].nt;
    return HLBM_OK;
}

int hlbm_batch_autotune(hlbm_batch *b, int *tile)
{
    NvtxRange nvtx_range("hlbm_batch_autotune");
    if (!b) return HLBM_ERR_ARG;
    if (cudaSetDevice(b->device) != cudaSuccess) return HLBM_ERR_CUDA;
    if (batch_parity(b) < 0) return HLBM_ERR_STATE;
    // snapshot every case (the trials advance the states)
    std::vector<void *> saved(b->cases.size(), nullptr);
    std::vector<size_t> sizes(b->cases.size());
    std::vector<int> cur(b->cases.size());
    std::vector<int64_t> steps(b->cases.size());
    int rc = HLBM_OK;
    for (size_t c = 0; c < b->cases.size() && rc == HLBM_OK; c++) {
        hlbm_handle *h = b->cases[c];
        sizes[c] = payload_bytes(h);
        cur[c] = h->cur;
        steps[c] = h->step;
        if (cudaMalloc(&saved[c], sizes[c]) != cudaSuccess) rc = HLBM_ERR_NOMEM;
        else if (cudaMemcpyAsync(saved[c], h->state[h->cur], sizes[c], cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
            rc = HLBM_ERR_CUDA;
    }
    float best = 1e30f;
    int best_tile = b->tile;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == HLBM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = HLBM_ERR_CUDA;
    for (int t = 0; t < kNumBatchKinds && rc == HLBM_OK; t++) {
        if (t >= kNumBatchTiles && !b->march_ok) break;
        b->tile = t;
        rc = batch_tables(b);
        if (rc != HLBM_OK) break;
        int par = batch_parity(b);
        for (int k = 0; k < 2 && rc == HLBM_OK; k++, par ^= 1)
            if (batch_launch_any(b, par) != cudaSuccess) rc = HLBM_ERR_CUDA;
        cudaEventRecord(e0, b->stream);
        for (int k = 0; k < 6 && rc == HLBM_OK; k++, par ^= 1)
            if (batch_launch_any(b, par) != cudaSuccess) rc = HLBM_ERR_CUDA;
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = HLBM_ERR_CUDA;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rc == HLBM_OK && ms < best) { best = ms; best_tile = t; }
    }
    // restore the states and the parity
    for (size_t c = 0; c < b->cases.size(); c++) {
        hlbm_handle *h = b->cases[c];
        if (saved[c] && rc == HLBM_OK &&
            cudaMemcpyAsync(h->state[cur[c]], saved[c], sizes[c], cudaMemcpyDeviceToDevice, b->stream) != cudaSuccess)
            rc = HLBM_ERR_CUDA;
        h->cur = cur[c];
        h->step = steps[c];
    }
    cudaStreamSynchronize(b->stream);
    for (void *p : saved) cudaFree(p);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    b->tile = best_tile;
    const int r2 = batch_tables(b);
    if (rc == HLBM_OK) rc = r2;
    if (tile) *tile = best_tile;
    return rc;
}

}  // extern "C"
