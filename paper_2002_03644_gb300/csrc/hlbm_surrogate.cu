// hlbm_surrogate.cu -- a learned K-step surrogate of the hybrid LBM step:
// a stack of periodic 3x3 convolutions (GELU between them, the output added
// to the input) trained on the GPU by the kernels of this file.
//
// Layout: activations NHWC (channels innermost), BF16, channel counts padded
// to a multiple of 16; FP32 master weights W[l][co][ci][tap] (tap = 3 (p+1) +
// (q+1) for the offset (p, q) in rows and columns) and their BF16 copies
// arranged for the tensor-core B operand: Wb[tap][co][ci] (forward) and
// Wd[tap][ci][co] (input gradient, read with the negated offset of the tap).
//
// Convolution = implicit GEMM on the BF16 tensor cores (mma.sync m16n8k16,
// FP32 accumulators): out[pixel, n] = sum_tap sum_k B[tap][n][k] *
// in[pixel + offset(tap), k].  One warp computes 16 pixels x 64 outputs; the
// epilogue adds the bias and, where the layer has one, applies GELU and
// keeps the pre-activation for the backward pass.
//
// Weight gradient: dW[co][ci][tap] = sum_pixels dz[pixel, co] *
// h[pixel + offset(tap), ci], a GEMM over pixels on the tensor cores
// (BF16 operands, FP32 accumulators), added to the FP32 gradient with
// atomics.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "hlbm.h"

namespace {

constexpr int MAX_LAYERS = 8;
constexpr int MAXC = 64;  // widest layer (padded channels)

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// GELU(x) = x Phi(x) = (x / 2) (1 + erf(x / sqrt 2)) and its derivative
// Phi(x) + x phi(x), with erf from Abramowitz & Stegun, Handbook of
// Mathematical Functions, formula 7.1.26: for z >= 0,
//   erf(z) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-z^2) + eps,
//   t = 1 / (1 + p z), |eps| <= 1.5e-7,
// extended to z < 0 by oddness.  With z = |x| / sqrt 2, exp(-z^2) is the
// Gaussian factor phi(x) sqrt(2 pi) that the derivative needs as well.  The
// reciprocal and the exponential are the PTX approximations (a few ulp); the
// result is rounded to BF16 (8 bits) by every caller, far above these errors.
__device__ __forceinline__ float rcp_fast(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2_fast(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// r = (1 - erf(|x| / sqrt 2)) / 2 = Phi(-|x|) and e = exp(-x^2 / 2)
__device__ __forceinline__ void normal_tail(float x, float &r, float &e)
{
    const float t = rcp_fast(fmaf(0.3275911f * 0.70710678118654752f, fabsf(x), 1.0f));
    const float q = t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f),
                             0.254829592f);
    e = ex2_fast(x * x * -0.72134752044448170f);  // exp(-x^2 / 2) = 2^(-x^2 / (2 ln 2))
    r = 0.5f * q * e;
}

__device__ __forceinline__ float gelu_f(float x)
{
    float r, e;
    normal_tail(x, r, e);
    return x * (x >= 0.0f ? 1.0f - r : r);
}

__device__ __forceinline__ float gelu_grad_f(float x)
{
    float r, e;
    normal_tail(x, r, e);
    return (x >= 0.0f ? 1.0f - r : r) + x * 0.3989422804014327f * e;
}

// Two FP32 values in one 64-bit register pair, for the packed .f32x2
// instructions (one instruction, two independent IEEE operations).
struct fp2 {
    float x, y;
};
__device__ __forceinline__ unsigned long long fp2_bits(fp2 a)
{
    unsigned long long u;
    asm("mov.b64 %0, {%1, %2};" : "=l"(u) : "f"(a.x), "f"(a.y));
    return u;
}
__device__ __forceinline__ fp2 fp2_of(unsigned long long u)
{
    fp2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(u));
    return r;
}
__device__ __forceinline__ fp2 bc2(float a) { return fp2{a, a}; }
__device__ __forceinline__ fp2 add2(fp2 a, fp2 b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(fp2_bits(a)), "l"(fp2_bits(b)));
    return fp2_of(d);
}
__device__ __forceinline__ fp2 sub2(fp2 a, fp2 b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(fp2_bits(a)), "l"(fp2_bits(b)));
    return fp2_of(d);
}
__device__ __forceinline__ fp2 mul2(fp2 a, fp2 b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(fp2_bits(a)), "l"(fp2_bits(b)));
    return fp2_of(d);
}
__device__ __forceinline__ fp2 fma2(fp2 a, fp2 b, fp2 c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(fp2_bits(a)), "l"(fp2_bits(b)), "l"(fp2_bits(c)));
    return fp2_of(d);
}

// normal_tail on two values: the same formula, with the factor 1/2 folded
// into the coefficients (exact: a power of two)
__device__ __forceinline__ void normal_tail2(fp2 x, fp2 &r, fp2 &e)
{
    const fp2 den = fma2(fp2{fabsf(x.x), fabsf(x.y)}, bc2(0.3275911f * 0.70710678118654752f), bc2(1.0f));
    const fp2 t{rcp_fast(den.x), rcp_fast(den.y)};
    fp2 q = fma2(t, bc2(0.5f * 1.061405429f), bc2(0.5f * -1.453152027f));
    q = fma2(t, q, bc2(0.5f * 1.421413741f));
    q = fma2(t, q, bc2(0.5f * -0.284496736f));
    q = fma2(t, q, bc2(0.5f * 0.254829592f));
    q = mul2(t, q);
    const fp2 g = mul2(mul2(x, x), bc2(-0.72134752044448170f));
    e = fp2{ex2_fast(g.x), ex2_fast(g.y)};
    r = mul2(q, e);
}

// Phi(x) for two values, from r = Phi(-|x|)
__device__ __forceinline__ fp2 cdf2(fp2 x, fp2 r)
{
    const fp2 c = sub2(bc2(1.0f), r);
    return fp2{x.x >= 0.0f ? c.x : r.x, x.y >= 0.0f ? c.y : r.y};
}

__device__ __forceinline__ fp2 gelu2(fp2 x)
{
    fp2 r, e;
    normal_tail2(x, r, e);
    return mul2(x, cdf2(x, r));
}

__device__ __forceinline__ fp2 gelu_grad2(fp2 x)
{
    fp2 r, e;
    normal_tail2(x, r, e);
    return fma2(mul2(x, bc2(0.3989422804014327f)), e, cdf2(x, r));
}

// Two floats rounded to BF16, low half first.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16 *p)
{
    return *reinterpret_cast<const uint32_t *>(p);
}

__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], const uint32_t b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// B fragments of two n tiles (x4) or one (x2) from shared memory.
__device__ __forceinline__ void ldsm_x4(uint32_t b[4], const void *p)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3]) : "r"(a));
}
__device__ __forceinline__ void ldsm_x2(uint32_t b[2], const void *p)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(b[0]), "=r"(b[1]) : "r"(a));
}

constexpr int CONV_THREADS = 256;  // 8 warps x 32 pixels = 256 pixels per tile

template <int CIN, int NOUT>
struct ConvGeom {
    static constexpr int LDB = CIN + 8;  // padded weight row (elements): conflict-free ldmatrix
    static constexpr size_t smem_bytes = (size_t)9 * NOUT * LDB * sizeof(__nv_bfloat16);
};

// in  [npix][CIN]  (NHWC, pixels n*H*W + i*W + j), CIN multiple of 16
// B   [9][NOUT][CIN] BF16, NOUT multiple of 8 and <= 64
// bias[nbias] FP32 added to the first nbias outputs (bias may be NULL)
// mode 0: z_f32 = z, out_bf16 = z (no activation)
// mode 1: z_f32 = z, out_bf16 = GELU(z)
// mode 2 (input gradient): g = z * GELU'(zprev) (or z when zprev is NULL);
//         z_f32 = g, out_bf16 = g
// flip: use offset -(p, q) for tap (p, q) (input gradient)
// A persistent CTA stages all nine taps' weights in shared memory once
// (rows padded by 8 elements so that the 8 rows an ldmatrix reads fall in
// different banks), then walks 256-pixel tiles; each warp computes 32
// pixels (two m16 tiles) x NOUT outputs, so every weight fragment feeds two
// MMAs.  A fragments are read from global memory (L1-resident neighbours).
template <int CIN, int NOUT>
__global__ void __launch_bounds__(CONV_THREADS, 2)
conv_mma_kernel(const __nv_bfloat16 *__restrict__ in, const __nv_bfloat16 *__restrict__ B,
                const float *__restrict__ bias, int nbias, __nv_bfloat16 *__restrict__ out_bf,
                float *__restrict__ z_f32, const float *__restrict__ zprev, int npix, int H, int W, int mode, int flip)
{
    constexpr int NT = NOUT / 8;  // n tiles of 8
    constexpr int LDB = ConvGeom<CIN, NOUT>::LDB;
    constexpr int CH = CIN / 8;   // 16-byte chunks per weight row
    extern __shared__ __align__(16) unsigned char conv_smem[];
    __nv_bfloat16 *Bs = reinterpret_cast<__nv_bfloat16 *>(conv_smem);  // [9][NOUT][LDB]
    for (int e = threadIdx.x; e < 9 * NOUT * CH; e += CONV_THREADS) {
        const int row = e / CH, c = e - row * CH;
        *reinterpret_cast<uint4 *>(Bs + row * LDB + c * 8) =
            *reinterpret_cast<const uint4 *>(B + (size_t)row * CIN + c * 8);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t4 = lane & 3;
    // ldmatrix row address of this lane: matrix j = lane / 8 (n tile j / 2,
    // k half j % 2), row lane % 8
    const int lj = lane >> 3, lr = lane & 7;
    const int HW = H * W;
    const int ntiles = (npix + CONV_THREADS - 1) / CONV_THREADS;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int pix0 = tile * CONV_THREADS + warp * 32;
        if (pix0 >= npix) continue;
        // pixel rows of this lane's A fragments: q = 2 mt + h -> pix0 + 16 mt + 8 h + g
        int pn[4], pi[4], pj[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int p = pix0 + 16 * (q >> 1) + 8 * (q & 1) + g;
            const int pp = p < npix ? p : npix - 1;
            pn[q] = pp / HW;
            const int rem = pp - pn[q] * HW;
            pi[q] = rem / W;
            pj[q] = rem - pi[q] * W;
        }
        float acc[2][NT][4];
#pragma unroll
        for (int m = 0; m < 2; m++)
#pragma unroll
            for (int n = 0; n < NT; n++)
#pragma unroll
                for (int k = 0; k < 4; k++) acc[m][n][k] = 0.0f;

#pragma unroll 1
        for (int tap = 0; tap < 9; tap++) {
            int dp = tap / 3 - 1, dq = tap % 3 - 1;
            if (flip) { dp = -dp; dq = -dq; }
            const __nv_bfloat16 *row[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int ii = wrap(pi[q] + dp, H), jj = wrap(pj[q] + dq, W);
                row[q] = in + ((size_t)pn[q] * HW + (size_t)ii * W + jj) * CIN;
            }
            const __nv_bfloat16 *Bt = Bs + tap * NOUT * LDB;
#pragma unroll
            for (int k0 = 0; k0 < CIN; k0 += 16) {
                uint32_t a[2][4];
#pragma unroll
                for (int m = 0; m < 2; m++) {
                    a[m][0] = ld_pair(row[2 * m] + k0 + 2 * t4);
                    a[m][1] = ld_pair(row[2 * m + 1] + k0 + 2 * t4);
                    a[m][2] = ld_pair(row[2 * m] + k0 + 8 + 2 * t4);
                    a[m][3] = ld_pair(row[2 * m + 1] + k0 + 8 + 2 * t4);
                }
#pragma unroll
                for (int n = 0; n < NT; n += 2) {
                    if (n + 1 < NT) {
                        uint32_t b[4];
                        ldsm_x4(b, Bt + (n * 8 + (lj >> 1) * 8 + lr) * LDB + k0 + (lj & 1) * 8);
#pragma unroll
                        for (int m = 0; m < 2; m++) {
                            mma_bf16(acc[m][n], a[m], b);
                            mma_bf16(acc[m][n + 1], a[m], b + 2);
                        }
                    } else {
                        uint32_t b[2];
                        ldsm_x2(b, Bt + (n * 8 + lr) * LDB + k0 + (lj & 1) * 8);
#pragma unroll
                        for (int m = 0; m < 2; m++) mma_bf16(acc[m][n], a[m], b);
                    }
                }
            }
        }
        // epilogue: C fragment rows g, g+8 of each m tile; columns 2 t4, 2 t4 + 1 of each n tile
#pragma unroll
        for (int m = 0; m < 2; m++) {
#pragma unroll
            for (int r = 0; r < 2; r++) {
                const int p = pix0 + 16 * m + g + 8 * r;
                if (p >= npix) continue;
#pragma unroll
                for (int n = 0; n < NT; n++) {
#pragma unroll
                    for (int e = 0; e < 2; e++) {
                        const int col = n * 8 + 2 * t4 + e;
                        float z = acc[m][n][2 * r + e] + ((bias && col < nbias) ? bias[col] : 0.0f);
                        const size_t idx = (size_t)p * NOUT + col;
                        if (mode == 2) {
                            if (zprev) z *= gelu_grad_f(zprev[idx]);
                            out_bf[idx] = __float2bfloat16_rn(z);
                            if (z_f32) z_f32[idx] = z;
                        } else {
                            if (z_f32) z_f32[idx] = z;
                            out_bf[idx] = __float2bfloat16_rn(mode == 1 ? gelu_f(z) : z);
                        }
                    }
                }
            }
        }
    }
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t b[4], const void *p)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3]) : "r"(a));
}

// Weight gradient on the tensor cores: for one tap, dW[co][ci] += sum over
// pixels p of dz[p, co] h[p + off(tap), ci], a GEMM with the pixels as its
// K dimension (M = output channels, N = input channels).  BF16 tiles of dz
// and of the shifted activations ([pixel][channel], rows padded by 8 for
// conflict-free ldmatrix) are staged in shared memory and read transposed
// into the A and B fragments of mma.sync m16n8k16; each of the 4 warps
// accumulates a 32 x 32 block of the (at most) 64 x 64 result in FP32 over
// its CTA's pixel chunk, then adds it to the FP32 gradient (real channels
// only).  The bias gradient (tap 4 CTAs) sums the FP32 dz.  One CTA per
// (chunk, tap).
constexpr int WG_THREADS = 128, WG_KC = 64;

template <int CIN, int COUT>
__global__ void __launch_bounds__(WG_THREADS)
wgrad_mma_kernel(const __nv_bfloat16 *__restrict__ h, const __nv_bfloat16 *__restrict__ dzb,
                 const float *__restrict__ dzf, int cin, int cout, int npix, int H, int W, int chunk,
                 float *__restrict__ dW, float *__restrict__ db)
{
    constexpr int LDA = COUT + 8, LDB = CIN + 8;
    constexpr int MT = COUT / 16, NTT = CIN / 8;
    constexpr int CA = COUT / 8, CB = CIN / 8;  // 16-byte chunks per staged row
    __shared__ __align__(16) __nv_bfloat16 sA[WG_KC * LDA];
    __shared__ __align__(16) __nv_bfloat16 sB[WG_KC * LDB];
    const int tap = blockIdx.y;
    const int dp = tap / 3 - 1, dq = tap % 3 - 1;
    const int p0 = blockIdx.x * chunk;
    const int p1 = min(p0 + chunk, npix);
    const int HW = H * W;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t4 = lane & 3, lj = lane >> 3, lr = lane & 7;
    const int mt0 = 2 * (warp >> 1), nt0 = 4 * (warp & 1);
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 4; j++)
#pragma unroll
            for (int k = 0; k < 4; k++) acc[i][j][k] = 0.0f;
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    for (int q0 = p0; q0 < p1; q0 += WG_KC) {
        __syncthreads();  // the previous sub-chunk's fragments are read
        for (int e = threadIdx.x; e < WG_KC * CA; e += WG_THREADS) {
            const int r = e / CA, c8 = e - r * CA;
            const int p = q0 + r;
            *reinterpret_cast<uint4 *>(sA + r * LDA + c8 * 8) =
                p < p1 ? *reinterpret_cast<const uint4 *>(dzb + (size_t)p * COUT + c8 * 8) : zero;
        }
        for (int e = threadIdx.x; e < WG_KC * CB; e += WG_THREADS) {
            const int r = e / CB, c8 = e - r * CB;
            const int p = q0 + r;
            uint4 v = zero;
            if (p < p1) {
                const int n = p / HW, rem = p - n * HW, i = rem / W, j = rem - i * W;
                const int src = n * HW + wrap(i + dp, H) * W + wrap(j + dq, W);
                v = *reinterpret_cast<const uint4 *>(h + (size_t)src * CIN + c8 * 8);
            }
            *reinterpret_cast<uint4 *>(sB + r * LDB + c8 * 8) = v;
        }
        __syncthreads();
#pragma unroll
        for (int k0 = 0; k0 < WG_KC; k0 += 16) {
            uint32_t a[2][4];
#pragma unroll
            for (int mi = 0; mi < 2; mi++)
                if (mt0 + mi < MT)
                    ldsm_x4_t(a[mi], sA + (k0 + (lj >> 1) * 8 + lr) * LDA + (mt0 + mi) * 16 + (lj & 1) * 8);
#pragma unroll
            for (int ni = 0; ni < 4; ni += 2) {
                if (nt0 + ni + 1 < NTT) {
                    uint32_t b[4];
                    ldsm_x4_t(b, sB + (k0 + (lj & 1) * 8 + lr) * LDB + (nt0 + ni) * 8 + (lj >> 1) * 8);
#pragma unroll
                    for (int mi = 0; mi < 2; mi++) {
                        if (mt0 + mi < MT) {
                            mma_bf16(acc[mi][ni], a[mi], b);
                            mma_bf16(acc[mi][ni + 1], a[mi], b + 2);
                        }
                    }
                }
            }
        }
    }
#pragma unroll
    for (int mi = 0; mi < 2; mi++) {
#pragma unroll
        for (int ni = 0; ni < 4; ni++) {
            if (mt0 + mi >= MT || nt0 + ni >= NTT) continue;
#pragma unroll
            for (int r = 0; r < 2; r++)
#pragma unroll
                for (int e = 0; e < 2; e++) {
                    const int co = (mt0 + mi) * 16 + g + 8 * r, ci = (nt0 + ni) * 8 + 2 * t4 + e;
                    if (co < cout && ci < cin) atomicAdd(&dW[((size_t)co * cin + ci) * 9 + tap], acc[mi][ni][2 * r + e]);
                }
        }
    }
    if (tap == 4 && (int)threadIdx.x < cout) {
        float bacc = 0.0f;
        for (int p = p0; p < p1; p++) bacc += dzf[(size_t)p * COUT + threadIdx.x];
        atomicAdd(&db[threadIdx.x], bacc);
    }
}

template <int CIN>
cudaError_t launch_wgrad_cin(int cout_pad, const __nv_bfloat16 *h, const __nv_bfloat16 *dzb, const float *dzf, int cin,
                             int cout, int npix, int H, int W, float *dW, float *db, cudaStream_t st)
{
    const int chunk = 16384;
    dim3 grid((npix + chunk - 1) / chunk, 9);
    switch (cout_pad) {
    case 16: wgrad_mma_kernel<CIN, 16><<<grid, WG_THREADS, 0, st>>>(h, dzb, dzf, cin, cout, npix, H, W, chunk, dW, db); break;
    case 32: wgrad_mma_kernel<CIN, 32><<<grid, WG_THREADS, 0, st>>>(h, dzb, dzf, cin, cout, npix, H, W, chunk, dW, db); break;
    case 48: wgrad_mma_kernel<CIN, 48><<<grid, WG_THREADS, 0, st>>>(h, dzb, dzf, cin, cout, npix, H, W, chunk, dW, db); break;
    case 64: wgrad_mma_kernel<CIN, 64><<<grid, WG_THREADS, 0, st>>>(h, dzb, dzf, cin, cout, npix, H, W, chunk, dW, db); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// cin_pad, cout_pad: padded channel counts (multiples of 16)
cudaError_t launch_wgrad(int cin_pad, int cout_pad, const __nv_bfloat16 *h, const __nv_bfloat16 *dzb, const float *dzf,
                         int cin, int cout, int npix, int H, int W, float *dW, float *db, cudaStream_t st)
{
    switch (cin_pad) {
    case 16: return launch_wgrad_cin<16>(cout_pad, h, dzb, dzf, cin, cout, npix, H, W, dW, db, st);
    case 32: return launch_wgrad_cin<32>(cout_pad, h, dzb, dzf, cin, cout, npix, H, W, dW, db, st);
    case 48: return launch_wgrad_cin<48>(cout_pad, h, dzb, dzf, cin, cout, npix, H, W, dW, db, st);
    case 64: return launch_wgrad_cin<64>(cout_pad, h, dzb, dzf, cin, cout, npix, H, W, dW, db, st);
    default: return cudaErrorInvalidValue;
    }
}

// y = x + net(x) with the FP32 input x, loss = mean((y - t)^2),
// dnet = dy = 2 (y - t) / n
__global__ void residual_loss_kernel(const float *__restrict__ xin, const float *__restrict__ zlast, int cpad_last,
                                     const float *__restrict__ target, int c_real, int npix, float *__restrict__ y,
                                     float *__restrict__ dz_last, double *__restrict__ loss_acc)
{
    double local = 0.0;
    const long long n = (long long)npix * c_real;
    const float inv_n2 = 2.0f / (float)n;
    // one pixel per thread: its c_real outputs
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
        const size_t e0 = (size_t)p * c_real;
        const float *zp = zlast + (size_t)p * cpad_last;
        for (int c = 0; c < c_real; c++) {
            const float yy = xin[e0 + c] + zp[c];
            y[e0 + c] = yy;
            if (target) {
                const float d = yy - target[e0 + c];
                local += (double)d * d;
                dz_last[(size_t)p * cpad_last + c] = d * inv_n2;
            }
        }
    }
    if (target) {
        __shared__ double red[256];
        red[threadIdx.x] = local;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) atomicAdd(loss_acc, red[0]);
    }
}

// FP32 NHWC (c_real channels) -> BF16 NHWC padded to cpad channels (zeros)
__global__ void pack_input_kernel(const float *__restrict__ x, int c_real, int cpad, int npix,
                                  __nv_bfloat16 *__restrict__ out)
{
    // one pixel per thread: c_real FP32 values in, cpad BF16 values out in
    // 16-byte pieces (cpad is a multiple of 16)
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
        const float *src = x + (size_t)p * c_real;
        uint4 *dst = reinterpret_cast<uint4 *>(out + (size_t)p * cpad);
        for (int c0 = 0; c0 < cpad; c0 += 8) {
            uint32_t w[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int c = c0 + 2 * k;
                w[k] = pack_bf16(c < c_real ? src[c] : 0.0f, c + 1 < c_real ? src[c + 1] : 0.0f);
            }
            dst[c0 / 8] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// FP32 [n] -> BF16 [n]
// dz_last[p][c] += dy[p][c] for c < c_real: an upstream gradient (from a
// later call of a rollout through the network) added to dL/dy.
__global__ void add_upstream_kernel(float *__restrict__ dz_last, int cpad_last, const float *__restrict__ dy,
                                    int c_real, int npix)
{
    const long long n = (long long)npix * c_real;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dz_last[(i / c_real) * cpad_last + i % c_real] += dy[i];
}

// dx[p][c] = g[p][c] for c < c_real, from a padded [npix][cpad] gradient;
// with add != 0, dx[p][c] += g[p][c].  The input gradient of y = x + net(x)
// is dL/dy (the identity) plus the network's part.
__global__ void gather_grad_kernel(const float *__restrict__ g, int cpad, int c_real, int npix, int add,
                                   float *__restrict__ dx)
{
    const long long n = (long long)npix * c_real;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float v = g[(i / c_real) * cpad + i % c_real];
        dx[i] = add ? dx[i] + v : v;
    }
}

__global__ void to_bf16_kernel(const float *__restrict__ x, long long n, __nv_bfloat16 *__restrict__ out)
{
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        out[e] = __float2bfloat16_rn(x[e]);
}

// master W[co][ci][tap] (real channels) -> Wb[tap][co_pad][ci_pad] and
// Wd[tap][ci_pad][co_pad] (the input-gradient pass negates the offset of
// the tap, not the tap index)
__global__ void arrange_weights_kernel(const float *__restrict__ Wm, int cout, int cin, int cout_pad, int cin_pad,
                                       __nv_bfloat16 *__restrict__ Wb, __nv_bfloat16 *__restrict__ Wd)
{
    const int n = 9 * cout_pad * cin_pad;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int tap = e / (cout_pad * cin_pad);
        const int rem = e - tap * cout_pad * cin_pad;
        const int co = rem / cin_pad, ci = rem - co * cin_pad;
        const float w = (co < cout && ci < cin) ? Wm[((size_t)co * cin + ci) * 9 + tap] : 0.0f;
        Wb[e] = __float2bfloat16_rn(w);
        Wd[((size_t)tap * cin_pad + ci) * cout_pad + co] = __float2bfloat16_rn(w);
    }
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2)
{
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float gg = g[e];
        const float mm = b1 * m[e] + (1.0f - b1) * gg;
        const float vv = b2 * v[e] + (1.0f - b2) * gg * gg;
        m[e] = mm;
        v[e] = vv;
        p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    }
}

int pad16(int c) { return (c + 15) / 16 * 16; }

struct ConvArgs {
    const __nv_bfloat16 *in, *B;
    const float *bias;
    int nbias;
    __nv_bfloat16 *out;
    float *z;
    const float *zprev;
    int npix, H, W, mode, flip;
};

// Staged form for images whose width is a multiple of STG_TW: a CTA of 4
// warps computes one 128-pixel segment of one image row.  It copies the
// three input rows a 3x3 tap reaches (periodic wrap, one pixel of halo on
// each side) into shared memory once with cp.async, and streams the
// weights one tap at a time through a double buffer (the copy of tap t+1
// overlaps the MMAs of tap t); both operands are read by ldmatrix.  Each
// warp computes 32 pixels x NOUT outputs.
constexpr int STG_TW = 128, STG_THREADS = 128;

template <int CIN, int NOUT>
struct StagedConvGeom {
    static constexpr int LDI = CIN + 8, LDB = CIN + 8, RW = STG_TW + 2;
    static constexpr size_t in_elems = (size_t)3 * RW * LDI;
    static constexpr size_t w_elems = (size_t)NOUT * LDB;  // one tap
    static constexpr size_t smem_bytes = (in_elems + 2 * w_elems) * sizeof(__nv_bfloat16);
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int CIN, int NOUT>
__global__ void __launch_bounds__(STG_THREADS)
conv_staged_kernel(const __nv_bfloat16 *__restrict__ in, const __nv_bfloat16 *__restrict__ B,
                   const float *__restrict__ bias, int nbias, __nv_bfloat16 *__restrict__ out_bf,
                   float *__restrict__ z_f32, const float *__restrict__ zprev, int H, int W, int mode, int flip)
{
    using G = StagedConvGeom<CIN, NOUT>;
    constexpr int NT = NOUT / 8, LDI = G::LDI, LDB = G::LDB, RW = G::RW, CH = CIN / 8;
    extern __shared__ __align__(16) unsigned char conv_smem[];
    __nv_bfloat16 *Is = reinterpret_cast<__nv_bfloat16 *>(conv_smem);  // [3][RW][LDI]
    __nv_bfloat16 *Ws = Is + G::in_elems;                               // [2][NOUT][LDB]
    const int nseg = W / STG_TW;
    const int seg = blockIdx.x % nseg, row = blockIdx.x / nseg;  // row = n H + i
    const int n = row / H, i = row - n * H;
    const int j0 = seg * STG_TW;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t4 = lane & 3, lj = lane >> 3, lr = lane & 7;
    // input rows i-1 .. i+1, columns j0-1 .. j0+STG_TW (wrapped)
    for (int e = threadIdx.x; e < 3 * RW * CH; e += STG_THREADS) {
        const int rr = e / (RW * CH), rem = e - rr * RW * CH;
        const int cc = rem / CH, c8 = rem - cc * CH;
        const int ii = wrap(i + rr - 1, H), jj = wrap(j0 + cc - 1, W);
        cp_async16(Is + (rr * RW + cc) * LDI + c8 * 8, in + (((size_t)n * H + ii) * W + jj) * CIN + c8 * 8);
    }
    auto load_w = [&](int tap, int buf) {
        for (int e = threadIdx.x; e < NOUT * CH; e += STG_THREADS) {
            const int r = e / CH, c8 = e - r * CH;
            cp_async16(Ws + buf * G::w_elems + r * LDB + c8 * 8, B + ((size_t)tap * NOUT + r) * CIN + c8 * 8);
        }
    };
    load_w(0, 0);
    cp_async_commit();
    float acc[2][NT][4];
#pragma unroll
    for (int m = 0; m < 2; m++)
#pragma unroll
        for (int q = 0; q < NT; q++)
#pragma unroll
            for (int k = 0; k < 4; k++) acc[m][q][k] = 0.0f;
#pragma unroll 1
    for (int tap = 0; tap < 9; tap++) {
        cp_async_wait0();
        __syncthreads();  // tap's weights (and the input rows) are in; tap-1's buffer is free
        if (tap + 1 < 9) {
            load_w(tap + 1, (tap + 1) & 1);
            cp_async_commit();
        }
        int dp = tap / 3 - 1, dq = tap % 3 - 1;
        if (flip) { dp = -dp; dq = -dq; }
        const __nv_bfloat16 *rowp = Is + (1 + dp) * RW * LDI;
        const __nv_bfloat16 *Bt = Ws + (tap & 1) * G::w_elems;
#pragma unroll
        for (int k0 = 0; k0 < CIN; k0 += 16) {
            uint32_t a[2][4];
#pragma unroll
            for (int m = 0; m < 2; m++)
                ldsm_x4(a[m], rowp + (32 * warp + 16 * m + (lj & 1) * 8 + lr + 1 + dq) * LDI + k0 + (lj >> 1) * 8);
#pragma unroll
            for (int q = 0; q < NT; q += 2) {
                if (q + 1 < NT) {
                    uint32_t b[4];
                    ldsm_x4(b, Bt + (q * 8 + (lj >> 1) * 8 + lr) * LDB + k0 + (lj & 1) * 8);
#pragma unroll
                    for (int m = 0; m < 2; m++) {
                        mma_bf16(acc[m][q], a[m], b);
                        mma_bf16(acc[m][q + 1], a[m], b + 2);
                    }
                } else {
                    uint32_t b[2];
                    ldsm_x2(b, Bt + (q * 8 + lr) * LDB + k0 + (lj & 1) * 8);
#pragma unroll
                    for (int m = 0; m < 2; m++) mma_bf16(acc[m][q], a[m], b);
                }
            }
        }
    }
    const size_t rowpix = (size_t)row * W + j0 + 32 * warp;
#pragma unroll
    for (int m = 0; m < 2; m++) {
#pragma unroll
        for (int r = 0; r < 2; r++) {
            const size_t p = rowpix + 16 * m + g + 8 * r;
#pragma unroll
            for (int q = 0; q < NT; q++) {
                // the two adjacent outputs of this thread, stored together
                const int col = q * 8 + 2 * t4;
                float z0 = acc[m][q][2 * r] + ((bias && col < nbias) ? bias[col] : 0.0f);
                float z1 = acc[m][q][2 * r + 1] + ((bias && col + 1 < nbias) ? bias[col + 1] : 0.0f);
                const size_t idx = p * NOUT + col;
                if (mode == 2 && zprev) {
                    const float2 zp = *reinterpret_cast<const float2 *>(zprev + idx);
                    const fp2 d = mul2(fp2{z0, z1}, gelu_grad2(fp2{zp.x, zp.y}));
                    z0 = d.x;
                    z1 = d.y;
                }
                if (z_f32) *reinterpret_cast<float2 *>(z_f32 + idx) = make_float2(z0, z1);
                if (mode == 1) {
                    const fp2 gv = gelu2(fp2{z0, z1});
                    z0 = gv.x;
                    z1 = gv.y;
                }
                *reinterpret_cast<uint32_t *>(out_bf + idx) = pack_bf16(z0, z1);
            }
        }
    }
}

// ---- 5th-generation tensor cores (tcgen05, TMEM accumulators) ---------------------
// The convolutions with CIN, NOUT in {16, 64} (padded channels) on images
// whose width is a multiple of 128, as a persistent kernel with one CTA of
// 17 warps per SM:
//   - the nine taps' weights stay in shared memory for the whole launch;
//   - each 128-pixel row segment is one M = 128 tile; a CTA walks down a
//     contiguous run of tiles of one column segment, so consecutive tiles
//     share two of their three input rows.  The rows live in a ring of five
//     shared-memory slots: the current tile's three, the next tile's new
//     row, and the row after it, copied two tiles ahead (a run that crosses
//     an image refills the ring);
//   - one thread issues a tile's 9 CIN / 16 MMAs (M = 128, N = NOUT, K = 16,
//     BF16 operands) into one of two TMEM accumulators of NOUT FP32 columns,
//     with tcgen05.commit signalling an mbarrier when they are done;
//   - while the MMAs of tile k run, all warps read tile k-1's accumulator
//     (tcgen05.ld), apply bias / GELU and store.
//   - warps 0-15 copy rows and run the epilogue; warp 16 only issues MMAs.
// Operands are K-major.  With 64 channels a pixel (or a weight row) is one
// 128-byte row of the 128-byte swizzle layout, so a tap's pixel shift moves
// the operand by whole aligned rows.  With 16 channels they use the layout
// without swizzle: 8-row x 16-byte core matrices, rows 16 bytes apart,
// 8-row groups SBO = 128 bytes apart (consecutive pixels are consecutive
// 16-byte rows and a pixel shift is a 16-byte offset of the start
// address), the two 8-channel halves of a K-slice LBO bytes apart.
constexpr int TC_THREADS = 544, TC_TW = 128, TC_RW = TC_TW + 2;
constexpr int TC_EPI = 512;        // warps 0-15: copies and epilogue; warp 16 issues the MMAs
constexpr int TC_MMA_TID = 512;
constexpr uint32_t TC_IN_LBO = TC_RW * 16;               // 2080: channel-chunk stride of a staged row
// Dynamic shared memory requested: the operands need at most 173.6 KB (64 ->
// 64); the rest is slack so that every address a descriptor can form stays
// inside the block.
constexpr uint32_t TC_SMEM = 220 * 1024;
constexpr long long TC_WAIT_CYCLES = 2000000000ll;       // about 1 s at 2 GHz

template <int CIN, int NOUT>
struct TcGeom {
    static constexpr int CH = CIN / 8;                         // 16-byte channel chunks per pixel
    // 64 channels: one pixel (or weight row) is one 128-byte row of the
    // 128-byte swizzle layout (16-byte chunk c of row r stored at chunk
    // c ^ (r % 8), rows 128 bytes apart, 8-row groups 1024 bytes apart), so a
    // tap's pixel shift moves the operand by whole rows.  16 channels: the
    // layout without swizzle.
    static constexpr bool SW = CIN == 64;
    static constexpr uint32_t W_LBO = NOUT * 16;               // chunk stride of one tap's weights (no swizzle)
    static constexpr uint32_t W_TAP = CH * W_LBO;              // one tap: [n][128 B] or [k / 8][n][8]
    static constexpr uint32_t W_BYTES = 9 * W_TAP;
    static constexpr uint32_t IN_ROW = SW ? (TC_RW * 128 + 1023) / 1024 * 1024  // [column][128 B]
                                          : CH * TC_IN_LBO;                       // [k / 8][column][8]
    static constexpr int SLOTS = 5;                              // row ring
    static constexpr uint32_t BAR_OFF = W_BYTES + SLOTS * IN_ROW;  // two mbarriers, then the TMEM address
    static constexpr uint32_t BIAS_OFF = BAR_OFF + 32;           // NOUT FP32 bias values
    static constexpr uint32_t TMEM_COLS = 2 * NOUT < 32 ? 32 : 2 * NOUT;  // two accumulators (allocation >= 32)
    static constexpr int COLS = NOUT / 4;                        // accumulator columns per warp in the epilogue
    // Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1),
    // BF16 A and B (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17,
    // M >> 4 at bit 24.
    static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NOUT >> 3) << 17) |
                                      ((uint32_t)(TC_TW >> 4) << 24);
    static_assert(BIAS_OFF + 4 * NOUT <= TC_SMEM, "shared memory");
    static_assert(!SW || (W_TAP % 1024 == 0 && W_BYTES % 1024 == 0 && IN_ROW % 1024 == 0), "swizzle atoms");
    static_assert(NOUT % 16 == 0 && CIN % 16 == 0, "shapes");
};

// Status of the tcgen05 kernel, read by hlbm_sur_synchronize: 1 when an
// mbarrier wait gave up, 2 when the shared memory was not 1024-byte aligned.
__device__ int g_tc_status = 0;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets (all >> 4), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// The same with the 128-byte swizzle (layout type 2): SBO = 1024 bytes
// between 8-row groups, LBO unused (16), base offset 0.  The swizzle phase
// follows the absolute shared-memory address (chunk bits 4-6 XOR row bits
// 7-9), so an operand may start at any 128-byte row of a 1024-byte aligned
// buffer, and 32-byte steps of the start address select the K-slice.
__device__ __forceinline__ uint64_t umma_desc_sw(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase; false (and the timeout flag set) after
// about a second.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > TC_WAIT_CYCLES) {
            atomicExch(&g_tc_status, 1);
            return false;
        }
    }
    return true;
}

// COLS TMEM columns of this warp's 32 lanes (one FP32 value per column).
template <int COLS>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float *v);
template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; k++) v[k] = __uint_as_float(r[k]);
}
template <>
__device__ __forceinline__ void tmem_ld<4>(uint32_t taddr, float *v)
{
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 4; k++) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 bytes: COLS / ... BF16 values of out (COLS = 4: 8 bytes)
template <int COLS>
__device__ __forceinline__ void store_bf16(__nv_bfloat16 *dst, const float *v)
{
    if constexpr (COLS == 4) {
        *reinterpret_cast<uint2 *>(dst) = make_uint2(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]));
    } else {
        uint4 *d = reinterpret_cast<uint4 *>(dst);
#pragma unroll
        for (int c = 0; c < COLS / 8; c++)
            d[c] = make_uint4(pack_bf16(v[8 * c], v[8 * c + 1]), pack_bf16(v[8 * c + 2], v[8 * c + 3]),
                              pack_bf16(v[8 * c + 4], v[8 * c + 5]), pack_bf16(v[8 * c + 6], v[8 * c + 7]));
    }
}

template <int CIN, int NOUT>
__global__ void __launch_bounds__(TC_THREADS, 1)
conv_tc_kernel(const __nv_bfloat16 *__restrict__ in, const __nv_bfloat16 *__restrict__ B,
               const float *__restrict__ bias, int nbias, __nv_bfloat16 *__restrict__ out_bf,
               float *__restrict__ z_f32, const float *__restrict__ zprev, int H, int W, int ntiles, int mode,
               int flip)
{
    using G = TcGeom<CIN, NOUT>;
    constexpr int CH = G::CH, COLS = G::COLS;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    const uint32_t sbase = smem_addr(tc_smem);
    const uint32_t w_s = sbase, ring_s = sbase + G::W_BYTES;
    auto bar = [&](int b) { return sbase + G::BAR_OFF + 8 * b; };
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tc_smem + G::BAR_OFF + 16);
    float *bias_s = reinterpret_cast<float *>(tc_smem + G::BIAS_OFF);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nseg = W / TC_TW;
    const int R = ntiles / nseg;  // image rows of the batch, B H
    // the swizzled layouts assume 1024-byte aligned shared memory
    if (G::SW && (sbase & 1023u) != 0) {
        if (tid == 0) atomicExch(&g_tc_status, 2);
        return;
    }
    if (tid < NOUT) bias_s[tid] = (bias && tid < nbias) ? bias[tid] : 0.0f;

    // TMEM for the two accumulators (one warp allocates), the mbarriers
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(G::TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar(0)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar(1)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // weights of all taps: B[tap][n][k] -> [tap][k / 8][n][8]
    for (int e = tid; e < 9 * NOUT * CH; e += TC_THREADS) {
        const int tap = e / (NOUT * CH), rem = e - tap * (NOUT * CH), nrow = rem / CH, kc = rem - nrow * CH;
        const uint32_t off = G::SW ? nrow * 128 + ((kc ^ (nrow & 7)) << 4) : kc * G::W_LBO + nrow * 16;
        cp_async16(tc_smem + tap * G::W_TAP + off, B + ((size_t)tap * NOUT + nrow) * CIN + kc * 8);
    }
    // Tiles are numbered column segment first: T = seg R + r, r = n H + i;
    // this CTA takes T in [t0, t0 + my_tiles).  Tile T + 1 shares two input
    // rows with T unless T is an image's last row (or the segment's).
    const int t0 = (int)(((long long)blockIdx.x * ntiles) / gridDim.x);
    const int my_tiles = (int)(((long long)(blockIdx.x + 1) * ntiles) / gridDim.x) - t0;
    auto successor = [&](int T) { return (T % H) != H - 1; };
    // input row i - 1 + d (wrapped in the image) of tile T, columns j0-1 ..
    // j0+128 -> ring slot [k / 8][column][8]: thread t copies channel chunk
    // t % CH of columns t / CH + (512 / CH) m
    const int s_kc = tid % CH, s_px = tid / CH;
    auto load_row = [&](int T, int d, int slot) {
        if (tid >= TC_EPI) return;
        const int seg = T / R, r = T - seg * R;
        const int n = r / H, i = r - n * H, j0 = seg * TC_TW;
        const __nv_bfloat16 *src = in + ((size_t)n * H + wrap(i - 1 + d, H)) * W * CIN + s_kc * 8;
        unsigned char *dst = tc_smem + G::W_BYTES + slot * G::IN_ROW;
#pragma unroll
        for (int m = 0; m < (TC_RW * CH + TC_EPI - 1) / TC_EPI; m++) {
            const int px = s_px + (TC_EPI / CH) * m;
            const uint32_t off = G::SW ? px * 128 + ((s_kc ^ (px & 7)) << 4) : s_kc * TC_IN_LBO + px * 16;
            if (px < TC_RW) cp_async16(dst + off, src + (size_t)wrap(j0 + px - 1, W) * CIN);
        }
    };
    cp_async_commit();
    cp_async_wait0();  // the weights
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // epilogue of local tile k (accumulator k & 1): warp w reads TMEM lanes
    // 32 (w % 4) .. +31 (pixels) and columns COLS (w / 4) .. +COLS-1 (outputs).
    // Once tile k's MMAs are complete, the ring slot of its first input row
    // is free: then() copies a later tile's row into it right away, so that
    // the copy overlaps the epilogue math.
    auto epilogue = [&](int k, auto then) -> bool {
        const int T = t0 + k;
        // the warp-wide TMEM load below needs the whole warp: agree on the outcome
        if (!__all_sync(0xffffffffu, mbar_wait(bar(k & 1), (k >> 1) & 1))) return false;
        then();
        tc_fence_after();
        const int q = warp & 3, h = warp >> 2;
        float v[COLS];
        tmem_ld<COLS>(tmem + ((uint32_t)(32 * q) << 16) + (k & 1) * NOUT + COLS * h, v);
        const int seg = T / R, r = T - seg * R;
        const size_t p = (size_t)r * W + seg * TC_TW + 32 * q + lane;
        const size_t o = p * NOUT + COLS * h;  // this thread's COLS outputs
        // pairs of adjacent outputs in packed FP32
        const float2 *bs = reinterpret_cast<const float2 *>(bias_s + COLS * h);
#pragma unroll
        for (int c = 0; c < COLS / 2; c++) {
            const float2 b2 = bs[c];
            const fp2 z = add2(fp2{v[2 * c], v[2 * c + 1]}, fp2{b2.x, b2.y});
            v[2 * c] = z.x;
            v[2 * c + 1] = z.y;
        }
        if (mode == 2 && zprev) {
            const float4 *zp = reinterpret_cast<const float4 *>(zprev + o);
#pragma unroll
            for (int c = 0; c < COLS / 4; c++) {
                const float4 g = zp[c];
                const fp2 d0 = mul2(fp2{v[4 * c], v[4 * c + 1]}, gelu_grad2(fp2{g.x, g.y}));
                const fp2 d1 = mul2(fp2{v[4 * c + 2], v[4 * c + 3]}, gelu_grad2(fp2{g.z, g.w}));
                v[4 * c] = d0.x; v[4 * c + 1] = d0.y; v[4 * c + 2] = d1.x; v[4 * c + 3] = d1.y;
            }
        }
        if (z_f32) {
            float4 *zd = reinterpret_cast<float4 *>(z_f32 + o);
#pragma unroll
            for (int c = 0; c < COLS / 4; c++) zd[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
        }
        if (mode == 1) {
#pragma unroll
            for (int c = 0; c < COLS / 2; c++) {
                const fp2 gv = gelu2(fp2{v[2 * c], v[2 * c + 1]});
                v[2 * c] = gv.x;
                v[2 * c + 1] = gv.y;
            }
        }
        store_bf16<COLS>(out_bf + o, v);
        return true;
    };

    // The MMAs of a tile whose input rows i-1, i, i+1 sit in ring slots
    // (base + 0, 1, 2) % 5: a K-slice of tap (dp, dq) starts at row slot
    // (base + 1 + dp), column 1 + dq; descriptors differ from the slot's
    // only in the start-address field (16-byte units).
    const uint64_t bdesc0 = G::SW ? umma_desc_sw(w_s) : umma_desc(w_s, G::W_LBO, 128);
    auto issue = [&](int b, int base, bool flipped) {
        const uint32_t d = tmem + b * NOUT;
        uint64_t rowdesc[3];
#pragma unroll
        for (int e = 0; e < 3; e++) {
            const uint32_t a = ring_s + ((base + e) % G::SLOTS) * G::IN_ROW;
            rowdesc[e] = G::SW ? umma_desc_sw(a) : umma_desc(a, TC_IN_LBO, 128);
        }
#pragma unroll
        for (int tap = 0; tap < 9; tap++) {
            const int dp = flipped ? 1 - tap / 3 : tap / 3 - 1, dq = flipped ? 1 - tap % 3 : tap % 3 - 1;
#pragma unroll
            for (int ks = 0; ks < CIN / 16; ks++) {
                // start-address offsets: the pixel shift (whole 128-byte rows
                // when swizzled) and the K-slice (32 bytes within the row)
                const uint32_t ao = G::SW ? ((1 + dq) * 128 + 32 * ks) >> 4 : ((1 + dq) * 16 + 2 * ks * TC_IN_LBO) >> 4;
                const uint32_t bo = G::SW ? (tap * G::W_TAP + 32 * ks) >> 4 : (tap * G::W_TAP + 2 * ks * G::W_LBO) >> 4;
                umma_f16(d, rowdesc[1 + dp] + ao, bdesc0 + bo, G::IDESC, (tap | ks) != 0);
            }
        }
        umma_commit(bar(b));
    };

    bool ok = true;
    int j0 = 0;  // local index of the tile that started the current run
    for (int k = 0; k < my_tiles && ok; k++) {
        const int T = t0 + k;
        if (k == 0 || !successor(T - 1)) {
            // a new run: wait until the ring is free (the previous tile's
            // MMAs are done), then copy this tile's three rows and the next
            // tile's new row
            if (k > 0) ok = __all_sync(0xffffffffu, mbar_wait(bar((k - 1) & 1), ((k - 1) >> 1) & 1));
            ok = __syncthreads_and(ok);
            if (!ok) break;
            j0 = k;
            for (int d = 0; d < 3; d++) load_row(T, d, d);
            if (k + 1 < my_tiles && successor(T)) load_row(T + 1, 2, 3);
            cp_async_commit();
            cp_async_wait0();
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
        }
        const int base = k - j0;
        if (tid == TC_MMA_TID) {
            // the MMAs of tile k into accumulator k & 1
            tc_fence_after();
            if (flip) issue(k & 1, base, true);
            else issue(k & 1, base, false);
        }
        // tile k+2's new row, into the slot tile k-1's MMAs release
        auto prefetch = [&]() {
            if (k + 2 < my_tiles && successor(T) && successor(T + 1)) load_row(T + 2, 2, (base + 4) % G::SLOTS);
        };
        // tile k-1's results while tile k's MMAs run (warps 0-15)
        if (tid < TC_EPI) {
            if (k > 0) {
                if (!epilogue(k - 1, prefetch)) ok = false;
            } else {
                prefetch();
            }
        }
        cp_async_commit();
        // tile k+1's new row (copied one iteration earlier) has arrived; the
        // row of tile k+2 may still be in flight
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        fence_async_smem();
        tc_fence_before();
        ok = __syncthreads_and(ok);
    }
    if (ok && my_tiles > 0 && tid < TC_EPI) epilogue(my_tiles - 1, [] {});
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G::TMEM_COLS) : "memory");
    }
}

// Persistent grid: two CTAs per SM (the weights of a 64 x 64 layer take
// 81 KB of shared memory), at most one CTA per 256-pixel tile.
// The tcgen05 kernel serves the layers with 16 or 64 padded input and
// output channels unless HLBM_SUR_TC=0 (then the staged mma.sync kernel
// does).
bool use_tc()
{
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("HLBM_SUR_TC");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

template <int CIN, int NOUT>
cudaError_t launch_conv_t(const ConvArgs &a, cudaStream_t st)
{
    using G = ConvGeom<CIN, NOUT>;
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(conv_mma_kernel<CIN, NOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)G::smem_bytes);
        if (e != cudaSuccess) { sms = 0; return e; }
    }
    if constexpr ((CIN == 16 || CIN == 64) && (NOUT == 16 || NOUT == 64)) {
        if (a.W % TC_TW == 0 && a.npix % (a.H * a.W) == 0 && use_tc()) {
            static bool tc_ready = false;
            if (!tc_ready) {
                const cudaError_t e = cudaFuncSetAttribute(conv_tc_kernel<CIN, NOUT>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
                if (e != cudaSuccess) return e;
                tc_ready = true;
            }
            const int ntiles = a.npix / TC_TW;
            const int blocks = ntiles < sms ? ntiles : sms;
            conv_tc_kernel<CIN, NOUT><<<blocks, TC_THREADS, TC_SMEM, st>>>(a.in, a.B, a.bias, a.nbias, a.out, a.z,
                                                                          a.zprev, a.H, a.W, ntiles, a.mode, a.flip);
            return cudaGetLastError();
        }
    }
    if (a.W % STG_TW == 0 && a.npix % (a.H * a.W) == 0) {
        using S = StagedConvGeom<CIN, NOUT>;
        static bool staged_ready = false;
        if (!staged_ready) {
            const cudaError_t e = cudaFuncSetAttribute(conv_staged_kernel<CIN, NOUT>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem_bytes);
            if (e != cudaSuccess) return e;
            staged_ready = true;
        }
        conv_staged_kernel<CIN, NOUT><<<a.npix / STG_TW, STG_THREADS, S::smem_bytes, st>>>(
            a.in, a.B, a.bias, a.nbias, a.out, a.z, a.zprev, a.H, a.W, a.mode, a.flip);
        return cudaGetLastError();
    }
    const int tiles = (a.npix + CONV_THREADS - 1) / CONV_THREADS;
    const int blocks = tiles < 2 * sms ? tiles : 2 * sms;
    conv_mma_kernel<CIN, NOUT><<<blocks, CONV_THREADS, G::smem_bytes, st>>>(a.in, a.B, a.bias, a.nbias, a.out, a.z,
                                                                          a.zprev, a.npix, a.H, a.W, a.mode, a.flip);
    return cudaGetLastError();
}

template <int CIN>
cudaError_t launch_conv_cin(int nout, const ConvArgs &a, cudaStream_t st)
{
    switch (nout) {
    case 8: return launch_conv_t<CIN, 8>(a, st);
    case 16: return launch_conv_t<CIN, 16>(a, st);
    case 32: return launch_conv_t<CIN, 32>(a, st);
    case 48: return launch_conv_t<CIN, 48>(a, st);
    case 64: return launch_conv_t<CIN, 64>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

// cin: padded input channels (multiple of 16); nout: padded outputs
cudaError_t launch_conv(int cin, int nout, const ConvArgs &a, cudaStream_t st)
{
    switch (cin) {
    case 16: return launch_conv_cin<16>(nout, a, st);
    case 32: return launch_conv_cin<32>(nout, a, st);
    case 48: return launch_conv_cin<48>(nout, a, st);
    case 64: return launch_conv_cin<64>(nout, a, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

struct hlbm_sur {
    int L = 0, H = 0, W = 0, bmax = 0;
    int width[MAX_LAYERS + 1];
    int cpad_in[MAX_LAYERS], cpad_out[MAX_LAYERS];  // padded channels (in: multiple of 16, out: of 8 / 16)
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t nparam = 0;
    size_t woff[MAX_LAYERS], boff[MAX_LAYERS];
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // FP32 master params / grads / Adam moments
    __nv_bfloat16 *Wb[MAX_LAYERS] = {nullptr}, *Wd[MAX_LAYERS] = {nullptr};
    __nv_bfloat16 *act[MAX_LAYERS + 1] = {nullptr};  // layer inputs h_l (BF16, padded)
    float *z[MAX_LAYERS] = {nullptr};                // pre-activations (FP32, padded out)
    __nv_bfloat16 *gbuf[2] = {nullptr, nullptr};     // BF16 gradient ping-pong
    float *dz = nullptr, *dz2 = nullptr;             // FP32 gradient ping-pong (pre-activations)
    float *y = nullptr;
    float *xin = nullptr;   // FP32 copy of the last forward input (residual path)
    double *loss = nullptr;
    int last_batch = 0;
    int64_t adam_t = 0;
};

extern "C" {

void hlbm_sur_destroy(hlbm_sur *s)
{
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    cudaFree(s->p); cudaFree(s->g); cudaFree(s->m); cudaFree(s->v);
    for (int l = 0; l < MAX_LAYERS; l++) { cudaFree(s->Wb[l]); cudaFree(s->Wd[l]); cudaFree(s->z[l]); }
    for (int l = 0; l <= MAX_LAYERS; l++) cudaFree(s->act[l]);
    cudaFree(s->gbuf[0]); cudaFree(s->gbuf[1]); cudaFree(s->dz); cudaFree(s->dz2); cudaFree(s->y); cudaFree(s->xin); cudaFree(s->loss);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

int hlbm_sur_create(int nlayer, const int *widths, int H, int W, int batch_max, void *stream, hlbm_sur **out)
{
    if (!out || !widths || nlayer < 1 || nlayer > MAX_LAYERS || H < 1 || W < 1 || batch_max < 1) return HLBM_ERR_ARG;
    *out = nullptr;
    for (int l = 0; l <= nlayer; l++)
        if (widths[l] < 1 || widths[l] > MAXC) return HLBM_ERR_ARG;
    if (widths[nlayer] != widths[0]) return HLBM_ERR_ARG;  // residual output
    hlbm_sur *s = new (std::nothrow) hlbm_sur();
    if (!s) return HLBM_ERR_NOMEM;
    s->L = nlayer; s->H = H; s->W = W; s->bmax = batch_max;
    for (int l = 0; l <= nlayer; l++) s->width[l] = widths[l];
    if (stream) {
        s->stream = static_cast<cudaStream_t>(stream);
    } else if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return HLBM_ERR_CUDA;
    } else {
        s->own_stream = true;
    }
    size_t off = 0;
    for (int l = 0; l < nlayer; l++) {
        // every padded count is a multiple of 16: it is the K dimension of
        // the next layer (forward) or of the input-gradient pass (backward)
        s->cpad_in[l] = pad16(widths[l]);
        s->cpad_out[l] = pad16(widths[l + 1]);
        s->woff[l] = off; off += (size_t)widths[l + 1] * widths[l] * 9;
        s->boff[l] = off; off += widths[l + 1];
    }
    s->nparam = off;
    const size_t npix = (size_t)batch_max * H * W;
    bool ok = cudaMalloc(&s->p, off * 4) == cudaSuccess && cudaMalloc(&s->g, off * 4) == cudaSuccess &&
              cudaMalloc(&s->m, off * 4) == cudaSuccess && cudaMalloc(&s->v, off * 4) == cudaSuccess &&
              cudaMalloc(&s->loss, sizeof(double)) == cudaSuccess &&
              cudaMalloc(&s->y, npix * widths[0] * 4) == cudaSuccess &&
              cudaMalloc(&s->xin, npix * widths[0] * 4) == cudaSuccess &&
              cudaMalloc(&s->dz, npix * MAXC * 4) == cudaSuccess && cudaMalloc(&s->dz2, npix * MAXC * 4) == cudaSuccess &&
              cudaMalloc(&s->gbuf[0], npix * MAXC * 2) == cudaSuccess &&
              cudaMalloc(&s->gbuf[1], npix * MAXC * 2) == cudaSuccess;
    for (int l = 0; l < nlayer && ok; l++) {
        ok = cudaMalloc(&s->Wb[l], (size_t)9 * s->cpad_out[l] * s->cpad_in[l] * 2) == cudaSuccess &&
             cudaMalloc(&s->Wd[l], (size_t)9 * s->cpad_out[l] * s->cpad_in[l] * 2) == cudaSuccess &&
             cudaMalloc(&s->z[l], npix * s->cpad_out[l] * 4) == cudaSuccess &&
             cudaMalloc(&s->act[l], npix * s->cpad_in[l] * 2) == cudaSuccess;
    }
    if (ok) ok = cudaMalloc(&s->act[nlayer], npix * s->cpad_out[nlayer - 1] * 2) == cudaSuccess;
    if (!ok) { cudaGetLastError(); hlbm_sur_destroy(s); return HLBM_ERR_NOMEM; }
    if (cudaMemsetAsync(s->m, 0, off * 4, s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->v, 0, off * 4, s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->p, 0, off * 4, s->stream) != cudaSuccess) {
        hlbm_sur_destroy(s);
        return HLBM_ERR_CUDA;
    }
    *out = s;
    return HLBM_OK;
}

int64_t hlbm_sur_param_count(const hlbm_sur *s) { return s ? (int64_t)s->nparam : -1; }

static int sur_arrange(hlbm_sur *s)
{
    for (int l = 0; l < s->L; l++) {
        const int n = 9 * s->cpad_out[l] * s->cpad_in[l];
        if (cudaMemsetAsync(s->Wd[l], 0, (size_t)n * 2, s->stream) != cudaSuccess) return HLBM_ERR_CUDA;
        arrange_weights_kernel<<<(n + 255) / 256, 256, 0, s->stream>>>(s->p + s->woff[l], s->width[l + 1], s->width[l],
                                                                       s->cpad_out[l], s->cpad_in[l], s->Wb[l], s->Wd[l]);
        if (cudaGetLastError() != cudaSuccess) return HLBM_ERR_CUDA;
    }
    return HLBM_OK;
}

int hlbm_sur_set_params(hlbm_sur *s, const float *params, int mem_kind)
{
    if (!s || !params) return HLBM_ERR_ARG;
    const cudaMemcpyKind k = mem_kind == HLBM_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaMemcpyAsync(s->p, params, s->nparam * 4, k, s->stream) != cudaSuccess) return HLBM_ERR_CUDA;
    if (cudaMemsetAsync(s->m, 0, s->nparam * 4, s->stream) != cudaSuccess ||
        cudaMemsetAsync(s->v, 0, s->nparam * 4, s->stream) != cudaSuccess)
        return HLBM_ERR_CUDA;
    s->adam_t = 0;
    const int r = sur_arrange(s);
    if (r != HLBM_OK) return r;
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? HLBM_OK : HLBM_ERR_CUDA;
}

int hlbm_sur_get_params(hlbm_sur *s, float *params, float *grads, int mem_kind)
{
    if (!s) return HLBM_ERR_ARG;
    const cudaMemcpyKind k = mem_kind == HLBM_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (params && cudaMemcpyAsync(params, s->p, s->nparam * 4, k, s->stream) != cudaSuccess) return HLBM_ERR_CUDA;
    if (grads && cudaMemcpyAsync(grads, s->g, s->nparam * 4, k, s->stream) != cudaSuccess) return HLBM_ERR_CUDA;
    return cudaStreamSynchronize(s->stream) == cudaSuccess ? HLBM_OK : HLBM_ERR_CUDA;
}

// x: device FP32 [B, H, W, C0] (NHWC); y: device FP32 [B, H, W, C0] or NULL.
// keep_z: store every layer's FP32 pre-activation (for the backward pass);
// otherwise only the last layer's, which the residual output needs.
static int sur_run(hlbm_sur *s, const float *x, float *y, int B, bool keep_z)
{
    if (!s || !x || B < 1 || B > s->bmax) return HLBM_ERR_ARG;
    const int npix = B * s->H * s->W;
    if (cudaMemcpyAsync(s->xin, x, (size_t)npix * s->width[0] * 4, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess)
        return HLBM_ERR_CUDA;
    pack_input_kernel<<<1024, 256, 0, s->stream>>>(x, s->width[0], s->cpad_in[0], npix, s->act[0]);
    if (cudaGetLastError() != cudaSuccess) return HLBM_ERR_CUDA;
    for (int l = 0; l < s->L; l++) {
        const bool last = l == s->L - 1;
        const ConvArgs a{s->act[l], s->Wb[l], s->p + s->boff[l], s->width[l + 1], s->act[l + 1],
                         (keep_z || last) ? s->z[l] : nullptr, nullptr, npix, s->H, s->W, last ? 0 : 1, 0};
        if (launch_conv(s->cpad_in[l], s->cpad_out[l], a, s->stream) != cudaSuccess) return HLBM_ERR_CUDA;
    }
    residual_loss_kernel<<<1024, 256, 0, s->stream>>>(s->xin, s->z[s->L - 1], s->cpad_out[s->L - 1], nullptr,
                                                      s->width[0], npix, s->y, nullptr, nullptr);
    if (cudaGetLastError() != cudaSuccess) return HLBM_ERR_CUDA;
    if (y && cudaMemcpyAsync(y, s->y, (size_t)npix * s->width[0] * 4, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess)
        return HLBM_ERR_CUDA;
    s->last_batch = keep_z ? B : 0;
    return HLBM_OK;
}

int hlbm_sur_forward(hlbm_sur *s, const float *x, float *y, int B)
{
    nvtxRangePushA("hlbm_sur_forward");
    const int rc = sur_run(s, x, y, B, true);
    nvtxRangePop();
    return rc;
}

// Inference only: the hidden layers' pre-activations are not stored.
int hlbm_sur_predict(hlbm_sur *s, const float *x, float *y, int B)
{
    nvtxRangePushA("hlbm_sur_predict");
    const int rc = sur_run(s, x, y, B, false);
    nvtxRangePop();
    return rc;
}

// After hlbm_sur_forward on the same batch: loss = mean((y - target)^2)
// (target FP32 NHWC [B, H, W, C0] on the device) and the gradient of every
// parameter into the gradient buffer.
// The backward pass after hlbm_sur_forward: dL/dy = 2 (y - target) / n (+
// dy); parameter gradients replace the stored ones, or are added to them
// with accumulate; dx (if non-NULL) receives dL/dx.
static int sur_backward(hlbm_sur *s, const float *target, const float *dy, int accumulate, float *dx,
                        double *loss_out)
{
    if (!s || !target || s->last_batch < 1) return HLBM_ERR_ARG;
    const int B = s->last_batch, npix = B * s->H * s->W;
    const int L = s->L;
    float *dzf[2] = {s->dz, s->dz2};
    int cur = 0;
    if ((!accumulate && cudaMemsetAsync(s->g, 0, s->nparam * 4, s->stream) != cudaSuccess) ||
        cudaMemsetAsync(s->loss, 0, sizeof(double), s->stream) != cudaSuccess ||
        cudaMemsetAsync(dzf[cur], 0, (size_t)npix * s->cpad_out[L - 1] * 4, s->stream) != cudaSuccess)
        return HLBM_ERR_CUDA;
    residual_loss_kernel<<<1024, 256, 0, s->stream>>>(s->xin, s->z[L - 1], s->cpad_out[L - 1], target, s->width[0],
                                                      npix, s->y, dzf[cur], s->loss);
    if (cudaGetLastError() != cudaSuccess) return HLBM_ERR_CUDA;
    if (dy) {
        add_upstream_kernel<<<1024, 256, 0, s->stream>>>(dzf[cur], s->cpad_out[L - 1], dy, s->width[0], npix);
        if (cudaGetLastError() != cudaSuccess) return HLBM_ERR_CUDA;
    }
    if (dx) {
        // the residual's identity: dL/dx starts as dL/dy
        gather_grad_kernel<<<1024, 256, 0, s->stream>>>(dzf[cur], s->cpad_out[L - 1], s->width[0], npix, 0, dx);
        if (cudaGetLastError() != cudaSuccess) return HLBM_ERR_CUDA;
    }
    // BF16 copy of the top gradient for the tensor-core input-gradient pass
    to_bf16_kernel<<<1024, 256, 0, s->stream>>>(dzf[cur], (long long)npix * s->cpad_out[L - 1], s->gbuf[0]);
    if (cudaGetLastError() != cudaSuccess) return HLBM_ERR_CUDA;
    int gb = 0;
    for (int l = L - 1; l >= 0; l--) {
        // weight gradient on the tensor cores from the BF16 copy of dz_l
        if (launch_wgrad(s->cpad_in[l], s->cpad_out[l], s->act[l], s->gbuf[gb], dzf[cur], s->width[l], s->width[l + 1],
                         npix, s->H, s->W, s->g + s->woff[l], s->g + s->boff[l], s->stream) != cudaSuccess)
            return HLBM_ERR_CUDA;
        if (l == 0) {
            if (dx) {
                // the network's part of dL/dx: W_0^T * dz_0, the transposed
                // convolution without GELU' (the input has no activation)
                const ConvArgs a{s->gbuf[gb], s->Wd[0], nullptr, 0, s->gbuf[gb ^ 1], dzf[cur ^ 1], nullptr, npix,
                                 s->H, s->W, 2, 1};
                if (launch_conv(s->cpad_out[0], s->cpad_in[0], a, s->stream) != cudaSuccess) return HLBM_ERR_CUDA;
                gather_grad_kernel<<<1024, 256, 0, s->stream>>>(dzf[cur ^ 1], s->cpad_in[0], s->width[0], npix, 1, dx);
                if (cudaGetLastError() != cudaSuccess) return HLBM_ERR_CUDA;
            }
            break;
        }
        // dz_{l-1} = (W_l^T * dz_l) . GELU'(z_{l-1}): the transposed
        // convolution on the tensor cores (dz read at p - offset(tap)),
        // GELU' in the epilogue, FP32 and BF16 results
        const ConvArgs a{s->gbuf[gb], s->Wd[l], nullptr, 0, s->gbuf[gb ^ 1], dzf[cur ^ 1], s->z[l - 1], npix, s->H,
                         s->W, 2, 1};
        if (launch_conv(s->cpad_out[l], s->cpad_in[l], a, s->stream) != cudaSuccess) return HLBM_ERR_CUDA;
        cur ^= 1;
        gb ^= 1;
    }
    if (loss_out) {
        double l2 = 0.0;
        if (cudaMemcpyAsync(&l2, s->loss, sizeof(double), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
            cudaStreamSynchronize(s->stream) != cudaSuccess)
            return HLBM_ERR_CUDA;
        *loss_out = l2 / ((double)npix * s->width[0]);
    }
    return HLBM_OK;
}

int hlbm_sur_backward(hlbm_sur *s, const float *target, double *loss_out)
{
    return sur_backward(s, target, nullptr, 0, nullptr, loss_out);
}

int hlbm_sur_backward_ex(hlbm_sur *s, const float *target, const float *dy, int accumulate, float *dx,
                         double *loss_out)
{
    return sur_backward(s, target, dy, accumulate, dx, loss_out);
}

// One Adam step (Kingma & Ba 2015) on all parameters from the gradient
// buffer; the BF16 copies are refreshed.
int hlbm_sur_adam(hlbm_sur *s, float lr, float beta1, float beta2, float eps)
{
    if (!s || !(lr > 0.0f)) return HLBM_ERR_ARG;
    s->adam_t++;
    const float c1 = 1.0f - powf(beta1, (float)s->adam_t), c2 = 1.0f - powf(beta2, (float)s->adam_t);
    adam_kernel<<<1024, 256, 0, s->stream>>>(s->p, s->g, s->m, s->v, (long long)s->nparam, lr, beta1, beta2, eps, c1, c2);
    if (cudaGetLastError() != cudaSuccess) return HLBM_ERR_CUDA;
    return sur_arrange(s);
}

int hlbm_sur_synchronize(hlbm_sur *s)
{
    if (!s) return HLBM_ERR_ARG;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return HLBM_ERR_CUDA;
    int st = 0;
    if (cudaMemcpyFromSymbol(&st, g_tc_status, sizeof(int)) != cudaSuccess) return HLBM_ERR_CUDA;
    return st == 0 ? HLBM_OK : (st == 1 ? HLBM_ERR_TIMEOUT : HLBM_ERR_CUDA);
}


}  // extern "C"
