// hlbm_tma.cuh -- persistent FP32 fused step with TMA double buffering.
//
// Same arithmetic as fused_step_kernel (hlbm_device.cuh), restructured for
// GB300: a persistent grid of CTAs walks the tiles; for every interior tile
// one elected thread issues three cp.async.bulk.tensor loads (the 9 F planes
// on tile + 2, s on tile + 3, a1 on tile + 1) into one of two shared-memory
// buffers, so the loads of tile k+1 run while tile k is computed.  Tiles
// that touch the domain edge are filled by ordinary loads through the
// boundary index map into the same layout.
//
// Shared layout of one buffer (floats), rows of BX = TX + 8 elements that
// start at x0 - 4 (a 16-byte-aligned x coordinate for TMA):
//   bF [9][TY + 4][BX]  rows y0-2 .. y0+TY+1   (R2 region at column 2)
//   bS [TY + 6][BX]     rows y0-3 .. y0+TY+2   (R3 region at column 1)
//   bA [3][TY + 2][BX]  rows y0-1 .. y0+TY     (R1 region at column 3)
//
// Every wait on an mbarrier is bounded: after about a second the kernel
// records an error in *err, stops issuing work and returns; the host turns
// the flag into HLBM_ERR_TIMEOUT.
#pragma once

#include <cuda.h>

#include "hlbm_device.cuh"

namespace hlbm {

template <int TX, int TY>
struct TmaGeom {
    static constexpr int BX = TX + 8;
    static constexpr int F_ROWS = TY + 4, S_ROWS = TY + 6, A_ROWS = TY + 2;
    static constexpr int F_ELEMS = 9 * F_ROWS * BX;
    static constexpr int S_ELEMS = S_ROWS * BX;
    static constexpr int A_ELEMS = 3 * A_ROWS * BX;
    static constexpr int round128(int bytes) { return (bytes + 127) / 128 * 128; }
    static constexpr int F_BYTES = F_ELEMS * 4, S_BYTES = S_ELEMS * 4, A_BYTES = A_ELEMS * 4;
    static constexpr int F_OFF = 0, S_OFF = round128(F_BYTES), A_OFF = S_OFF + round128(S_BYTES);
    static constexpr int BUF_BYTES = A_OFF + round128(A_BYTES);
    static constexpr int TX_BYTES = F_BYTES + S_BYTES + A_BYTES;  // bytes one tile's TMA delivers
    // level-n macros on tile + 2 and level-(n+1) values on tile + 1
    static constexpr int R2X = TX + 4, N2 = R2X * (TY + 4);
    static constexpr int R1X = TX + 2, N1 = R1X * (TY + 2);
    static constexpr int M_OFF = 2 * BUF_BYTES;
    static constexpr int N_OFF = M_OFF + round128(4 * N2 * 4);
    static constexpr int BAR_OFF = N_OFF + round128(5 * N1 * 4);
    static constexpr size_t smem_bytes = BAR_OFF + 64;  // 2 barriers + abort flag
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity; false after ~1 s (2^31 cycles).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > (1ll << 31)) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

struct TmaMaps {
    CUtensorMap f, s, a;
};

template <int TX, int TY, int NT>
__global__ void __launch_bounds__(NT)
fused_step_tma_kernel(const __grid_constant__ TmaMaps maps, const float *__restrict__ in, float *__restrict__ out,
                      const KParams kp, int *err)
{
    using G = TmaGeom<TX, TY>;
    constexpr int BX = G::BX, R2X = G::R2X, N2 = G::N2, R1X = G::R1X, N1 = G::N1;
    constexpr int FR = G::F_ROWS, SR = G::S_ROWS, AR = G::A_ROWS;
    extern __shared__ __align__(128) unsigned char smem[];
    float *mRho = reinterpret_cast<float *>(smem + G::M_OFF), *mUx = mRho + N2, *mUy = mUx + N2, *mTh = mUy + N2;
    float *nRho = reinterpret_cast<float *>(smem + G::N_OFF), *nUx = nRho + N1, *nUy = nUx + N1, *nTh = nUy + N1,
          *nS = nTh + N1;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + G::BAR_OFF);
    int &s_abort = *reinterpret_cast<int *>(smem + G::BAR_OFF + 32);

    Consts<float> cs;
    cs.load(kp);
    const Side<float> side{kp};
    const float third = 1.0f / 3.0f;
    const int pitch = kp.pitch;
    const long long P = kp.plane;
    const int tiles_x = (kp.nx + TX - 1) / TX, tiles_y = (kp.ny + TY - 1) / TY;
    const int ntiles = tiles_x * tiles_y;

    auto is_interior = [&](int t) {
        const int x0 = (t % tiles_x) * TX, y0 = (t / tiles_x) * TY;
        return x0 >= 4 && y0 >= 3 && x0 + TX + 4 <= kp.nx && y0 + TY + 3 <= kp.ny;
    };
    auto issue = [&](int t, int b) {
        const int x0 = (t % tiles_x) * TX, y0 = (t / tiles_x) * TY;
        unsigned char *buf = smem + b * G::BUF_BYTES;
        mbar_expect_tx(&bar[b], G::TX_BYTES);
        tma_load_3d(buf + G::F_OFF, &maps.f, x0 - 4, y0 - 2, 0, &bar[b]);
        tma_load_3d(buf + G::S_OFF, &maps.s, x0 - 4, y0 - 3, P_S, &bar[b]);
        tma_load_3d(buf + G::A_OFF, &maps.a, x0 - 4, y0 - 1, P_AXX, &bar[b]);
    };

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    __syncthreads();

    uint32_t phase_bits = 0;  // parity of the next completion of bar[0], bar[1]
    uint32_t inflight = 0;    // thread 0: buffers with a load in flight
    int b = 0;
    int t = blockIdx.x;
    if (t < ntiles && threadIdx.x == 0 && is_interior(t)) { issue(t, 0); inflight |= 1u; }

    for (; t < ntiles; t += gridDim.x) {
        const int x0 = (t % tiles_x) * TX, y0 = (t / tiles_x) * TY;
        const bool interior = is_interior(t);
        const int tn = t + gridDim.x;
        if (threadIdx.x == 0 && tn < ntiles && is_interior(tn)) {
            fence_proxy_async_smem();  // earlier generic accesses to the other buffer are done
            issue(tn, b ^ 1);
            inflight |= 1u << (b ^ 1);
        }
        float *bF = reinterpret_cast<float *>(smem + b * G::BUF_BYTES + G::F_OFF);
        float *bS = reinterpret_cast<float *>(smem + b * G::BUF_BYTES + G::S_OFF);
        float *bA = reinterpret_cast<float *>(smem + b * G::BUF_BYTES + G::A_OFF);
        if (interior) {
            if (!mbar_wait_bounded(&bar[b], (phase_bits >> b) & 1u)) {
                atomicExch(err, 1);
                s_abort = 1;
            } else {
                inflight &= ~(1u << b);
            }
            phase_bits ^= 1u << b;
        } else {
            // ordinary loads through the boundary index map, same layout
            for (int c = threadIdx.x; c < FR * BX; c += NT) {
                const int r = c / BX, col = c - r * BX;
                const int o = locate(x0 - 4 + col, y0 - 2 + r, kp, pitch);
#pragma unroll
                for (int i = 0; i < 9; i++) bF[i * FR * BX + c] = o >= 0 ? __ldg(in + i * P + o) : side.F(-o - 1, i);
            }
            for (int c = threadIdx.x; c < SR * BX; c += NT) {
                const int r = c / BX, col = c - r * BX;
                const int o = locate(x0 - 4 + col, y0 - 3 + r, kp, pitch);
                bS[c] = o >= 0 ? __ldg(in + P_S * P + o) : side.s_(-o - 1);
            }
            for (int c = threadIdx.x; c < AR * BX; c += NT) {
                const int r = c / BX, col = c - r * BX;
                const int o = locate(x0 - 4 + col, y0 - 1 + r, kp, pitch);
#pragma unroll
                for (int i = 0; i < 3; i++) bA[i * AR * BX + c] = o >= 0 ? __ldg(in + (P_AXX + i) * P + o) : 0.0f;
            }
        }
        __syncthreads();
        if (s_abort) break;

        // phase 1: level-n rho, u, theta on tile + 2 (R2 cell (lx, ly) is at
        // F-buffer row ly, column lx + 2, and s-buffer row ly + 1, column lx + 2)
        for (int c = threadIdx.x; c < N2; c += NT) {
            const int ly = c / R2X, lx = c - ly * R2X;
            float rho, ux, uy, th;
            bool dirichlet = false;
            int sd = 0;
            if (!interior) {
                const int o = locate(x0 - 2 + lx, y0 - 2 + ly, kp, pitch);
                if (o < 0) { dirichlet = true; sd = -o - 1; }
            }
            if (!dirichlet) {
                const int kb = ly * BX + lx + 2;
                float f[9];
#pragma unroll
                for (int i = 0; i < 9; i++) f[i] = bF[i * FR * BX + kb];
                float jx, jy;
                moments(f, rho, jx, jy);
                const float ir = fdiv(1.0f, rho);
                ux = jx * ir; uy = jy * ir;
                th = cs.theta(rho, bS[(ly + 1) * BX + lx + 2]);
            } else {
                rho = side.rho(sd); ux = side.ux(sd); uy = side.uy(sd); th = side.th(sd);
            }
            mRho[c] = rho; mUx[c] = ux; mUy[c] = uy; mTh[c] = th;
        }
        __syncthreads();

        // phase 2: level n+1 on tile + 1
        for (int c = threadIdx.x; c < N1; c += NT) {
            const int ly = c / R1X, lx = c - ly * R1X;
            const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
            if (!interior) {
                int sd = 0;
                const int kind = classify_r1(gx, gy, kp, &sd);
                if (kind == 1) {
                    nRho[c] = side.rho(sd); nUx[c] = side.ux(sd); nUy[c] = side.uy(sd);
                    nTh[c] = side.th(sd); nS[c] = side.s_(sd);
                    continue;
                }
                if (kind == 2) continue;
            }
            const int k2 = (ly + 1) * R2X + lx + 1;
            const float rho0 = mRho[k2], th0 = mTh[k2], ux0 = mUx[k2], uy0 = mUy[k2];
            const float dxux = 0.5f * (mUx[k2 + 1] - mUx[k2 - 1]);
            const float dyux = 0.5f * (mUx[k2 + R2X] - mUx[k2 - R2X]);
            const float dxuy = 0.5f * (mUy[k2 + 1] - mUy[k2 - 1]);
            const float dyuy = 0.5f * (mUy[k2 + R2X] - mUy[k2 - R2X]);
            const float lap = (mTh[k2 + 1] + mTh[k2 - 1]) + (mTh[k2 + R2X] + mTh[k2 - R2X]) - 4.0f * th0;
            const int k3 = (ly + 2) * BX + lx + 3;  // s of this cell in the buffer
            const float s0 = bS[k3];
            const float adv = muscl_adv(ux0, bS[k3 - 2], bS[k3 - 1], s0, bS[k3 + 1], bS[k3 + 2])
                            + muscl_adv(uy0, bS[k3 - 2 * BX], bS[k3 - BX], s0, bS[k3 + BX], bS[k3 + 2 * BX]);
            const float rt = rho0 * th0;
            const float p0 = rt * third;
            float phi;
            if (kp.phi_mode == 0) {
                const int ka = ly * BX + lx + 3;
                const float axx = bA[ka], axy = bA[AR * BX + ka], ayy = bA[2 * AR * BX + ka];
                phi = -fdiv(cs.two_mu, cs.two_mu + p0) * (axx * dxux + axy * (dyux + dxuy) + ayy * dyuy);
            } else {
                const float d1 = dxux - dyuy, d2 = dyux + dxuy;
                phi = cs.mu * (d1 * d1 + d2 * d2);
            }
            const float s1 = s0 - adv + fdiv(cs.lam * lap + phi, rt);
            const int kb = (ly + 1) * BX + lx + 3;  // this cell in the F buffer
            float f[9];
#pragma unroll
            for (int i = 0; i < 9; i++) f[i] = bF[i * FR * BX + kb - cxi(i) - cyi(i) * BX];
            float rho1, jx, jy;
            moments(f, rho1, jx, jy);
            const float ir = fdiv(1.0f, rho1);
            nRho[c] = rho1; nUx[c] = jx * ir; nUy[c] = jy * ir;
            nTh[c] = cs.theta(rho1, s1);
            nS[c] = s1;
        }
        __syncthreads();

        if (!interior) {
            for (int c = threadIdx.x; c < N1; c += NT) {
                const int ly = c / R1X, lx = c - ly * R1X;
                const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
                int sd = 0;
                if (classify_r1(gx, gy, kp, &sd) != 2) continue;
                int sx = gx, sy = gy;
                if ((gx < 0 || gx >= kp.nx) && kp.bc[gx < 0 ? 0 : 1] == BC_ZEROGRAD) sx = gx < 0 ? 0 : kp.nx - 1;
                if ((gy < 0 || gy >= kp.ny) && kp.bc[gy < 0 ? 2 : 3] == BC_ZEROGRAD) sy = gy < 0 ? 0 : kp.ny - 1;
                const int src = (sy - (y0 - 1)) * R1X + (sx - (x0 - 1));
                nRho[c] = nRho[src]; nUx[c] = nUx[src]; nUy[c] = nUy[src]; nTh[c] = nTh[src]; nS[c] = nS[src];
            }
            __syncthreads();
        }

        // phase 3: psi, f^eq, a1 and the collision on the tile
        for (int c = threadIdx.x; c < TX * TY; c += NT) {
            const int ly = c / TX, lx = c - ly * TX;
            const int gx = x0 + lx, gy = y0 + ly;
            if (gx >= kp.nx || gy >= kp.ny) continue;
            const int k = (ly + 1) * R1X + lx + 1;
            const float rho = nRho[k], ux = nUx[k], uy = nUy[k], th = nTh[k];
            const float uxm = nUx[k - 1], uxp = nUx[k + 1], uym = nUy[k - R1X], uyp = nUy[k + R1X];
            const float dxux = 0.5f * (uxp - uxm);
            const float dyux = 0.5f * (nUx[k + R1X] - nUx[k - R1X]);
            const float dxuy = 0.5f * (nUy[k + 1] - nUy[k - 1]);
            const float dyuy = 0.5f * (uyp - uym);
            const float p = rho * th * third;
            const float gxc = gamma_defect(rho, ux, th), gyc = gamma_defect(rho, uy, th);
            const float gxm = gamma_defect(nRho[k - 1], uxm, nTh[k - 1]);
            const float gxp = gamma_defect(nRho[k + 1], uxp, nTh[k + 1]);
            const float gym = gamma_defect(nRho[k - R1X], uym, nTh[k - R1X]);
            const float gyp = gamma_defect(nRho[k + R1X], uyp, nTh[k + R1X]);
            const bool cen = kp.e1_centred != 0;
            const float e1xx = (ux > 0.0f && !cen) ? gxc - gxm : ((ux < 0.0f && !cen) ? gxp - gxc : 0.5f * (gxp - gxm));
            const float e1yy = (uy > 0.0f && !cen) ? gyc - gym : ((uy < 0.0f && !cen) ? gyp - gyc : 0.5f * (gyp - gym));
            const float e2 = p * cs.two_m_gamma * (dxux + dyuy);
            const float ex = e1xx + e2, ey = e1yy + e2;
            const float cfd = -(cs.mu + 0.5f * p);
            const float fdxx = cfd * (dxux - dyuy), fdxy = cfd * (dyux + dxuy);
            float axx, axy, ayy;
            if (kp.sigma_nonzero) {
                const int kb = (ly + 2) * BX + lx + 4;
                float f[9];
#pragma unroll
                for (int i = 0; i < 9; i++) f[i] = bF[i * FR * BX + kb - cxi(i) - cyi(i) * BX];
                const float diag = (f[5] + f[6]) + (f[7] + f[8]);
                const float mxx = (f[1] + f[3]) + diag, myy = (f[2] + f[4]) + diag;
                const float mxy = (f[5] - f[6]) + (f[7] - f[8]);
                const float prxx = mxx - rho * ux * ux - p + 0.5f * ex;
                const float pryy = myy - rho * uy * uy - p + 0.5f * ey;
                const float prxy = mxy - rho * ux * uy;
                axx = cs.sigma * prxx + cs.one_m_sigma * fdxx;
                ayy = cs.sigma * pryy - cs.one_m_sigma * fdxx;
                axy = cs.sigma * prxy + cs.one_m_sigma * fdxy;
            } else {
                axx = fdxx; ayy = -fdxx; axy = fdxy;
            }
            const float omega = fdiv(cs.two_mu - p, cs.two_mu + p);
            float f[9];
            build_populations(rho, ux, uy, th, axx, axy, ayy, ex, ey, omega, f);
            const int o = gy * pitch + gx;
#pragma unroll
            for (int i = 0; i < 9; i++) out[i * P + o] = f[i];
            out[P_S * P + o] = nS[k];
            out[P_AXX * P + o] = axx;
            out[P_AXY * P + o] = axy;
            out[P_AYY * P + o] = ayy;
        }
        __syncthreads();  // every thread is done with buffer b and the m/n arrays
        b ^= 1;
    }

    if (s_abort) {
        // a load never arrived: wait (bounded) for the copies this CTA still
        // has in flight before leaving, so no TMA writes after exit
        if (threadIdx.x == 0) {
            for (int q = 0; q < 2; q++)
                if (inflight & (1u << q)) mbar_wait_bounded(&bar[q], ((phase_bits >> q) & 1u) ^ (q == b ? 1u : 0u));
        }
    }
}

}  // namespace hlbm
