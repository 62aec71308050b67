// hlbm_device.cuh -- sm_103a kernels of the hybrid lattice Boltzmann step of
// Renard, Feng, Boussuge and Sagaut (arXiv 2002.03644), Algorithm 1.
//
// State layout in HBM (one copy per ping-pong side): 13 planes of
// [ny][pitch] elements of T (float or double), in the order
//   0..8  post-collision populations F_i of the current level (eq. streamalgo,
//         before propagation), D2Q9 order c_x = {0,1,0,-1,0,1,-1,-1,1},
//         c_y = {0,0,1,0,-1,1,1,-1,-1} (Sec. 2.1)
//   9     entropy s (eq. Entropie expression)
//   10-12 a1_xx, a1_xy, a1_yy (eq. a1sigalgo)
// pitch is nx rounded up to 32 elements so that every row starts on a
// 128-byte boundary.  rho and u of a level are never stored: they are the
// moments of F (collision invariants, eqs. rhoalgo, ualgo); theta follows
// from s and rho.
//
// One launch of fused_step_kernel performs Algorithm 1 steps 5-11 for a tile
// of TX x TY cells:
//   phase 0: s(n) on the tile plus a 3-cell halo -> shared memory
//   phase 1: rho, u, theta at level n on tile + 2 (local moments of F(n))
//   phase 2: on tile + 1: the entropy update (step 7, MUSCL / Van Albada,
//            Fourier, viscous heating), pull-streaming and moments (steps
//            5-6), theta (step 8), closure defect Gamma (Sec. 3.2)
//   phase 3: on the tile: E1 (upwind) and E2 (centred) -> psi (step 9),
//            f^eq (step 10), a1 = sigma a1^PR + (1 - sigma) a1^FD with the
//            recurrence (step 11), and the regularised collision of the next
//            step, written as F(n+1), s(n+1), a1(n+1).
// The populations are rebuilt from their nine raw moments with a 1-D x 1-D
// inverse transform (the D2Q9 lattice is the tensor product of two D1Q3
// lattices); the equilibrium is the product of two D1Q3 equilibria, which is
// the same function as the fourth-order Hermite form restricted to the
// D2Q9 basis (Sec. 2.3).
//
// Boundaries are index maps applied wherever a coordinate leaves the domain:
// periodic sides wrap, zero-gradient sides clamp to the nearest interior
// cell, Dirichlet sides return a fixed state.  A value of level n+1 outside
// the domain is the value at the mapped cell; for clamped sides it is copied
// from the tile's own edge after phase 2.  A Dirichlet y side wins at a
// corner, then a Dirichlet x side.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hlbm {

constexpr int NPLANE = 13;
constexpr int P_S = 9, P_AXX = 10, P_AXY = 11, P_AYY = 12;
enum { BC_PERIODIC = 0, BC_ZEROGRAD = 1, BC_DIRICHLET = 2 };

struct KParams {
    int nx, ny, pitch;
    long long plane;           // elements per plane = pitch * ny
    int bc[4];                 // x-, x+, y-, y+
    int phi_mode;              // 0 regularised, 1 finite differences
    int sigma_nonzero;
    double mu, sigma, lambda;  // lambda = mu c_p / Pr
    double gm1, inv_cv, cv, two_minus_gamma, gamma;
    // Dirichlet side constants: macros, entropy, closure defect, populations
    double d_rho[4], d_ux[4], d_uy[4], d_th[4], d_s[4], d_gx[4], d_gy[4];
    double d_F[4][9];
};

__device__ __forceinline__ constexpr int cxi(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0); }
__device__ __forceinline__ constexpr int cyi(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0); }

__device__ __forceinline__ int wrapi(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

// Offset gy * pitch + gx of the cell that (gx, gy) maps to, or -(side + 1)
// when it falls on a Dirichlet side.
__device__ __forceinline__ int locate(int gx, int gy, const KParams &kp, int pitch)
{
    if (gy < 0 || gy >= kp.ny) {
        const int s = gy < 0 ? 2 : 3;
        const int b = kp.bc[s];
        if (b == BC_DIRICHLET) return -(s + 1);
        gy = (b == BC_PERIODIC) ? wrapi(gy, kp.ny) : (gy < 0 ? 0 : kp.ny - 1);
    }
    if (gx < 0 || gx >= kp.nx) {
        const int s = gx < 0 ? 0 : 1;
        const int b = kp.bc[s];
        if (b == BC_DIRICHLET) return -(s + 1);
        gx = (b == BC_PERIODIC) ? wrapi(gx, kp.nx) : (gx < 0 ? 0 : kp.nx - 1);
    }
    return gy * pitch + gx;
}

// ---- precision-dependent helpers -------------------------------------------
template <typename T> struct Consts;

template <> struct Consts<float> {
    float gm1, s2exp, mu, two_mu, lam, sigma, one_m_sigma, two_m_gamma;
    __device__ void load(const KParams &kp)
    {
        gm1 = (float)kp.gm1;
        s2exp = (float)(kp.inv_cv * 1.4426950408889634);  // 1 / (c_v ln 2)
        mu = (float)kp.mu; two_mu = 2.0f * mu; lam = (float)kp.lambda;
        sigma = (float)kp.sigma; one_m_sigma = (float)(1.0 - kp.sigma);
        two_m_gamma = (float)kp.two_minus_gamma;
    }
    // theta = rho^(gamma-1) exp(s / c_v) = 2^((gamma-1) log2 rho + s / (c_v ln 2))
    __device__ __forceinline__ float theta(float rho, float s) const { return exp2f(fmaf(gm1, __log2f(rho), s * s2exp)); }
};

template <> struct Consts<double> {
    double gm1, s2exp, mu, two_mu, lam, sigma, one_m_sigma, two_m_gamma;
    __device__ void load(const KParams &kp)
    {
        gm1 = kp.gm1; s2exp = kp.inv_cv; mu = kp.mu; two_mu = 2.0 * kp.mu; lam = kp.lambda;
        sigma = kp.sigma; one_m_sigma = 1.0 - kp.sigma; two_m_gamma = kp.two_minus_gamma;
    }
    __device__ __forceinline__ double theta(double rho, double s) const { return exp(fma(gm1, log(rho), s * s2exp)); }
};

// rho and momentum of nine populations.  The momentum sums pair mirror
// directions so that a mirror-symmetric set gives exactly zero.
template <typename T>
__device__ __forceinline__ void moments(const T f[9], T &rho, T &jx, T &jy)
{
    rho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    jy = (f[2] - f[4]) + (f[5] - f[8]) + (f[6] - f[7]);
}

// Van Albada limited slope from the two one-sided differences; zero at an
// extremum (a b <= 0).
template <typename T>
__device__ __forceinline__ T va_slope(T a, T b)
{
    const T ab = a * b;
    return ab > T(0) ? ab * (a + b) / (a * a + b * b) : T(0);
}

// u ds/dx from limited, upwinded face values (non-conservative advection of
// Sec. 3.4).  For u > 0 the term is u [(s0 + d0/2) - (sm + dm/2)]; for u < 0
// the same expression on the mirrored stencil (sm <-> sp, smm <-> spp) times
// |u|, since the limited slope is odd in its arguments.  u = 0 gives zero.
template <typename T>
__device__ __forceinline__ T muscl_adv(T u, T smm, T sm, T s0, T sp, T spp)
{
    const bool pos = u > T(0);
    const T q2 = pos ? smm : spp, q1 = pos ? sm : sp, qm = pos ? sp : sm;
    const T d10 = s0 - q1;
    const T dd = d10 + T(0.5) * (va_slope(d10, qm - s0) - va_slope(q1 - q2, d10));
    return fabs(u) * dd;
}

// Post-collision populations from level quantities: F = f^eq + omega f1 +
// psi / 2 (eq. streamalgo), built from raw moments R_ab = sum c_x^a c_y^b F.
//   f^eq : R_ab = rho m_a(u_x) m_b(u_y), m_0 = 1, m_1 = u, m_2 = u^2 + theta/3
//   f1   : Hermite coefficients a1_xx, a1_xy, a1_yy and, by the recurrence of
//          Sec. 3.3, a1_xxy, a1_yyx, a1_xxyy
//   psi  : Hermite coefficients E_x = E1_xx + E2, E_y = E1_yy + E2 (eq. Psialgo)
template <typename T>
__device__ __forceinline__ void build_populations(T rho, T ux, T uy, T th, T axx, T axy, T ayy,
                                                  T ex, T ey, T omega, T f[9])
{
    const T third = T(1) / T(3);
    const T t3 = th * third;
    const T mx2 = ux * ux + t3, my2 = uy * uy + t3;
    const T axxy = uy * axx + T(2) * ux * axy;
    const T ayyx = ux * ayy + T(2) * uy * axy;
    const T cth = (th - T(1)) * third;
    const T axxyy = T(2) * (ux * ayyx + uy * axxy) + (cth - ux * ux) * ayy + (cth - uy * uy) * axx
                  - T(4) * ux * uy * axy;
    const T rux = rho * ux, ruy = rho * uy;
    const T R00 = rho, R10 = rux, R01 = ruy;
    const T R20 = rho * mx2 + omega * axx + T(0.5) * ex;
    const T R02 = rho * my2 + omega * ayy + T(0.5) * ey;
    const T R11 = rux * uy + omega * axy;
    const T R21 = rho * mx2 * uy + omega * axxy;
    const T R12 = rux * my2 + omega * ayyx;
    const T R22 = rho * mx2 * my2 + omega * (axxyy + (axx + ayy) * third) + (ex + ey) * (T(0.5) * third);
    // D1Q3 inverse along x: (M0, M1, M2) -> f(0) = M0 - M2, f(+-1) = (M2 +- M1) / 2
    const T X0z = R00 - R20, X0p = T(0.5) * (R20 + R10), X0m = T(0.5) * (R20 - R10);
    const T X1z = R01 - R21, X1p = T(0.5) * (R21 + R11), X1m = T(0.5) * (R21 - R11);
    const T X2z = R02 - R22, X2p = T(0.5) * (R22 + R12), X2m = T(0.5) * (R22 - R12);
    // and along y
    f[0] = X0z - X2z;
    f[1] = X0p - X2p;
    f[3] = X0m - X2m;
    f[2] = T(0.5) * (X2z + X1z);
    f[4] = T(0.5) * (X2z - X1z);
    f[5] = T(0.5) * (X2p + X1p);
    f[8] = T(0.5) * (X2p - X1p);
    f[6] = T(0.5) * (X2m + X1m);
    f[7] = T(0.5) * (X2m - X1m);
}

// ---- the fused step ------------------------------------------------------------
template <typename T, int TX, int TY>
struct TileGeom {
    static constexpr int R3X = TX + 6, R3Y = TY + 6, N3 = R3X * R3Y;
    static constexpr int R2X = TX + 4, R2Y = TY + 4, N2 = R2X * R2Y;
    static constexpr int R1X = TX + 2, R1Y = TY + 2, N1 = R1X * R1Y;
    static constexpr size_t smem_bytes = sizeof(T) * (size_t)(N3 + 4 * N2 + 10 * N1);
};

// Classification of a tile + 1 cell for phase 2: 0 compute, 1 Dirichlet
// constant (side in *side), 2 copy from the clamped cell.
__device__ __forceinline__ int classify_r1(int gx, int gy, const KParams &kp, int *side)
{
    const bool outx = gx < 0 || gx >= kp.nx, outy = gy < 0 || gy >= kp.ny;
    if (!outx && !outy) return 0;
    const int o = locate(gx, gy, kp, kp.pitch);
    if (o < 0) { *side = -o - 1; return 1; }
    const bool cx = outx && kp.bc[gx < 0 ? 0 : 1] == BC_ZEROGRAD;
    const bool cy = outy && kp.bc[gy < 0 ? 2 : 3] == BC_ZEROGRAD;
    return (cx || cy) ? 2 : 0;
}

template <typename T, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT)
fused_step_kernel(const T *__restrict__ in, T *__restrict__ out, const KParams kp)
{
    using Geo = TileGeom<T, TX, TY>;
    constexpr int R3X = Geo::R3X, N3 = Geo::N3, R2X = Geo::R2X, N2 = Geo::N2, R1X = Geo::R1X, N1 = Geo::N1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sS = reinterpret_cast<T *>(smem_raw);
    T *mRho = sS + N3, *mUx = mRho + N2, *mUy = mUx + N2, *mTh = mUy + N2;
    T *nRho = mTh + N2, *nUx = nRho + N1, *nUy = nUx + N1, *nTh = nUy + N1, *nS = nTh + N1;
    T *nGx = nS + N1, *nGy = nGx + N1, *nMxx = nGy + N1, *nMxy = nMxx + N1, *nMyy = nMxy + N1;

    Consts<T> cs;
    cs.load(kp);
    const T third = T(1) / T(3);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int pitch = kp.pitch;
    const long long P = kp.plane;
    const bool interior = x0 >= 3 && y0 >= 3 && x0 + TX + 3 <= kp.nx && y0 + TY + 3 <= kp.ny;

    // phase 0: s(n) on tile + 3
    for (int c = threadIdx.x; c < N3; c += NT) {
        const int ly = c / R3X, lx = c - ly * R3X;
        const int gx = x0 - 3 + lx, gy = y0 - 3 + ly;
        const int o = interior ? gy * pitch + gx : locate(gx, gy, kp, pitch);
        sS[c] = o >= 0 ? __ldg(in + P_S * P + o) : T(kp.d_s[-o - 1]);
    }
    __syncthreads();

    // phase 1: rho, u, theta of level n on tile + 2
    for (int c = threadIdx.x; c < N2; c += NT) {
        const int ly = c / R2X, lx = c - ly * R2X;
        const int gx = x0 - 2 + lx, gy = y0 - 2 + ly;
        const int o = interior ? gy * pitch + gx : locate(gx, gy, kp, pitch);
        T rho, ux, uy, th;
        if (o >= 0) {
            T f[9];
#pragma unroll
            for (int i = 0; i < 9; i++) f[i] = __ldg(in + i * P + o);
            T jx, jy;
            moments(f, rho, jx, jy);
            const T ir = T(1) / rho;
            ux = jx * ir; uy = jy * ir;
            th = cs.theta(rho, sS[(ly + 1) * R3X + lx + 1]);
        } else {
            const int sd = -o - 1;
            rho = T(kp.d_rho[sd]); ux = T(kp.d_ux[sd]); uy = T(kp.d_uy[sd]); th = T(kp.d_th[sd]);
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
                nRho[c] = T(kp.d_rho[sd]); nUx[c] = T(kp.d_ux[sd]); nUy[c] = T(kp.d_uy[sd]);
                nTh[c] = T(kp.d_th[sd]); nS[c] = T(kp.d_s[sd]);
                nGx[c] = T(kp.d_gx[sd]); nGy[c] = T(kp.d_gy[sd]);
                nMxx[c] = T(0); nMxy[c] = T(0); nMyy[c] = T(0);
                continue;
            }
            if (kind == 2) continue;
        }
        // step 7: entropy update from level-n fields
        const int k2 = (ly + 1) * R2X + lx + 1;
        const T rho0 = mRho[k2], th0 = mTh[k2], ux0 = mUx[k2], uy0 = mUy[k2];
        const T dxux = T(0.5) * (mUx[k2 + 1] - mUx[k2 - 1]);
        const T dyux = T(0.5) * (mUx[k2 + R2X] - mUx[k2 - R2X]);
        const T dxuy = T(0.5) * (mUy[k2 + 1] - mUy[k2 - 1]);
        const T dyuy = T(0.5) * (mUy[k2 + R2X] - mUy[k2 - R2X]);
        const T lap = (mTh[k2 + 1] + mTh[k2 - 1]) + (mTh[k2 + R2X] + mTh[k2 - R2X]) - T(4) * th0;
        const int k3 = (ly + 2) * R3X + lx + 2;
        const T s0 = sS[k3];
        const T adv = muscl_adv(ux0, sS[k3 - 2], sS[k3 - 1], s0, sS[k3 + 1], sS[k3 + 2])
                    + muscl_adv(uy0, sS[k3 - 2 * R3X], sS[k3 - R3X], s0, sS[k3 + R3X], sS[k3 + 2 * R3X]);
        const T rt = rho0 * th0;
        const T p0 = rt * third;
        T phi;
        if (kp.phi_mode == 0) {
            const int o = interior ? gy * pitch + gx : locate(gx, gy, kp, pitch);
            T axx = T(0), axy = T(0), ayy = T(0);
            if (o >= 0) {
                axx = __ldg(in + P_AXX * P + o); axy = __ldg(in + P_AXY * P + o); ayy = __ldg(in + P_AYY * P + o);
            }
            phi = -(cs.two_mu / (cs.two_mu + p0)) * (axx * dxux + axy * (dyux + dxuy) + ayy * dyuy);
        } else {
            const T d1 = dxux - dyuy, d2 = dyux + dxuy;
            phi = cs.mu * (d1 * d1 + d2 * d2);
        }
        const T s1 = s0 - adv + (cs.lam * lap + phi) / rt;
        // steps 5-6: pull the post-collision populations, moments
        T f[9];
        if (interior) {
            const int o = gy * pitch + gx;
#pragma unroll
            for (int i = 0; i < 9; i++) f[i] = __ldg(in + i * P + (o - cyi(i) * pitch - cxi(i)));
        } else {
#pragma unroll
            for (int i = 0; i < 9; i++) {
                const int o = locate(gx - cxi(i), gy - cyi(i), kp, pitch);
                f[i] = o >= 0 ? __ldg(in + i * P + o) : T(kp.d_F[-o - 1][i]);
            }
        }
        T rho1, jx, jy;
        moments(f, rho1, jx, jy);
        const T ir = T(1) / rho1;
        const T ux1 = jx * ir, uy1 = jy * ir;
        const T th1 = cs.theta(rho1, s1);  // step 8
        nRho[c] = rho1; nUx[c] = ux1; nUy[c] = uy1; nTh[c] = th1; nS[c] = s1;
        nGx[c] = rho1 * ux1 * (T(1) - th1 - ux1 * ux1);
        nGy[c] = rho1 * uy1 * (T(1) - th1 - uy1 * uy1);
        if (kp.sigma_nonzero) {
            const T diag = (f[5] + f[6]) + (f[7] + f[8]);
            nMxx[c] = (f[1] + f[3]) + diag;
            nMyy[c] = (f[2] + f[4]) + diag;
            nMxy[c] = (f[5] - f[6]) + (f[7] - f[8]);
        }
    }
    __syncthreads();

    if (!interior) {
        // zero-gradient sides: level n+1 outside the domain equals the value
        // at the clamped cell of the tile's edge
        for (int c = threadIdx.x; c < N1; c += NT) {
            const int ly = c / R1X, lx = c - ly * R1X;
            const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
            int sd = 0;
            if (classify_r1(gx, gy, kp, &sd) != 2) continue;
            int sx = gx, sy = gy;
            if ((gx < 0 || gx >= kp.nx) && kp.bc[gx < 0 ? 0 : 1] == BC_ZEROGRAD) sx = gx < 0 ? 0 : kp.nx - 1;
            if ((gy < 0 || gy >= kp.ny) && kp.bc[gy < 0 ? 2 : 3] == BC_ZEROGRAD) sy = gy < 0 ? 0 : kp.ny - 1;
            const int src = (sy - (y0 - 1)) * R1X + (sx - (x0 - 1));
            nRho[c] = nRho[src]; nUx[c] = nUx[src]; nUy[c] = nUy[src]; nTh[c] = nTh[src];
            nS[c] = nS[src]; nGx[c] = nGx[src]; nGy[c] = nGy[src];
            nMxx[c] = nMxx[src]; nMxy[c] = nMxy[src]; nMyy[c] = nMyy[src];
        }
        __syncthreads();
    }

    // phase 3: steps 9-11 and the collision of the next step on the tile
    for (int c = threadIdx.x; c < TX * TY; c += NT) {
        const int ly = c / TX, lx = c - ly * TX;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= kp.nx || gy >= kp.ny) continue;
        const int k = (ly + 1) * R1X + lx + 1;
        const T rho = nRho[k], ux = nUx[k], uy = nUy[k], th = nTh[k];
        const T dxux = T(0.5) * (nUx[k + 1] - nUx[k - 1]);
        const T dyux = T(0.5) * (nUx[k + R1X] - nUx[k - R1X]);
        const T dxuy = T(0.5) * (nUy[k + 1] - nUy[k - 1]);
        const T dyuy = T(0.5) * (nUy[k + R1X] - nUy[k - R1X]);
        const T p = rho * th * third;
        // E1: upwind difference of Gamma by the sign of the cell's velocity
        const T gxc = nGx[k], gyc = nGy[k];
        const T e1xx = ux > T(0) ? gxc - nGx[k - 1]
                     : (ux < T(0) ? nGx[k + 1] - gxc : T(0.5) * (nGx[k + 1] - nGx[k - 1]));
        const T e1yy = uy > T(0) ? gyc - nGy[k - R1X]
                     : (uy < T(0) ? nGy[k + R1X] - gyc : T(0.5) * (nGy[k + R1X] - nGy[k - R1X]));
        const T e2 = p * cs.two_m_gamma * (dxux + dyuy);
        const T ex = e1xx + e2, ey = e1yy + e2;
        // a1^FD = -tau_bar p (grad u + grad u^T - div u I), tau_bar p = mu + p/2
        const T cfd = -(cs.mu + T(0.5) * p);
        const T fdxx = cfd * (dxux - dyuy), fdxy = cfd * (dyux + dxuy);
        T axx, axy, ayy;
        if (kp.sigma_nonzero) {
            const T prxx = nMxx[k] - rho * ux * ux - p + T(0.5) * ex;
            const T pryy = nMyy[k] - rho * uy * uy - p + T(0.5) * ey;
            const T prxy = nMxy[k] - rho * ux * uy;
            axx = cs.sigma * prxx + cs.one_m_sigma * fdxx;
            ayy = cs.sigma * pryy - cs.one_m_sigma * fdxx;
            axy = cs.sigma * prxy + cs.one_m_sigma * fdxy;
        } else {
            axx = fdxx; ayy = -fdxx; axy = fdxy;
        }
        // 1 - 1 / tau_bar with tau = mu / p
        const T omega = (cs.two_mu - p) / (cs.two_mu + p);
        T f[9];
        build_populations(rho, ux, uy, th, axx, axy, ayy, ex, ey, omega, f);
        const int o = gy * pitch + gx;
#pragma unroll
        for (int i = 0; i < 9; i++) out[i * P + o] = f[i];
        out[P_S * P + o] = nS[k];
        out[P_AXX * P + o] = axx;
        out[P_AXY * P + o] = axy;
        out[P_AYY * P + o] = ayy;
    }
}

// ---- initialisation (Algorithm 1, steps 1-4) -----------------------------------
// In FP64 from FP64 caller fields (row-major [ny][nx]); writes the state in T.
template <typename T>
__global__ void init_kernel(const double *__restrict__ rho, const double *__restrict__ ux,
                            const double *__restrict__ uy, const double *__restrict__ th,
                            const double *__restrict__ a1, T *__restrict__ out, const KParams kp)
{
    const int gx = blockIdx.x * blockDim.x + threadIdx.x;
    const int gy = blockIdx.y * blockDim.y + threadIdx.y;
    if (gx >= kp.nx || gy >= kp.ny) return;
    const int n = kp.nx * kp.ny;
    auto at = [&](int dx, int dy, double &r, double &u, double &v, double &t) {
        const int o = locate(gx + dx, gy + dy, kp, kp.nx);
        if (o >= 0) { r = rho[o]; u = ux[o]; v = uy[o]; t = th[o]; }
        else { const int s = -o - 1; r = kp.d_rho[s]; u = kp.d_ux[s]; v = kp.d_uy[s]; t = kp.d_th[s]; }
    };
    double r0, u0, v0, t0, rxm, uxm, vxm, txm, rxp, uxp, vxp, txp, rym, uym, vym, tym, ryp, uyp, vyp, typ;
    at(0, 0, r0, u0, v0, t0);
    at(-1, 0, rxm, uxm, vxm, txm); at(1, 0, rxp, uxp, vxp, txp);
    at(0, -1, rym, uym, vym, tym); at(0, 1, ryp, uyp, vyp, typ);
    const double p = r0 * t0 / 3.0;
    const double dxux = 0.5 * (uxp - uxm), dyux = 0.5 * (uyp - uym);
    const double dxuy = 0.5 * (vxp - vxm), dyuy = 0.5 * (vyp - vym);
    double axx, axy, ayy;
    const int c = gy * kp.nx + gx;
    if (a1) {
        axx = a1[c]; axy = a1[n + c]; ayy = a1[2 * n + c];
    } else {
        const double cfd = -(kp.mu + 0.5 * p);
        axx = cfd * (dxux - dyuy); axy = cfd * (dyux + dxuy); ayy = -axx;
    }
    auto gam = [](double r, double u, double t) { return r * u * (1.0 - t - u * u); };
    const double gxc = gam(r0, u0, t0), gyc = gam(r0, v0, t0);
    const double e1xx = u0 > 0.0 ? gxc - gam(rxm, uxm, txm)
                      : (u0 < 0.0 ? gam(rxp, uxp, txp) - gxc : 0.5 * (gam(rxp, uxp, txp) - gam(rxm, uxm, txm)));
    const double e1yy = v0 > 0.0 ? gyc - gam(rym, vym, tym)
                      : (v0 < 0.0 ? gam(ryp, vyp, typ) - gyc : 0.5 * (gam(ryp, vyp, typ) - gam(rym, vym, tym)));
    const double e2 = p * kp.two_minus_gamma * (dxux + dyuy);
    const double omega = (2.0 * kp.mu - p) / (2.0 * kp.mu + p);
    double f[9];
    build_populations<double>(r0, u0, v0, t0, axx, axy, ayy, e1xx + e2, e1yy + e2, omega, f);
    const long long P = kp.plane;
    const int o = gy * kp.pitch + gx;
#pragma unroll
    for (int i = 0; i < 9; i++) out[i * P + o] = (T)f[i];
    out[P_S * P + o] = (T)(kp.cv * (log(t0) - kp.gm1 * log(r0)));
    out[P_AXX * P + o] = (T)axx;
    out[P_AXY * P + o] = (T)axy;
    out[P_AYY * P + o] = (T)ayy;
}

// ---- field extraction ----------------------------------------------------------
template <typename T>
__global__ void macros_kernel(const T *__restrict__ in, double *rho, double *ux, double *uy, double *th,
                              double *s, double *a1, double *F, const KParams kp)
{
    const int gx = blockIdx.x * blockDim.x + threadIdx.x;
    const int gy = blockIdx.y * blockDim.y + threadIdx.y;
    if (gx >= kp.nx || gy >= kp.ny) return;
    Consts<T> cs;
    cs.load(kp);
    const long long P = kp.plane;
    const int o = gy * kp.pitch + gx;
    const int c = gy * kp.nx + gx;
    const size_t n = (size_t)kp.nx * kp.ny;
    T f[9];
#pragma unroll
    for (int i = 0; i < 9; i++) f[i] = in[i * P + o];
    T r, jx, jy;
    moments(f, r, jx, jy);
    const T sv = in[P_S * P + o];
    if (rho) rho[c] = (double)r;
    if (ux) ux[c] = (double)(jx / r);
    if (uy) uy[c] = (double)(jy / r);
    if (th) th[c] = (double)cs.theta(r, sv);
    if (s) s[c] = (double)sv;
    if (a1) {
        a1[c] = (double)in[P_AXX * P + o];
        a1[n + c] = (double)in[P_AXY * P + o];
        a1[2 * n + c] = (double)in[P_AYY * P + o];
    }
    if (F) {
#pragma unroll
        for (int i = 0; i < 9; i++) F[i * n + c] = (double)f[i];
    }
}

// ---- diagnostics: FP64 block partials, then one block folds them ----------------
constexpr int DIAG_NT = 256;
constexpr int DIAG_NV = 8;

template <typename T>
__global__ void __launch_bounds__(DIAG_NT)
diag_partial_kernel(const T *__restrict__ in, double *__restrict__ partial, const KParams kp)
{
    Consts<T> cs;
    cs.load(kp);
    const long long P = kp.plane;
    const long long ncell = (long long)kp.nx * kp.ny;
    double acc[DIAG_NV] = {0.0, 0.0, 0.0, 0.0, 1e300, 1e300, 0.0, 0.0};
    for (long long c = (long long)blockIdx.x * DIAG_NT + threadIdx.x; c < ncell; c += (long long)gridDim.x * DIAG_NT) {
        const int gy = (int)(c / kp.nx), gx = (int)(c - (long long)gy * kp.nx);
        const int o = gy * kp.pitch + gx;
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

__global__ void __launch_bounds__(DIAG_NT)
diag_final_kernel(const double *__restrict__ partial, int nblocks, double *__restrict__ out)
{
    __shared__ double red[DIAG_NV][DIAG_NT];
    double acc[DIAG_NV] = {0.0, 0.0, 0.0, 0.0, 1e300, 1e300, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += DIAG_NT) {
#pragma unroll
        for (int k = 0; k < DIAG_NV; k++) {
            const double v = partial[b * DIAG_NV + k];
            acc[k] = (k == 4 || k == 5) ? fmin(acc[k], v) : (k == 6 ? fmax(acc[k], v) : acc[k] + v);
        }
    }
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
    if (threadIdx.x < DIAG_NV) out[threadIdx.x] = red[threadIdx.x][0];
}

}  // namespace hlbm
