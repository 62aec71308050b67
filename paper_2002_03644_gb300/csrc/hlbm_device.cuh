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
// 128-byte boundary.  rho and u of a level are the moments of F (collision
// invariants, eqs. rhoalgo, ualgo) and theta follows from s and rho; only the
// FP64 row-marching form also stores them, in four planes behind these
// (A_RHO .. A_TH), so that no step recomputes them.
//
// This file holds the tiled form of the step (FP64, and FP32 grids of up to
// 768^2 cells) with the scalar cell arithmetic; hlbm_march.cuh holds the
// row-marching form (the FP32 default on larger grids, the batched form's
// marching shapes, and the moment-state form).
//
// One launch of fused_step_kernel performs one time step of Algorithm 1 for a tile
// of TX x TY cells:
//   phase 0: s(n) on the tile plus a 3-cell halo -> shared memory
//   phase 1: rho, u, theta at level n on tile + 2 (local moments of F(n))
//   phase 2: on tile + 1: the entropy update (eq sequaalgo, MUSCL / Van Albada,
//            Fourier, viscous heating), pull-streaming and moments (eqs
//            rhoalgo, ualgo), theta (eq Entropie expression), closure defect Gamma (Sec. 3.2)
//   phase 3: on the tile: E1 (upwind) and E2 (centred) -> psi (eq Psialgo),
//            f^eq (eq Equilibrium), a1 = sigma a1^PR + (1 - sigma) a1^FD with the
//            recurrence (eq a1sigalgo, Sec. 3.3), and the regularised collision of the next
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
// Wall sides (tiled kernel): a no-slip, fixed-temperature wall half-way
// between the first ghost layer and the first interior layer.  Ghost layer g
// mirrors interior layer g - 1: u reflected about the wall velocity, theta
// about the wall temperature, the pressure of the mirrored cell (rho_g
// theta_g = rho theta), s of that rho and theta, and post-collision
// populations rebuilt from them and the mirrored cell's a1 by the collision
// formula without psi.  A wall or Dirichlet y side wins at a corner; the
// x ghosts of a wall row's mirrored row are taken first (an x wall's ghost
// is mirrored once more).  wall_ghost_kernel writes the level-n ghost layers
// to a small buffer before each step; the level-(n+1) ghosts are mirrored
// inside the tile after phase 2.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace hlbm {

// ---- index checks of the debug build (HLBM_DEBUG) --------------------------------
// Built with -DHLBM_DEBUG, the marching and tiled kernels check the cell of
// every global access against the grid (and the vector accesses' partner
// column) and their ring slots against the ring depths.  The first failing
// check records (site, first value, second value) in dbg_first and the
// access is skipped (a load gives zero); no kernel traps.  hlbm_debug_check
// reads and clears the record.  In the release build every check is the
// constant true and costs nothing.
#ifdef HLBM_DEBUG
static __device__ unsigned long long dbg_first;  // 0: no failed check
__device__ __noinline__ void dbg_record(int site, long long a, long long b)
{
    const unsigned long long v = ((unsigned long long)(site & 0xFF) << 56) |
                                 ((unsigned long long)(a & 0xFFFFFFF) << 28) | (unsigned long long)(b & 0xFFFFFFF);
    atomicCAS(&dbg_first, 0ull, v | (1ull << 63));
}
// (row, col) inside the grid, and col + width - 1 too
__device__ __forceinline__ bool dbg_cell(int row, int col, int width, int nx, int ny, int site)
{
    if (row >= 0 && row < ny && col >= 0 && col + width - 1 < nx) return true;
    dbg_record(site, row, col);
    return false;
}
__device__ __forceinline__ bool dbg_range(long long v, long long n, int site)
{
    if (v >= 0 && v < n) return true;
    dbg_record(site, v, n);
    return false;
}
#define HLBM_CELL_OK(row, col, width, kp, site) ::hlbm::dbg_cell((row), (col), (width), (kp).nx, (kp).ny, (site))
#define HLBM_RANGE_OK(v, n, site) ::hlbm::dbg_range((v), (n), (site))
#else
#define HLBM_CELL_OK(row, col, width, kp, site) true
#define HLBM_RANGE_OK(v, n, site) true
#endif

constexpr int NPLANE = 13;
constexpr int P_S = 9, P_AXX = 10, P_AXY = 11, P_AYY = 12;
enum { BC_PERIODIC = 0, BC_ZEROGRAD = 1, BC_DIRICHLET = 2, BC_WALL = 3 };

struct KParams {
    int nx, ny, pitch;
    long long plane;           // elements per plane = pitch * ny
    int bc[4];                 // x-, x+, y-, y+
    int phi_mode;              // 0 regularised, 1 finite differences
    int sigma_nonzero;
    int e1_centred;            // 1: E1 by centred differences (ablation)
    double mu, sigma, lambda;  // lambda = mu c_p / Pr
    double gm1, inv_cv, cv, two_minus_gamma, gamma;
    // Dirichlet side constants: macros, entropy, closure defect, populations
    double d_rho[4], d_ux[4], d_uy[4], d_th[4], d_s[4], d_gx[4], d_gy[4];
    double d_F[4][9];
    // the same constants rounded to FP32 on the host, so that FP32 kernels
    // never touch the (slow) FP64 pipe
    float f_gm1, f_s2exp, f_mu, f_lam, f_sigma, f_one_m_sigma, f_two_m_gamma;
    float f_d_rho[4], f_d_ux[4], f_d_uy[4], f_d_th[4], f_d_s[4];
    float f_d_F[4][9];
    // reference populations subtracted before 16-bit storage (precision
    // forms HLBM_FP32_F16POP / HLBM_FP32_BF16POP; unused otherwise)
    float f_ref[9];
    // wall ghost layers of level n (arithmetic type): 10 planes (F_0..F_8,
    // s), each of 4 rows (y- depth 1, 2; y+ depth 1, 2) of wall_p = nx + 4
    // columns (x = -2 .. nx + 1), then 4 columns (x- depth 1, 2; x+ depth 1,
    // 2) of wall_q = ny + 4 rows (y = -2 .. ny + 1); null without wall sides
    void *wall_g;
    int wall_p, wall_q;
};

// ---- population storage ----------------------------------------------------------
// The nine population planes are stored as S::raw; the four auxiliary planes
// (s, a1_xx, a1_xy, a1_yy) always in the arithmetic type T.  Full storage
// keeps F_i itself; the 16-bit forms keep F_i - f_ref_i, the difference from
// one reference equilibrium per case, rounded to FP16 or BF16.
// raw2 holds two horizontally adjacent stored values (one aligned access).
template <typename T> struct Vec2;
template <> struct Vec2<float> {
    using type = float2;
    static __device__ __forceinline__ float2 make(float a, float b) { return make_float2(a, b); }
};
template <> struct Vec2<double> {
    using type = double2;
    static __device__ __forceinline__ double2 make(double a, double b) { return make_double2(a, b); }
};
template <typename T> struct FullStore {
    using raw = T;
    using raw2 = typename Vec2<T>::type;
    static __device__ __forceinline__ T get(raw r, int, const KParams &) { return r; }
    static __device__ __forceinline__ raw put(T v, int, const KParams &) { return v; }
    static __device__ __forceinline__ raw2 pack(raw a, raw b) { return Vec2<T>::make(a, b); }
};
struct HalfStore {
    using raw = __half;
    using raw2 = __half2;
    static __device__ __forceinline__ float get(raw r, int i, const KParams &kp) { return __half2float(r) + kp.f_ref[i]; }
    static __device__ __forceinline__ raw put(float v, int i, const KParams &kp) { return __float2half_rn(v - kp.f_ref[i]); }
    static __device__ __forceinline__ raw2 pack(raw a, raw b) { return __halves2half2(a, b); }
};
struct BF16Store {
    using raw = __nv_bfloat16;
    using raw2 = __nv_bfloat162;
    static __device__ __forceinline__ float get(raw r, int i, const KParams &kp) { return __bfloat162float(r) + kp.f_ref[i]; }
    static __device__ __forceinline__ raw put(float v, int i, const KParams &kp) { return __float2bfloat16_rn(v - kp.f_ref[i]); }
    static __device__ __forceinline__ raw2 pack(raw a, raw b) { return __halves2bfloat162(a, b); }
};
// auxiliary plane indices
constexpr int A_S = 0, A_XX = 1, A_XY = 2, A_YY = 3;
// FP64 row-marching form only: four more planes behind the auxiliary ones
// hold each cell's level-n rho, u_x, u_y, theta.  They are derived state, so
// a checkpoint leaves them out: the step that ends a level stores the values
// its phase 2 computed, and the next step's load phase reads them instead of
// taking the moments of F(n) and recovering theta again.
constexpr int A_RHO = 4, A_UX = 5, A_UY = 6, A_TH = 7, A_NCACHE = 4;

// Dirichlet constants in the kernel's precision.
template <typename T> struct Side;
template <> struct Side<float> {
    const KParams &k;
    __device__ float rho(int s) const { return k.f_d_rho[s]; }
    __device__ float ux(int s) const { return k.f_d_ux[s]; }
    __device__ float uy(int s) const { return k.f_d_uy[s]; }
    __device__ float th(int s) const { return k.f_d_th[s]; }
    __device__ float s_(int s) const { return k.f_d_s[s]; }
    __device__ float F(int s, int i) const { return k.f_d_F[s][i]; }
};
template <> struct Side<double> {
    const KParams &k;
    __device__ double rho(int s) const { return k.d_rho[s]; }
    __device__ double ux(int s) const { return k.d_ux[s]; }
    __device__ double uy(int s) const { return k.d_uy[s]; }
    __device__ double th(int s) const { return k.d_th[s]; }
    __device__ double s_(int s) const { return k.d_s[s]; }
    __device__ double F(int s, int i) const { return k.d_F[s][i]; }
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

// locate() with wall sides: a coordinate beyond a wall maps to the wall
// ghost buffer, returned as -(kWallCode + index).  A y wall (checked first,
// so that it wins at a corner) gives index = row * wall_p + x + 2 (row =
// (side - 2) * 2 + depth - 1, x clamped to [-2, nx + 1]); otherwise y is
// mapped and an x wall gives index = 4 wall_p + col * wall_q + y + 2 (col =
// side * 2 + depth - 1).  Depths are clamped to 2, which covers every ghost
// value a tile reads.
constexpr int kWallCode = 8;
constexpr int kWallPlanes = 10;
__device__ __forceinline__ int locate_w(int gx, int gy, const KParams &kp, int pitch)
{
    if (gy < 0 || gy >= kp.ny) {
        const int s = gy < 0 ? 2 : 3;
        const int b = kp.bc[s];
        if (b == BC_WALL) {
            const int d = min(gy < 0 ? -gy : gy - kp.ny + 1, 2);
            const int x = min(max(gx, -2), kp.nx + 1);
            return -(kWallCode + ((s - 2) * 2 + d - 1) * kp.wall_p + x + 2);
        }
        if (b == BC_DIRICHLET) return -(s + 1);
        gy = (b == BC_PERIODIC) ? wrapi(gy, kp.ny) : (gy < 0 ? 0 : kp.ny - 1);
    }
    if ((gx < 0 || gx >= kp.nx) && kp.bc[gx < 0 ? 0 : 1] == BC_WALL) {
        const int s = gx < 0 ? 0 : 1;
        const int d = min(gx < 0 ? -gx : gx - kp.nx + 1, 2);
        return -(kWallCode + 4 * kp.wall_p + (s * 2 + d - 1) * kp.wall_q + gy + 2);
    }
    return locate(gx, gy, kp, pitch);
}

// Whether a wall code belongs to an x wall.
__device__ __forceinline__ bool wall_is_x(int o, const KParams &kp) { return -o - kWallCode >= 4 * kp.wall_p; }

// Plane q (0..8 populations, 9 entropy) of wall ghost index w.
template <typename T>
__device__ __forceinline__ T wall_val(const KParams &kp, int w, int q)
{
    return static_cast<const T *>(kp.wall_g)[(size_t)q * (4 * kp.wall_p + 4 * kp.wall_q) + w];
}

// ---- FP32 hardware approximations ------------------------------------------
// The PTX approximate reciprocal, base-2 logarithm and base-2 exponential
// (relative error of a few ulp, denormals flushed).  The state never holds
// denormal or huge values, so the range handling of the library functions
// is not needed; the FP32 parity bound (1e-4) is far above these errors.
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float lg2_approx(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ---- precision-dependent helpers -------------------------------------------
template <typename T> struct Consts;

template <> struct Consts<float> {
    float gm1, s2exp, mu, two_mu, lam, sigma, one_m_sigma, two_m_gamma;
    __device__ void load(const KParams &kp)
    {
        gm1 = kp.f_gm1; s2exp = kp.f_s2exp;  // 1 / (c_v ln 2)
        mu = kp.f_mu; two_mu = 2.0f * mu; lam = kp.f_lam;
        sigma = kp.f_sigma; one_m_sigma = kp.f_one_m_sigma; two_m_gamma = kp.f_two_m_gamma;
    }
    // theta = rho^(gamma-1) exp(s / c_v) = 2^((gamma-1) log2 rho + s / (c_v ln 2))
    __device__ __forceinline__ float theta(float rho, float s) const { return ex2_approx(fmaf(gm1, lg2_approx(rho), s * s2exp)); }
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
// Shared memory per tile (elements of T):
//   sS  s(n) on tile + 3                      (TX+6)(TY+6)
//   sF  F_i(n) on tile + 2, 9 planes          9 (TX+4)(TY+4)
//   m*  rho, u_x, u_y, theta of level n on tile + 2   4 (TX+4)(TY+4)
//   n*  rho, u_x, u_y, theta, s of level n+1 on tile + 1   5 (TX+2)(TY+2)
// F(n) is read from HBM once (phase 1, coalesced rows) and every later use --
// the pull of phase 2 and the projection of phase 3 -- reads shared memory.
template <typename T, int TX, int TY>
struct TileGeom {
    static constexpr int R3X = TX + 6, R3Y = TY + 6, N3 = R3X * R3Y;
    static constexpr int R2X = TX + 4, R2Y = TY + 4, N2 = R2X * R2Y;
    static constexpr int R1X = TX + 2, R1Y = TY + 2, N1 = R1X * R1Y;
    static constexpr size_t smem_bytes = sizeof(T) * (size_t)(N3 + 13 * N2 + 5 * N1);
};

// Classification of a tile + 1 cell for phase 2: 0 compute, 1 Dirichlet
// constant (side in *side), 2 copy from the clamped cell, 3 mirror of the
// first interior row across a y wall, 4 of the first interior column across
// an x wall.
__device__ __forceinline__ int classify_r1(int gx, int gy, const KParams &kp, int *side)
{
    const bool outx = gx < 0 || gx >= kp.nx, outy = gy < 0 || gy >= kp.ny;
    if (!outx && !outy) return 0;
    const int o = locate_w(gx, gy, kp, kp.pitch);
    if (o <= -kWallCode) return wall_is_x(o, kp) ? 4 : 3;
    if (o < 0) { *side = -o - 1; return 1; }
    const bool cx = outx && kp.bc[gx < 0 ? 0 : 1] == BC_ZEROGRAD;
    const bool cy = outy && kp.bc[gy < 0 ? 2 : 3] == BC_ZEROGRAD;
    return (cx || cy) ? 2 : 0;
}

// Division: a times the approximate reciprocal in FP32 (about 2 ulp, well
// inside the FP32 parity bound), IEEE division in FP64.
__device__ __forceinline__ float fdiv(float a, float b) { return a * rcp_approx(b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }

// Van Albada limited slope from the two one-sided differences; zero at an
// extremum (a b <= 0).
template <typename T>
__device__ __forceinline__ T va_slope(T a, T b)
{
    const T ab = a * b;
    return ab > T(0) ? fdiv(ab * (a + b), a * a + b * b) : T(0);
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

// closure defect Gamma_a = rho u_a (1 - theta - u_a^2) (Sec. 2.3)
template <typename T>
__device__ __forceinline__ T gamma_defect(T rho, T ua, T th)
{
    return rho * ua * (T(1) - th - ua * ua);
}

// One tile of one time step of Algorithm 1 (all threads of the CTA take part;
// the caller separates consecutive tiles with a barrier).
template <typename T, typename S, int TX, int TY, int NT>
__device__ __forceinline__ void step_tile(const typename S::raw *__restrict__ inF, const T *__restrict__ inA,
                                          typename S::raw *__restrict__ outF, T *__restrict__ outA,
                                          const KParams &kp, const int x0, const int y0, unsigned char *smem_raw)
{
    using Geo = TileGeom<T, TX, TY>;
    constexpr int R3X = Geo::R3X, N3 = Geo::N3, R2X = Geo::R2X, N2 = Geo::N2, R1X = Geo::R1X, N1 = Geo::N1;
    T *sS = reinterpret_cast<T *>(smem_raw);
    T *sF = sS + N3;
    T *mRho = sF + 9 * N2, *mUx = mRho + N2, *mUy = mUx + N2, *mTh = mUy + N2;
    T *nRho = mTh + N2, *nUx = nRho + N1, *nUy = nUx + N1, *nTh = nUy + N1, *nS = nTh + N1;

    Consts<T> cs;
    cs.load(kp);
    const Side<T> side{kp};
    const T third = T(1) / T(3);
    const int pitch = kp.pitch;
    const long long P = kp.plane;
    const bool interior = x0 >= 3 && y0 >= 3 && x0 + TX + 3 <= kp.nx && y0 + TY + 3 <= kp.ny;

    // phase 0 + 1 loads: s(n) on tile + 3 and F(n) on tile + 2 go to shared
    // memory first, with all of a thread's loads in flight together
    for (int c = threadIdx.x; c < N3; c += NT) {
        const int ly = c / R3X, lx = c - ly * R3X;
        const int gx = x0 - 3 + lx, gy = y0 - 3 + ly;
        const int o = interior ? gy * pitch + gx : locate_w(gx, gy, kp, pitch);
        sS[c] = o >= 0 ? (HLBM_CELL_OK(o / pitch, o % pitch, 1, kp, 10) ? __ldg(inA + A_S * P + o) : T(0))
                       : (o > -kWallCode ? side.s_(-o - 1) : wall_val<T>(kp, -o - kWallCode, 9));
    }
    {
        constexpr int ITER = (N2 + NT - 1) / NT;
        T f[ITER][9];
        int oc[ITER];
#pragma unroll
        for (int it = 0; it < ITER; it++) {
            const int c = threadIdx.x + it * NT;
            oc[it] = 0;
            if (c < N2) {
                const int ly = c / R2X, lx = c - ly * R2X;
                const int gx = x0 - 2 + lx, gy = y0 - 2 + ly;
                const int o = interior ? gy * pitch + gx : locate_w(gx, gy, kp, pitch);
                oc[it] = o;
                if (o >= 0) {
                    const bool ok = HLBM_CELL_OK(o / pitch, o % pitch, 1, kp, 11);
#pragma unroll
                    for (int i = 0; i < 9; i++) f[it][i] = ok ? S::get(inF[i * P + o], i, kp) : T(0);
                } else if (o > -kWallCode) {
#pragma unroll
                    for (int i = 0; i < 9; i++) f[it][i] = side.F(-o - 1, i);
                } else {
#pragma unroll
                    for (int i = 0; i < 9; i++) f[it][i] = wall_val<T>(kp, -o - kWallCode, i);
                }
            }
        }
#pragma unroll
        for (int it = 0; it < ITER; it++) {
            const int c = threadIdx.x + it * NT;
            if (c < N2) {
#pragma unroll
                for (int i = 0; i < 9; i++) sF[i * N2 + c] = f[it][i];
            }
        }
        (void)oc;
    }
    __syncthreads();

    // phase 1: the level-n rho, u, theta on tile + 2
    for (int c = threadIdx.x; c < N2; c += NT) {
        const int ly = c / R2X, lx = c - ly * R2X;
        T rho, ux, uy, th;
        bool dirichlet = false;
        int sd = 0;
        if (!interior) {
            // wall ghosts take their macros from their populations like cells
            const int o = locate_w(x0 - 2 + lx, y0 - 2 + ly, kp, pitch);
            if (o < 0 && o > -kWallCode) { dirichlet = true; sd = -o - 1; }
        }
        if (!dirichlet) {
            T f[9];
#pragma unroll
            for (int i = 0; i < 9; i++) f[i] = sF[i * N2 + c];
            T jx, jy;
            moments(f, rho, jx, jy);
            const T ir = fdiv(T(1), rho);
            ux = jx * ir; uy = jy * ir;
            th = cs.theta(rho, sS[(ly + 1) * R3X + lx + 1]);
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
            if (kind >= 2) continue;
        }
        // a1(n) of this cell (phi_mode 0): issued first so the loads overlap
        // the stencil arithmetic below
        T axx = T(0), axy = T(0), ayy = T(0);
        if (kp.phi_mode == 0) {
            const int o = interior ? gy * pitch + gx : locate(gx, gy, kp, pitch);
            if (o >= 0) {
                axx = __ldg(inA + A_XX * P + o); axy = __ldg(inA + A_XY * P + o); ayy = __ldg(inA + A_YY * P + o);
            }
        }
        // entropy update from level-n fields (eq sequaalgo)
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
            phi = -fdiv(cs.two_mu, cs.two_mu + p0) * (axx * dxux + axy * (dyux + dxuy) + ayy * dyuy);
        } else {
            const T d1 = dxux - dyuy, d2 = dyux + dxuy;
            phi = cs.mu * (d1 * d1 + d2 * d2);
        }
        const T s1 = s0 - adv + fdiv(cs.lam * lap + phi, rt);
        // pull the post-collision populations (shared memory), moments (eqs rhoalgo, ualgo)
        T f[9];
#pragma unroll
        for (int i = 0; i < 9; i++) f[i] = sF[i * N2 + k2 - cxi(i) - cyi(i) * R2X];
        T rho1, jx, jy;
        moments(f, rho1, jx, jy);
        const T ir = fdiv(T(1), rho1);
        nRho[c] = rho1; nUx[c] = jx * ir; nUy[c] = jy * ir;
        nTh[c] = cs.theta(rho1, s1);  // eq (Entropie expression)
        nS[c] = s1;
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
            nRho[c] = nRho[src]; nUx[c] = nUx[src]; nUy[c] = nUy[src]; nTh[c] = nTh[src]; nS[c] = nS[src];
        }
        __syncthreads();
        if (kp.wall_g) {
            // wall sides: mirror the first interior column (x walls, after
            // the clamped copies, which the mirrored column may hold at a
            // corner), then the first interior row (y walls, whose mirrored
            // row may hold x-wall ghosts)
            for (int pass = 4; pass >= 3; pass--) {
                for (int c = threadIdx.x; c < N1; c += NT) {
                    const int ly = c / R1X, lx = c - ly * R1X;
                    const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
                    int sd = 0;
                    if (classify_r1(gx, gy, kp, &sd) != pass) continue;
                    const int ws = pass == 4 ? (gx < 0 ? 0 : 1) : (gy < 0 ? 2 : 3);
                    // columns 0 / nx - 1, rows 0 / ny - 1
                    const int src = pass == 4 ? c + (gx < 0 ? 1 : -1) : c + (gy < 0 ? R1X : -R1X);
                    const T th = T(2) * side.th(ws) - nTh[src];
                    nTh[c] = th;
                    nRho[c] = fdiv(nRho[src] * nTh[src], th);
                    nUx[c] = T(2) * side.ux(ws) - nUx[src];
                    nUy[c] = T(2) * side.uy(ws) - nUy[src];
                    nS[c] = T(0);  // not read: phase 3 uses the entropy of its own cell only
                }
                __syncthreads();
            }
        }
    }

    // phase 3: psi, f^eq, a1 and the collision of the next step on the tile
    for (int c = threadIdx.x; c < TX * TY; c += NT) {
        const int ly = c / TX, lx = c - ly * TX;
        const int gx = x0 + lx, gy = y0 + ly;
        if (gx >= kp.nx || gy >= kp.ny) continue;
        const int k = (ly + 1) * R1X + lx + 1;
        const T rho = nRho[k], ux = nUx[k], uy = nUy[k], th = nTh[k];
        const T uxm = nUx[k - 1], uxp = nUx[k + 1], uym = nUy[k - R1X], uyp = nUy[k + R1X];
        const T dxux = T(0.5) * (uxp - uxm);
        const T dyux = T(0.5) * (nUx[k + R1X] - nUx[k - R1X]);
        const T dxuy = T(0.5) * (nUy[k + 1] - nUy[k - 1]);
        const T dyuy = T(0.5) * (uyp - uym);
        const T p = rho * th * third;
        // E1: upwind difference of Gamma by the sign of the cell's velocity
        const T gxc = gamma_defect(rho, ux, th), gyc = gamma_defect(rho, uy, th);
        const T gxm = gamma_defect(nRho[k - 1], uxm, nTh[k - 1]);
        const T gxp = gamma_defect(nRho[k + 1], uxp, nTh[k + 1]);
        const T gym = gamma_defect(nRho[k - R1X], uym, nTh[k - R1X]);
        const T gyp = gamma_defect(nRho[k + R1X], uyp, nTh[k + R1X]);
        const bool cen = kp.e1_centred != 0;
        const T e1xx = (ux > T(0) && !cen) ? gxc - gxm : ((ux < T(0) && !cen) ? gxp - gxc : T(0.5) * (gxp - gxm));
        const T e1yy = (uy > T(0) && !cen) ? gyc - gym : ((uy < T(0) && !cen) ? gyp - gyc : T(0.5) * (gyp - gym));
        const T e2 = p * cs.two_m_gamma * (dxux + dyuy);
        const T ex = e1xx + e2, ey = e1yy + e2;
        // a1^FD = -tau_bar p (grad u + grad u^T - div u I), tau_bar p = mu + p/2
        const T cfd = -(cs.mu + T(0.5) * p);
        const T fdxx = cfd * (dxux - dyuy), fdxy = cfd * (dyux + dxuy);
        T axx, axy, ayy;
        if (kp.sigma_nonzero) {
            // second raw moments of the pulled populations of this cell
            const int k2 = (ly + 2) * R2X + lx + 2;
            T f[9];
#pragma unroll
            for (int i = 0; i < 9; i++) f[i] = sF[i * N2 + k2 - cxi(i) - cyi(i) * R2X];
            const T diag = (f[5] + f[6]) + (f[7] + f[8]);
            const T mxx = (f[1] + f[3]) + diag, myy = (f[2] + f[4]) + diag;
            const T mxy = (f[5] - f[6]) + (f[7] - f[8]);
            const T prxx = mxx - rho * ux * ux - p + T(0.5) * ex;
            const T pryy = myy - rho * uy * uy - p + T(0.5) * ey;
            const T prxy = mxy - rho * ux * uy;
            axx = cs.sigma * prxx + cs.one_m_sigma * fdxx;
            ayy = cs.sigma * pryy - cs.one_m_sigma * fdxx;
            axy = cs.sigma * prxy + cs.one_m_sigma * fdxy;
        } else {
            axx = fdxx; ayy = -fdxx; axy = fdxy;
        }
        // 1 - 1 / tau_bar with tau = mu / p
        const T omega = fdiv(cs.two_mu - p, cs.two_mu + p);
        T f[9];
        build_populations(rho, ux, uy, th, axx, axy, ayy, ex, ey, omega, f);
        const int o = gy * pitch + gx;
        if (!HLBM_CELL_OK(gy, gx, 1, kp, 12)) continue;
#pragma unroll
        for (int i = 0; i < 9; i++) outF[i * P + o] = S::put(f[i], i, kp);
        outA[A_S * P + o] = nS[k];
        outA[A_XX * P + o] = axx;
        outA[A_XY * P + o] = axy;
        outA[A_YY * P + o] = ayy;
    }
}

// One case: one CTA per tile.
template <typename T, typename S, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT)
fused_step_kernel(const typename S::raw *__restrict__ inF, const T *__restrict__ inA,
                  typename S::raw *__restrict__ outF, T *__restrict__ outA, const KParams kp)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    step_tile<T, S, TX, TY, NT>(inF, inA, outF, outA, kp, blockIdx.x * TX, blockIdx.y * TY, smem_raw);
}

// ---- many cases in one persistent launch (FP32) -----------------------------------
// Every case keeps its own ping-pong state and parameters; the tiles of all
// cases form one list that a grid of resident CTAs walks.  The parameters
// of the current case are copied to shared memory once per tile.
struct CasePlanes {
    const float *inF[2], *inA[2];  // read planes for parity 0 / 1
    float *outF[2], *outA[2];      // written planes for parity 0 / 1
};

struct BatchTables {
    const KParams *kps;       // [ncase]
    const CasePlanes *planes; // [ncase]
    const int *tile_case;     // [ntiles] case of each tile
    const int *tile_first;    // [ncase] first tile index of each case
    int ntiles;
};

template <int TX, int TY, int NT>
__global__ void __launch_bounds__(NT)
batched_step_kernel(const BatchTables tab, const int parity)
{
    using Geo = TileGeom<float, TX, TY>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    KParams &skp = *reinterpret_cast<KParams *>(smem_raw + (Geo::smem_bytes + 15) / 16 * 16);
    for (int t = blockIdx.x; t < tab.ntiles; t += gridDim.x) {
        const int c = tab.tile_case[t];
        {
            const int *src = reinterpret_cast<const int *>(tab.kps + c);
            int *dst = reinterpret_cast<int *>(&skp);
            for (int w = threadIdx.x; w < (int)(sizeof(KParams) / sizeof(int)); w += NT) dst[w] = __ldg(src + w);
        }
        __syncthreads();
        const int local = t - tab.tile_first[c];
        const int tiles_x = (skp.nx + TX - 1) / TX;
        const int x0 = (local % tiles_x) * TX, y0 = (local / tiles_x) * TY;
        const CasePlanes &pl = tab.planes[c];
        step_tile<float, FullStore<float>, TX, TY, NT>(pl.inF[parity], pl.inA[parity], pl.outF[parity],
                                                      pl.outA[parity], skp, x0, y0, smem_raw);
        __syncthreads();
    }
}

// ---- wall ghost layers of level n -----------------------------------------------
// One thread per ghost cell (blockIdx.x, threadIdx.x along the wall;
// blockIdx.y = layer): layers 0-3 are the y walls' rows (side 2 + layer / 2,
// depth layer % 2 + 1) over x = -2 .. nx + 1, layers 4-7 the x walls'
// columns (side (layer - 4) / 2, depth layer % 2 + 1) over y = -2 .. ny + 1.
// The mirrored cell's rho and u are the moments of its F(n), theta follows
// from its s(n), a1 is its own.  A cell beyond an x side takes the x side's
// map: a Dirichlet x side gives its constants and a1 = 0, an x wall the
// reflection of the cell it mirrors (so a y wall's corner ghost is mirrored
// twice).
template <typename T>
struct WallCell {
    T rho, ux, uy, th, axx, axy, ayy;
};

template <typename T>
__device__ __forceinline__ void wall_reflect(const Side<T> &side, int ws, WallCell<T> &c)
{
    const T tg = T(2) * side.th(ws) - c.th;
    c.rho = fdiv(c.rho * c.th, tg);
    c.th = tg;
    c.ux = T(2) * side.ux(ws) - c.ux;
    c.uy = T(2) * side.uy(ws) - c.uy;
}

template <typename T, typename S>
__global__ void wall_ghost_kernel(const typename S::raw *__restrict__ inF, const T *__restrict__ inA,
                                  const KParams kp)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int layer = blockIdx.y;
    const bool xw = layer >= 4;
    const int ws = xw ? (layer - 4) / 2 : 2 + layer / 2, depth = layer % 2 + 1;
    if (i >= (xw ? kp.wall_q : kp.wall_p) || kp.bc[ws] != BC_WALL) return;
    Consts<T> cs;
    cs.load(kp);
    const Side<T> side{kp};
    const long long P = kp.plane;
    // the interior cell this ghost mirrors: (column, row)
    int mx, my;
    if (xw) {
        mx = ws == 0 ? depth - 1 : kp.nx - depth;
        my = i - 2;
    } else {
        mx = i - 2;
        my = ws == 2 ? depth - 1 : kp.ny - depth;
    }
    // beyond an x wall (a y wall's corner): mirror across it first
    int xwall = -1;
    if (!xw && (mx < 0 || mx >= kp.nx) && kp.bc[mx < 0 ? 0 : 1] == BC_WALL) {
        xwall = mx < 0 ? 0 : 1;
        mx = mx < 0 ? -mx - 1 : 2 * kp.nx - 1 - mx;
    }
    const int o = locate(mx, my, kp, kp.pitch);
    WallCell<T> c;
    c.axx = c.axy = c.ayy = T(0);
    if (o >= 0) {
        T f[9];
#pragma unroll
        for (int q = 0; q < 9; q++) f[q] = S::get(inF[q * P + o], q, kp);
        T jx, jy;
        moments(f, c.rho, jx, jy);
        const T ir = fdiv(T(1), c.rho);
        c.ux = jx * ir;
        c.uy = jy * ir;
        c.th = cs.theta(c.rho, inA[A_S * P + o]);
        c.axx = inA[A_XX * P + o];
        c.axy = inA[A_XY * P + o];
        c.ayy = inA[A_YY * P + o];
    } else {
        const int sd = -o - 1;
        c.rho = side.rho(sd); c.ux = side.ux(sd); c.uy = side.uy(sd); c.th = side.th(sd);
    }
    if (xwall >= 0) wall_reflect(side, xwall, c);
    const T p = c.rho * c.th * (T(1) / T(3));  // the pressure is kept by every reflection
    wall_reflect(side, ws, c);
    const T omega = fdiv(cs.two_mu - p, cs.two_mu + p);
    T f[9];
    build_populations(c.rho, c.ux, c.uy, c.th, c.axx, c.axy, c.ayy, T(0), T(0), omega, f);
    T *wg = static_cast<T *>(kp.wall_g);
    const size_t w = xw ? (size_t)4 * kp.wall_p + (size_t)(layer - 4) * kp.wall_q + i : (size_t)layer * kp.wall_p + i;
    const size_t stride = (size_t)4 * kp.wall_p + (size_t)4 * kp.wall_q;
#pragma unroll
    for (int q = 0; q < 9; q++) wg[q * stride + w] = f[q];
    wg[9 * stride + w] = (T)(kp.cv * (log((double)c.th) - kp.gm1 * log((double)c.rho)));
}

// ---- initialisation (Sec. 3.5: f^eq, a1^FD and psi of the input state) --------
// Entropy of an initial cell, s = c_v (ln theta - (gamma - 1) ln rho), in the
// arithmetic type of the state.
__device__ __forceinline__ double init_entropy(const KParams &kp, double rho, double th)
{
    return kp.cv * (log(th) - kp.gm1 * log(rho));
}
__device__ __forceinline__ float init_entropy(const KParams &kp, float rho, float th)
{
    return (float)kp.cv * (logf(th) - kp.f_gm1 * logf(rho));
}

// From FP64 caller fields (row-major [ny][nx]); writes the state in T.  The
// arithmetic is in T as well: the FP32-arithmetic forms round the fields to
// FP32 on load, as their step does with every level, and FP64 computes in
// FP64 throughout.
template <typename T, typename S>
__global__ void init_kernel(const double *__restrict__ rho, const double *__restrict__ ux,
                            const double *__restrict__ uy, const double *__restrict__ th,
                            const double *__restrict__ a1, typename S::raw *__restrict__ outF,
                            T *__restrict__ outA, const KParams kp)
{
    const int gx = blockIdx.x * blockDim.x + threadIdx.x;
    const int gy = blockIdx.y * blockDim.y + threadIdx.y;
    if (gx >= kp.nx || gy >= kp.ny) return;
    const int n = kp.nx * kp.ny;
    auto at = [&](int dx, int dy, T &r, T &u, T &v, T &t) {
        int xx = gx + dx, yy = gy + dy;  // one of them at most is outside
        int ws = -1;
        // beyond a wall: the mirrored interior cell, reflected (see wall_ghost_kernel)
        if ((yy < 0 || yy >= kp.ny) && kp.bc[yy < 0 ? 2 : 3] == BC_WALL) {
            ws = yy < 0 ? 2 : 3;
            yy = yy < 0 ? -yy - 1 : 2 * kp.ny - 1 - yy;
        } else if ((xx < 0 || xx >= kp.nx) && kp.bc[xx < 0 ? 0 : 1] == BC_WALL) {
            ws = xx < 0 ? 0 : 1;
            xx = xx < 0 ? -xx - 1 : 2 * kp.nx - 1 - xx;
        }
        const int o = locate(xx, yy, kp, kp.nx);
        if (o >= 0) { r = (T)rho[o]; u = (T)ux[o]; v = (T)uy[o]; t = (T)th[o]; }
        else { const int s = -o - 1; r = (T)kp.d_rho[s]; u = (T)kp.d_ux[s]; v = (T)kp.d_uy[s]; t = (T)kp.d_th[s]; }
        if (ws >= 0) {
            const T tg = T(2) * (T)kp.d_th[ws] - t;
            r = r * t / tg;
            t = tg;
            u = T(2) * (T)kp.d_ux[ws] - u;
            v = T(2) * (T)kp.d_uy[ws] - v;
        }
    };
    T r0, u0, v0, t0, rxm, uxm, vxm, txm, rxp, uxp, vxp, txp, rym, uym, vym, tym, ryp, uyp, vyp, typ;
    at(0, 0, r0, u0, v0, t0);
    at(-1, 0, rxm, uxm, vxm, txm); at(1, 0, rxp, uxp, vxp, txp);
    at(0, -1, rym, uym, vym, tym); at(0, 1, ryp, uyp, vyp, typ);
    const T mu = (T)kp.mu;
    const T p = r0 * t0 / T(3);
    const T dxux = T(0.5) * (uxp - uxm), dyux = T(0.5) * (uyp - uym);
    const T dxuy = T(0.5) * (vxp - vxm), dyuy = T(0.5) * (vyp - vym);
    T axx, axy, ayy;
    const int c = gy * kp.nx + gx;
    if (a1) {
        axx = (T)a1[c]; axy = (T)a1[n + c]; ayy = (T)a1[2 * n + c];
    } else {
        const T cfd = -(mu + T(0.5) * p);
        axx = cfd * (dxux - dyuy); axy = cfd * (dyux + dxuy); ayy = -axx;
    }
    auto gam = [](T r, T u, T t) { return r * u * (T(1) - t - u * u); };
    const T gxc = gam(r0, u0, t0), gyc = gam(r0, v0, t0);
    const bool cen = kp.e1_centred != 0;
    const T e1xx = (u0 > T(0) && !cen) ? gxc - gam(rxm, uxm, txm)
                 : ((u0 < T(0) && !cen) ? gam(rxp, uxp, txp) - gxc : T(0.5) * (gam(rxp, uxp, txp) - gam(rxm, uxm, txm)));
    const T e1yy = (v0 > T(0) && !cen) ? gyc - gam(rym, vym, tym)
                 : ((v0 < T(0) && !cen) ? gam(ryp, vyp, typ) - gyc : T(0.5) * (gam(ryp, vyp, typ) - gam(rym, vym, tym)));
    const T e2 = p * (T)kp.two_minus_gamma * (dxux + dyuy);
    const T omega = (T(2) * mu - p) / (T(2) * mu + p);
    T f[9];
    build_populations<T>(r0, u0, v0, t0, axx, axy, ayy, e1xx + e2, e1yy + e2, omega, f);
    const long long P = kp.plane;
    const int o = gy * kp.pitch + gx;
#pragma unroll
    for (int i = 0; i < 9; i++) outF[i * P + o] = S::put(f[i], i, kp);
    outA[A_S * P + o] = init_entropy(kp, r0, t0);
    outA[A_XX * P + o] = axx;
    outA[A_XY * P + o] = axy;
    outA[A_YY * P + o] = ayy;
}

// ---- field extraction ----------------------------------------------------------
template <typename T, typename S>
__global__ void macros_kernel(const typename S::raw *__restrict__ inF, const T *__restrict__ inA, double *rho,
                              double *ux, double *uy, double *th, double *s, double *a1, double *F,
                              const KParams kp)
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
    for (int i = 0; i < 9; i++) f[i] = S::get(inF[i * P + o], i, kp);
    T r, jx, jy;
    moments(f, r, jx, jy);
    const T sv = inA[A_S * P + o];
    if (rho) rho[c] = (double)r;
    if (ux) ux[c] = (double)(jx / r);
    if (uy) uy[c] = (double)(jy / r);
    if (th) th[c] = (double)cs.theta(r, sv);
    if (s) s[c] = (double)sv;
    if (a1) {
        a1[c] = (double)inA[A_XX * P + o];
        a1[n + c] = (double)inA[A_XY * P + o];
        a1[2 * n + c] = (double)inA[A_YY * P + o];
    }
    if (F) {
#pragma unroll
        for (int i = 0; i < 9; i++) F[i * n + c] = (double)f[i];
    }
}

// ---- diagnostics: FP64 block partials, then one block folds them ----------------
constexpr int DIAG_NT = 256;
constexpr int DIAG_NV = 8;

template <typename T, typename S>
__global__ void __launch_bounds__(DIAG_NT)
diag_partial_kernel(const typename S::raw *__restrict__ inF, const T *__restrict__ inA,
                    double *__restrict__ partial, const KParams kp)
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
        for (int i = 0; i < 9; i++) f[i] = S::get(inF[i * P + o], i, kp);
        T r, jx, jy;
        moments(f, r, jx, jy);
        const double rho = (double)r;
        const double u = (double)jx / rho, v = (double)jy / rho;
        const double th = (double)cs.theta(r, inA[A_S * P + o]);
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

// Sums of rho, rho u_x, rho u_y and theta over FP64 caller fields (for the
// reference equilibrium of the 16-bit storage forms); same partial layout as
// diag_partial_kernel so that diag_final_kernel folds them.
__global__ void __launch_bounds__(DIAG_NT)
field_sums_partial_kernel(const double *__restrict__ rho, const double *__restrict__ ux,
                          const double *__restrict__ uy, const double *__restrict__ th, long long n,
                          double *__restrict__ partial)
{
    double acc[DIAG_NV] = {0.0, 0.0, 0.0, 0.0, 1e300, 1e300, 0.0, 0.0};
    for (long long c = (long long)blockIdx.x * DIAG_NT + threadIdx.x; c < n; c += (long long)gridDim.x * DIAG_NT) {
        acc[0] += rho[c]; acc[1] += rho[c] * ux[c]; acc[2] += rho[c] * uy[c]; acc[3] += th[c];
    }
    __shared__ double red[4][DIAG_NT];
#pragma unroll
    for (int k = 0; k < 4; k++) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = DIAG_NT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
#pragma unroll
            for (int k = 0; k < 4; k++) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x < DIAG_NV)
        partial[blockIdx.x * DIAG_NV + threadIdx.x] = threadIdx.x < 4 ? red[threadIdx.x][0] : acc[threadIdx.x];
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
