// hlbm_march.cuh -- the fused step of Algorithm 1 (steps 5-11) as a
// row-marching kernel: each CTA owns a strip of W columns and walks down a
// segment of rows, so that only the x halo is loaded and computed twice.
//
// Per row r of the segment one iteration does, separated by two barriers:
//   load:    F(n) of row r+2 on columns x0-2 .. x0+W+1 and s(n) of row r+3
//            on x0-3 .. x0+W+2 (prefetched into registers one iteration
//            earlier), the level-n rho, u, theta of row r+2 (local moments
//            of F(n), theta from s(n) of the same cell)
//   phase 2: level n+1 of row r+1 on x0-1 .. x0+W: the entropy update
//            (step 7), pull-streaming and moments (steps 5-6), theta
//            (step 8), and the second moments of the pulled populations
//            when sigma > 0
//   phase 3: row r on x0 .. x0+W-1: E1, E2, a1 and the regularised
//            collision (steps 9-11), written as F(n+1), s(n+1), a1(n+1).
// Rows live in shared-memory rings: 3 rows of F and of the level-n macros,
// 5 rows of s, 3 rows of level-(n+1) values.  A segment starts four rows
// early to fill them.  The arithmetic of every cell is that of the tiled
// kernel, term by term, so both give the same numbers.
//
// Boundaries use the index maps of the tiled kernel: a row or column off
// the domain maps to its periodic image, to the nearest edge cell
// (zero-gradient) or to the constants of a Dirichlet side (the y side wins
// at a corner).  Level-(n+1) values beyond a zero-gradient side are read
// from the edge cell itself in phase 3.
#pragma once

#include "hlbm_device.cuh"

namespace hlbm {

template <typename T, int W>
struct MarchGeom {
    static constexpr int NT = W + 32;       // the last warp covers the x halo
    static constexpr int FC = W + 4;        // F and level-n macro columns
    static constexpr int SC = W + 6;        // s columns
    static constexpr int NC = W + 2;        // level-(n+1) columns
    static constexpr int NQ = 8;            // rho, u_x, u_y, theta, s, m_xx, m_yy, m_xy
    static constexpr int OFF_F = 0;                      // [3][9][FC]
    static constexpr int OFF_M = OFF_F + 3 * 9 * FC;     // [3][4][FC]
    static constexpr int OFF_S = OFF_M + 3 * 4 * FC;     // [5][SC]
    static constexpr int OFF_N = OFF_S + 5 * SC;         // [3][NQ][NC]
    static constexpr int N = OFF_N + 3 * NQ * NC;
    static constexpr size_t smem_bytes = sizeof(T) * (size_t)N;
};

// Row (or column) of the cell that gy (gx) maps to, or -(side + 1) on a
// Dirichlet side.
__device__ __forceinline__ int map_row(int gy, const KParams &kp)
{
    if (gy >= 0 && gy < kp.ny) return gy;
    const int s = gy < 0 ? 2 : 3;
    const int b = kp.bc[s];
    if (b == BC_DIRICHLET) return -(s + 1);
    return b == BC_PERIODIC ? wrapi(gy, kp.ny) : (gy < 0 ? 0 : kp.ny - 1);
}

__device__ __forceinline__ int map_col(int gx, const KParams &kp)
{
    if (gx >= 0 && gx < kp.nx) return gx;
    const int s = gx < 0 ? 0 : 1;
    const int b = kp.bc[s];
    if (b == BC_DIRICHLET) return -(s + 1);
    return b == BC_PERIODIC ? wrapi(gx, kp.nx) : (gx < 0 ? 0 : kp.nx - 1);
}

// Offset of (mapped row, mapped column), or -(side + 1); a Dirichlet y side
// wins over a Dirichlet x side, as in locate().
__device__ __forceinline__ int join_map(int mr, int mc, int pitch)
{
    return mr < 0 ? mr : (mc < 0 ? mc : mr * pitch + mc);
}

// Row segment k of nseg: rows [k ny / nseg, (k + 1) ny / nseg).
__device__ __forceinline__ int seg_start(int k, int nseg, int ny)
{
    return (int)(((long long)k * ny) / nseg);
}

template <typename T, typename S, int W>
__global__ void __launch_bounds__(W + 32)
march_step_kernel(const typename S::raw *__restrict__ inF, const T *__restrict__ inA,
                  typename S::raw *__restrict__ outF, T *__restrict__ outA, const KParams kp, const int nseg)
{
    using G = MarchGeom<T, W>;
    constexpr int FC = G::FC, SC = G::SC, NC = G::NC, NQ = G::NQ;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *const rF = reinterpret_cast<T *>(smem_raw) + G::OFF_F;
    T *const rM = reinterpret_cast<T *>(smem_raw) + G::OFF_M;
    T *const rS = reinterpret_cast<T *>(smem_raw) + G::OFF_S;
    T *const rN = reinterpret_cast<T *>(smem_raw) + G::OFF_N;

    Consts<T> cs;
    cs.load(kp);
    const Side<T> side{kp};
    const T third = T(1) / T(3);
    const long long P = kp.plane;
    const int pitch = kp.pitch;
    const int t = threadIdx.x;
    const int x0 = blockIdx.x * W;
    const int ys = seg_start(blockIdx.y, nseg, kp.ny), ye = seg_start(blockIdx.y + 1, nseg, kp.ny);
    const int base = ys - 4;  // ring slots count rows from here (all used rows lie above it)

    // load-phase column (s on t < SC, F and macros on 1 <= t < SC - 1)
    const int mcL = map_col(x0 - 3 + t, kp);
    const bool doS = t < SC, doF = t >= 1 && t < SC - 1;
    // phase-2 column
    const int gx2 = x0 - 1 + t;
    const int mc2 = map_col(gx2, kp);
    const bool do2 = t < NC;
    const bool out2x = gx2 < 0 || gx2 >= kp.nx;
    const int side2x = gx2 < 0 ? 0 : 1;
    const bool dir2x = out2x && kp.bc[side2x] == BC_DIRICHLET;
    const bool zg2x = out2x && kp.bc[side2x] == BC_ZEROGRAD;
    // phase-3 column and its neighbours in the level-(n+1) ring
    const int gx3 = x0 + t;
    const bool do3 = t < W && gx3 < kp.nx;
    const int cl = (gx3 == 0 && kp.bc[0] == BC_ZEROGRAD) ? t + 1 : t;
    const int cr = (gx3 == kp.nx - 1 && kp.bc[1] == BC_ZEROGRAD) ? t + 1 : t + 2;

    // prefetch registers: F(n) of row r+2, s(n) of row r+3, a1(n) of row r+1
    T pF[9], pS = T(0), pA0 = T(0), pA1 = T(0), pA2 = T(0);
#pragma unroll
    for (int i = 0; i < 9; i++) pF[i] = T(0);
    auto fetch = [&](int r) {
        if (doF) {
            const int o = join_map(map_row(r + 2, kp), mcL, pitch);
            if (o >= 0) {
                const typename S::raw *src = inF + o;
#pragma unroll
                for (int i = 0; i < 9; i++) pF[i] = S::get(src[i * P], i, kp);
            } else {
#pragma unroll
                for (int i = 0; i < 9; i++) pF[i] = side.F(-o - 1, i);
            }
        }
        if (doS) {
            const int o = join_map(map_row(r + 3, kp), mcL, pitch);
            pS = o >= 0 ? __ldg(inA + A_S * P + o) : side.s_(-o - 1);
        }
        if (kp.phi_mode == 0 && do2) {
            const int o = join_map(map_row(r + 1, kp), mc2, pitch);
            if (o >= 0) {
                pA0 = __ldg(inA + A_XX * P + o);
                pA1 = __ldg(inA + A_XY * P + o);
                pA2 = __ldg(inA + A_YY * P + o);
            }
        }
    };

    // s(n) of rows ys-3 and ys-2; the latter stays in a register for the
    // level-n theta of row ys-2
    T s_prev = T(0);
    if (doS) {
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const int gy = ys - 3 + k;
            const int o = join_map(map_row(gy, kp), mcL, pitch);
            const T v = o >= 0 ? __ldg(inA + A_S * P + o) : side.s_(-o - 1);
            rS[((gy - base) % 5) * SC + t] = v;
            s_prev = v;
        }
    }
    fetch(base);

    for (int r = base; r < ye; r++) {
        // ---- load phase: row r+2 of F(n) and of the level-n macros, row r+3 of s(n)
        T f[9];
#pragma unroll
        for (int i = 0; i < 9; i++) f[i] = pF[i];
        const T snew = pS, a_xx = pA0, a_xy = pA1, a_yy = pA2;
        if (r + 1 < ye) fetch(r + 1);
        if (doF) {
            const int yF = r + 2;
            const int sl = (yF - base) % 3;
            const int c = t - 1;
#pragma unroll
            for (int i = 0; i < 9; i++) rF[(sl * 9 + i) * FC + c] = f[i];
            const int o = join_map(map_row(yF, kp), mcL, pitch);
            T rho, ux, uy, th;
            if (o >= 0) {
                T jx, jy;
                moments(f, rho, jx, jy);
                const T ir = fdiv(T(1), rho);
                ux = jx * ir;
                uy = jy * ir;
                th = cs.theta(rho, s_prev);
            } else {
                const int sd = -o - 1;
                rho = side.rho(sd); ux = side.ux(sd); uy = side.uy(sd); th = side.th(sd);
            }
            T *m = rM + sl * 4 * FC + c;
            m[0] = rho; m[FC] = ux; m[2 * FC] = uy; m[3 * FC] = th;
        }
        if (doS) {
            rS[((r + 3 - base) % 5) * SC + t] = snew;
            s_prev = snew;
        }
        __syncthreads();

        // ---- phase 2: level n+1 of row r+1
        const int y2 = r + 1;
        if (y2 >= ys - 1 && do2) {
            const bool out2y = y2 < 0 || y2 >= kp.ny;
            const int side2y = y2 < 0 ? 2 : 3;
            const bool dir2y = out2y && kp.bc[side2y] == BC_DIRICHLET;
            const bool zg2y = out2y && kp.bc[side2y] == BC_ZEROGRAD;
            T *n = rN + ((y2 - base) % 3) * NQ * NC + t;
            if (dir2y || dir2x) {
                const int sd = dir2y ? side2y : side2x;
                n[0] = side.rho(sd); n[NC] = side.ux(sd); n[2 * NC] = side.uy(sd);
                n[3 * NC] = side.th(sd); n[4 * NC] = side.s_(sd);
            } else if (!(zg2y || zg2x)) {
                const int m0 = (y2 - base) % 3, mm = (y2 - 1 - base) % 3, mp = (y2 + 1 - base) % 3;
                const int cF = t + 1;
                const T *M0 = rM + m0 * 4 * FC + cF, *Mm = rM + mm * 4 * FC + cF, *Mp = rM + mp * 4 * FC + cF;
                const T rho0 = M0[0], ux0 = M0[FC], uy0 = M0[2 * FC], th0 = M0[3 * FC];
                const T dxux = T(0.5) * (M0[FC + 1] - M0[FC - 1]);
                const T dyux = T(0.5) * (Mp[FC] - Mm[FC]);
                const T dxuy = T(0.5) * (M0[2 * FC + 1] - M0[2 * FC - 1]);
                const T dyuy = T(0.5) * (Mp[2 * FC] - Mm[2 * FC]);
                const T lap = (M0[3 * FC + 1] + M0[3 * FC - 1]) + (Mp[3 * FC] + Mm[3 * FC]) - T(4) * th0;
                const int cS = t + 2;
                const T *S0 = rS + ((y2 - base) % 5) * SC + cS;
                const T s0 = S0[0];
                const T sym2 = rS[((y2 - 2 - base) % 5) * SC + cS], sym = rS[((y2 - 1 - base) % 5) * SC + cS];
                const T syp = rS[((y2 + 1 - base) % 5) * SC + cS], syp2 = rS[((y2 + 2 - base) % 5) * SC + cS];
                const T adv = muscl_adv(ux0, S0[-2], S0[-1], s0, S0[1], S0[2]) + muscl_adv(uy0, sym2, sym, s0, syp, syp2);
                const T rt = rho0 * th0;
                const T p0 = rt * third;
                T phi;
                if (kp.phi_mode == 0) {
                    phi = -fdiv(cs.two_mu, cs.two_mu + p0) * (a_xx * dxux + a_xy * (dyux + dxuy) + a_yy * dyuy);
                } else {
                    const T d1 = dxux - dyuy, d2 = dyux + dxuy;
                    phi = cs.mu * (d1 * d1 + d2 * d2);
                }
                const T s1 = s0 - adv + fdiv(cs.lam * lap + phi, rt);
                // pull: F_i from (x - c_ix, y - c_iy)
                T g[9];
#pragma unroll
                for (int i = 0; i < 9; i++) {
                    const int sl = cyi(i) > 0 ? mm : (cyi(i) < 0 ? mp : m0);
                    g[i] = rF[(sl * 9 + i) * FC + cF - cxi(i)];
                }
                T rho1, jx, jy;
                moments(g, rho1, jx, jy);
                const T ir = fdiv(T(1), rho1);
                n[0] = rho1; n[NC] = jx * ir; n[2 * NC] = jy * ir;
                n[3 * NC] = cs.theta(rho1, s1);
                n[4 * NC] = s1;
                if (kp.sigma_nonzero) {
                    const T diag = (g[5] + g[6]) + (g[7] + g[8]);
                    n[5 * NC] = (g[1] + g[3]) + diag;
                    n[6 * NC] = (g[2] + g[4]) + diag;
                    n[7 * NC] = (g[5] - g[6]) + (g[7] - g[8]);
                }
            }
        }
        __syncthreads();

        // ---- phase 3: steps 9-11 and the next collision on row r
        if (r >= ys && do3) {
            const int n0 = (r - base) % 3;
            const int nm = (r == 0 && kp.bc[2] == BC_ZEROGRAD) ? n0 : (r - 1 - base) % 3;
            const int np = (r == kp.ny - 1 && kp.bc[3] == BC_ZEROGRAD) ? n0 : (r + 1 - base) % 3;
            const T *N0 = rN + n0 * NQ * NC, *Nm = rN + nm * NQ * NC, *Np = rN + np * NQ * NC;
            const int k = t + 1;
            const T rho = N0[k], ux = N0[NC + k], uy = N0[2 * NC + k], th = N0[3 * NC + k];
            const T uxm = N0[NC + cl], uxp = N0[NC + cr], uym = Nm[2 * NC + k], uyp = Np[2 * NC + k];
            const T dxux = T(0.5) * (uxp - uxm);
            const T dyux = T(0.5) * (Np[NC + k] - Nm[NC + k]);
            const T dxuy = T(0.5) * (N0[2 * NC + cr] - N0[2 * NC + cl]);
            const T dyuy = T(0.5) * (uyp - uym);
            const T p = rho * th * third;
            const T gxc = gamma_defect(rho, ux, th), gyc = gamma_defect(rho, uy, th);
            const T gxm = gamma_defect(N0[cl], uxm, N0[3 * NC + cl]);
            const T gxp = gamma_defect(N0[cr], uxp, N0[3 * NC + cr]);
            const T gym = gamma_defect(Nm[k], uym, Nm[3 * NC + k]);
            const T gyp = gamma_defect(Np[k], uyp, Np[3 * NC + k]);
            const bool cen = kp.e1_centred != 0;
            const T e1xx = (ux > T(0) && !cen) ? gxc - gxm : ((ux < T(0) && !cen) ? gxp - gxc : T(0.5) * (gxp - gxm));
            const T e1yy = (uy > T(0) && !cen) ? gyc - gym : ((uy < T(0) && !cen) ? gyp - gyc : T(0.5) * (gyp - gym));
            const T e2 = p * cs.two_m_gamma * (dxux + dyuy);
            const T ex = e1xx + e2, ey = e1yy + e2;
            const T cfd = -(cs.mu + T(0.5) * p);
            const T fdxx = cfd * (dxux - dyuy), fdxy = cfd * (dyux + dxuy);
            T axx, axy, ayy;
            if (kp.sigma_nonzero) {
                const T prxx = N0[5 * NC + k] - rho * ux * ux - p + T(0.5) * ex;
                const T pryy = N0[6 * NC + k] - rho * uy * uy - p + T(0.5) * ey;
                const T prxy = N0[7 * NC + k] - rho * ux * uy;
                axx = cs.sigma * prxx + cs.one_m_sigma * fdxx;
                ayy = cs.sigma * pryy - cs.one_m_sigma * fdxx;
                axy = cs.sigma * prxy + cs.one_m_sigma * fdxy;
            } else {
                axx = fdxx; ayy = -fdxx; axy = fdxy;
            }
            const T omega = fdiv(cs.two_mu - p, cs.two_mu + p);
            T fo[9];
            build_populations(rho, ux, uy, th, axx, axy, ayy, ex, ey, omega, fo);
            const long long o = (long long)r * pitch + gx3;
            typename S::raw *dF = outF + o;
#pragma unroll
            for (int i = 0; i < 9; i++) dF[i * P] = S::put(fo[i], i, kp);
            T *dA = outA + o;
            dA[A_S * P] = N0[4 * NC + k];
            dA[A_XX * P] = axx;
            dA[A_XY * P] = axy;
            dA[A_YY * P] = ayy;
        }
    }
}

}  // namespace hlbm
