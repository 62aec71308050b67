// hlbm_march.cuh -- the fused step of Algorithm 1 (steps 5-11) as a
// row-marching kernel: each CTA owns a strip of columns and walks down a
// segment of rows, so that only the x halo is loaded and computed twice
// (a tiled kernel recomputes a halo in both directions).
//
// Per row r of the segment one iteration does, separated by two barriers:
//   load:    F(n) of row r+2 and s(n) of row r+3 (prefetched into registers
//            one iteration earlier), the level-n rho, u, theta of row r+2
//            (local moments of F(n), theta from s(n) of the same cell)
//   phase 2: level n+1 of row r+1: the entropy update (step 7),
//            pull-streaming and moments (steps 5-6), theta (step 8), and
//            the second moments of the pulled populations when sigma > 0
//   phase 3: row r: E1, E2, a1 and the regularised collision (steps 9-11),
//            written as F(n+1), s(n+1), a1(n+1).
// Rows live in shared-memory rings; a segment starts four rows early to
// fill them.  The arithmetic of every cell is that of the tiled kernel,
// term by term.
//
// Boundaries use the index maps of the tiled kernel: a row or column off
// the domain maps to its periodic image, to the nearest edge cell
// (zero-gradient) or to the constants of a Dirichlet side (the y side wins
// at a corner).  Level-(n+1) values beyond a zero-gradient side are read
// from the edge cell itself in phase 3.
#pragma once

#include "hlbm_device.cuh"

namespace hlbm {

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

// ---- paired-column form -----------------------------------------------------------
// The same pipeline with each thread owning two horizontally adjacent
// columns: global and shared-memory traffic moves in 2-element accesses, a
// cell's x neighbours come from its partner or one neighbouring pair, and a
// cell's own level-(n+1) values stay in the registers of the thread that
// computed them until its collision one iteration later.
//   NT threads; ring columns x0-4 .. x0+2NT-5 (pair t = columns 2t, 2t+1);
//   load phase on every pair, phase 2 on pairs 1 .. NT-2 (x0-2 .. x0+W+1),
//   phase 3 on pairs 2 .. NT-3 (the W = 2 (NT - 4) output columns).
// The pull reads population i of row y - c_iy only, so the F rows are kept
// by population group: (4, 7, 8) for one row (they stream from y + 1),
// (0, 1, 3) for two, (2, 5, 6) for three (they stream from y - 1).
// SIG (sigma > 0) and PHI0 (regularised Phi) are compile-time choices.

// Level-n+1 values of one cell and the second moments of its pulled
// populations (used by a1^PR when sigma > 0).
template <typename T>
struct CellN1 {
    T rho, ux, uy, th, s, mxx, myy, mxy;
};

// Steps 5-8 for one cell (the arithmetic of phase 2 of the tiled kernel).
// W/E/S/N = x-1, x+1, y-1, y+1; g[] the pulled populations.
template <typename T, bool SIG, bool PHI0>
__device__ __forceinline__ CellN1<T> level_np1(const Consts<T> &cs, T rho0, T ux0, T uy0, T th0, T uxW, T uxE,
                                              T uxS, T uxN, T uyW, T uyE, T uyS, T uyN, T thW, T thE, T thS, T thN,
                                              T sWW, T sW, T s0, T sE, T sEE, T sSS, T sS, T sN, T sNN, T a_xx,
                                              T a_xy, T a_yy, const T g[9])
{
    const T third = T(1) / T(3);
    const T dxux = T(0.5) * (uxE - uxW);
    const T dyux = T(0.5) * (uxN - uxS);
    const T dxuy = T(0.5) * (uyE - uyW);
    const T dyuy = T(0.5) * (uyN - uyS);
    const T lap = (thE + thW) + (thN + thS) - T(4) * th0;
    const T adv = muscl_adv(ux0, sWW, sW, s0, sE, sEE) + muscl_adv(uy0, sSS, sS, s0, sN, sNN);
    const T rt = rho0 * th0;
    const T p0 = rt * third;
    T phi;
    if (PHI0) {
        phi = -fdiv(cs.two_mu, cs.two_mu + p0) * (a_xx * dxux + a_xy * (dyux + dxuy) + a_yy * dyuy);
    } else {
        const T d1 = dxux - dyuy, d2 = dyux + dxuy;
        phi = cs.mu * (d1 * d1 + d2 * d2);
    }
    CellN1<T> o;
    o.s = s0 - adv + fdiv(cs.lam * lap + phi, rt);
    T jx, jy;
    moments(g, o.rho, jx, jy);
    const T ir = fdiv(T(1), o.rho);
    o.ux = jx * ir;
    o.uy = jy * ir;
    o.th = cs.theta(o.rho, o.s);
    if (SIG) {
        const T diag = (g[5] + g[6]) + (g[7] + g[8]);
        o.mxx = (g[1] + g[3]) + diag;
        o.myy = (g[2] + g[4]) + diag;
        o.mxy = (g[5] - g[6]) + (g[7] - g[8]);
    } else {
        o.mxx = o.myy = o.mxy = T(0);
    }
    return o;
}

// Steps 9-11 and the next collision for one cell (phase 3 of the tiled
// kernel) from its level-(n+1) values and those of its four neighbours.
template <typename T, bool SIG>
__device__ __forceinline__ void collide_cell(const Consts<T> &cs, bool cen, const CellN1<T> &c, T rW, T uxW, T uyW,
                                             T thW, T rE, T uxE, T uyE, T thE, T rS, T uxS, T uyS, T thS, T rN,
                                             T uxN, T uyN, T thN, T f[9], T &axx, T &axy, T &ayy)
{
    const T third = T(1) / T(3);
    const T rho = c.rho, ux = c.ux, uy = c.uy, th = c.th;
    const T dxux = T(0.5) * (uxE - uxW);
    const T dyux = T(0.5) * (uxN - uxS);
    const T dxuy = T(0.5) * (uyE - uyW);
    const T dyuy = T(0.5) * (uyN - uyS);
    const T p = rho * th * third;
    const T gxc = gamma_defect(rho, ux, th), gyc = gamma_defect(rho, uy, th);
    const T gxm = gamma_defect(rW, uxW, thW), gxp = gamma_defect(rE, uxE, thE);
    const T gym = gamma_defect(rS, uyS, thS), gyp = gamma_defect(rN, uyN, thN);
    const T e1xx = (ux > T(0) && !cen) ? gxc - gxm : ((ux < T(0) && !cen) ? gxp - gxc : T(0.5) * (gxp - gxm));
    const T e1yy = (uy > T(0) && !cen) ? gyc - gym : ((uy < T(0) && !cen) ? gyp - gyc : T(0.5) * (gyp - gym));
    const T e2 = p * cs.two_m_gamma * (dxux + dyuy);
    const T ex = e1xx + e2, ey = e1yy + e2;
    const T cfd = -(cs.mu + T(0.5) * p);
    const T fdxx = cfd * (dxux - dyuy), fdxy = cfd * (dyux + dxuy);
    if (SIG) {
        const T prxx = c.mxx - rho * ux * ux - p + T(0.5) * ex;
        const T pryy = c.myy - rho * uy * uy - p + T(0.5) * ey;
        const T prxy = c.mxy - rho * ux * uy;
        axx = cs.sigma * prxx + cs.one_m_sigma * fdxx;
        ayy = cs.sigma * pryy - cs.one_m_sigma * fdxx;
        axy = cs.sigma * prxy + cs.one_m_sigma * fdxy;
    } else {
        axx = fdxx; ayy = -fdxx; axy = fdxy;
    }
    const T omega = fdiv(cs.two_mu - p, cs.two_mu + p);
    build_populations(rho, ux, uy, th, axx, axy, ayy, ex, ey, omega, f);
}

template <typename T, int NT>
struct PairGeom {
    static constexpr int NP = NT - 4;   // output pairs
    static constexpr int W = 2 * NP;    // output columns
    static constexpr int CW = 2 * NT;   // ring columns
    static constexpr int OFF_GA = 0;                     // [3][CW]     F_4, F_7, F_8 of row r+2
    static constexpr int OFF_GB = OFF_GA + 3 * CW;       // [2][3][CW]  F_0, F_1, F_3 of rows r+1, r+2
    static constexpr int OFF_GC = OFF_GB + 6 * CW;       // [3][3][CW]  F_2, F_5, F_6 of rows r .. r+2
    static constexpr int OFF_M = OFF_GC + 9 * CW;        // [3][4][CW]  rho, u_x, u_y, theta (level n)
    static constexpr int OFF_S = OFF_M + 12 * CW;        // [5][CW]
    static constexpr int OFF_N = OFF_S + 5 * CW;         // [3][4][CW]  rho, u_x, u_y, theta (level n+1)
    static constexpr int N = OFF_N + 12 * CW;
    static constexpr size_t smem_bytes = sizeof(T) * (size_t)N;
};

// One strip (columns x0 .. x0+W-1) and one row segment [ys, ye) of one
// case; all NT threads of the CTA take part (the caller separates
// consecutive segments with a barrier).
template <typename T, typename S, int NT, bool SIG, bool PHI0>
__device__ __forceinline__ void march_pair_segment(const typename S::raw *__restrict__ inF,
                                                   const T *__restrict__ inA, typename S::raw *__restrict__ outF,
                                                   T *__restrict__ outA, const KParams &kp, const int x0,
                                                   const int ys, const int ye, unsigned char *smem_raw)
{
    using G = PairGeom<T, NT>;
    using V = typename Vec2<T>::type;
    using raw = typename S::raw;
    using raw2 = typename S::raw2;
    T *const sm = reinterpret_cast<T *>(smem_raw);
    V *const gA = reinterpret_cast<V *>(sm + G::OFF_GA);  // [3][NT] pairs
    V *const gB = reinterpret_cast<V *>(sm + G::OFF_GB);  // [2][3][NT]
    V *const gC = reinterpret_cast<V *>(sm + G::OFF_GC);  // [3][3][NT]
    V *const rM = reinterpret_cast<V *>(sm + G::OFF_M);   // [3][4][NT]
    V *const rS = reinterpret_cast<V *>(sm + G::OFF_S);   // [5][NT]
    V *const rN = reinterpret_cast<V *>(sm + G::OFF_N);   // [3][4][NT]

    Consts<T> cs;
    cs.load(kp);
    const Side<T> side{kp};
    const bool cen = kp.e1_centred != 0;
    const long long P = kp.plane;
    const int pitch = kp.pitch;
    const int t = threadIdx.x;
    const int base = ys - 4;

    // load-phase pair t: columns gxL, gxL + 1
    const int gxL = x0 - 4 + 2 * t;
    const int mcLa = map_col(gxL, kp), mcLb = map_col(gxL + 1, kp);
    const bool vecL = gxL >= 0 && gxL + 1 < kp.nx;
    // phase-2 / phase-3 pair q = t + 1: columns gx2, gx2 + 1
    const int gx2 = gxL + 2;
    const bool do2 = t < NT - 2;
    const int mc2a = map_col(gx2, kp), mc2b = map_col(gx2 + 1, kp);
    const bool vec2 = gx2 >= 0 && gx2 + 1 < kp.nx;
    // Dirichlet x sides: level n+1 beyond them is the side's state
    bool dir2[2];
    int side2[2];
#pragma unroll
    for (int c = 0; c < 2; c++) {
        const int gx = gx2 + c;
        side2[c] = gx < 0 ? 0 : 1;
        dir2[c] = (gx < 0 || gx >= kp.nx) && kp.bc[side2[c]] == BC_DIRICHLET;
    }
    const bool do3 = t >= 1 && t <= G::NP;
    const bool v3a = do3 && gx2 < kp.nx, v3b = do3 && gx2 + 1 < kp.nx;
    // zero-gradient x sides: the neighbour beyond the edge is the edge cell itself
    const bool zgW = gx2 == 0 && kp.bc[0] == BC_ZEROGRAD;             // west of cell a
    const bool zgEa = gx2 == kp.nx - 1 && kp.bc[1] == BC_ZEROGRAD;    // east of cell a
    const bool zgEb = gx2 + 1 == kp.nx - 1 && kp.bc[1] == BC_ZEROGRAD; // east of cell b

    // prefetch registers: F(n) of row r+2, s(n) of row r+3 (load pair),
    // a1(n) of row r+1 (phase-2 pair)
    T pFa[9], pFb[9], pSa = T(0), pSb = T(0), pA[2][3];
#pragma unroll
    for (int i = 0; i < 9; i++) { pFa[i] = T(0); pFb[i] = T(0); }
#pragma unroll
    for (int c = 0; c < 2; c++) { pA[c][0] = T(0); pA[c][1] = T(0); pA[c][2] = T(0); }

    auto load_F = [&](int mr, T *fa, T *fb) {
        if (mr >= 0 && vecL) {
            const raw *src = inF + ((long long)mr * pitch + gxL);
#pragma unroll
            for (int i = 0; i < 9; i++) {
                const raw2 v = *reinterpret_cast<const raw2 *>(src + i * P);
                fa[i] = S::get(v.x, i, kp);
                fb[i] = S::get(v.y, i, kp);
            }
        } else {
            const int oa = join_map(mr, mcLa, pitch), ob = join_map(mr, mcLb, pitch);
#pragma unroll
            for (int i = 0; i < 9; i++) {
                fa[i] = oa >= 0 ? S::get(inF[oa + i * P], i, kp) : side.F(-oa - 1, i);
                fb[i] = ob >= 0 ? S::get(inF[ob + i * P], i, kp) : side.F(-ob - 1, i);
            }
        }
    };
    auto load_s = [&](int mr, T &sa, T &sb) {
        if (mr >= 0 && vecL) {
            const V v = *reinterpret_cast<const V *>(inA + A_S * P + ((long long)mr * pitch + gxL));
            sa = v.x;
            sb = v.y;
        } else {
            const int oa = join_map(mr, mcLa, pitch), ob = join_map(mr, mcLb, pitch);
            sa = oa >= 0 ? inA[A_S * P + oa] : side.s_(-oa - 1);
            sb = ob >= 0 ? inA[A_S * P + ob] : side.s_(-ob - 1);
        }
    };
    auto fetch = [&](int r) {
        load_F(map_row(r + 2, kp), pFa, pFb);
        load_s(map_row(r + 3, kp), pSa, pSb);
        if (PHI0 && do2) {
            const int mr = map_row(r + 1, kp);
            if (mr >= 0 && vec2) {
                const T *src = inA + ((long long)mr * pitch + gx2);
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    const V v = *reinterpret_cast<const V *>(src + (A_XX + k) * P);
                    pA[0][k] = v.x;
                    pA[1][k] = v.y;
                }
            } else {
                const int oa = join_map(mr, mc2a, pitch), ob = join_map(mr, mc2b, pitch);
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    pA[0][k] = oa >= 0 ? inA[(A_XX + k) * P + oa] : T(0);
                    pA[1][k] = ob >= 0 ? inA[(A_XX + k) * P + ob] : T(0);
                }
            }
        }
    };

    // s(n) of rows ys-3 and ys-2 (the latter kept for the level-n theta of row ys-2)
    T sPa = T(0), sPb = T(0);
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int gy = ys - 3 + k;
        load_s(map_row(gy, kp), sPa, sPb);
        rS[((gy - base) % 5) * NT + t] = Vec2<T>::make(sPa, sPb);
    }
    fetch(base);

    // ring slots: level-n rows r .. r+2 (fs*, also F_2,5,6), F_0,1,3 rows r+1 / r+2
    // (bs*), s rows r-1 .. r+3 (ss*), level n+1 rows r-1 .. r+1 (ns*)
    int fs0 = 0, fs1 = 1, fs2 = 2;
    int bs1 = 1, bs2 = 0;
    int ss0 = 4, ss1 = 0, ss2 = 1, ss3 = 2, ss4 = 3;
    int ns0 = 2, ns1 = 0, ns2 = 1;
    CellN1<T> cur[2], nxt[2];
#pragma unroll
    for (int c = 0; c < 2; c++) cur[c] = nxt[c] = CellN1<T>{T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};

    for (int r = base; r < ye; r++) {
        {
            // ---- load phase: row r+2 of F(n) and the level-n macros, row r+3 of s(n)
            T fa[9], fb[9];
#pragma unroll
            for (int i = 0; i < 9; i++) { fa[i] = pFa[i]; fb[i] = pFb[i]; }
            const T sna = pSa, snb = pSb;
            T a2[2][3];
#pragma unroll
            for (int c = 0; c < 2; c++)
#pragma unroll
                for (int k = 0; k < 3; k++) a2[c][k] = pA[c][k];
            if (r + 1 < ye) fetch(r + 1);
            gA[0 * NT + t] = Vec2<T>::make(fa[4], fb[4]);
            gA[1 * NT + t] = Vec2<T>::make(fa[7], fb[7]);
            gA[2 * NT + t] = Vec2<T>::make(fa[8], fb[8]);
            gB[(bs2 * 3 + 0) * NT + t] = Vec2<T>::make(fa[0], fb[0]);
            gB[(bs2 * 3 + 1) * NT + t] = Vec2<T>::make(fa[1], fb[1]);
            gB[(bs2 * 3 + 2) * NT + t] = Vec2<T>::make(fa[3], fb[3]);
            gC[(fs2 * 3 + 0) * NT + t] = Vec2<T>::make(fa[2], fb[2]);
            gC[(fs2 * 3 + 1) * NT + t] = Vec2<T>::make(fa[5], fb[5]);
            gC[(fs2 * 3 + 2) * NT + t] = Vec2<T>::make(fa[6], fb[6]);
            const int mr = map_row(r + 2, kp);
            T m[2][4];
            auto macros = [&](const T *f, T sv, int o, T *mm) {
                if (o >= 0) {
                    T jx, jy;
                    moments(f, mm[0], jx, jy);
                    const T ir = fdiv(T(1), mm[0]);
                    mm[1] = jx * ir;
                    mm[2] = jy * ir;
                    mm[3] = cs.theta(mm[0], sv);
                } else {
                    const int sd = -o - 1;
                    mm[0] = side.rho(sd); mm[1] = side.ux(sd); mm[2] = side.uy(sd); mm[3] = side.th(sd);
                }
            };
            macros(fa, sPa, join_map(mr, mcLa, pitch), m[0]);
            macros(fb, sPb, join_map(mr, mcLb, pitch), m[1]);
#pragma unroll
            for (int k = 0; k < 4; k++) rM[(fs2 * 4 + k) * NT + t] = Vec2<T>::make(m[0][k], m[1][k]);
            rS[ss4 * NT + t] = Vec2<T>::make(sna, snb);
            sPa = sna;
            sPb = snb;
            __syncthreads();

            // ---- phase 2: level n+1 of row r+1 on pair q = t + 1
            const int y2 = r + 1;
            if (y2 >= ys - 1 && do2) {
                const int q = t + 1;
                // level-n macros: rho at the pair, u and theta at pairs q-1, q, q+1 and rows y2 +- 1
                const V rho0 = rM[(fs1 * 4 + 0) * NT + q];
                V mc[3][3], ms[3], mn[3];  // [field ux, uy, th][pair q-1, q, q+1]
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    mc[k][0] = rM[(fs1 * 4 + 1 + k) * NT + q - 1];
                    mc[k][1] = rM[(fs1 * 4 + 1 + k) * NT + q];
                    mc[k][2] = rM[(fs1 * 4 + 1 + k) * NT + q + 1];
                    ms[k] = rM[(fs0 * 4 + 1 + k) * NT + q];
                    mn[k] = rM[(fs2 * 4 + 1 + k) * NT + q];
                }
                // s: pairs q-1 .. q+1 of row y2, pair q of rows y2-2 .. y2+2
                const V sc0 = rS[ss2 * NT + q - 1], sc1 = rS[ss2 * NT + q], sc2 = rS[ss2 * NT + q + 1];
                const V sS2 = rS[ss0 * NT + q], sS1 = rS[ss1 * NT + q], sN1 = rS[ss3 * NT + q], sN2 = rS[ss4 * NT + q];
                // pull: F_i from (x - c_ix, y - c_iy): F_0,1,3 of row y2 (bs1), F_2,5,6 of
                // row y2-1 (fs0), F_4,7,8 of row y2+1
                T ga[9], gb[9];
                {
                    const V f0 = gB[(bs1 * 3 + 0) * NT + q], f2 = gC[(fs0 * 3 + 0) * NT + q], f4 = gA[0 * NT + q];
                    ga[0] = f0.x; gb[0] = f0.y;
                    ga[2] = f2.x; gb[2] = f2.y;
                    ga[4] = f4.x; gb[4] = f4.y;
                    // c_x = +1 (1, 5, 8): from x-1
                    const V f1l = gB[(bs1 * 3 + 1) * NT + q - 1], f1c = gB[(bs1 * 3 + 1) * NT + q];
                    const V f5l = gC[(fs0 * 3 + 1) * NT + q - 1], f5c = gC[(fs0 * 3 + 1) * NT + q];
                    const V f8l = gA[2 * NT + q - 1], f8c = gA[2 * NT + q];
                    ga[1] = f1l.y; gb[1] = f1c.x;
                    ga[5] = f5l.y; gb[5] = f5c.x;
                    ga[8] = f8l.y; gb[8] = f8c.x;
                    // c_x = -1 (3, 6, 7): from x+1
                    const V f3c = gB[(bs1 * 3 + 2) * NT + q], f3r = gB[(bs1 * 3 + 2) * NT + q + 1];
                    const V f6c = gC[(fs0 * 3 + 2) * NT + q], f6r = gC[(fs0 * 3 + 2) * NT + q + 1];
                    const V f7c = gA[1 * NT + q], f7r = gA[1 * NT + q + 1];
                    ga[3] = f3c.y; gb[3] = f3r.x;
                    ga[6] = f6c.y; gb[6] = f6r.x;
                    ga[7] = f7c.y; gb[7] = f7r.x;
                }
                nxt[0] = level_np1<T, SIG, PHI0>(cs, rho0.x, mc[0][1].x, mc[1][1].x, mc[2][1].x,
                                                 mc[0][0].y, mc[0][1].y, ms[0].x, mn[0].x,
                                                 mc[1][0].y, mc[1][1].y, ms[1].x, mn[1].x,
                                                 mc[2][0].y, mc[2][1].y, ms[2].x, mn[2].x,
                                                 sc0.x, sc0.y, sc1.x, sc1.y, sc2.x, sS2.x, sS1.x, sN1.x, sN2.x,
                                                 a2[0][0], a2[0][1], a2[0][2], ga);
                nxt[1] = level_np1<T, SIG, PHI0>(cs, rho0.y, mc[0][1].y, mc[1][1].y, mc[2][1].y,
                                                 mc[0][1].x, mc[0][2].x, ms[0].y, mn[0].y,
                                                 mc[1][1].x, mc[1][2].x, ms[1].y, mn[1].y,
                                                 mc[2][1].x, mc[2][2].x, ms[2].y, mn[2].y,
                                                 sc0.y, sc1.x, sc1.y, sc2.x, sc2.y, sS2.y, sS1.y, sN1.y, sN2.y,
                                                 a2[1][0], a2[1][1], a2[1][2], gb);
                // Dirichlet cells hold the side's constants
                const bool out2y = y2 < 0 || y2 >= kp.ny;
                const int side2y = y2 < 0 ? 2 : 3;
                const bool dir2y = out2y && kp.bc[side2y] == BC_DIRICHLET;
#pragma unroll
                for (int c = 0; c < 2; c++) {
                    if (dir2y || dir2[c]) {
                        const int sd = dir2y ? side2y : side2[c];
                        nxt[c].rho = side.rho(sd); nxt[c].ux = side.ux(sd); nxt[c].uy = side.uy(sd);
                        nxt[c].th = side.th(sd); nxt[c].s = side.s_(sd);
                    }
                }
                rN[(ns2 * 4 + 0) * NT + q] = Vec2<T>::make(nxt[0].rho, nxt[1].rho);
                rN[(ns2 * 4 + 1) * NT + q] = Vec2<T>::make(nxt[0].ux, nxt[1].ux);
                rN[(ns2 * 4 + 2) * NT + q] = Vec2<T>::make(nxt[0].uy, nxt[1].uy);
                rN[(ns2 * 4 + 3) * NT + q] = Vec2<T>::make(nxt[0].th, nxt[1].th);
            }
        }
        __syncthreads();

        // ---- phase 3: row r on pair q = t + 1 (own values from the previous iteration)
        if (r >= ys && do3) {
            const int q = t + 1;
            const bool zS = r == 0 && kp.bc[2] == BC_ZEROGRAD;
            const bool zN = r == kp.ny - 1 && kp.bc[3] == BC_ZEROGRAD;
            V nW[4], nE[4], nS[4], nN[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                nW[k] = rN[(ns1 * 4 + k) * NT + q - 1];
                nE[k] = rN[(ns1 * 4 + k) * NT + q + 1];
                nS[k] = rN[(ns0 * 4 + k) * NT + q];
                nN[k] = rN[(ns2 * 4 + k) * NT + q];
            }
            const CellN1<T> &A = cur[0], &B = cur[1];
            // cell a: west = pair q-1 (.y), east = cell b; cell b: west = cell a, east = pair q+1 (.x)
            const T aWr = zgW ? A.rho : nW[0].y, aWux = zgW ? A.ux : nW[1].y, aWuy = zgW ? A.uy : nW[2].y,
                    aWth = zgW ? A.th : nW[3].y;
            const T aEr = zgEa ? A.rho : B.rho, aEux = zgEa ? A.ux : B.ux, aEuy = zgEa ? A.uy : B.uy,
                    aEth = zgEa ? A.th : B.th;
            const T bEr = zgEb ? B.rho : nE[0].x, bEux = zgEb ? B.ux : nE[1].x, bEuy = zgEb ? B.uy : nE[2].x,
                    bEth = zgEb ? B.th : nE[3].x;
            T fa[9], fb[9], aa[3], ab[3];
            if (v3a) {
                collide_cell<T, SIG>(cs, cen, A, aWr, aWux, aWuy, aWth, aEr, aEux, aEuy, aEth,
                                     zS ? A.rho : nS[0].x, zS ? A.ux : nS[1].x, zS ? A.uy : nS[2].x, zS ? A.th : nS[3].x,
                                     zN ? A.rho : nN[0].x, zN ? A.ux : nN[1].x, zN ? A.uy : nN[2].x, zN ? A.th : nN[3].x,
                                     fa, aa[0], aa[1], aa[2]);
            }
            if (v3b) {
                collide_cell<T, SIG>(cs, cen, B, A.rho, A.ux, A.uy, A.th, bEr, bEux, bEuy, bEth,
                                     zS ? B.rho : nS[0].y, zS ? B.ux : nS[1].y, zS ? B.uy : nS[2].y, zS ? B.th : nS[3].y,
                                     zN ? B.rho : nN[0].y, zN ? B.ux : nN[1].y, zN ? B.uy : nN[2].y, zN ? B.th : nN[3].y,
                                     fb, ab[0], ab[1], ab[2]);
            }
            const long long o = (long long)r * pitch + gx2;
            if (v3a && v3b) {
                raw *dF = outF + o;
#pragma unroll
                for (int i = 0; i < 9; i++)
                    *reinterpret_cast<raw2 *>(dF + i * P) = S::pack(S::put(fa[i], i, kp), S::put(fb[i], i, kp));
                T *dA = outA + o;
                *reinterpret_cast<V *>(dA + A_S * P) = Vec2<T>::make(A.s, B.s);
#pragma unroll
                for (int k = 0; k < 3; k++) *reinterpret_cast<V *>(dA + (A_XX + k) * P) = Vec2<T>::make(aa[k], ab[k]);
            } else if (v3a) {
                raw *dF = outF + o;
#pragma unroll
                for (int i = 0; i < 9; i++) dF[i * P] = S::put(fa[i], i, kp);
                T *dA = outA + o;
                dA[A_S * P] = A.s;
#pragma unroll
                for (int k = 0; k < 3; k++) dA[(A_XX + k) * P] = aa[k];
            }
        }
        // next row: the values computed in phase 2 become the cells' own
#pragma unroll
        for (int c = 0; c < 2; c++) cur[c] = nxt[c];
        {
            const int f = fs0; fs0 = fs1; fs1 = fs2; fs2 = f;
            const int b = bs1; bs1 = bs2; bs2 = b;
            const int sx = ss0; ss0 = ss1; ss1 = ss2; ss2 = ss3; ss3 = ss4; ss4 = sx;
            const int n = ns0; ns0 = ns1; ns1 = ns2; ns2 = n;
        }
    }
}

// One case: blockIdx.x picks the strip, blockIdx.y the row segment.
template <typename T, typename S, int NT, int MINB, bool SIG, bool PHI0>
__global__ void __launch_bounds__(NT, MINB)
march_pair_kernel(const typename S::raw *__restrict__ inF, const T *__restrict__ inA,
                  typename S::raw *__restrict__ outF, T *__restrict__ outA, const KParams kp, const int nseg)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ys = seg_start(blockIdx.y, nseg, kp.ny), ye = seg_start(blockIdx.y + 1, nseg, kp.ny);
    march_pair_segment<T, S, NT, SIG, PHI0>(inF, inA, outF, outA, kp, blockIdx.x * PairGeom<T, NT>::W, ys, ye,
                                            smem_raw);
}

// ---- many cases in one persistent launch (FP32) ---------------------------------
// The (case, strip, segment) items of all cases form one list that a grid
// of resident CTAs walks; the parameters of an item's case are copied to
// shared memory behind the rings.
struct MarchItem {
    int c, x0, ys, ye;
};

struct MarchTables {
    const KParams *kps;        // [ncase]
    const CasePlanes *planes;  // [ncase]
    const MarchItem *items;    // [nitems]
    int nitems;
};

template <int NT, int MINB, bool SIG, bool PHI0>
__global__ void __launch_bounds__(NT, MINB)
batched_march_kernel(const MarchTables tab, const int parity)
{
    using G = PairGeom<float, NT>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    KParams &skp = *reinterpret_cast<KParams *>(smem_raw + (G::smem_bytes + 15) / 16 * 16);
    int loaded = -1;
    for (int i = blockIdx.x; i < tab.nitems; i += gridDim.x) {
        const MarchItem it = tab.items[i];
        __syncthreads();  // the previous segment is done with the rings and the parameters
        if (it.c != loaded) {
            const int *src = reinterpret_cast<const int *>(tab.kps + it.c);
            int *dst = reinterpret_cast<int *>(&skp);
            for (int w = threadIdx.x; w < (int)(sizeof(KParams) / sizeof(int)); w += NT) dst[w] = __ldg(src + w);
            loaded = it.c;
            __syncthreads();
        }
        const CasePlanes &pl = tab.planes[it.c];
        march_pair_segment<float, FullStore<float>, NT, SIG, PHI0>(pl.inF[parity], pl.inA[parity], pl.outF[parity],
                                                                  pl.outA[parity], skp, it.x0, it.ys, it.ye,
                                                                  smem_raw);
    }
}

}  // namespace hlbm
