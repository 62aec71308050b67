// hlbm_march.cuh -- the fused time step of Algorithm 1 as a
// row-marching kernel: each CTA owns a strip of columns and walks down a
// segment of rows, so that only the x halo is loaded and computed twice
// (a tiled kernel recomputes a halo in both directions).
//
// Per row r of the segment one iteration does, separated by two barriers:
//   load:    F(n) of row r+2 and s(n) of row r+3 (prefetched into registers
//            one iteration earlier), the level-n rho, u, theta of row r+2
//            (local moments of F(n), theta from s(n) of the same cell)
//   phase 2: level n+1 of row r+1: the entropy update (eq sequaalgo),
//            pull-streaming and moments (eqs streamalgo, rhoalgo, ualgo),
//            theta (eq Entropie expression), and
//            the second moments of the pulled populations when sigma > 0
//   phase 3: row r: E1, E2, a1 and the regularised collision (eqs Psialgo,
//            Equilibrium, a1sigalgo, streamalgo),
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

#include <type_traits>

#include "hlbm_device.cuh"
#include "hlbm_pack.cuh"

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

// The periodic image of i in [0, n) (a division only for i outside).
__device__ __forceinline__ int wrap_per(int i, int n) { return (unsigned)i < (unsigned)n ? i : wrapi(i, n); }

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

// Pull, moments, entropy and theta of level n+1 for one cell (the arithmetic
// of phase 2 of the tiled kernel).
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

// psi, f^eq, a1 and the next collision for one cell (phase 3 of the tiled
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
template <typename T, typename S, int NT, bool SIG, bool PHI0, bool PER>
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
    // PER (all four sides periodic, ny >= 4): every index map is a wrap, and
    // the boundary selections below are compiled out; the rows a segment
    // reads lie within [-3, ny + 3), one period from the domain at most
    auto mrow = [&](int gy) {
        return PER ? (gy < 0 ? gy + kp.ny : (gy >= kp.ny ? gy - kp.ny : gy)) : map_row(gy, kp);
    };

    // load-phase pair t: columns gxL, gxL + 1
    const int gxL = x0 - 4 + 2 * t;
    const int mcLa = PER ? wrap_per(gxL, kp.nx) : map_col(gxL, kp), mcLb = PER ? wrap_per(gxL + 1, kp.nx) : map_col(gxL + 1, kp);
    const bool vecL = gxL >= 0 && gxL + 1 < kp.nx;
    // phase-2 / phase-3 pair q = t + 1: columns gx2, gx2 + 1
    const int gx2 = gxL + 2;
    const bool do2 = t < NT - 2;
    const int mc2a = PER ? wrap_per(gx2, kp.nx) : map_col(gx2, kp), mc2b = PER ? wrap_per(gx2 + 1, kp.nx) : map_col(gx2 + 1, kp);
    const bool vec2 = gx2 >= 0 && gx2 + 1 < kp.nx;
    // Dirichlet x sides: level n+1 beyond them is the side's state
    bool dir2[2];
    int side2[2];
#pragma unroll
    for (int c = 0; c < 2; c++) {
        const int gx = gx2 + c;
        side2[c] = gx < 0 ? 0 : 1;
        dir2[c] = !PER && (gx < 0 || gx >= kp.nx) && kp.bc[side2[c]] == BC_DIRICHLET;
    }
    const bool do3 = t >= 1 && t <= G::NP;
    const bool v3a = do3 && gx2 < kp.nx, v3b = do3 && gx2 + 1 < kp.nx;
    // zero-gradient x sides: the neighbour beyond the edge is the edge cell itself
    const bool zgW = !PER && gx2 == 0 && kp.bc[0] == BC_ZEROGRAD;             // west of cell a
    const bool zgEa = !PER && gx2 == kp.nx - 1 && kp.bc[1] == BC_ZEROGRAD;    // east of cell a
    const bool zgEb = !PER && gx2 + 1 == kp.nx - 1 && kp.bc[1] == BC_ZEROGRAD; // east of cell b

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
            const bool ok = HLBM_CELL_OK(mr, gxL, 2, kp, 1);
#pragma unroll
            for (int i = 0; i < 9; i++) {
                const raw2 v = ok ? *reinterpret_cast<const raw2 *>(src + i * P) : S::pack(S::put(T(0), i, kp), S::put(T(0), i, kp));
                fa[i] = S::get(v.x, i, kp);
                fb[i] = S::get(v.y, i, kp);
            }
        } else {
            const int oa = join_map(mr, mcLa, pitch), ob = join_map(mr, mcLb, pitch);
            const bool oka = oa < 0 || HLBM_CELL_OK(oa / pitch, oa % pitch, 1, kp, 1);
            const bool okb = ob < 0 || HLBM_CELL_OK(ob / pitch, ob % pitch, 1, kp, 1);
#pragma unroll
            for (int i = 0; i < 9; i++) {
                fa[i] = oa >= 0 ? (oka ? S::get(inF[oa + i * P], i, kp) : T(0)) : side.F(-oa - 1, i);
                fb[i] = ob >= 0 ? (okb ? S::get(inF[ob + i * P], i, kp) : T(0)) : side.F(-ob - 1, i);
            }
        }
    };
    auto load_s = [&](int mr, T &sa, T &sb) {
        if (mr >= 0 && vecL) {
            const bool ok = HLBM_CELL_OK(mr, gxL, 2, kp, 2);
            const V v = ok ? *reinterpret_cast<const V *>(inA + A_S * P + ((long long)mr * pitch + gxL))
                           : Vec2<T>::make(T(0), T(0));
            sa = v.x;
            sb = v.y;
        } else {
            const int oa = join_map(mr, mcLa, pitch), ob = join_map(mr, mcLb, pitch);
            const bool oka = oa < 0 || HLBM_CELL_OK(oa / pitch, oa % pitch, 1, kp, 2);
            const bool okb = ob < 0 || HLBM_CELL_OK(ob / pitch, ob % pitch, 1, kp, 2);
            sa = oa >= 0 ? (oka ? inA[A_S * P + oa] : T(0)) : side.s_(-oa - 1);
            sb = ob >= 0 ? (okb ? inA[A_S * P + ob] : T(0)) : side.s_(-ob - 1);
        }
    };
    auto fetch = [&](int r) {
        load_F(mrow(r + 2), pFa, pFb);
        load_s(mrow(r + 3), pSa, pSb);
        if (PHI0 && do2) {
            const int mr = mrow(r + 1);
            if (mr >= 0 && vec2) {
                const T *src = inA + ((long long)mr * pitch + gx2);
                const bool ok = HLBM_CELL_OK(mr, gx2, 2, kp, 3);
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    const V v = ok ? *reinterpret_cast<const V *>(src + (A_XX + k) * P) : Vec2<T>::make(T(0), T(0));
                    pA[0][k] = v.x;
                    pA[1][k] = v.y;
                }
            } else {
                const int oa = join_map(mr, mc2a, pitch), ob = join_map(mr, mc2b, pitch);
                const bool oka = oa >= 0 && HLBM_CELL_OK(oa / pitch, oa % pitch, 1, kp, 3);
                const bool okb = ob >= 0 && HLBM_CELL_OK(ob / pitch, ob % pitch, 1, kp, 3);
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    pA[0][k] = oka ? inA[(A_XX + k) * P + oa] : T(0);
                    pA[1][k] = okb ? inA[(A_XX + k) * P + ob] : T(0);
                }
            }
        }
    };

    // s(n) of rows ys-3 and ys-2 (the latter kept for the level-n theta of row ys-2)
    T sPa = T(0), sPb = T(0);
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const int gy = ys - 3 + k;
        load_s(mrow(gy), sPa, sPb);
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
#ifdef HLBM_DEBUG
        // ring slots within their rings; the neighbour pairs of phases 2 and 3 inside the CTA
        {
            const int slots[14] = {fs0, fs1, fs2, bs1, bs2, ss0, ss1, ss2, ss3, ss4, ns0, ns1, ns2, 0};
            const int depth[14] = {3, 3, 3, 2, 2, 5, 5, 5, 5, 5, 3, 3, 3, 1};
            for (int k = 0; k < 14; k++) HLBM_RANGE_OK(slots[k], depth[k], 5);
        }
        if (do2) HLBM_RANGE_OK(t + 2, NT, 6);  // phase 2 reads pairs q - 1 .. q + 1, q = t + 1
#endif
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
            const int mr = mrow(r + 2);
            T m[2][4];
            // FP64: the level-n rho, u, theta of a cell are the level-(n+1)
            // values that phase 2 of the previous step computed (the
            // collision conserves rho and rho u, eqs. rhoalgo, ualgo), kept in
            // the cache planes A_RHO .. A_TH; a Dirichlet position holds the
            // side's state
            auto cached = [&](int o, T *mm) {
                if (o >= 0) {
                    const bool ok = HLBM_CELL_OK(o / pitch, o % pitch, 1, kp, 1);
#pragma unroll
                    for (int k = 0; k < 4; k++) mm[k] = ok ? inA[(A_RHO + k) * P + o] : T(0);
                } else {
                    const int sd = -o - 1;
                    mm[0] = side.rho(sd); mm[1] = side.ux(sd); mm[2] = side.uy(sd); mm[3] = side.th(sd);
                }
            };
            if constexpr (std::is_same<T, float>::value) {
                // both cells at once (packed FP32)
                f2 g[9];
#pragma unroll
                for (int i = 0; i < 9; i++) g[i] = mk2(fa[i], fb[i]);
                f2 rho, jx, jy;
                moments2(g, rho, jx, jy);
                const f2 ir = rcp2(rho);
                const f2 ux = jx * ir, uy = jy * ir, th = theta2(cs, rho, mk2(sPa, sPb));
                m[0][0] = rho.x; m[0][1] = ux.x; m[0][2] = uy.x; m[0][3] = th.x;
                m[1][0] = rho.y; m[1][1] = ux.y; m[1][2] = uy.y; m[1][3] = th.y;
                const int oa = join_map(mr, mcLa, pitch), ob = join_map(mr, mcLb, pitch);
                if (!PER && oa < 0) { const int sd = -oa - 1; m[0][0] = side.rho(sd); m[0][1] = side.ux(sd); m[0][2] = side.uy(sd); m[0][3] = side.th(sd); }
                if (!PER && ob < 0) { const int sd = -ob - 1; m[1][0] = side.rho(sd); m[1][1] = side.ux(sd); m[1][2] = side.uy(sd); m[1][3] = side.th(sd); }
            } else {
                cached(join_map(mr, mcLa, pitch), m[0]);
                cached(join_map(mr, mcLb, pitch), m[1]);
            }
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
                if constexpr (std::is_same<T, float>::value) {
                    // both cells at once (packed FP32): lane x = cell a, lane y = cell b
                    f2 C[3], Wv[3], Ev[3], Sv[3], Nv[3];
#pragma unroll
                    for (int k = 0; k < 3; k++) {
                        C[k] = from2(mc[k][1]);
                        Wv[k] = mk2(mc[k][0].y, mc[k][1].x);
                        Ev[k] = mk2(mc[k][1].y, mc[k][2].x);
                        Sv[k] = from2(ms[k]);
                        Nv[k] = from2(mn[k]);
                    }
                    f2 g2[9];
#pragma unroll
                    for (int i = 0; i < 9; i++) g2[i] = mk2(ga[i], gb[i]);
                    const CellN1x2 n2 = level_np1_2<SIG, PHI0>(
                        cs, from2(rho0), C[0], C[1], C[2], Wv[0], Ev[0], Sv[0], Nv[0], Wv[1], Ev[1], Sv[1], Nv[1], Wv[2],
                        Ev[2], Sv[2], Nv[2], from2(sc0), mk2(sc0.y, sc1.x), from2(sc1), mk2(sc1.y, sc2.x), from2(sc2),
                        from2(sS2), from2(sS1), from2(sN1), from2(sN2), mk2(a2[0][0], a2[1][0]), mk2(a2[0][1], a2[1][1]),
                        mk2(a2[0][2], a2[1][2]), g2);
                    nxt[0] = CellN1<T>{n2.rho.x, n2.ux.x, n2.uy.x, n2.th.x, n2.s.x, n2.mxx.x, n2.myy.x, n2.mxy.x};
                    nxt[1] = CellN1<T>{n2.rho.y, n2.ux.y, n2.uy.y, n2.th.y, n2.s.y, n2.mxx.y, n2.myy.y, n2.mxy.y};
                } else {
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
                }
                // Dirichlet cells hold the side's constants
                const bool out2y = y2 < 0 || y2 >= kp.ny;
                const int side2y = y2 < 0 ? 2 : 3;
                const bool dir2y = !PER && out2y && kp.bc[side2y] == BC_DIRICHLET;
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
            const bool zS = !PER && r == 0 && kp.bc[2] == BC_ZEROGRAD;
            const bool zN = !PER && r == kp.ny - 1 && kp.bc[3] == BC_ZEROGRAD;
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
            if constexpr (std::is_same<T, float>::value) {
                // both cells at once (packed FP32); the neighbours of cell a are (W, E) =
                // (west pair or a, b) and of cell b (a, east pair or b)
                const f2 cr = mk2(A.rho, B.rho), cux = mk2(A.ux, B.ux), cuy = mk2(A.uy, B.uy), cth = mk2(A.th, B.th);
                const f2 wr = mk2(aWr, A.rho), wux = mk2(aWux, A.ux), wuy = mk2(aWuy, A.uy), wth = mk2(aWth, A.th);
                const f2 er = mk2(aEr, bEr), eux = mk2(aEux, bEux), euy = mk2(aEuy, bEuy), eth = mk2(aEth, bEth);
                const f2 sr = zS ? cr : from2(nS[0]), sux = zS ? cux : from2(nS[1]), suy = zS ? cuy : from2(nS[2]),
                         sth = zS ? cth : from2(nS[3]);
                const f2 nr = zN ? cr : from2(nN[0]), nux = zN ? cux : from2(nN[1]), nuy = zN ? cuy : from2(nN[2]),
                         nth = zN ? cth : from2(nN[3]);
                const f2 half = bc2(0.5f);
                const f2 dxux = half * (eux - wux), dyux = half * (nux - sux);
                const f2 dxuy = half * (euy - wuy), dyuy = half * (nuy - suy);
                f2 ex, ey, om;
                closure_terms2(cs, cen, cr, cux, cuy, cth, wr, wux, wth, er, eux, eth, sr, suy, sth, nr, nuy, nth, ex, ey,
                               om);
                const CellN1x2 c2{cr, cux, cuy, cth, mk2(A.s, B.s), mk2(A.mxx, B.mxx), mk2(A.myy, B.myy),
                                  mk2(A.mxy, B.mxy)};
                f2 axx, axy, ayy, fo[9];
                a1_next2<SIG>(cs, c2, dxux, dyux, dxuy, dyuy, ex, ey, axx, axy, ayy);
                build_populations2(cr, cux, cuy, cth, axx, axy, ayy, ex, ey, om, fo);
#pragma unroll
                for (int i = 0; i < 9; i++) { fa[i] = fo[i].x; fb[i] = fo[i].y; }
                aa[0] = axx.x; aa[1] = axy.x; aa[2] = ayy.x;
                ab[0] = axx.y; ab[1] = axy.y; ab[2] = ayy.y;
            } else {
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
            }
            const long long o = (long long)r * pitch + gx2;
            const bool okst = !v3a || HLBM_CELL_OK(r, gx2, v3b ? 2 : 1, kp, 4);  // checked where a store happens
            if (!okst) {
            } else if (v3a && v3b) {
                raw *dF = outF + o;
#pragma unroll
                for (int i = 0; i < 9; i++)
                    *reinterpret_cast<raw2 *>(dF + i * P) = S::pack(S::put(fa[i], i, kp), S::put(fb[i], i, kp));
                T *dA = outA + o;
                *reinterpret_cast<V *>(dA + A_S * P) = Vec2<T>::make(A.s, B.s);
#pragma unroll
                for (int k = 0; k < 3; k++) *reinterpret_cast<V *>(dA + (A_XX + k) * P) = Vec2<T>::make(aa[k], ab[k]);
                if constexpr (std::is_same<T, double>::value) {
                    // the cache planes: this row's level n+1, the next step's level n
                    *reinterpret_cast<V *>(dA + A_RHO * P) = Vec2<T>::make(A.rho, B.rho);
                    *reinterpret_cast<V *>(dA + A_UX * P) = Vec2<T>::make(A.ux, B.ux);
                    *reinterpret_cast<V *>(dA + A_UY * P) = Vec2<T>::make(A.uy, B.uy);
                    *reinterpret_cast<V *>(dA + A_TH * P) = Vec2<T>::make(A.th, B.th);
                }
            } else if (v3a) {
                raw *dF = outF + o;
#pragma unroll
                for (int i = 0; i < 9; i++) dF[i * P] = S::put(fa[i], i, kp);
                T *dA = outA + o;
                dA[A_S * P] = A.s;
#pragma unroll
                for (int k = 0; k < 3; k++) dA[(A_XX + k) * P] = aa[k];
                if constexpr (std::is_same<T, double>::value) {
                    dA[A_RHO * P] = A.rho; dA[A_UX * P] = A.ux; dA[A_UY * P] = A.uy; dA[A_TH * P] = A.th;
                }
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

// One case: blockIdx.x picks the strip, blockIdx.y the row segment.  PER:
// all four sides periodic and ny >= 4 (the boundary selections compiled
// out).
template <typename T, typename S, int NT, int MINB, bool SIG, bool PHI0, bool PER = false>
__global__ void __launch_bounds__(NT, MINB)
march_pair_kernel(const typename S::raw *__restrict__ inF, const T *__restrict__ inA,
                  typename S::raw *__restrict__ outF, T *__restrict__ outA, const KParams kp, const int nseg)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ys = seg_start(blockIdx.y, nseg, kp.ny), ye = seg_start(blockIdx.y + 1, nseg, kp.ny);
    march_pair_segment<T, S, NT, SIG, PHI0, PER>(inF, inA, outF, outA, kp, blockIdx.x * PairGeom<T, NT>::W, ys, ye,
                                                 smem_raw);
}

// FP64 row-marching form: the cache planes of a state whose level-n values
// no step has stored yet (after init or a checkpoint is set).  Per cell,
// rho and u are the moments of F(n) (eqs. rhoalgo, ualgo) and theta follows
// from rho and s(n) (eq. Entropie expression): the arithmetic the load phase
// would do.  One thread per cell of the interior; pad columns stay as they are.
__global__ void cache_macros_kernel(const double *__restrict__ F, double *__restrict__ A, const KParams kp)
{
    const long long n = (long long)kp.nx * kp.ny;
    const long long P = kp.plane;
    Consts<double> cs;
    cs.load(kp);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / kp.nx), x = (int)(i % kp.nx);
        const long long o = (long long)y * kp.pitch + x;
        double f[9], rho, jx, jy;
#pragma unroll
        for (int k = 0; k < 9; k++) f[k] = F[o + k * P];
        moments(f, rho, jx, jy);
        const double ir = fdiv(1.0, rho);
        A[A_RHO * P + o] = rho;
        A[A_UX * P + o] = jx * ir;
        A[A_UY * P + o] = jy * ir;
        A[A_TH * P + o] = cs.theta(rho, A[A_S * P + o]);
    }
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

template <int NT, int MINB, bool SIG, bool PHI0, bool PER = false>
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
        march_pair_segment<float, FullStore<float>, NT, SIG, PHI0, PER>(pl.inF[parity], pl.inA[parity],
                                                                       pl.outF[parity], pl.outA[parity], skp, it.x0,
                                                                       it.ys, it.ye, smem_raw);
    }
}

// ---- moment-state form (HLBM_FP32_MOMENTS) -------------------------------------------
// The state holds 7 FP32 planes per cell instead of 13: rho, u_x, u_y, s,
// a1_xx, a1_xy, a1_yy (56 B read + written per cell-update instead of 104).
// In the regularised scheme the post-collision populations are a function
// of the level's macros and a1 (Sec. 3.4: only a1 needs keeping), so each
// step rebuilds F(n) once per cell from the stored moments -- the arithmetic
// of the collision that ended the previous step -- and ends with a1(n+1)
// instead of a collision.  Per row r of the segment, three barriers apart:
//   load:    rho, u, s, a1 of row r+3 (prefetched one iteration earlier);
//            theta; the level-n macros of row r+3
//   rebuild: F(n) of row r+2 from the level-n macros of rows r+1 .. r+3
//            (E1, E2, omega) and its own a1; a Dirichlet position holds
//            the side's equilibrium
//   phase 2: level n+1 of row r+1 (as in the population form); a pull
//            from beyond a zero-gradient side reads the edge cell, which is
//            where the population form's index map takes the populations
//   phase 3: a1(n+1) of row r (a1^FD, blended with a1^PR when sigma > 0),
//            written with rho, u and s of level n+1.
// Ring columns x0-6 .. x0+2NT-7: load on pairs 0 .. NT-1, rebuild on
// 1 .. NT-2, phase 2 on 2 .. NT-3, phase 3 on the W = 2 (NT - 6) columns of
// pairs 3 .. NT-4.
constexpr int MS_RHO = 0, MS_UX = 1, MS_UY = 2, MS_S = 3, MS_AXX = 4, MS_AXY = 5, MS_AYY = 6, MS_NPLANE = 7;

template <int NT>
struct MomGeom {
    static constexpr int NP = NT - 6;
    static constexpr int W = 2 * NP;
    static constexpr int CW = 2 * NT;
    static constexpr int OFF_GA = 0;                  // [2][3][CW]  F_4, F_7, F_8 of rows r+1, r+2
    static constexpr int OFF_GB = OFF_GA + 6 * CW;    // [2][3][CW]  F_0, F_1, F_3 of rows r+1, r+2
    static constexpr int OFF_GC = OFF_GB + 6 * CW;    // [3][3][CW]  F_2, F_5, F_6 of rows r .. r+2
    static constexpr int OFF_M = OFF_GC + 9 * CW;     // [4][4][CW]  rho, u_x, u_y, theta of rows r .. r+3
    static constexpr int OFF_S = OFF_M + 16 * CW;     // [5][CW]     s of rows r-1 .. r+3
    static constexpr int OFF_N = OFF_S + 5 * CW;      // [3][4][CW]  level n+1 of rows r-1 .. r+1
    static constexpr int N = OFF_N + 12 * CW;
    static constexpr size_t smem_bytes = sizeof(float) * (size_t)N;
};

template <int NT, bool SIG, bool PHI0, bool PER>
__device__ __forceinline__ void moment_segment(const float *__restrict__ in, float *__restrict__ out,
                                               const KParams &kp, const int x0, const int ys, const int ye,
                                               unsigned char *smem_raw)
{
    using G = MomGeom<NT>;
    using V = float2;
    float *const sm = reinterpret_cast<float *>(smem_raw);
    V *const gA = reinterpret_cast<V *>(sm + G::OFF_GA);  // [2][3][NT]
    V *const gB = reinterpret_cast<V *>(sm + G::OFF_GB);  // [2][3][NT]
    V *const gC = reinterpret_cast<V *>(sm + G::OFF_GC);  // [3][3][NT]
    V *const rM = reinterpret_cast<V *>(sm + G::OFF_M);   // [4][4][NT]
    V *const rS = reinterpret_cast<V *>(sm + G::OFF_S);   // [5][NT]
    V *const rN = reinterpret_cast<V *>(sm + G::OFF_N);   // [3][4][NT]

    Consts<float> cs;
    cs.load(kp);
    const Side<float> side{kp};
    const bool cen = kp.e1_centred != 0;
    const long long P = kp.plane;
    const int pitch = kp.pitch;
    const int t = threadIdx.x;
    const int base = ys - 6;
    // PER (all four sides periodic): every index map is a wrap, and the
    // boundary selections below are compiled out
    auto mrow = [&](int gy) { return PER ? wrap_per(gy, kp.ny) : map_row(gy, kp); };

    // load / rebuild pair t: columns gxL, gxL + 1
    const int gxL = x0 - 6 + 2 * t;
    const int mcLa = PER ? wrap_per(gxL, kp.nx) : map_col(gxL, kp), mcLb = PER ? wrap_per(gxL + 1, kp.nx) : map_col(gxL + 1, kp);
    const bool vecL = gxL >= 0 && gxL + 1 < kp.nx;
    const bool doR = t >= 1 && t <= NT - 2;
    // phase-2 / phase-3 pair q = t + 2: columns gx2, gx2 + 1
    const int q = t + 2;
    const int gx2 = gxL + 4;
    const bool do2 = t <= NT - 5;
    const int mc2a = PER ? wrap_per(gx2, kp.nx) : map_col(gx2, kp), mc2b = PER ? wrap_per(gx2 + 1, kp.nx) : map_col(gx2 + 1, kp);
    const bool vec2 = gx2 >= 0 && gx2 + 1 < kp.nx;
    bool dir2[2];
    int side2[2];
#pragma unroll
    for (int c = 0; c < 2; c++) {
        const int gx = gx2 + c;
        side2[c] = gx < 0 ? 0 : 1;
        dir2[c] = !PER && (gx < 0 || gx >= kp.nx) && kp.bc[side2[c]] == BC_DIRICHLET;
    }
    const bool do3 = t >= 1 && t <= G::NP;
    const bool v3a = do3 && gx2 < kp.nx, v3b = do3 && gx2 + 1 < kp.nx;
    // zero-gradient x sides: a neighbour (phase 3) or a pull source (phase 2)
    // beyond the edge is the edge cell itself
    const bool zgW = !PER && gx2 == 0 && kp.bc[0] == BC_ZEROGRAD;             // west of cell a
    const bool zgEa = !PER && gx2 == kp.nx - 1 && kp.bc[1] == BC_ZEROGRAD;    // east of cell a
    const bool zgEb = !PER && gx2 + 1 == kp.nx - 1 && kp.bc[1] == BC_ZEROGRAD; // east of cell b

    // prefetch registers: moments of row r+4 (load pair), a1 of row r+2 (phase-2 pair)
    float pM[2][4], pA[2][3], pA2[2][3];
#pragma unroll
    for (int c = 0; c < 2; c++) {
#pragma unroll
        for (int k = 0; k < 4; k++) pM[c][k] = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; k++) { pA[c][k] = 0.0f; pA2[c][k] = 0.0f; }
    }
    // moments of row y at the load pair; a Dirichlet position gives the side's
    // state with a1 = 0
    auto load_row = [&](int y) {
        const int mr = mrow(y);
        if (mr >= 0 && vecL && HLBM_CELL_OK(mr, gxL, 2, kp, 21)) {
            const float *src = in + ((long long)mr * pitch + gxL);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const V v = *reinterpret_cast<const V *>(src + k * P);
                pM[0][k] = v.x; pM[1][k] = v.y;
            }
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const V v = *reinterpret_cast<const V *>(src + (MS_AXX + k) * P);
                pA[0][k] = v.x; pA[1][k] = v.y;
            }
        } else {
#pragma unroll
            for (int c = 0; c < 2; c++) {
                const int o = join_map(mr, c ? mcLb : mcLa, pitch);
                if ((PER || o >= 0) && HLBM_CELL_OK(o / pitch, o % pitch, 1, kp, 21)) {
#pragma unroll
                    for (int k = 0; k < 4; k++) pM[c][k] = in[k * P + o];
#pragma unroll
                    for (int k = 0; k < 3; k++) pA[c][k] = in[(MS_AXX + k) * P + o];
                } else {
                    const int sd = -o - 1;
                    pM[c][0] = side.rho(sd); pM[c][1] = side.ux(sd); pM[c][2] = side.uy(sd); pM[c][3] = side.s_(sd);
                    pA[c][0] = pA[c][1] = pA[c][2] = 0.0f;
                }
            }
        }
    };
    // a1(n) of row y at the phase-2 pair (for Phi)
    auto load_a2 = [&](int y) {
        if (!PHI0 || !do2) return;
        const int mr = mrow(y);
        if (mr >= 0 && vec2 && HLBM_CELL_OK(mr, gx2, 2, kp, 22)) {
            const float *src = in + ((long long)mr * pitch + gx2);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const V v = *reinterpret_cast<const V *>(src + (MS_AXX + k) * P);
                pA2[0][k] = v.x; pA2[1][k] = v.y;
            }
        } else {
#pragma unroll
            for (int c = 0; c < 2; c++) {
                const int o = join_map(mr, c ? mc2b : mc2a, pitch);
                const bool ok = (PER || o >= 0) && HLBM_CELL_OK(o / pitch, o % pitch, 1, kp, 22);
#pragma unroll
                for (int k = 0; k < 3; k++) pA2[c][k] = ok ? in[(MS_AXX + k) * P + o] : 0.0f;
            }
        }
    };
    load_row(base + 3);
    load_a2(base + 1);

    float aCur[2][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};  // a1(n) of the rebuild row
    CellN1<float> cur[2], nxt[2];
#pragma unroll
    for (int c = 0; c < 2; c++) cur[c] = nxt[c] = CellN1<float>{0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};

    for (int r = base; r < ye; r++) {
        const int rel = r - base;
        // ---- load: level-n macros and s of row r+3
        float mv[2][4], an[2][3], a2[2][3];
#pragma unroll
        for (int c = 0; c < 2; c++) {
#pragma unroll
            for (int k = 0; k < 4; k++) mv[c][k] = pM[c][k];
#pragma unroll
            for (int k = 0; k < 3; k++) { an[c][k] = pA[c][k]; a2[c][k] = pA2[c][k]; }
        }
        if (r + 1 < ye) {
            load_row(r + 4);
            load_a2(r + 2);
        }
        {
            const int mr = mrow(r + 3);
            float th[2];
#pragma unroll
            for (int c = 0; c < 2; c++) {
                const int o = join_map(mr, c ? mcLb : mcLa, pitch);
                th[c] = (PER || o >= 0) ? cs.theta(mv[c][0], mv[c][3]) : side.th(-o - 1);
            }
            const int m3 = (rel + 3) & 3;
            rM[(m3 * 4 + 0) * NT + t] = V{mv[0][0], mv[1][0]};
            rM[(m3 * 4 + 1) * NT + t] = V{mv[0][1], mv[1][1]};
            rM[(m3 * 4 + 2) * NT + t] = V{mv[0][2], mv[1][2]};
            rM[(m3 * 4 + 3) * NT + t] = V{th[0], th[1]};
            rS[((rel + 3) % 5) * NT + t] = V{mv[0][3], mv[1][3]};
        }
        __syncthreads();

        // ---- rebuild: F(n) of row r+2 on pair t
        if (rel >= 2 && doR) {
            const int m1 = (rel + 1) & 3, m2 = (rel + 2) & 3, m3 = (rel + 3) & 3;
            const V *M2 = rM + m2 * 4 * NT, *M1 = rM + m1 * 4 * NT, *M3 = rM + m3 * 4 * NT;
            V c0[4], cw[4], ce[4], cS[4], cN[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                c0[k] = M2[k * NT + t];
                cw[k] = M2[k * NT + t - 1];
                ce[k] = M2[k * NT + t + 1];
                cS[k] = M1[k * NT + t];
                cN[k] = M3[k * NT + t];
            }
            const int mr = mrow(r + 2);
            float fa[9], fb[9];
            {
                // both cells at once (packed FP32): west of a is pair t-1, east of b pair t+1
                f2 ex, ey, om, fo[9];
                closure_terms2(cs, cen, from2(c0[0]), from2(c0[1]), from2(c0[2]), from2(c0[3]),
                               mk2(cw[0].y, c0[0].x), mk2(cw[1].y, c0[1].x), mk2(cw[3].y, c0[3].x),
                               mk2(c0[0].y, ce[0].x), mk2(c0[1].y, ce[1].x), mk2(c0[3].y, ce[3].x),
                               from2(cS[0]), from2(cS[2]), from2(cS[3]), from2(cN[0]), from2(cN[2]), from2(cN[3]),
                               ex, ey, om);
                build_populations2(from2(c0[0]), from2(c0[1]), from2(c0[2]), from2(c0[3]), mk2(aCur[0][0], aCur[1][0]),
                                   mk2(aCur[0][1], aCur[1][1]), mk2(aCur[0][2], aCur[1][2]), ex, ey, om, fo);
#pragma unroll
                for (int i = 0; i < 9; i++) { fa[i] = fo[i].x; fb[i] = fo[i].y; }
            }
            const int oa = join_map(mr, mcLa, pitch), ob = join_map(mr, mcLb, pitch);
            if (!PER && oa < 0) {
#pragma unroll
                for (int i = 0; i < 9; i++) fa[i] = side.F(-oa - 1, i);
            }
            if (!PER && ob < 0) {
#pragma unroll
                for (int i = 0; i < 9; i++) fb[i] = side.F(-ob - 1, i);
            }
            const int a2s = (rel + 2) & 1, c2s = (rel + 2) % 3;
            gA[(a2s * 3 + 0) * NT + t] = V{fa[4], fb[4]};
            gA[(a2s * 3 + 1) * NT + t] = V{fa[7], fb[7]};
            gA[(a2s * 3 + 2) * NT + t] = V{fa[8], fb[8]};
            gB[(a2s * 3 + 0) * NT + t] = V{fa[0], fb[0]};
            gB[(a2s * 3 + 1) * NT + t] = V{fa[1], fb[1]};
            gB[(a2s * 3 + 2) * NT + t] = V{fa[3], fb[3]};
            gC[(c2s * 3 + 0) * NT + t] = V{fa[2], fb[2]};
            gC[(c2s * 3 + 1) * NT + t] = V{fa[5], fb[5]};
            gC[(c2s * 3 + 2) * NT + t] = V{fa[6], fb[6]};
        }
        __syncthreads();

        // ---- phase 2: level n+1 of row r+1 on pair q
        const int y2 = r + 1;
        if (rel >= 4 && do2) {
            const int m0 = rel & 3, m1 = (rel + 1) & 3, m2 = (rel + 2) & 3;
            const V rho0 = rM[(m1 * 4 + 0) * NT + q];
            V mc[3][3], ms[3], mn[3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                mc[k][0] = rM[(m1 * 4 + 1 + k) * NT + q - 1];
                mc[k][1] = rM[(m1 * 4 + 1 + k) * NT + q];
                mc[k][2] = rM[(m1 * 4 + 1 + k) * NT + q + 1];
                ms[k] = rM[(m0 * 4 + 1 + k) * NT + q];
                mn[k] = rM[(m2 * 4 + 1 + k) * NT + q];
            }
            const int s0 = (rel - 1) % 5, s1 = rel % 5, s2 = (rel + 1) % 5, s3 = (rel + 2) % 5, s4 = (rel + 3) % 5;
            const V sc0 = rS[s2 * NT + q - 1], sc1 = rS[s2 * NT + q], sc2 = rS[s2 * NT + q + 1];
            const V sS2 = rS[s0 * NT + q], sS1 = rS[s1 * NT + q], sN1 = rS[s3 * NT + q], sN2 = rS[s4 * NT + q];
            // pull sources: F_0,1,3 of row y2, F_2,5,6 of row y2-1, F_4,7,8 of row y2+1;
            // beyond a zero-gradient side, the edge row / column itself
            const bool zS = !PER && y2 == 0 && kp.bc[2] == BC_ZEROGRAD;
            const bool zN = !PER && y2 == kp.ny - 1 && kp.bc[3] == BC_ZEROGRAD;
            const int bsl = (rel + 1) & 1;                               // row y2 in gB
            const int csl = zS ? (rel + 1) % 3 : rel % 3;                // row y2-1 (or y2) in gC
            const int asl = zN ? (rel + 1) & 1 : (rel + 2) & 1;          // row y2+1 (or y2) in gA
            const V *GB = gB + bsl * 3 * NT, *GC = gC + csl * 3 * NT, *GA = gA + asl * 3 * NT;
            float ga[9], gb[9];
            {
                const V f0 = GB[0 * NT + q], f2 = GC[0 * NT + q], f4 = GA[0 * NT + q];
                ga[0] = f0.x; gb[0] = f0.y;
                ga[2] = f2.x; gb[2] = f2.y;
                ga[4] = f4.x; gb[4] = f4.y;
                // c_x = +1 (1, 5, 8): from x-1 (cell a: pair q-1, or itself at a zero-gradient edge)
                const V f1l = GB[1 * NT + q - 1], f1c = GB[1 * NT + q];
                const V f5l = GC[1 * NT + q - 1], f5c = GC[1 * NT + q];
                const V f8l = GA[2 * NT + q - 1], f8c = GA[2 * NT + q];
                ga[1] = zgW ? f1c.x : f1l.y; gb[1] = f1c.x;
                ga[5] = zgW ? f5c.x : f5l.y; gb[5] = f5c.x;
                ga[8] = zgW ? f8c.x : f8l.y; gb[8] = f8c.x;
                // c_x = -1 (3, 6, 7): from x+1
                const V f3c = GB[2 * NT + q], f3r = GB[2 * NT + q + 1];
                const V f6c = GC[2 * NT + q], f6r = GC[2 * NT + q + 1];
                const V f7c = GA[1 * NT + q], f7r = GA[1 * NT + q + 1];
                ga[3] = zgEa ? f3c.x : f3c.y; gb[3] = zgEb ? f3c.y : f3r.x;
                ga[6] = zgEa ? f6c.x : f6c.y; gb[6] = zgEb ? f6c.y : f6r.x;
                ga[7] = zgEa ? f7c.x : f7c.y; gb[7] = zgEb ? f7c.y : f7r.x;
            }
            {
                f2 C[3], Wv[3], Ev[3], Sv[3], Nv[3];
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    C[k] = from2(mc[k][1]);
                    Wv[k] = mk2(mc[k][0].y, mc[k][1].x);
                    Ev[k] = mk2(mc[k][1].y, mc[k][2].x);
                    Sv[k] = from2(ms[k]);
                    Nv[k] = from2(mn[k]);
                }
                f2 g2[9];
#pragma unroll
                for (int i = 0; i < 9; i++) g2[i] = mk2(ga[i], gb[i]);
                const CellN1x2 n2 = level_np1_2<SIG, PHI0>(
                    cs, from2(rho0), C[0], C[1], C[2], Wv[0], Ev[0], Sv[0], Nv[0], Wv[1], Ev[1], Sv[1], Nv[1], Wv[2], Ev[2],
                    Sv[2], Nv[2], from2(sc0), mk2(sc0.y, sc1.x), from2(sc1), mk2(sc1.y, sc2.x), from2(sc2), from2(sS2),
                    from2(sS1), from2(sN1), from2(sN2), mk2(a2[0][0], a2[1][0]), mk2(a2[0][1], a2[1][1]),
                    mk2(a2[0][2], a2[1][2]), g2);
                nxt[0] = CellN1<float>{n2.rho.x, n2.ux.x, n2.uy.x, n2.th.x, n2.s.x, n2.mxx.x, n2.myy.x, n2.mxy.x};
                nxt[1] = CellN1<float>{n2.rho.y, n2.ux.y, n2.uy.y, n2.th.y, n2.s.y, n2.mxx.y, n2.myy.y, n2.mxy.y};
            }
            const bool out2y = y2 < 0 || y2 >= kp.ny;
            const int side2y = y2 < 0 ? 2 : 3;
            const bool dir2y = !PER && out2y && kp.bc[side2y] == BC_DIRICHLET;
#pragma unroll
            for (int c = 0; c < 2; c++) {
                if (dir2y || dir2[c]) {
                    const int sd = dir2y ? side2y : side2[c];
                    nxt[c].rho = side.rho(sd); nxt[c].ux = side.ux(sd); nxt[c].uy = side.uy(sd);
                    nxt[c].th = side.th(sd); nxt[c].s = side.s_(sd);
                }
            }
            const int ns2 = (rel + 1) % 3;
            rN[(ns2 * 4 + 0) * NT + q] = V{nxt[0].rho, nxt[1].rho};
            rN[(ns2 * 4 + 1) * NT + q] = V{nxt[0].ux, nxt[1].ux};
            rN[(ns2 * 4 + 2) * NT + q] = V{nxt[0].uy, nxt[1].uy};
            rN[(ns2 * 4 + 3) * NT + q] = V{nxt[0].th, nxt[1].th};
        }
        __syncthreads();

        // ---- phase 3: a1(n+1) of row r; write the level-(n+1) moments
        if (r >= ys && do3) {
            const int ns0 = (rel + 2) % 3, ns1 = rel % 3, ns2 = (rel + 1) % 3;  // rows r-1, r, r+1
            const bool zS = !PER && r == 0 && kp.bc[2] == BC_ZEROGRAD;
            const bool zN = !PER && r == kp.ny - 1 && kp.bc[3] == BC_ZEROGRAD;
            V nW[4], nE[4], nS[4], nN[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                nW[k] = rN[(ns1 * 4 + k) * NT + q - 1];
                nE[k] = rN[(ns1 * 4 + k) * NT + q + 1];
                nS[k] = rN[(ns0 * 4 + k) * NT + q];
                nN[k] = rN[(ns2 * 4 + k) * NT + q];
            }
            const CellN1<float> &A = cur[0], &B = cur[1];
            const float aWr = zgW ? A.rho : nW[0].y, aWux = zgW ? A.ux : nW[1].y, aWuy = zgW ? A.uy : nW[2].y,
                        aWth = zgW ? A.th : nW[3].y;
            const float aEr = zgEa ? A.rho : B.rho, aEux = zgEa ? A.ux : B.ux, aEuy = zgEa ? A.uy : B.uy,
                        aEth = zgEa ? A.th : B.th;
            const float bEr = zgEb ? B.rho : nE[0].x, bEux = zgEb ? B.ux : nE[1].x, bEuy = zgEb ? B.uy : nE[2].x,
                        bEth = zgEb ? B.th : nE[3].x;
            float aa[3], ab[3];
            {
                // both cells at once (packed FP32)
                const f2 cr = mk2(A.rho, B.rho), cux = mk2(A.ux, B.ux), cuy = mk2(A.uy, B.uy), cth = mk2(A.th, B.th);
                const f2 wr = mk2(aWr, A.rho), wux = mk2(aWux, A.ux), wuy = mk2(aWuy, A.uy), wth = mk2(aWth, A.th);
                const f2 er = mk2(aEr, bEr), eux = mk2(aEux, bEux), euy = mk2(aEuy, bEuy), eth = mk2(aEth, bEth);
                const f2 sr = zS ? cr : from2(nS[0]), sux = zS ? cux : from2(nS[1]), suy = zS ? cuy : from2(nS[2]),
                         sth = zS ? cth : from2(nS[3]);
                const f2 nr = zN ? cr : from2(nN[0]), nux = zN ? cux : from2(nN[1]), nuy = zN ? cuy : from2(nN[2]),
                         nth = zN ? cth : from2(nN[3]);
                const f2 half = bc2(0.5f);
                const f2 dxux = half * (eux - wux), dyux = half * (nux - sux);
                const f2 dxuy = half * (euy - wuy), dyuy = half * (nuy - suy);
                f2 ex = bc2(0.0f), ey = bc2(0.0f), om;
                if (SIG)
                    closure_terms2(cs, cen, cr, cux, cuy, cth, wr, wux, wth, er, eux, eth, sr, suy, sth, nr, nuy, nth, ex,
                                   ey, om);
                const CellN1x2 c2{cr, cux, cuy, cth, mk2(A.s, B.s), mk2(A.mxx, B.mxx), mk2(A.myy, B.myy),
                                  mk2(A.mxy, B.mxy)};
                f2 axx, axy, ayy;
                a1_next2<SIG>(cs, c2, dxux, dyux, dxuy, dyuy, ex, ey, axx, axy, ayy);
                aa[0] = axx.x; aa[1] = axy.x; aa[2] = ayy.x;
                ab[0] = axx.y; ab[1] = axy.y; ab[2] = ayy.y;
            }
            const long long o = (long long)r * pitch + gx2;
            float *d = out + o;
            if (v3a && !HLBM_CELL_OK(r, gx2, v3b ? 2 : 1, kp, 24)) {
            } else if (v3a && v3b) {
                *reinterpret_cast<V *>(d + MS_RHO * P) = V{A.rho, B.rho};
                *reinterpret_cast<V *>(d + MS_UX * P) = V{A.ux, B.ux};
                *reinterpret_cast<V *>(d + MS_UY * P) = V{A.uy, B.uy};
                *reinterpret_cast<V *>(d + MS_S * P) = V{A.s, B.s};
#pragma unroll
                for (int k = 0; k < 3; k++) *reinterpret_cast<V *>(d + (MS_AXX + k) * P) = V{aa[k], ab[k]};
            } else if (v3a) {
                d[MS_RHO * P] = A.rho; d[MS_UX * P] = A.ux; d[MS_UY * P] = A.uy; d[MS_S * P] = A.s;
#pragma unroll
                for (int k = 0; k < 3; k++) d[(MS_AXX + k) * P] = aa[k];
            }
        }
#pragma unroll
        for (int c = 0; c < 2; c++) {
            cur[c] = nxt[c];
#pragma unroll
            for (int k = 0; k < 3; k++) aCur[c][k] = an[c][k];
        }
    }
}

template <int NT, int MINB, bool SIG, bool PHI0, bool PER = false>
__global__ void __launch_bounds__(NT, MINB)
march_moment_kernel(const float *__restrict__ in, float *__restrict__ out, const KParams kp, const int nseg)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ys = seg_start(blockIdx.y, nseg, kp.ny), ye = seg_start(blockIdx.y + 1, nseg, kp.ny);
    moment_segment<NT, SIG, PHI0, PER>(in, out, kp, blockIdx.x * MomGeom<NT>::W, ys, ye, smem_raw);
}

// Moment state from FP64 caller fields (the initialisation of Sec. 3.5): rho, u, s
// and a1 (given, or a1^FD of the initial fields as in init_kernel), computed
// in FP32 from the fields rounded to FP32, as init_kernel does for FP32.
__global__ void init_moments_kernel(const double *__restrict__ rho, const double *__restrict__ ux,
                                    const double *__restrict__ uy, const double *__restrict__ th,
                                    const double *__restrict__ a1, float *__restrict__ out, const KParams kp)
{
    const int gx = blockIdx.x * blockDim.x + threadIdx.x;
    const int gy = blockIdx.y * blockDim.y + threadIdx.y;
    if (gx >= kp.nx || gy >= kp.ny) return;
    const int n = kp.nx * kp.ny;
    const int c = gy * kp.nx + gx;
    const long long P = kp.plane;
    const int o = gy * kp.pitch + gx;
    const float r0 = (float)rho[c], t0 = (float)th[c];
    float axx, axy, ayy;
    if (a1) {
        axx = (float)a1[c]; axy = (float)a1[n + c]; ayy = (float)a1[2 * n + c];
    } else {
        auto vel = [&](int dx, int dy, float &u, float &v) {
            const int q = locate(gx + dx, gy + dy, kp, kp.nx);
            if (q >= 0) { u = (float)ux[q]; v = (float)uy[q]; }
            else { u = (float)kp.d_ux[-q - 1]; v = (float)kp.d_uy[-q - 1]; }
        };
        float uxm, vxm, uxp, vxp, uym, vym, uyp, vyp;
        vel(-1, 0, uxm, vxm); vel(1, 0, uxp, vxp); vel(0, -1, uym, vym); vel(0, 1, uyp, vyp);
        const float p = r0 * t0 / 3.0f;
        const float cfd = -((float)kp.mu + 0.5f * p);
        axx = cfd * (0.5f * (uxp - uxm) - 0.5f * (vyp - vym));
        axy = cfd * (0.5f * (uyp - uym) + 0.5f * (vxp - vxm));
        ayy = -axx;
    }
    out[MS_RHO * P + o] = r0;
    out[MS_UX * P + o] = (float)ux[c];
    out[MS_UY * P + o] = (float)uy[c];
    out[MS_S * P + o] = init_entropy(kp, r0, t0);
    out[MS_AXX * P + o] = axx;
    out[MS_AXY * P + o] = axy;
    out[MS_AYY * P + o] = ayy;
}

// Caller fields from the moment state (theta recomputed from rho and s).
__global__ void moments_macros_kernel(const float *__restrict__ in, double *rho, double *ux, double *uy,
                                      double *th, double *s, double *a1, const KParams kp)
{
    const int gx = blockIdx.x * blockDim.x + threadIdx.x;
    const int gy = blockIdx.y * blockDim.y + threadIdx.y;
    if (gx >= kp.nx || gy >= kp.ny) return;
    Consts<float> cs;
    cs.load(kp);
    const long long P = kp.plane;
    const int o = gy * kp.pitch + gx;
    const int c = gy * kp.nx + gx;
    const size_t n = (size_t)kp.nx * kp.ny;
    const float r = in[MS_RHO * P + o], sv = in[MS_S * P + o];
    if (rho) rho[c] = (double)r;
    if (ux) ux[c] = (double)in[MS_UX * P + o];
    if (uy) uy[c] = (double)in[MS_UY * P + o];
    if (th) th[c] = (double)cs.theta(r, sv);
    if (s) s[c] = (double)sv;
    if (a1) {
        a1[c] = (double)in[MS_AXX * P + o];
        a1[n + c] = (double)in[MS_AXY * P + o];
        a1[2 * n + c] = (double)in[MS_AYY * P + o];
    }
}

// Diagnostics of the moment state: the same 8 values as diag_partial_kernel.
__global__ void __launch_bounds__(DIAG_NT)
moments_diag_partial_kernel(const float *__restrict__ in, double *__restrict__ partial, const KParams kp)
{
    Consts<float> cs;
    cs.load(kp);
    const long long P = kp.plane;
    const long long ncell = (long long)kp.nx * kp.ny;
    double acc[DIAG_NV] = {0.0, 0.0, 0.0, 0.0, 1e300, 1e300, 0.0, 0.0};
    for (long long c = (long long)blockIdx.x * DIAG_NT + threadIdx.x; c < ncell; c += (long long)gridDim.x * DIAG_NT) {
        const int gy = (int)(c / kp.nx), gx = (int)(c - (long long)gy * kp.nx);
        const int o = gy * kp.pitch + gx;
        const float r = in[MS_RHO * P + o];
        const double rho = (double)r;
        const double u = (double)in[MS_UX * P + o], v = (double)in[MS_UY * P + o];
        const double th = (double)cs.theta(r, in[MS_S * P + o]);
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

}  // namespace hlbm
