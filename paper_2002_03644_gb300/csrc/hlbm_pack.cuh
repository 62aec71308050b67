// hlbm_pack.cuh -- the per-cell arithmetic of the fused step on two cells
// at once, with the packed FP32 instructions of sm_100-class GPUs
// (add / sub / mul / fma .f32x2: one instruction, two independent IEEE
// operations).  The paired-column kernels give each thread two horizontally
// adjacent cells with the same instruction stream, so lane x is the cell at
// even ring column and lane y its right partner.  Comparisons, selections
// and the MUFU approximations stay per lane.
//
// The formulas are those of level_np1 / collide_cell / build_populations in
// hlbm_march.cuh and hlbm_device.cuh term by term; multiply-adds are written
// as explicit fused operations, so results may differ from the scalar
// kernels by FP32 rounding only.
#pragma once

#include "hlbm_device.cuh"

namespace hlbm {

struct f2 {
    float x, y;
};

__device__ __forceinline__ unsigned long long f2_bits(f2 a)
{
    unsigned long long u;
    asm("mov.b64 %0, {%1, %2};" : "=l"(u) : "f"(a.x), "f"(a.y));
    return u;
}
__device__ __forceinline__ f2 f2_from_bits(unsigned long long u)
{
    f2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(u));
    return r;
}
__device__ __forceinline__ f2 mk2(float a, float b) { return f2{a, b}; }
__device__ __forceinline__ f2 bc2(float a) { return f2{a, a}; }
__device__ __forceinline__ f2 from2(float2 v) { return f2{v.x, v.y}; }

__device__ __forceinline__ f2 operator+(f2 a, f2 b)
{
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from_bits(d);
}
__device__ __forceinline__ f2 operator-(f2 a, f2 b)
{
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from_bits(d);
}
__device__ __forceinline__ f2 operator*(f2 a, f2 b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
    return f2_from_bits(d);
}
// a * b + c, one rounding per lane
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
    return f2_from_bits(d);
}
__device__ __forceinline__ f2 operator*(float a, f2 b) { return bc2(a) * b; }

// per-lane helpers
__device__ __forceinline__ f2 sel2(bool px, bool py, f2 a, f2 b) { return f2{px ? a.x : b.x, py ? a.y : b.y}; }
__device__ __forceinline__ f2 abs2(f2 a) { return f2{fabsf(a.x), fabsf(a.y)}; }
__device__ __forceinline__ f2 rcp2(f2 a) { return f2{rcp_approx(a.x), rcp_approx(a.y)}; }
__device__ __forceinline__ f2 div2(f2 a, f2 b) { return a * rcp2(b); }

// theta = 2^((gamma-1) log2 rho + s / (c_v ln 2))
__device__ __forceinline__ f2 theta2(const Consts<float> &cs, f2 rho, f2 s)
{
    const f2 e = fma2(bc2(cs.gm1), f2{lg2_approx(rho.x), lg2_approx(rho.y)}, s * bc2(cs.s2exp));
    return f2{ex2_approx(e.x), ex2_approx(e.y)};
}

// rho and momentum; mirror directions paired as in moments()
__device__ __forceinline__ void moments2(const f2 f[9], f2 &rho, f2 &jx, f2 &jy)
{
    rho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    jy = (f[2] - f[4]) + (f[5] - f[8]) + (f[6] - f[7]);
}

__device__ __forceinline__ f2 va_slope2(f2 a, f2 b)
{
    const f2 ab = a * b;
    const f2 r = div2(ab * (a + b), fma2(a, a, b * b));
    return sel2(ab.x > 0.0f, ab.y > 0.0f, r, bc2(0.0f));
}

// u ds/dx, upwinded by the sign of u (muscl_adv)
__device__ __forceinline__ f2 muscl_adv2(f2 u, f2 smm, f2 sm, f2 s0, f2 sp, f2 spp)
{
    const bool px = u.x > 0.0f, py = u.y > 0.0f;
    const f2 q2 = sel2(px, py, smm, spp), q1 = sel2(px, py, sm, sp), qm = sel2(px, py, sp, sm);
    const f2 d10 = s0 - q1;
    const f2 dd = fma2(bc2(0.5f), va_slope2(d10, qm - s0) - va_slope2(q1 - q2, d10), d10);
    return abs2(u) * dd;
}

__device__ __forceinline__ f2 gamma_defect2(f2 rho, f2 ua, f2 th)
{
    return rho * ua * (bc2(1.0f) - th - ua * ua);
}

// Post-collision populations from level quantities (build_populations).
__device__ __forceinline__ void build_populations2(f2 rho, f2 ux, f2 uy, f2 th, f2 axx, f2 axy, f2 ayy, f2 ex, f2 ey,
                                                   f2 omega, f2 f[9])
{
    const f2 third = bc2(1.0f / 3.0f), half = bc2(0.5f), two = bc2(2.0f);
    const f2 t3 = th * third;
    const f2 mx2 = fma2(ux, ux, t3), my2 = fma2(uy, uy, t3);
    const f2 axxy = fma2(uy, axx, two * ux * axy);
    const f2 ayyx = fma2(ux, ayy, two * uy * axy);
    const f2 cth = (th - bc2(1.0f)) * third;
    const f2 axxyy = fma2(two, fma2(ux, ayyx, uy * axxy), fma2(cth - ux * ux, ayy, (cth - uy * uy) * axx))
                   - bc2(4.0f) * ux * uy * axy;
    const f2 rux = rho * ux, ruy = rho * uy;
    const f2 R00 = rho, R10 = rux, R01 = ruy;
    const f2 R20 = fma2(rho, mx2, fma2(omega, axx, half * ex));
    const f2 R02 = fma2(rho, my2, fma2(omega, ayy, half * ey));
    const f2 R11 = fma2(rux, uy, omega * axy);
    const f2 R21 = fma2(rho * mx2, uy, omega * axxy);
    const f2 R12 = fma2(rux, my2, omega * ayyx);
    const f2 R22 = fma2(rho * mx2, my2, fma2(omega, fma2(axx + ayy, third, axxyy), (ex + ey) * bc2(0.5f / 3.0f)));
    const f2 X0z = R00 - R20, X0p = half * (R20 + R10), X0m = half * (R20 - R10);
    const f2 X1z = R01 - R21, X1p = half * (R21 + R11), X1m = half * (R21 - R11);
    const f2 X2z = R02 - R22, X2p = half * (R22 + R12), X2m = half * (R22 - R12);
    f[0] = X0z - X2z;
    f[1] = X0p - X2p;
    f[3] = X0m - X2m;
    f[2] = half * (X2z + X1z);
    f[4] = half * (X2z - X1z);
    f[5] = half * (X2p + X1p);
    f[8] = half * (X2p - X1p);
    f[6] = half * (X2m + X1m);
    f[7] = half * (X2m - X1m);
}

// Level-(n+1) values of two cells (CellN1 per lane).
struct CellN1x2 {
    f2 rho, ux, uy, th, s, mxx, myy, mxy;
};

// Pull, moments, entropy and theta of level n+1 for two cells (level_np1).
template <bool SIG, bool PHI0>
__device__ __forceinline__ CellN1x2 level_np1_2(const Consts<float> &cs, f2 rho0, f2 ux0, f2 uy0, f2 th0, f2 uxW,
                                               f2 uxE, f2 uxS, f2 uxN, f2 uyW, f2 uyE, f2 uyS, f2 uyN, f2 thW,
                                               f2 thE, f2 thS, f2 thN, f2 sWW, f2 sW, f2 s0, f2 sE, f2 sEE, f2 sSS,
                                               f2 sS, f2 sN, f2 sNN, f2 a_xx, f2 a_xy, f2 a_yy, const f2 g[9])
{
    const f2 half = bc2(0.5f);
    const f2 dxux = half * (uxE - uxW);
    const f2 dyux = half * (uxN - uxS);
    const f2 dxuy = half * (uyE - uyW);
    const f2 dyuy = half * (uyN - uyS);
    const f2 lap = fma2(bc2(-4.0f), th0, (thE + thW) + (thN + thS));
    const f2 adv = muscl_adv2(ux0, sWW, sW, s0, sE, sEE) + muscl_adv2(uy0, sSS, sS, s0, sN, sNN);
    const f2 rt = rho0 * th0;
    const f2 p0 = rt * bc2(1.0f / 3.0f);
    f2 phi;
    if (PHI0) {
        const f2 two_mu = bc2(cs.two_mu);
        const f2 contr = fma2(a_xx, dxux, fma2(a_xy, dyux + dxuy, a_yy * dyuy));
        phi = bc2(0.0f) - div2(two_mu, two_mu + p0) * contr;
    } else {
        const f2 d1 = dxux - dyuy, d2 = dyux + dxuy;
        phi = bc2(cs.mu) * fma2(d1, d1, d2 * d2);
    }
    CellN1x2 o;
    o.s = s0 - adv + div2(fma2(bc2(cs.lam), lap, phi), rt);
    f2 jx, jy;
    moments2(g, o.rho, jx, jy);
    const f2 ir = rcp2(o.rho);
    o.ux = jx * ir;
    o.uy = jy * ir;
    o.th = theta2(cs, o.rho, o.s);
    if (SIG) {
        const f2 diag = (g[5] + g[6]) + (g[7] + g[8]);
        o.mxx = (g[1] + g[3]) + diag;
        o.myy = (g[2] + g[4]) + diag;
        o.mxy = (g[5] - g[6]) + (g[7] - g[8]);
    } else {
        o.mxx = o.myy = o.mxy = bc2(0.0f);
    }
    return o;
}

// E_x, E_y (E1 upwind or centred, plus E2) and omega of two cells from their
// macros and those of their four neighbours (the first half of collide_cell).
__device__ __forceinline__ void closure_terms2(const Consts<float> &cs, bool cen, f2 rho, f2 ux, f2 uy, f2 th, f2 rW,
                                               f2 uxW, f2 thW, f2 rE, f2 uxE, f2 thE, f2 rS, f2 uyS, f2 thS, f2 rN,
                                               f2 uyN, f2 thN, f2 &ex, f2 &ey, f2 &omega)
{
    const f2 half = bc2(0.5f);
    const f2 dxux = half * (uxE - uxW);
    const f2 dyuy = half * (uyN - uyS);
    const f2 p = rho * th * bc2(1.0f / 3.0f);
    const f2 gxc = gamma_defect2(rho, ux, th), gyc = gamma_defect2(rho, uy, th);
    const f2 gxm = gamma_defect2(rW, uxW, thW), gxp = gamma_defect2(rE, uxE, thE);
    const f2 gym = gamma_defect2(rS, uyS, thS), gyp = gamma_defect2(rN, uyN, thN);
    // upwind by the sign of the cell's velocity; u = 0 (or the centred
    // ablation) gives the centred difference
    const f2 cx = half * (gxp - gxm), cy = half * (gyp - gym);
    const f2 bx = gxc - gxm, fx = gxp - gxc, by = gyc - gym, fy = gyp - gyc;
    const f2 e1xx = sel2(ux.x > 0.0f && !cen, ux.y > 0.0f && !cen, bx, sel2(ux.x < 0.0f && !cen, ux.y < 0.0f && !cen, fx, cx));
    const f2 e1yy = sel2(uy.x > 0.0f && !cen, uy.y > 0.0f && !cen, by, sel2(uy.x < 0.0f && !cen, uy.y < 0.0f && !cen, fy, cy));
    const f2 e2 = p * bc2(cs.two_m_gamma) * (dxux + dyuy);
    ex = e1xx + e2;
    ey = e1yy + e2;
    const f2 two_mu = bc2(cs.two_mu);
    omega = div2(two_mu - p, two_mu + p);
}

// a1(n+1) of two cells: a1^FD, blended with a1^PR when SIG (collide_cell's
// first half); ex, ey are needed only for a1^PR.
template <bool SIG>
__device__ __forceinline__ void a1_next2(const Consts<float> &cs, const CellN1x2 &c, f2 dxux, f2 dyux, f2 dxuy,
                                         f2 dyuy, f2 ex, f2 ey, f2 &axx, f2 &axy, f2 &ayy)
{
    const f2 p = c.rho * c.th * bc2(1.0f / 3.0f);
    const f2 cfd = bc2(0.0f) - fma2(bc2(0.5f), p, bc2(cs.mu));
    const f2 fdxx = cfd * (dxux - dyuy), fdxy = cfd * (dyux + dxuy);
    if (SIG) {
        const f2 prxx = fma2(bc2(0.5f), ex, c.mxx - c.rho * c.ux * c.ux - p);
        const f2 pryy = fma2(bc2(0.5f), ey, c.myy - c.rho * c.uy * c.uy - p);
        const f2 prxy = c.mxy - c.rho * c.ux * c.uy;
        const f2 sg = bc2(cs.sigma), om = bc2(cs.one_m_sigma);
        axx = fma2(sg, prxx, om * fdxx);
        ayy = fma2(sg, pryy, bc2(0.0f) - om * fdxx);
        axy = fma2(sg, prxy, om * fdxy);
    } else {
        axx = fdxx;
        ayy = bc2(0.0f) - fdxx;
        axy = fdxy;
    }
}

}  // namespace hlbm
