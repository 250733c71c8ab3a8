// models.cuh -- the two comparison collision models the paper sets beside the
// cascaded one, on the same D3Q19 layout and deviation variables h = f - w:
//
//   SRT-LBM (Sec. III.A): f*_i = f_i - s (f_i - f_D,i) + (1 - s/2) R_G,i with
//     s = s2, the second-order discrete equilibrium
//     f_D,i = w_i rho [1 + 3 e_i.u + 9/2 (e_i.u)^2 - 3/2 u.u]   (Sec. II.B)
//     and Guo's forcing term
//     R_G,i = w_i [3 (e_i - u) + 9 (e_i.u) e_i] . F             (Appendix B),
//     evaluated as the MRT collision below with every rate equal to s.
//
//   Non-orthogonal MRT-LBM (Appendix B): raw moments T = M f of Eq. A4,
//     T* = T - S (T - M f_D) + (I - S/2) M R_G, f* = M^-1 T*, with the
//     block-diagonal S of Eq. A3, evaluated in moment space with the raw
//     moments of f_D and R_G in closed form. The conserved components come
//     out as rho and rho u + F/2 for any s0, s1 (Eq. 9's u carries F/2), so
//     s0 and s1 do not enter.
//
// u is Eq. 9's velocity (with F/2) in both.
#pragma once

#include "d3q19.cuh"

namespace clbm {

// Non-orthogonal MRT collision on deviations h, in place. Returns rho - 1.
// Evaluated in raw-moment space: T - M w = M h (raw_moments), the raw moments
// of f_D - w and of R_G in closed form (D3Q19 lattice sums: sum w e_a^2 e_b^2
// = 1/9 for a != b, sum w e_x^4 e_y^2 = 1/9, no corners):
//   f_D:  rho u_a u_b (a != b), rho u_a^2 + drho/3, rho u_x / 3 (k_120 and the
//         other third-order moments alike), drho/9 + rho ((u_x^2 + u_y^2)/2 - u.u/6)
//         (k_220 alike);
//   R_G:  u_a F_b + u_b F_a, 2 u_a F_a, F_x / 3, u_x F_x + u_y F_y - u.F / 3;
// then T* = T_eq + (I - S)(T - T_eq) + (I - S/2) G and h* = M^-1 (T* - M w).
template <bool FR = false>
__device__ __forceinline__ float collide_mrt(float (&h)[kQ], float Fx, float Fy, float Fz, const Rates &r) {
    Moments k;
    raw_moments(h, k);
    const float drho = k.m000;
    const float rho = 1.0f + drho, inv = recip_of<FR>(rho);
    const float jx = fmaf(0.5f, Fx, k.m100), jy = fmaf(0.5f, Fy, k.m010), jz = fmaf(0.5f, Fz, k.m001);
    const float ux = jx * inv, uy = jy * inv, uz = jz * inv;
    const float X = ux * ux, Y = uy * uy, Z = uz * uz;
    const float u6 = (X + Y + Z) * (1.0f / 6.0f);
    const float uF3 = fmaf(ux, Fx, fmaf(uy, Fy, uz * Fz)) * kC;
    const float xF = ux * Fx, yF = uy * Fy, zF = uz * Fz;
    const float h2 = 0.5f * (1.0f + r.om2), h4 = 0.5f * (1.0f + r.om4);  // 1 - s/2
    Moments q;
    q.m000 = drho;
    q.m100 = jx + 0.5f * Fx; q.m010 = jy + 0.5f * Fy; q.m001 = jz + 0.5f * Fz;
    {
        const float e110 = jx * uy, e101 = jx * uz, e011 = jy * uz;
        q.m110 = fmaf(r.om2, k.m110 - e110, fmaf(h2, fmaf(ux, Fy, uy * Fx), e110));
        q.m101 = fmaf(r.om2, k.m101 - e101, fmaf(h2, fmaf(ux, Fz, uz * Fx), e101));
        q.m011 = fmaf(r.om2, k.m011 - e011, fmaf(h2, fmaf(uy, Fz, uz * Fy), e011));
    }
    {
        const float e200 = fmaf(jx, ux, drho * kC), e020 = fmaf(jy, uy, drho * kC), e002 = fmaf(jz, uz, drho * kC);
        const float n200 = k.m200 - e200, n020 = k.m020 - e020, n002 = k.m002 - e002;
        const float tr = r.cb * (n200 + n020 + n002);
        const float gtr = r.cb * (xF + yF + zF);  // (s_-/2) times the trace of G = 2 u.F
        q.m200 = fmaf(r.om2, n200, e200) - tr + fmaf(2.0f * h2, xF, -gtr);
        q.m020 = fmaf(r.om2, n020, e020) - tr + fmaf(2.0f * h2, yF, -gtr);
        q.m002 = fmaf(r.om2, n002, e002) - tr + fmaf(2.0f * h2, zF, -gtr);
    }
    {
        const float ex = jx * kC, ey = jy * kC, ez = jz * kC;
        q.m120 = fmaf(r.om3, k.m120 - ex, fmaf(r.c3, Fx, ex));
        q.m102 = fmaf(r.om3, k.m102 - ex, fmaf(r.c3, Fx, ex));
        q.m210 = fmaf(r.om3, k.m210 - ey, fmaf(r.c3, Fy, ey));
        q.m012 = fmaf(r.om3, k.m012 - ey, fmaf(r.c3, Fy, ey));
        q.m201 = fmaf(r.om3, k.m201 - ez, fmaf(r.c3, Fz, ez));
        q.m021 = fmaf(r.om3, k.m021 - ez, fmaf(r.c3, Fz, ez));
    }
    {
        const float d9 = drho * kC2;
        const float e220 = fmaf(rho, fmaf(0.5f, X + Y, -u6), d9);
        const float e202 = fmaf(rho, fmaf(0.5f, X + Z, -u6), d9);
        const float e022 = fmaf(rho, fmaf(0.5f, Y + Z, -u6), d9);
        q.m220 = fmaf(r.om4, k.m220 - e220, fmaf(h4, xF + yF - uF3, e220));
        q.m202 = fmaf(r.om4, k.m202 - e202, fmaf(h4, xF + zF - uF3, e202));
        q.m022 = fmaf(r.om4, k.m022 - e022, fmaf(h4, yF + zF - uF3, e022));
    }
    inverse_moments(q, h);
    return drho;
}

// SRT collision on deviations h, in place; s = s2. The GMRT framework with
// every rate equal is the SRT-LBM (Sec. II.A), so this is the MRT collision
// with all rates set to s2; in moment space mass and momentum come out
// exactly. (A per-population form, f + s (f_D - f) + (1 - s/2) R_G, rounds
// the equilibrium's mass and momentum in FP32 the same way every step on a
// nearly steady flow, and drifted from the FP64 oracle by 3e-5 in 1000 steps
// of a shear wave at u = 0.17.)
template <bool FR = false>
__device__ __forceinline__ float collide_srt(float (&h)[kQ], float Fx, float Fy, float Fz, const Rates &r) {
    Rates e;
    e.om2 = r.om2;
    e.cb = 0.0f;
    e.om3 = r.om2;
    e.c3 = 0.5f * (1.0f + r.om2) * kC;
    e.om4 = r.om2;
    return collide_mrt<FR>(h, Fx, Fy, Fz, e);
}

}  // namespace clbm
