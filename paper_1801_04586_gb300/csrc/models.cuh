// models.cuh -- the two comparison collision models the paper sets beside the
// cascaded one, on the same D3Q19 layout and deviation variables h = f - w:
//
//   SRT-LBM (Sec. III.A): f*_i = f_i - s (f_i - f_D,i) + (1 - s/2) R_G,i with
//     s = s2, the second-order discrete equilibrium
//     f_D,i = w_i rho [1 + 3 e_i.u + 9/2 (e_i.u)^2 - 3/2 u.u]   (Sec. II.B)
//     and Guo's forcing term
//     R_G,i = w_i [3 (e_i - u) + 9 (e_i.u) e_i] . F             (Appendix B).
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

// Macroscopic moments of deviations h (Eq. 9): drho = sum h, j = sum e h + F/2.
__device__ __forceinline__ float moments_eq9(const float (&h)[kQ], float Fx, float Fy, float Fz, float &jx,
                                             float &jy, float &jz) {
    float d = 0.0f, ax = 0.0f, ay = 0.0f, az = 0.0f;
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        d += h[i];
        if (ex19(i)) ax += ex19(i) > 0 ? h[i] : -h[i];
        if (ey19(i)) ay += ey19(i) > 0 ? h[i] : -h[i];
        if (ez19(i)) az += ez19(i) > 0 ? h[i] : -h[i];
    }
    jx = fmaf(0.5f, Fx, ax);
    jy = fmaf(0.5f, Fy, ay);
    jz = fmaf(0.5f, Fz, az);
    return d;
}

// f_D,i - w_i and R_G,i for population i at (drho, rho, u, F); a = drho - 3/2 rho u.u
// and uF = u.F are shared by all i.
template <int I>
__device__ __forceinline__ void feq_guo(float rho, float a, float ux, float uy, float uz, float uF, float Fx,
                                        float Fy, float Fz, float &heq, float &R) {
    constexpr float w = rest_weight(I);
    float eu = 0.0f, eF = 0.0f;
    if (ex19(I)) { eu += ex19(I) * ux; eF += ex19(I) * Fx; }
    if (ey19(I)) { eu += ey19(I) * uy; eF += ey19(I) * Fy; }
    if (ez19(I)) { eu += ez19(I) * uz; eF += ez19(I) * Fz; }
    heq = w * fmaf(rho * eu, fmaf(4.5f, eu, 3.0f), a);
    R = w * fmaf(9.0f * eu, eF, 3.0f * (eF - uF));
}

template <int I>
__device__ __forceinline__ void srt_one(float (&h)[kQ], float rho, float a, float ux, float uy, float uz, float uF,
                                        float Fx, float Fy, float Fz, float s, float cf) {
    float heq, R;
    feq_guo<I>(rho, a, ux, uy, uz, uF, Fx, Fy, Fz, heq, R);
    h[I] = fmaf(cf, R, fmaf(s, heq - h[I], h[I]));
}

template <int I>
__device__ __forceinline__ void srt_all(float (&h)[kQ], float rho, float a, float ux, float uy, float uz, float uF,
                                        float Fx, float Fy, float Fz, float s, float cf) {
    srt_one<I>(h, rho, a, ux, uy, uz, uF, Fx, Fy, Fz, s, cf);
    if constexpr (I + 1 < kQ) srt_all<I + 1>(h, rho, a, ux, uy, uz, uF, Fx, Fy, Fz, s, cf);
}

// SRT collision on deviations h, in place; s = s2 = 1 - r.om2. Returns rho - 1.
__device__ __forceinline__ float collide_srt(float (&h)[kQ], float Fx, float Fy, float Fz, const Rates &r) {
    float jx, jy, jz;
    const float drho = moments_eq9(h, Fx, Fy, Fz, jx, jy, jz);
    const float rho = 1.0f + drho, inv = 1.0f / rho;
    const float ux = jx * inv, uy = jy * inv, uz = jz * inv;
    const float uu = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
    const float uF = fmaf(ux, Fx, fmaf(uy, Fy, uz * Fz));
    const float a = fmaf(-1.5f * rho, uu, drho);
    const float s = 1.0f - r.om2, cf = 1.0f - 0.5f * s;
    srt_all<0>(h, rho, a, ux, uy, uz, uF, Fx, Fy, Fz, s, cf);
    return drho;
}

// Non-orthogonal MRT collision on deviations h, in place. Returns rho - 1.
// Evaluated in raw-moment space: T - M w = M h (raw_moments), the raw moments
// of f_D - w and of R_G in closed form (D3Q19 lattice sums: sum w e_a^2 e_b^2
// = 1/9 for a != b, sum w e_x^4 e_y^2 = 1/9, no corners):
//   f_D:  rho u_a u_b (a != b), rho u_a^2 + drho/3, rho u_x / 3 (k_120 and the
//         other third-order moments alike), drho/9 + rho ((u_x^2 + u_y^2)/2 - u.u/6)
//         (k_220 alike);
//   R_G:  u_a F_b + u_b F_a, 2 u_a F_a, F_x / 3, u_x F_x + u_y F_y - u.F / 3;
// then T* = T_eq + (I - S)(T - T_eq) + (I - S/2) G and h* = M^-1 (T* - M w).
__device__ __forceinline__ float collide_mrt(float (&h)[kQ], float Fx, float Fy, float Fz, const Rates &r) {
    Moments k;
    raw_moments(h, k);
    const float drho = k.m000;
    const float rho = 1.0f + drho, inv = 1.0f / rho;
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

}  // namespace clbm
