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
//     block-diagonal S of Eq. A3. Written as
//       A = M (f - f_D + R_G/2),  f* = f_D + R_G/2 + M^-1 (I - S) A,
//     which is the same update: (I - S)(D + G/2) + G/2 = (I - S) D + (I - S/2) G.
//     The conserved components of A vanish (mass; momentum, since Eq. 9's
//     u carries F/2), so s0 and s1 do not enter.
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

template <int I>
__device__ __forceinline__ void mrt_pre(float (&h)[kQ], float (&b)[kQ], float rho, float a, float ux, float uy,
                                        float uz, float uF, float Fx, float Fy, float Fz) {
    float heq, R;
    feq_guo<I>(rho, a, ux, uy, uz, uF, Fx, Fy, Fz, heq, R);
    b[I] = fmaf(0.5f, R, heq);         // f_D - w + R/2
    h[I] = fmaf(0.5f, R, h[I] - heq);  // f - f_D + R/2
    if constexpr (I + 1 < kQ) mrt_pre<I + 1>(h, b, rho, a, ux, uy, uz, uF, Fx, Fy, Fz);
}

// Non-orthogonal MRT collision on deviations h, in place. Returns rho - 1.
__device__ __forceinline__ float collide_mrt(float (&h)[kQ], float Fx, float Fy, float Fz, const Rates &r) {
    float jx, jy, jz;
    const float drho = moments_eq9(h, Fx, Fy, Fz, jx, jy, jz);
    const float rho = 1.0f + drho, inv = 1.0f / rho;
    const float ux = jx * inv, uy = jy * inv, uz = jz * inv;
    const float uu = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
    const float uF = fmaf(ux, Fx, fmaf(uy, Fy, uz * Fz));
    const float a = fmaf(-1.5f * rho, uu, drho);
    float b[kQ];
    mrt_pre<0>(h, b, rho, a, ux, uy, uz, uF, Fx, Fy, Fz);
    Moments A;
    raw_moments(h, A);
    // (I - S) A; the conserved components vanish
    A.m000 = 0.0f; A.m100 = 0.0f; A.m010 = 0.0f; A.m001 = 0.0f;
    A.m110 *= r.om2; A.m101 *= r.om2; A.m011 *= r.om2;
    {
        const float tr = r.cb * (A.m200 + A.m020 + A.m002);
        A.m200 = fmaf(r.om2, A.m200, -tr);
        A.m020 = fmaf(r.om2, A.m020, -tr);
        A.m002 = fmaf(r.om2, A.m002, -tr);
    }
    A.m120 *= r.om3; A.m102 *= r.om3; A.m210 *= r.om3;
    A.m201 *= r.om3; A.m012 *= r.om3; A.m021 *= r.om3;
    A.m220 *= r.om4; A.m202 *= r.om4; A.m022 *= r.om4;
    inverse_moments(A, h);
#pragma unroll
    for (int i = 0; i < kQ; ++i) h[i] += b[i];
    return drho;
}

}  // namespace clbm
