// models27.cuh -- the SRT-LBM and non-orthogonal MRT comparison collisions
// (models.cuh) on the D3Q27 lattice of Sec. II; Appendix B runs the MRT one
// on D3Q27. Same definitions: the second-order discrete equilibrium f_D of
// Sec. II.B, Guo's forcing term R_G, s = s2 for SRT; for MRT the raw moments
// of Eq. 14 relaxed with the S of Eq. 13.
//
// The D3Q27 weights factor per axis (2/3 for e = 0, 1/6 for e = +-1), so the
// raw moments of f_D and R_G are sums of products of the 1D lattice moments
// mu_k = sum_e w(e) e^k = 1, 0, 1/3, 0, 1/3 (k = 0..4):
//   M_abc f_D = rho [W (1 - 3/2 u.u) + 3 sum_d u_d W_d + 9/2 sum_dd' u_d u_d' W_dd']
//   M_abc R_G = 3 sum_d F_d W_d - 3 u.F W + 9 sum_dd' u_d F_d' W_dd'
// with W = mu_a mu_b mu_c and W_d, W_dd' the same with the exponent of axis d
// (and d') raised by one. The exponents are compile-time constants, so every
// W is a constant and the vanishing terms drop out.
#pragma once

#include "d3q27.cuh"

namespace clbm {

__host__ __device__ constexpr float mu1(int k) { return k == 0 ? 1.0f : ((k & 1) ? 0.0f : (1.0f / 3.0f)); }
__host__ __device__ constexpr float w27(int a, int b, int c) { return mu1(a) * mu1(b) * mu1(c); }

// Raw moment (a, b, c) of f_D - w (teq) and of R_G (g).
__device__ __forceinline__ void feq_guo_moment27(int a, int b, int c, float drho, float rho, const float (&u)[3],
                                                 const float (&F)[3], float uu, float uF, float &teq, float &g) {
    const int ex[3] = {a, b, c};
    const float W = w27(a, b, c);
    float s = 0.0f, gs = 0.0f;
    if (W != 0.0f) {
        s = -1.5f * uu * W;
        gs = -3.0f * uF * W;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float Wd = w27(ex[0] + (d == 0), ex[1] + (d == 1), ex[2] + (d == 2));
        if (Wd != 0.0f) {
            s = fmaf(3.0f * Wd, u[d], s);
            gs = fmaf(3.0f * Wd, F[d], gs);
        }
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const float Wdd = w27(ex[0] + (d == 0) + (e == 0), ex[1] + (d == 1) + (e == 1),
                                  ex[2] + (d == 2) + (e == 2));
            if (Wdd != 0.0f) {
                s = fmaf(4.5f * Wdd * u[d], u[e], s);
                gs = fmaf(9.0f * Wdd * u[d], F[e], gs);
            }
        }
    }
    teq = W != 0.0f ? fmaf(rho, s, drho * W) : rho * s;
    g = gs;
}

// Relaxation rate (1 - s) of raw moment (a, b, c) under Eq. 13, other than
// the conserved moments and the 3 x 3 block of the normal second moments.
__device__ __forceinline__ float om27(int a, int b, int c, const Rates27 &r) {
    const int n1 = (a == 1) + (b == 1) + (c == 1), n2 = (a == 2) + (b == 2) + (c == 2);
    if (n1 == 2 && n2 == 0) return r.om2;   // k110, k101, k011
    if (n1 == 1 && n2 == 1) return r.om3;   // k120, ...
    if (n1 == 3) return r.om3b;             // k111
    if (n1 == 0 && n2 == 2) return r.om4;   // k220, ...
    if (n1 == 2 && n2 == 1) return r.om4b;  // k211, ...
    if (n1 == 1 && n2 == 2) return r.om5;   // k122, ...
    return r.om6;                           // k222
}

// Non-orthogonal MRT on D3Q27 deviations h (cube by velocity code), in place:
// T* = T_eq + (I - S)(T - T_eq) + (I - S/2) G, h* = M^-1 (T* - M w).
template <bool FR = false>
__device__ __forceinline__ float collide_mrt27(float (&h)[3][3][3], float Fx, float Fy, float Fz,
                                               const Rates27 &r) {
    float m[3][3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) m[a][b][c] = h[a][b][c];
    raw_axis<0>(m);
    raw_axis<1>(m);
    raw_axis<2>(m);
    const float drho = m[0][0][0];
    const float rho = 1.0f + drho, inv = recip_of<FR>(rho);
    const float jx = fmaf(0.5f, Fx, m[1][0][0]), jy = fmaf(0.5f, Fy, m[0][1][0]), jz = fmaf(0.5f, Fz, m[0][0][1]);
    const float u[3] = {jx * inv, jy * inv, jz * inv};
    const float F[3] = {Fx, Fy, Fz};
    const float uu = fmaf(u[0], u[0], fmaf(u[1], u[1], u[2] * u[2]));
    const float uF = fmaf(u[0], Fx, fmaf(u[1], Fy, u[2] * Fz));
    // the 3 x 3 block of the normal second moments
    float te[3], gn[3], nn[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int a = d == 0 ? 2 : 0, b = d == 1 ? 2 : 0, c = d == 2 ? 2 : 0;
        feq_guo_moment27(a, b, c, drho, rho, u, F, uu, uF, te[d], gn[d]);
        nn[d] = m[a][b][c] - te[d];
    }
    {
        const float h2 = 0.5f * (1.0f + r.om2);
        const float tr = r.cb * (nn[0] + nn[1] + nn[2]), gtr = 0.5f * r.cb * (gn[0] + gn[1] + gn[2]);
        m[2][0][0] = fmaf(r.om2, nn[0], te[0]) - tr + fmaf(h2, gn[0], -gtr);
        m[0][2][0] = fmaf(r.om2, nn[1], te[1]) - tr + fmaf(h2, gn[1], -gtr);
        m[0][0][2] = fmaf(r.om2, nn[2], te[2]) - tr + fmaf(h2, gn[2], -gtr);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int n1 = (a == 1) + (b == 1) + (c == 1), n2 = (a == 2) + (b == 2) + (c == 2);
                if (n1 + n2 <= 1 || (n1 == 0 && n2 == 1)) continue;  // conserved or the block
                float teq, g;
                feq_guo_moment27(a, b, c, drho, rho, u, F, uu, uF, teq, g);
                const float om = om27(a, b, c, r);
                m[a][b][c] = fmaf(om, m[a][b][c] - teq, fmaf(0.5f * (1.0f + om), g, teq));
            }
    m[0][0][0] = drho;
    m[1][0][0] = jx + 0.5f * Fx;
    m[0][1][0] = jy + 0.5f * Fy;
    m[0][0][1] = jz + 0.5f * Fz;
    inverse_axis<2>(m);
    inverse_axis<1>(m);
    inverse_axis<0>(m);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) h[a][b][c] = m[a][b][c];
    return drho;
}

// SRT on D3Q27 deviations: the MRT collision with every rate equal to s2
// (Sec. II.A), so mass and momentum come out exactly (see collide_srt in
// models.cuh for why not per population).
template <bool FR = false>
__device__ __forceinline__ float collide_srt27(float (&h)[3][3][3], float Fx, float Fy, float Fz,
                                               const Rates27 &r) {
    const float om = r.om2;
    Rates27 e;
    e.om2 = om;
    e.cb = 0.0f;
    e.om3 = om;
    e.c3 = 0.5f * (1.0f + om) * kC;
    e.om3b = om;
    e.om4 = om;
    e.om4b = om;
    e.om5 = om;
    e.c5 = 0.5f * (1.0f + om) * kC2;
    e.om6 = om;
    return collide_mrt27<FR>(h, Fx, Fy, Fz, e);
}

}  // namespace clbm
