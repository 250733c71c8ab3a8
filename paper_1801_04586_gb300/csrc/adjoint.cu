// adjoint.cu -- hand-written reverse of one stream-and-collide step, for
// gradients of a loss on the final velocity with respect to the body force.
//
// Forward step (Eq. 8 after Eqs. 5, 7, 9; see d3q19.cuh): f^{t+1} = P C(f^t, F),
// with C the node collision and P the streaming permutation (periodic wrap or
// halfway bounce-back). Its adjoint, per node x:
//   lam*(x)  = lam^{t+1} read at the slot (x, i) streams into: (i, x + e_i), or
//              (ibar, x) when x + e_i lies beyond a wall face   (P transposed)
//   lam^t(x) = J_f(x)^T lam*(x),  dL/dF(x) += J_F(x)^T lam*(x)
// where J is the Jacobian of the deviation-form collision. The collision is
// recomputed from f^t and differentiated by hand in reverse order:
//   h* = M^-1 q,  q = R* + e',  R* = N(-u) D*,  D* = Lam D + C~(F),
//   D = N(u) r,  r = M h - e',  e' = raw moments of the generalized
//   equilibrium minus those of the rest state, u = (M_1 h + F/2)/rho.
// Transposed shifts are applied as transposed triplet factors in reverse
// order. The velocity derivative of a shifted moment vector is a lower-order
// moment of the same vector: d/du_x of N(-u) D* at (m,n,p) is
// m R*_{m-1,n,p}, and of N(u) r it is -m D_{m-1,n,p}; so only D and R* are
// kept from the forward recomputation.
#include "kernels.cuh"

namespace clbm {

// Transposed triplet factors. Unshift (c -> k with velocity v) has matrix
// [[1,0,0],[v,1,0],[v^2,2v,1]]; its transpose maps (a0,a1,a2) to
// (a0 + v a1 + v^2 a2, a1 + 2 v a2, a2). The shift is the unshift with -v.
__device__ __forceinline__ void unshiftT(float &a0, float &a1, float a2, float v) {
    const float t = fmaf(v, a2, a1);
    a1 = fmaf(v, a2, t);
    a0 = fmaf(v, t, a0);
}

// Adjoint of the 15 generalized-equilibrium deviations e (eq_dev) with
// respect to drho, rho, j and u, accumulated.
__device__ __forceinline__ void eq_dev_adjoint(const Moments &eb, float rho, float jx, float jy, float jz, float ux,
                                               float uy, float uz, float &b_drho, float &b_rho, float &b_jx,
                                               float &b_jy, float &b_jz, float &b_ux, float &b_uy, float &b_uz) {
    const float X = ux * ux, Y = uy * uy, Z = uz * uz;
    // e110 = jx uy, e101 = jx uz, e011 = jy uz
    b_jx += eb.m110 * uy + eb.m101 * uz;
    b_jy += eb.m011 * uz;
    b_uy += eb.m110 * jx;
    b_uz += eb.m101 * jx + eb.m011 * jy;
    // e200 = jx ux + drho/3 (and y, z)
    b_jx += eb.m200 * ux; b_ux += eb.m200 * jx;
    b_jy += eb.m020 * uy; b_uy += eb.m020 * jy;
    b_jz += eb.m002 * uz; b_uz += eb.m002 * jz;
    b_drho += kC * (eb.m200 + eb.m020 + eb.m002);
    // third order: e120 = jx (Y + c), e102 = jx (Z + c), e210 = jy (X + c),
    //              e201 = jz (X + c), e012 = jy (Z + c), e021 = jz (Y + c)
    b_jx += eb.m120 * (Y + kC) + eb.m102 * (Z + kC);
    b_jy += eb.m210 * (X + kC) + eb.m012 * (Z + kC);
    b_jz += eb.m201 * (X + kC) + eb.m021 * (Y + kC);
    b_ux += 2.0f * ux * (eb.m210 * jy + eb.m201 * jz);
    b_uy += 2.0f * uy * (eb.m120 * jx + eb.m021 * jz);
    b_uz += 2.0f * uz * (eb.m102 * jx + eb.m012 * jy);
    // fourth order: e220 = rho (X Y + c (X + Y)) + drho/9, ...
    b_rho += eb.m220 * fmaf(X, Y, kC * (X + Y)) + eb.m202 * fmaf(X, Z, kC * (X + Z)) +
             eb.m022 * fmaf(Y, Z, kC * (Y + Z));
    b_drho += kC2 * (eb.m220 + eb.m202 + eb.m022);
    b_ux += 2.0f * rho * ux * (eb.m220 * (Y + kC) + eb.m202 * (Z + kC));
    b_uy += 2.0f * rho * uy * (eb.m220 * (X + kC) + eb.m022 * (Z + kC));
    b_uz += 2.0f * rho * uz * (eb.m202 * (X + kC) + eb.m022 * (Y + kC));
}

// lam = M^T kb (Eq. A4 transposed): lam_i = sum_j kb_j e_i^(m_j, n_j, p_j).
__device__ __forceinline__ void moments_transpose(const Moments &kb, float (&lam)[kQ]) {
    const float b0 = kb.m000;
    const float ax = b0 + kb.m200, ay = b0 + kb.m020, az = b0 + kb.m002;
    lam[0] = b0;
    lam[1] = ax + kb.m100; lam[2] = ax - kb.m100;
    lam[3] = ay + kb.m010; lam[4] = ay - kb.m010;
    lam[5] = az + kb.m001; lam[6] = az - kb.m001;
    // xy plane: terms in ex (100, 120), ey (010, 210), ex ey (110), even (000, 200, 020, 220)
    {
        const float ev = b0 + kb.m200 + kb.m020 + kb.m220;
        const float sx = kb.m100 + kb.m120, sy = kb.m010 + kb.m210;
        lam[7] = ev + sx + sy + kb.m110;
        lam[8] = ev - sx + sy - kb.m110;
        lam[9] = ev + sx - sy - kb.m110;
        lam[10] = ev - sx - sy + kb.m110;
    }
    {
        const float ev = b0 + kb.m200 + kb.m002 + kb.m202;
        const float sx = kb.m100 + kb.m102, sz = kb.m001 + kb.m201;
        lam[11] = ev + sx + sz + kb.m101;
        lam[12] = ev - sx + sz - kb.m101;
        lam[13] = ev + sx - sz - kb.m101;
        lam[14] = ev - sx - sz + kb.m101;
    }
    {
        const float ev = b0 + kb.m020 + kb.m002 + kb.m022;
        const float sy = kb.m010 + kb.m012, sz = kb.m001 + kb.m021;
        lam[15] = ev + sy + sz + kb.m011;
        lam[16] = ev - sy + sz - kb.m011;
        lam[17] = ev + sy - sz - kb.m011;
        lam[18] = ev - sy - sz + kb.m011;
    }
}

// qb = M^-T lam (transpose of inverse_moments in d3q19.cuh).
__device__ __forceinline__ void inverse_moments_transpose(const float (&l)[kQ], Moments &qb) {
    const float P1 = l[1] + l[2], M1 = l[1] - l[2];
    const float P2 = l[3] + l[4], M2 = l[3] - l[4];
    const float P3 = l[5] + l[6], M3 = l[5] - l[6];
    const float Sxy = (l[7] + l[8]) + (l[9] + l[10]), Axy = (l[7] + l[8]) - (l[9] + l[10]);
    const float Bxy = (l[7] + l[9]) - (l[8] + l[10]), Cxy = (l[7] + l[10]) - (l[8] + l[9]);
    const float Sxz = (l[11] + l[12]) + (l[13] + l[14]), Axz = (l[11] + l[12]) - (l[13] + l[14]);
    const float Bxz = (l[11] + l[13]) - (l[12] + l[14]), Cxz = (l[11] + l[14]) - (l[12] + l[13]);
    const float Syz = (l[15] + l[16]) + (l[17] + l[18]), Ayz = (l[15] + l[16]) - (l[17] + l[18]);
    const float Byz = (l[15] + l[17]) - (l[16] + l[18]), Cyz = (l[15] + l[18]) - (l[16] + l[17]);
    qb.m000 = l[0];
    qb.m200 = 0.5f * P1 - l[0]; qb.m020 = 0.5f * P2 - l[0]; qb.m002 = 0.5f * P3 - l[0];
    qb.m100 = 0.5f * M1; qb.m010 = 0.5f * M2; qb.m001 = 0.5f * M3;
    qb.m220 = l[0] - 0.5f * (P1 + P2) + 0.25f * Sxy;
    qb.m202 = l[0] - 0.5f * (P1 + P3) + 0.25f * Sxz;
    qb.m022 = l[0] - 0.5f * (P2 + P3) + 0.25f * Syz;
    qb.m120 = 0.25f * Bxy - 0.5f * M1; qb.m102 = 0.25f * Bxz - 0.5f * M1;
    qb.m210 = 0.25f * Axy - 0.5f * M2; qb.m012 = 0.25f * Byz - 0.5f * M2;
    qb.m201 = 0.25f * Axz - 0.5f * M3; qb.m021 = 0.25f * Ayz - 0.5f * M3;
    qb.m110 = 0.25f * Cxy; qb.m101 = 0.25f * Cxz; qb.m011 = 0.25f * Cyz;
}

// Reverse of collide(): given h (pre-collision deviations, Eq. 9 state) and
// lam = dL/dh*, returns lam <- dL/dh and accumulates dL/dF.
__device__ __forceinline__ void collide_adjoint(const float (&h)[kQ], float (&lam)[kQ], float Fx, float Fy,
                                                float Fz, const Rates &r, float &gFx, float &gFy, float &gFz) {
    // ---------------- forward recomputation (as collide()), keeping D and R*
    Moments k;
    raw_moments(h, k);
    const float drho = k.m000;
    const float rho = 1.0f + drho;
    const float inv = 1.0f / rho;
    const float jx = fmaf(0.5f, Fx, k.m100), jy = fmaf(0.5f, Fy, k.m010), jz = fmaf(0.5f, Fz, k.m001);
    const float ux = jx * inv, uy = jy * inv, uz = jz * inv;
    EqDev e;
    eq_dev(drho, rho, jx, jy, jz, ux, uy, uz, e);
    const float hFx = 0.5f * Fx, hFy = 0.5f * Fy, hFz = 0.5f * Fz;
    Moments D;  // central non-equilibrium moments (D000 = 0, D1 = -F/2)
    D.m110 = k.m110 - e.d110; D.m101 = k.m101 - e.d101; D.m011 = k.m011 - e.d011;
    D.m200 = k.m200 - e.d200; D.m020 = k.m020 - e.d020; D.m002 = k.m002 - e.d002;
    D.m120 = k.m120 - e.d120; D.m102 = k.m102 - e.d102; D.m210 = k.m210 - e.d210;
    D.m201 = k.m201 - e.d201; D.m012 = k.m012 - e.d012; D.m021 = k.m021 - e.d021;
    D.m220 = k.m220 - e.d220; D.m202 = k.m202 - e.d202; D.m022 = k.m022 - e.d022;
    D.m200 = fmaf(ux, Fx, D.m200);
    shift3(-hFy, D.m110, D.m210, ux);
    shift3(-hFz, D.m101, D.m201, ux);
    shift3(D.m020, D.m120, D.m220, ux);
    shift3(D.m002, D.m102, D.m202, ux);
    D.m020 = fmaf(uy, Fy, D.m020);
    shift3(-hFx, D.m110, D.m120, uy);
    shift3(-hFz, D.m011, D.m021, uy);
    shift3(D.m200, D.m210, D.m220, uy);
    shift3(D.m002, D.m012, D.m022, uy);
    D.m002 = fmaf(uz, Fz, D.m002);
    shift3(-hFx, D.m101, D.m102, uz);
    shift3(-hFy, D.m011, D.m012, uz);
    shift3(D.m200, D.m201, D.m202, uz);
    shift3(D.m020, D.m021, D.m022, uz);
    Moments R;  // becomes R* = N(-u) D* (R000 = 0, R1 = F/2)
    R.m110 = r.om2 * D.m110; R.m101 = r.om2 * D.m101; R.m011 = r.om2 * D.m011;
    {
        const float tr = r.cb * (D.m200 + D.m020 + D.m002);
        R.m200 = fmaf(r.om2, D.m200, -tr);
        R.m020 = fmaf(r.om2, D.m020, -tr);
        R.m002 = fmaf(r.om2, D.m002, -tr);
    }
    R.m120 = fmaf(r.om3, D.m120, r.c3 * Fx);
    R.m102 = fmaf(r.om3, D.m102, r.c3 * Fx);
    R.m210 = fmaf(r.om3, D.m210, r.c3 * Fy);
    R.m201 = fmaf(r.om3, D.m201, r.c3 * Fz);
    R.m012 = fmaf(r.om3, D.m012, r.c3 * Fy);
    R.m021 = fmaf(r.om3, D.m021, r.c3 * Fz);
    R.m220 = r.om4 * D.m220; R.m202 = r.om4 * D.m202; R.m022 = r.om4 * D.m022;
    R.m002 = fmaf(uz, Fz, R.m002);
    unshift3(hFx, R.m101, R.m102, uz);
    unshift3(hFy, R.m011, R.m012, uz);
    unshift3(R.m200, R.m201, R.m202, uz);
    unshift3(R.m020, R.m021, R.m022, uz);
    R.m020 = fmaf(uy, Fy, R.m020);
    unshift3(hFx, R.m110, R.m120, uy);
    unshift3(hFz, R.m011, R.m021, uy);
    unshift3(R.m200, R.m210, R.m220, uy);
    unshift3(R.m002, R.m012, R.m022, uy);
    R.m200 = fmaf(ux, Fx, R.m200);
    unshift3(hFy, R.m110, R.m210, ux);
    unshift3(hFz, R.m101, R.m201, ux);
    unshift3(R.m020, R.m120, R.m220, ux);
    unshift3(R.m002, R.m102, R.m202, ux);

    // ---------------- reverse
    float b_drho = 0.f, b_rho = 0.f, b_jx = 0.f, b_jy = 0.f, b_jz = 0.f, b_ux = 0.f, b_uy = 0.f, b_uz = 0.f;
    float bFx = 0.f, bFy = 0.f, bFz = 0.f;
    Moments B;  // adjoint vector, reused: q-bar -> R*-bar -> D*-bar -> D-bar -> r-bar
    inverse_moments_transpose(lam, B);
    // q000 = drho, q1 = j + F/2, q_other = R*_other + e_other
    b_drho += B.m000;
    b_jx += B.m100; b_jy += B.m010; b_jz += B.m001;
    bFx += 0.5f * B.m100; bFy += 0.5f * B.m010; bFz += 0.5f * B.m001;
    eq_dev_adjoint(B, rho, jx, jy, jz, ux, uy, uz, b_drho, b_rho, b_jx, b_jy, b_jz, b_ux, b_uy, b_uz);
    B.m000 = 0.f; B.m100 = 0.f; B.m010 = 0.f; B.m001 = 0.f;  // R*000, R*1 are not outputs
    // d/du of R* = N(-u) D*: m R*_{m-1} (R*000 = 0, R*1 = F/2)
    b_ux += B.m110 * hFy + B.m101 * hFz + 2.f * B.m200 * hFx + B.m120 * R.m020 + B.m102 * R.m002 +
            2.f * (B.m210 * R.m110 + B.m201 * R.m101 + B.m220 * R.m120 + B.m202 * R.m102);
    b_uy += B.m110 * hFx + B.m011 * hFz + 2.f * B.m020 * hFy + B.m210 * R.m200 + B.m012 * R.m002 +
            2.f * (B.m120 * R.m110 + B.m021 * R.m011 + B.m220 * R.m210 + B.m022 * R.m012);
    b_uz += B.m101 * hFx + B.m011 * hFy + 2.f * B.m002 * hFz + B.m201 * R.m200 + B.m021 * R.m020 +
            2.f * (B.m102 * R.m101 + B.m012 * R.m011 + B.m202 * R.m201 + B.m022 * R.m021);
    // D*-bar = N(-u)^T R*-bar: x factors first, then y, then z
    unshiftT(B.m000, B.m100, B.m200, ux);
    unshiftT(B.m010, B.m110, B.m210, ux);
    unshiftT(B.m001, B.m101, B.m201, ux);
    unshiftT(B.m020, B.m120, B.m220, ux);
    unshiftT(B.m002, B.m102, B.m202, ux);
    unshiftT(B.m000, B.m010, B.m020, uy);
    unshiftT(B.m100, B.m110, B.m120, uy);
    unshiftT(B.m001, B.m011, B.m021, uy);
    unshiftT(B.m200, B.m210, B.m220, uy);
    unshiftT(B.m002, B.m012, B.m022, uy);
    unshiftT(B.m000, B.m001, B.m002, uz);
    unshiftT(B.m100, B.m101, B.m102, uz);
    unshiftT(B.m010, B.m011, B.m012, uz);
    unshiftT(B.m200, B.m201, B.m202, uz);
    unshiftT(B.m020, B.m021, B.m022, uz);
    // D*000 = 0, D*1 = F/2, third order carries c3 F
    bFx += 0.5f * B.m100 + r.c3 * (B.m120 + B.m102);
    bFy += 0.5f * B.m010 + r.c3 * (B.m210 + B.m012);
    bFz += 0.5f * B.m001 + r.c3 * (B.m201 + B.m021);
    // D-bar = Lam D*-bar (Lam symmetric; zero on the conserved moments)
    B.m000 = 0.f; B.m100 = 0.f; B.m010 = 0.f; B.m001 = 0.f;
    B.m110 *= r.om2; B.m101 *= r.om2; B.m011 *= r.om2;
    {
        const float tr = r.cb * (B.m200 + B.m020 + B.m002);
        B.m200 = fmaf(r.om2, B.m200, -tr);
        B.m020 = fmaf(r.om2, B.m020, -tr);
        B.m002 = fmaf(r.om2, B.m002, -tr);
    }
    B.m120 *= r.om3; B.m102 *= r.om3; B.m210 *= r.om3; B.m201 *= r.om3; B.m012 *= r.om3; B.m021 *= r.om3;
    B.m220 *= r.om4; B.m202 *= r.om4; B.m022 *= r.om4;
    // d/du of D = N(u) r: -m D_{m-1} (D000 = 0, D1 = -F/2)
    b_ux -= -B.m110 * hFy - B.m101 * hFz - 2.f * B.m200 * hFx + B.m120 * D.m020 + B.m102 * D.m002 +
            2.f * (B.m210 * D.m110 + B.m201 * D.m101 + B.m220 * D.m120 + B.m202 * D.m102);
    b_uy -= -B.m110 * hFx - B.m011 * hFz - 2.f * B.m020 * hFy + B.m210 * D.m200 + B.m012 * D.m002 +
            2.f * (B.m120 * D.m110 + B.m021 * D.m011 + B.m220 * D.m210 + B.m022 * D.m012);
    b_uz -= -B.m101 * hFx - B.m011 * hFy - 2.f * B.m002 * hFz + B.m201 * D.m200 + B.m021 * D.m020 +
            2.f * (B.m102 * D.m101 + B.m012 * D.m011 + B.m202 * D.m201 + B.m022 * D.m021);
    // r-bar = N(u)^T D-bar: z factors first, then y, then x (shift = unshift with -v)
    unshiftT(B.m000, B.m001, B.m002, -uz);
    unshiftT(B.m100, B.m101, B.m102, -uz);
    unshiftT(B.m010, B.m011, B.m012, -uz);
    unshiftT(B.m200, B.m201, B.m202, -uz);
    unshiftT(B.m020, B.m021, B.m022, -uz);
    unshiftT(B.m000, B.m010, B.m020, -uy);
    unshiftT(B.m100, B.m110, B.m120, -uy);
    unshiftT(B.m001, B.m011, B.m021, -uy);
    unshiftT(B.m200, B.m210, B.m220, -uy);
    unshiftT(B.m002, B.m012, B.m022, -uy);
    unshiftT(B.m000, B.m100, B.m200, -ux);
    unshiftT(B.m010, B.m110, B.m210, -ux);
    unshiftT(B.m001, B.m101, B.m201, -ux);
    unshiftT(B.m020, B.m120, B.m220, -ux);
    unshiftT(B.m002, B.m102, B.m202, -ux);
    // r000 = 0, r1 = -F/2, r_other = k_other - e_other
    bFx -= 0.5f * B.m100; bFy -= 0.5f * B.m010; bFz -= 0.5f * B.m001;
    {
        Moments neg;
        neg.m110 = -B.m110; neg.m101 = -B.m101; neg.m011 = -B.m011;
        neg.m200 = -B.m200; neg.m020 = -B.m020; neg.m002 = -B.m002;
        neg.m120 = -B.m120; neg.m102 = -B.m102; neg.m210 = -B.m210;
        neg.m201 = -B.m201; neg.m012 = -B.m012; neg.m021 = -B.m021;
        neg.m220 = -B.m220; neg.m202 = -B.m202; neg.m022 = -B.m022;
        eq_dev_adjoint(neg, rho, jx, jy, jz, ux, uy, uz, b_drho, b_rho, b_jx, b_jy, b_jz, b_ux, b_uy, b_uz);
    }
    // u = j / rho, rho = 1 + drho, j = k1 + F/2, drho = k000
    b_jx += b_ux * inv; b_jy += b_uy * inv; b_jz += b_uz * inv;
    b_rho -= (b_ux * ux + b_uy * uy + b_uz * uz) * inv;
    b_drho += b_rho;
    bFx += 0.5f * b_jx; bFy += 0.5f * b_jy; bFz += 0.5f * b_jz;
    B.m000 = b_drho;
    B.m100 = b_jx; B.m010 = b_jy; B.m001 = b_jz;
    moments_transpose(B, lam);
    gFx += bFx; gFy += bFy; gFz += bFz;
}

template <int FM>
__device__ __forceinline__ void force_adj(const ForceArgs &F, const Geom &g, int z, uint32_t self, float &fx,
                                          float &fy, float &fz) {
    if (FM == kForceUniform) {
        fx = F.fx; fy = F.fy; fz = F.fz;
    } else if (FM == kForceProfileZ) {
        fx = __ldg(F.profile + z); fy = __ldg(F.profile + g.nz + z); fz = __ldg(F.profile + 2 * g.nz + z);
    } else {
        fx = __ldg(F.field + self); fy = __ldg(F.field + F.n + self); fz = __ldg(F.field + 2 * F.n + self);
    }
    fx *= F.scale;
    fy *= F.scale;
    fz *= F.scale;
}

// push_targets on a z-slab (Geom::slab): z walls only at faces that are not
// halo faces, and a population leaving across a halo face (not bounced back at
// an x or y wall) has its target in the neighbour's first or last plane. The
// adjoint of that target comes from the receive planes appended to the lambda
// array (pop = kQ, off within them): planes 0-4 the lower neighbour's last
// plane (e_z = -1 at z = 0), planes 5-9 the upper neighbour's first plane
// (e_z = +1 at z = nz - 1), in the order of zface_index.
template <bool WALLS>
__device__ __forceinline__ void push_targets_slab(const Geom &g, int x, int y, int z, uint32_t (&off)[kQ],
                                                  int (&pop)[kQ]) {
    push_targets<false>(g, x, y, z, off, pop);  // periodic targets
    const uint32_t plane = (uint32_t)g.nx * (uint32_t)g.ny;
    const uint32_t self = (uint32_t)z * plane + (uint32_t)y * (uint32_t)g.nx + (uint32_t)x;
    bool bb[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) bb[i] = false;
    if (WALLS) {
        const bool wx = g.walls & 1u, wy = g.walls & 2u, wz = g.walls & 4u;
        const bool xl = wx && x == 0, xh = wx && x == g.nx - 1;  // leaving through x- (ex = -1) / x+ (ex = +1)
        const bool yl = wy && y == 0, yh = wy && y == g.ny - 1;
        const bool zl = wz && z == 0 && !(g.slab & 1u), zh = wz && z == g.nz - 1 && !(g.slab & 2u);
        const bool w[kQ] = {false,
                            xh, xl, yh, yl, zh, zl,
                            xh || yh, xl || yh, xh || yl, xl || yl,
                            xh || zh, xl || zh, xh || zl, xl || zl,
                            yh || zh, yl || zh, yh || zl, yl || zl};
#pragma unroll
        for (int i = 1; i < kQ; ++i) {
            bb[i] = w[i];
            if (w[i]) {
                pop[i] = opposite(i);
                off[i] = self;
            }
        }
    }
    const int zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;
    if ((g.slab & 1u) && z == 0) {
#pragma unroll
        for (int i = 1; i < kQ; ++i)
            if (ez19(i) < 0 && !bb[i]) {
                pop[i] = kQ;
                off[i] = (uint32_t)zface_index(i) * plane + (off[i] - (uint32_t)zm * plane);
            }
    }
    if ((g.slab & 2u) && z == g.nz - 1) {
#pragma unroll
        for (int i = 1; i < kQ; ++i)
            if (ez19(i) > 0 && !bb[i]) {
                pop[i] = kQ;
                off[i] = (uint32_t)(5 + zface_index(i)) * plane + (off[i] - (uint32_t)zp * plane);
            }
    }
}

// A z-slab's outgoing adjoint faces, after the 10 receive planes of the lambda
// array: its first plane's lambda of the e_z = +1 populations (send planes
// 10-14, for the lower neighbour, whose last plane pushes them into this one)
// and its last plane's lambda of the e_z = -1 populations (15-19, for the upper
// neighbour).
__device__ __forceinline__ void send_adjoint_faces(float *lam, const Geom &g, int64_t n, int z, uint32_t self,
                                                   const float (&l)[kQ]) {
    const uint32_t plane = (uint32_t)g.nx * (uint32_t)g.ny, ps = self - (uint32_t)z * plane;
    float *send = lam + (size_t)kQ * n + (size_t)10 * plane + ps;
    if ((g.slab & 1u) && z == 0) {
#pragma unroll
        for (int i = 1; i < kQ; ++i)
            if (ez19(i) > 0) send[(size_t)zface_index(i) * plane] = l[i];
    }
    if ((g.slab & 2u) && z == g.nz - 1) {
#pragma unroll
        for (int i = 1; i < kQ; ++i)
            if (ez19(i) < 0) send[(size_t)(5 + zface_index(i)) * plane] = l[i];
    }
}

// One adjoint step. state: raw buffer whose pull gives f^t; lam_next: adjoint
// of f^{t+1} (19 x n, post-streaming layout); lam: adjoint of f^t (19 x n);
// gF: dL/dF accumulated (3 x n). The node's three gF values are read first,
// beside its gathers, so their latency is hidden behind the collision instead
// of adding a second memory round trip at the end; 80 registers keep three
// blocks per SM (a few bytes spill): 0.94 against 0.82 of the copy roofline.
// SLAB: a z-slab (pull through the halo map, gathers across halo faces from
// lam_next's receive planes, send planes of lam written).
template <typename S, int FM, bool WALLS, bool SLAB>
__global__ void __launch_bounds__(256, 3) k_adjoint_step(const S *__restrict__ state, const float *__restrict__ lam_next,
                                                      float *__restrict__ lam, float *__restrict__ gF, Geom g,
                                                      Rates r, ForceArgs F, int64_t n) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const uint32_t self0 = ((uint32_t)z * g.ny + y) * g.nx + x;
    const float g0x = gF[self0], g0y = gF[n + self0], g0z = gF[2 * n + self0];
    float l[kQ];
    {
        uint32_t off[kQ];
        int pop[kQ];
        if (SLAB)
            push_targets_slab<WALLS>(g, x, y, z, off, pop);
        else
            push_targets<WALLS>(g, x, y, z, off, pop);
#pragma unroll
        for (int i = 0; i < kQ; ++i) l[i] = __ldg(lam_next + (size_t)pop[i] * n + off[i]);
    }
    float h[kQ];
    uint32_t self;
    {
        uint32_t off[kQ];
        int pop[kQ];
        pull_sources<WALLS, false, SLAB>(g, x, y, z, off, pop);
#pragma unroll
        for (int i = 0; i < kQ; ++i) h[i] = Codec<S>::load(state + (size_t)pop[i] * g.stride + off[i]);
        self = off[0];
    }
    float fx, fy, fz;
    force_adj<FM>(F, g, z, self, fx, fy, fz);
    float gx = 0.f, gy = 0.f, gz = 0.f;
    collide_adjoint(h, l, fx, fy, fz, r, gx, gy, gz);
#pragma unroll
    for (int i = 0; i < kQ; ++i) lam[(size_t)i * n + self] = l[i];
    if (SLAB) send_adjoint_faces(lam, g, n, z, self, l);
    gF[self] = g0x + gx;
    gF[n + self] = g0y + gy;
    gF[2 * n + self] = g0z + gz;
}

// Seed from a cotangent gu (3 x n) on the Eq. 9 velocity of the state in
// `state`: lam_i = sum_a gu_a (e_ia - u_a)/rho, gF = gu/(2 rho) (written).
template <typename S, int FM, bool WALLS, bool SLAB>
__global__ void k_adjoint_seed(const S *__restrict__ state, const float *__restrict__ gu, float *__restrict__ lam,
                               float *__restrict__ gF, Geom g, ForceArgs F, int64_t n) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    uint32_t off[kQ];
    int pop[kQ];
    pull_sources<WALLS, false, SLAB>(g, x, y, z, off, pop);
    float h[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) h[i] = Codec<S>::load(state + (size_t)pop[i] * g.stride + off[i]);
    const uint32_t self = off[0];
    float fx, fy, fz, jx, jy, jz;
    force_adj<FM>(F, g, z, self, fx, fy, fz);
    const float rho = 1.0f + macros_dev(h, fx, fy, fz, jx, jy, jz);
    const float inv = 1.0f / rho;
    const float ux = jx * inv, uy = jy * inv, uz = jz * inv;
    const float ax = gu[self] * inv, ay = gu[n + self] * inv, az = gu[2 * n + self] * inv;
    const float base = -(ax * ux + ay * uy + az * uz);
    // lam_i = base + ax e_ix + ay e_iy + az e_iz
    const float l[kQ] = {base,
                         base + ax, base - ax, base + ay, base - ay, base + az, base - az,
                         base + ax + ay, base - ax + ay, base + ax - ay, base - ax - ay,
                         base + ax + az, base - ax + az, base + ax - az, base - ax - az,
                         base + ay + az, base - ay + az, base + ay - az, base - ay - az};
#pragma unroll
    for (int i = 0; i < kQ; ++i) lam[(size_t)i * n + self] = l[i];
    if (SLAB) send_adjoint_faces(lam, g, n, z, self, l);
    gF[self] = 0.5f * ax;
    gF[n + self] = 0.5f * ay;
    gF[2 * n + self] = 0.5f * az;
}

#define CLBM_ADJ_LAUNCH(FMODE, walls, slab, KERNEL, ...)                                                     \
    do {                                                                                                    \
        if (slab) {                                                                                         \
            if (walls) KERNEL<S, FMODE, true, true><<<L.grid, L.block, 0, L.stream>>>(__VA_ARGS__);         \
            else KERNEL<S, FMODE, false, true><<<L.grid, L.block, 0, L.stream>>>(__VA_ARGS__);              \
        } else {                                                                                            \
            if (walls) KERNEL<S, FMODE, true, false><<<L.grid, L.block, 0, L.stream>>>(__VA_ARGS__);        \
            else KERNEL<S, FMODE, false, false><<<L.grid, L.block, 0, L.stream>>>(__VA_ARGS__);             \
        }                                                                                                   \
    } while (0)

#define CLBM_ADJ_DISPATCH(storage, fmode, walls, slab, KERNEL, ...)                                          \
    do {                                                                                                    \
        if ((storage) != 0) return cudaErrorInvalidValue;                                                   \
        using S = float;                                                                                    \
        switch (fmode) {                                                                                    \
            case kForceUniform: CLBM_ADJ_LAUNCH(kForceUniform, walls, slab, KERNEL, __VA_ARGS__); break;     \
            case kForceProfileZ: CLBM_ADJ_LAUNCH(kForceProfileZ, walls, slab, KERNEL, __VA_ARGS__); break;   \
            default: CLBM_ADJ_LAUNCH(kForceField, walls, slab, KERNEL, __VA_ARGS__); break;                  \
        }                                                                                                   \
    } while (0)

cudaError_t launch_adjoint_step(int storage, const Launch &L, const void *state, const float *lam_next, float *lam,
                                float *gF, const Rates &r, const ForceArgs &F, int64_t n) {
    CLBM_ADJ_DISPATCH(storage, F.mode, L.g.walls, L.g.slab, k_adjoint_step, (const S *)state, lam_next, lam, gF, L.g,
                      r, F, n);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_seed(int storage, const Launch &L, const void *state, const float *gu, float *lam,
                                float *gF, const ForceArgs &F, int64_t n) {
    CLBM_ADJ_DISPATCH(storage, F.mode, L.g.walls, L.g.slab, k_adjoint_seed, (const S *)state, gu, lam, gF, L.g, F,
                      n);
    return cudaGetLastError();
}

}  // namespace clbm
