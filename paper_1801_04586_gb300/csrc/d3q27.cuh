// d3q27.cuh -- device-side D3Q27 cascaded-LBM node arithmetic (Sec. II of
// Fei, Luo & Li, arXiv:1801.04586: velocities Eq. 1, moment set Eq. 12,
// relaxation matrix Eq. 13, equilibria Eq. 15, forcing terms Eq. 16).
//
// The D3Q27 moment set holds every exponent triple (m, n, p) in {0,1,2}^3, so
// M = Mx (x) My (x) Mz is a tensor product of one 3 x 3 map per axis acting on
// the three populations of a line with e = 0, +1, -1:
//   (f0, f+, f-) -> (k0, k1, k2) = (f0 + f+ + f-, f+ - f-, f+ + f-),
// and M^-1 is the inverse per axis: f0 = k0 - k2, f+ = (k2 + k1)/2,
// f- = (k2 - k1)/2. The shift N(u) factors per axis as in d3q19.cuh
// (shift3 / unshift3 on every line). Populations are held as a cube
// c[ix][iy][iz] (index 0: e = 0, 1: e = +1, 2: e = -1), moments as a cube
// m[a][b][c] of exponents. Arithmetic is on deviations from the rest weights,
// as in d3q19.cuh: R = M f - rho G(u) with rho G(u) = rho g_a(ux) g_b(uy)
// g_c(uz), g = (1, u, u^2 + c_s^2).
#pragma once

#include "d3q19.cuh"

namespace clbm {

constexpr int kQ27 = 27;

// Eq. 1 velocity index of the population with components (e_x, e_y, e_z),
// each coded 0 (zero), 1 (+1), 2 (-1).
__host__ __device__ constexpr int q27_index(int ix, int iy, int iz) {
    // rest, axes, xy / xz / yz edges, corners in the order of Eq. 1
    return (ix | iy | iz) == 0 ? 0
         : (iy == 0 && iz == 0) ? (ix == 1 ? 1 : 2)
         : (ix == 0 && iz == 0) ? (iy == 1 ? 3 : 4)
         : (ix == 0 && iy == 0) ? (iz == 1 ? 5 : 6)
         : iz == 0 ? 7 + (ix == 1 ? 0 : 1) + (iy == 1 ? 0 : 2)
         : iy == 0 ? 11 + (ix == 1 ? 0 : 1) + (iz == 1 ? 0 : 2)
         : ix == 0 ? 15 + (iy == 1 ? 0 : 1) + (iz == 1 ? 0 : 2)
         : 19 + (ix == 1 ? 0 : 1) + (iy == 1 ? 0 : 2) + (iz == 1 ? 0 : 4);
}
__host__ __device__ constexpr int e_of(int code) { return code == 0 ? 0 : (code == 1 ? 1 : -1); }

// Rest weights: products of the 1D weights 2/3 (e = 0) and 1/6 (e = +-1).
__host__ __device__ constexpr float rest_weight27_code(int ix, int iy, int iz) {
    return (ix ? 1.0f / 6.0f : 2.0f / 3.0f) * (iy ? 1.0f / 6.0f : 2.0f / 3.0f) * (iz ? 1.0f / 6.0f : 2.0f / 3.0f);
}

struct Rates27 {
    float om2, cb, om3, c3;  // as Rates (second- and third-order of Eq. 13)
    float om3b;              // 1 - s3b: k~111
    float om4;               // 1 - s4: k~220, k~202, k~022
    float om4b;              // 1 - s4b: k~211, k~121, k~112
    float om5, c5;           // 1 - s5 and (1 - s5/2) c_s^4: k~122, k~212, k~221 (Eq. 16)
    float om6;               // 1 - s6: k~222
};

// Pull sources of the 27 populations arriving at (x, y, z), population index
// by cube code: periodic wrap, or halfway bounce-back (the opposite population
// at the node itself) when x - e lies beyond a wall face. SWAP = true gives
// the opposite population index at the same offsets: the slots of the
// in-place (AA) pattern's odd step (as pull_sources in d3q19.cuh).
template <bool WALLS, bool SWAP = false>
__device__ __forceinline__ void pull_sources27(const Geom &g, int x, int y, int z, uint32_t (&off)[3][3][3],
                                               int (&pop)[3][3][3]) {
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    // source coordinate for e = 0, +1, -1
    const int xs[3] = {x, x == 0 ? nx - 1 : x - 1, x == nx - 1 ? 0 : x + 1};
    const int ys[3] = {y, y == 0 ? ny - 1 : y - 1, y == ny - 1 ? 0 : y + 1};
    const int zs[3] = {z, z == 0 ? nz - 1 : z - 1, z == nz - 1 ? 0 : z + 1};
    bool bx[3] = {false, false, false}, by[3] = {false, false, false}, bz[3] = {false, false, false};
    if (WALLS) {
        bx[1] = (g.walls & 1u) && x == 0; bx[2] = (g.walls & 1u) && x == nx - 1;
        by[1] = (g.walls & 2u) && y == 0; by[2] = (g.walls & 2u) && y == ny - 1;
        bz[1] = (g.walls & 4u) && z == 0; bz[2] = (g.walls & 4u) && z == nz - 1;
    }
    const uint32_t self = ((uint32_t)z * ny + y) * nx + x;
#pragma unroll
    for (int iz = 0; iz < 3; ++iz)
#pragma unroll
        for (int iy = 0; iy < 3; ++iy) {
            const uint32_t row = ((uint32_t)zs[iz] * ny + ys[iy]) * nx;
#pragma unroll
            for (int ix = 0; ix < 3; ++ix) {
                const bool bb = WALLS && (bx[ix] || by[iy] || bz[iz]);
                // opposite: swap codes 1 <-> 2 on every axis
                const int ox = ix == 0 ? 0 : 3 - ix, oy = iy == 0 ? 0 : 3 - iy, oz = iz == 0 ? 0 : 3 - iz;
                pop[ix][iy][iz] = (bb != SWAP) ? q27_index(ox, oy, oz) : q27_index(ix, iy, iz);
                off[ix][iy][iz] = bb ? self : row + xs[ix];
            }
        }
}

// Per-axis transforms on a cube. Axis A, line (i, j) over the other two axes.
#define CLBM_CUBE_LINE(c, A, i, j, k) (A == 0 ? c[k][i][j] : (A == 1 ? c[i][k][j] : c[i][j][k]))

template <int A>
__device__ __forceinline__ void raw_axis(float (&c)[3][3][3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float &f0 = CLBM_CUBE_LINE(c, A, i, j, 0), &fp = CLBM_CUBE_LINE(c, A, i, j, 1),
                  &fm = CLBM_CUBE_LINE(c, A, i, j, 2);
            const float k2 = fp + fm, k1 = fp - fm;
            f0 = f0 + k2;
            fp = k1;
            fm = k2;
        }
}

template <int A>
__device__ __forceinline__ void inverse_axis(float (&c)[3][3][3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float &k0 = CLBM_CUBE_LINE(c, A, i, j, 0), &k1 = CLBM_CUBE_LINE(c, A, i, j, 1),
                  &k2 = CLBM_CUBE_LINE(c, A, i, j, 2);
            const float fp = 0.5f * (k2 + k1), fm = 0.5f * (k2 - k1);
            k0 = k0 - k2;
            k1 = fp;
            k2 = fm;
        }
}

template <int A>
__device__ __forceinline__ void shift_axis(float (&c)[3][3][3], float v) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            shift3(CLBM_CUBE_LINE(c, A, i, j, 0), CLBM_CUBE_LINE(c, A, i, j, 1), CLBM_CUBE_LINE(c, A, i, j, 2), v);
}

template <int A>
__device__ __forceinline__ void unshift_axis(float (&c)[3][3][3], float v) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            unshift3(CLBM_CUBE_LINE(c, A, i, j, 0), CLBM_CUBE_LINE(c, A, i, j, 1), CLBM_CUBE_LINE(c, A, i, j, 2), v);
}

// rho G(u) - M w for the cube, telescoped so every term carries a small
// factor: with g = e + d per axis (e = (1, 0, c_s^2), d = (0, u, u^2)),
// rho g_a g_b g_c - e_a e_b e_c = drho g_a g_b g_c + d_a g_b g_c + e_a d_b g_c + e_a e_b d_c.
__device__ __forceinline__ void eq_dev27(float drho, float ux, float uy, float uz, float (&q)[3][3][3]) {
    const float gx[3] = {1.0f, ux, fmaf(ux, ux, kC)}, gy[3] = {1.0f, uy, fmaf(uy, uy, kC)},
                gz[3] = {1.0f, uz, fmaf(uz, uz, kC)};
    const float dx[3] = {0.0f, ux, ux * ux}, dy[3] = {0.0f, uy, uy * uy}, dz[3] = {0.0f, uz, uz * uz};
    const float e[3] = {1.0f, 0.0f, kC};
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float gbc = gy[b] * gz[c];
                q[a][b][c] = fmaf(drho, gx[a] * gbc, fmaf(dx[a], gbc, e[a] * fmaf(dy[b], gz[c], e[b] * dz[c])));
            }
}

// One collision on deviations h (cube by velocity code), in place; returns
// drho of the pre-collision state (Eq. 9).
template <bool FR = false>
__device__ __forceinline__ float collide27(float (&h)[3][3][3], float Fx, float Fy, float Fz, const Rates27 &r) {
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
    const float rho = 1.0f + drho;
    const float inv = recip_of<FR>(rho);
    const float jx = fmaf(0.5f, Fx, m[1][0][0]), jy = fmaf(0.5f, Fy, m[0][1][0]), jz = fmaf(0.5f, Fz, m[0][0][1]);
    const float ux = jx * inv, uy = jy * inv, uz = jz * inv;
    float e[3][3][3];
    eq_dev27(drho, ux, uy, uz, e);
    // non-equilibrium raw moments; exact values on the conserved ones
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) m[a][b][c] -= e[a][b][c];
    const float hFx = 0.5f * Fx, hFy = 0.5f * Fy, hFz = 0.5f * Fz;
    m[0][0][0] = 0.0f;
    m[1][0][0] = -hFx; m[0][1][0] = -hFy; m[0][0][1] = -hFz;
    // D = N(u) R
    shift_axis<0>(m, ux);
    shift_axis<1>(m, uy);
    shift_axis<2>(m, uz);
    // Eq. 5 on non-equilibrium central moments (s0 = s1 = 1)
    m[0][0][0] = 0.0f;
    m[1][0][0] = hFx; m[0][1][0] = hFy; m[0][0][1] = hFz;
    m[1][1][0] *= r.om2; m[1][0][1] *= r.om2; m[0][1][1] *= r.om2;
    {
        const float tr = r.cb * (m[2][0][0] + m[0][2][0] + m[0][0][2]);
        m[2][0][0] = fmaf(r.om2, m[2][0][0], -tr);
        m[0][2][0] = fmaf(r.om2, m[0][2][0], -tr);
        m[0][0][2] = fmaf(r.om2, m[0][0][2], -tr);
    }
    m[1][2][0] = fmaf(r.om3, m[1][2][0], r.c3 * Fx);
    m[1][0][2] = fmaf(r.om3, m[1][0][2], r.c3 * Fx);
    m[2][1][0] = fmaf(r.om3, m[2][1][0], r.c3 * Fy);
    m[2][0][1] = fmaf(r.om3, m[2][0][1], r.c3 * Fz);
    m[0][1][2] = fmaf(r.om3, m[0][1][2], r.c3 * Fy);
    m[0][2][1] = fmaf(r.om3, m[0][2][1], r.c3 * Fz);
    m[1][1][1] *= r.om3b;
    m[2][2][0] *= r.om4; m[2][0][2] *= r.om4; m[0][2][2] *= r.om4;
    m[2][1][1] *= r.om4b; m[1][2][1] *= r.om4b; m[1][1][2] *= r.om4b;
    m[1][2][2] = fmaf(r.om5, m[1][2][2], r.c5 * Fx);
    m[2][1][2] = fmaf(r.om5, m[2][1][2], r.c5 * Fy);
    m[2][2][1] = fmaf(r.om5, m[2][2][1], r.c5 * Fz);
    m[2][2][2] *= r.om6;
    // R* = N(-u) D*, then Q = R* + (rho G - M w); first order exactly j + F/2
    unshift_axis<2>(m, uz);
    unshift_axis<1>(m, uy);
    unshift_axis<0>(m, ux);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) m[a][b][c] += e[a][b][c];
    m[0][0][0] = drho;
    m[1][0][0] = jx + hFx; m[0][1][0] = jy + hFy; m[0][0][1] = jz + hFz;
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

// Deviations of the generalized local equilibrium at (rho, u).
__device__ __forceinline__ void equilibrium_dev27(float rho, float ux, float uy, float uz, float (&h)[3][3][3]) {
    eq_dev27(rho - 1.0f, ux, uy, uz, h);
    inverse_axis<2>(h);
    inverse_axis<1>(h);
    inverse_axis<0>(h);
}

// Eq. 9 on deviations: drho and rho*u (with F/2).
__device__ __forceinline__ float macros_dev27(const float (&h)[3][3][3], float Fx, float Fy, float Fz, float &jx,
                                              float &jy, float &jz) {
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
    jx = fmaf(0.5f, Fx, m[1][0][0]);
    jy = fmaf(0.5f, Fy, m[0][1][0]);
    jz = fmaf(0.5f, Fz, m[0][0][1]);
    return m[0][0][0];
}

}  // namespace clbm
