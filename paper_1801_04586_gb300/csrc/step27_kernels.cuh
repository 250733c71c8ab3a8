// step27_kernels.cuh -- the D3Q27 step kernels (A/B pull and in-place AA),
// templated on the collision: a policy C with
//   static float run(float (&h)[3][3][3], float Fx, float Fy, float Fz, const Rates27 &r)
// that collides the deviations h (cube by velocity code) in place and returns
// rho - 1 (Eq. 9): the cascaded collision of Sec. II (step27.cu) or the SRT
// and non-orthogonal MRT comparison models (models27.cuh; step27_srt.cu,
// step27_mrt.cu). Same layout and conventions as the D3Q19 kernels.
#pragma once

#include "d3q27.cuh"
#include "kernels.cuh"
#include "step_tma.cuh"

namespace clbm {

template <int FM>
__device__ __forceinline__ void force27(const ForceArgs &F, const Geom &g, int z, uint32_t self, float &fx, float &fy,
                                        float &fz) {
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

__device__ __forceinline__ bool node27(const Geom &g, int &x, int &y, int &z) {
    x = blockIdx.x * blockDim.x + threadIdx.x;
    y = blockIdx.y * blockDim.y + threadIdx.y;
    z = blockIdx.z;
    return x < g.nx && y < g.ny;
}

template <typename S, bool WALLS>
__device__ __forceinline__ uint32_t pull27(const S *src, const Geom &g, int x, int y, int z, float (&h)[3][3][3]) {
    uint32_t off[3][3][3];
    int pop[3][3][3];
    pull_sources27<WALLS>(g, x, y, z, off, pop);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) h[a][b][c] = Codec<S>::load(src + CLBM_IDX(g, (size_t)pop[a][b][c] * g.stride + off[a][b][c]));
    return ((uint32_t)z * g.ny + y) * g.nx + x;
}

// cube (by velocity code) -> population order of Eq. 1
__device__ __forceinline__ void flatten27(const float (&h)[3][3][3], float (&f)[kQ27]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) f[q27_index(a, b, c)] = h[a][b][c];
}

template <typename C, typename S, int FM, bool WALLS>
__global__ void __launch_bounds__(256, 4) k_step27(const S *__restrict__ src, S *__restrict__ dst, Geom g, Rates27 r,
                                                ForceArgs F, int *__restrict__ flag, uint32_t key) {
    int x, y, z;
    if (!node27(g, x, y, z)) return;
    float h[3][3][3];
    const uint32_t self = pull27<S, WALLS>(src, g, x, y, z, h);
    float fx, fy, fz;
    force27<FM>(F, g, z, self, fx, fy, fz);
    const float drho = C::template run<sizeof(S) == 2>(h, fx, fy, fz, r);
    if (!(fabsf(drho) < 0.9f)) *flag = 1;
    float f[kQ27];
    flatten27(h, f);
    store_node<S, kQ27>(dst + CLBM_SLOTS(g, self, (kQ27 - 1) * g.stride), g.stride, f, self, key);
}

// In-place (AA) pattern, as k_step_aa in step_kernels.cuh: the even kind
// reads the node's natural slots and writes population (a,b,c) to the
// opposite slot at the node; the odd kind reads the swapped pull slots and
// writes population (a,b,c) to the slot the opposite direction was read from.
// A node writes exactly the slots it read; a slot is read once, by the thread
// that later overwrites it, so loads may take the read-only path.
template <typename C, typename S, int FM, bool WALLS, bool ODD>
__global__ void __launch_bounds__(256) k_step27_aa(S *f, Geom g, Rates27 r, ForceArgs F, int *__restrict__ flag,
                                                   uint32_t key) {
    int x, y, z;
    if (!node27(g, x, y, z)) return;
    const uint32_t self = ((uint32_t)z * g.ny + y) * g.nx + x;
    uint32_t off[3][3][3];
    int pop[3][3][3];
    if (ODD) {
        pull_sources27<WALLS, true>(g, x, y, z, off, pop);
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int c = 0; c < 3; ++c) { off[a][b][c] = self; pop[a][b][c] = q27_index(a, b, c); }
    }
    float h[3][3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) h[a][b][c] = Codec<S>::load(f + CLBM_IDX(g, (size_t)pop[a][b][c] * g.stride + off[a][b][c]));
    float fx, fy, fz;
    force27<FM>(F, g, z, self, fx, fy, fz);
    const float drho = C::template run<sizeof(S) == 2>(h, fx, fy, fz, r);
    if (!(fabsf(drho) < 0.9f)) *flag = 1;
    if (ODD) {
        // recompute the slots from coordinates the compiler must treat as new
        // and as depending on the collision's outputs, so that 27 offsets do
        // not stay live through the collision
        int xs = x, ys = y, zs = z;
        asm volatile("" : "+r"(xs), "+r"(ys), "+r"(zs) : "f"(h[0][0][0]), "f"(h[2][2][2]));
        pull_sources27<WALLS, true>(g, xs, ys, zs, off, pop);
    }
    // destination of population q27_index(a,b,c): the slot read for the opposite code
    float v[kQ27];
    uint32_t doff[kQ27];
    int dpop[kQ27];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int p = q27_index(a, b, c);
                const int oa = a ? 3 - a : 0, ob = b ? 3 - b : 0, oc = c ? 3 - c : 0;
                v[p] = h[a][b][c];
                doff[p] = off[oa][ob][oc];
                dpop[p] = pop[oa][ob][oc];
            }
    store_each<S, kQ27>(v, self, key, [&](int p) { return f + CLBM_IDX(g, (size_t)dpop[p] * g.stride + doff[p]); });
}

// ---- dispatch: storage x force mode x walls
#define CLBM_Q27_STORE(storage, ...)                                                  \
    switch (storage) {                                                                \
        case 0: { using S = float; __VA_ARGS__; } break;                              \
        case 1: { using S = __half; __VA_ARGS__; } break;                             \
        case 2: { using S = __nv_bfloat16; __VA_ARGS__; } break;                      \
        case 3: { using S = HalfSR; __VA_ARGS__; } break;                             \
        default: { using S = BF16SR; __VA_ARGS__; } break;                            \
    }
// state kernels round to nearest: stochastic formats share the 16-bit bits
#define CLBM_Q27_STATE(storage, ...)                                                  \
    switch (storage) {                                                                \
        case 0: { using S = float; __VA_ARGS__; } break;                              \
        case 1: case 3: { using S = __half; __VA_ARGS__; } break;                     \
        default: { using S = __nv_bfloat16; __VA_ARGS__; } break;                     \
    }
#define CLBM_Q27_FM(mode, ...)                                                        \
    switch (mode) {                                                                   \
        case kForceUniform: { constexpr int FM = kForceUniform; __VA_ARGS__; } break; \
        case kForceProfileZ: { constexpr int FM = kForceProfileZ; __VA_ARGS__; } break; \
        default: { constexpr int FM = kForceField; __VA_ARGS__; } break;              \
    }

template <typename C>
cudaError_t launch_step27_with(int storage, const Launch &L, const void *src, void *dst, const Rates27 &r,
                               const ForceArgs &F, int *flag, uint32_t key) {
    CLBM_Q27_STORE(storage, CLBM_Q27_FM(F.mode, {
        bool staged = false;
        if constexpr (sizeof(S) == 2) {  // 16-bit storage: rows staged in shared memory where they apply
            cudaError_t e = cudaSuccess;
            staged = L.staged && launch_step_tma<27, C, S, FM>(L, src, dst, r, F, flag, key, e);
            if (staged && e != cudaSuccess) return e;
        }
        if (staged)
            ;
        else if (L.g.walls)
            k_step27<C, S, FM, true><<<L.grid, L.block, 0, L.stream>>>((const S *)src, (S *)dst, L.g, r, F, flag, key);
        else
            k_step27<C, S, FM, false><<<L.grid, L.block, 0, L.stream>>>((const S *)src, (S *)dst, L.g, r, F, flag, key);
    }))
    return cudaGetLastError();
}

template <typename C>
cudaError_t launch_step27_aa_with(int storage, const Launch &L, void *f, const Rates27 &r, const ForceArgs &F,
                                  int *flag, uint32_t key, bool odd) {
    CLBM_Q27_STORE(storage, CLBM_Q27_FM(F.mode, {
        if (!odd)
            k_step27_aa<C, S, FM, false, false><<<L.grid, L.block, 0, L.stream>>>((S *)f, L.g, r, F, flag, key);
        else if (L.g.walls)
            k_step27_aa<C, S, FM, true, true><<<L.grid, L.block, 0, L.stream>>>((S *)f, L.g, r, F, flag, key);
        else
            k_step27_aa<C, S, FM, false, true><<<L.grid, L.block, 0, L.stream>>>((S *)f, L.g, r, F, flag, key);
    }))
    return cudaGetLastError();
}

}  // namespace clbm
