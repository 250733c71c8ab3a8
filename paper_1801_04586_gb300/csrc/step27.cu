// step27.cu -- D3Q27 kernels: the cascaded collision's step kernels (collision
// in d3q27.cuh, kernels in step27_kernels.cuh) and the state kernels around
// them (initial equilibrium, import / export of post-streaming populations,
// Eq. 9 read-out, fixed-point conservation sums). Same layout and conventions
// as the D3Q19 kernels: structure of arrays, 27 arrays of `stride` elements,
// deviations from the rest weights in the storage format S.
#include "block_reduce.cuh"
#include "step27_kernels.cuh"

namespace clbm {

// The paper's cascaded collision on D3Q27 (Sec. II).
struct Cascaded27 {
    template <bool FR = false>
    static __device__ __forceinline__ float run(float (&h)[3][3][3], float Fx, float Fy, float Fz,
                                                const Rates27 &r) {
        return collide27<FR>(h, Fx, Fy, Fz, r);
    }
};

cudaError_t launch_step27(int storage, const Launch &L, const void *src, void *dst, const Rates27 &r,
                          const ForceArgs &F, int *flag, uint32_t key) {
    return launch_step27_with<Cascaded27>(storage, L, src, dst, r, F, flag, key);
}

cudaError_t launch_step27_aa(int storage, const Launch &L, void *f, const Rates27 &r, const ForceArgs &F, int *flag,
                             uint32_t key, bool odd) {
    return launch_step27_aa_with<Cascaded27>(storage, L, f, r, F, flag, key, odd);
}

// Slots of the post-streaming populations of (x, y, z) in a state buffer, by
// cube code. map 0: A/B pull map; 1: in-place pattern after an even number of
// steps (natural order at the node); 2: after an odd number (swapped pull map).
template <bool WALLS>
__device__ __forceinline__ void state_slots27(const Geom &g, int x, int y, int z, int map, uint32_t (&off)[3][3][3],
                                              int (&pop)[3][3][3]) {
    if (map == 1) {
        const uint32_t self = ((uint32_t)z * g.ny + y) * g.nx + x;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int c = 0; c < 3; ++c) { off[a][b][c] = self; pop[a][b][c] = q27_index(a, b, c); }
    } else if (map == 2) {
        pull_sources27<WALLS, true>(g, x, y, z, off, pop);
    } else {
        pull_sources27<WALLS>(g, x, y, z, off, pop);
    }
}

template <typename S, bool WALLS>
__device__ __forceinline__ uint32_t state_load27(const S *src, const Geom &g, int x, int y, int z, int map,
                                                 float (&h)[3][3][3]) {
    uint32_t off[3][3][3];
    int pop[3][3][3];
    state_slots27<WALLS>(g, x, y, z, map, off, pop);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                h[a][b][c] = Codec<S>::load_plain(src + CLBM_IDX(g, (size_t)pop[a][b][c] * g.stride + off[a][b][c]));
    return ((uint32_t)z * g.ny + y) * g.nx + x;
}

// Write a post-streaming state (cube by velocity code) where the next step finds it.
template <typename S, bool WALLS>
__device__ __forceinline__ void scatter27(S *dst, const Geom &g, int x, int y, int z, int map,
                                          const float (&h)[3][3][3]) {
    uint32_t off[3][3][3];
    int pop[3][3][3];
    state_slots27<WALLS>(g, x, y, z, map, off, pop);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) dst[CLBM_IDX(g, (size_t)pop[a][b][c] * g.stride + off[a][b][c])] = Codec<S>::from_f(h[a][b][c]);
}

template <typename S, int FM, bool WALLS>
__global__ void k_init27(S *dst, Geom g, int map, const float *__restrict__ rho, const float *__restrict__ u,
                         int64_t n, ForceArgs F) {
    int x, y, z;
    if (!node27(g, x, y, z)) return;
    const uint32_t self = ((uint32_t)z * g.ny + y) * g.nx + x;
    const float r = rho ? rho[self] : 1.0f;
    float fx, fy, fz;
    force27<FM>(F, g, z, self, fx, fy, fz);
    const float hi = 0.5f / r;
    float h[3][3][3];
    equilibrium_dev27(r, (u ? u[self] : 0.0f) - fx * hi, (u ? u[n + self] : 0.0f) - fy * hi,
                      (u ? u[2 * n + self] : 0.0f) - fz * hi, h);
    scatter27<S, WALLS>(dst, g, x, y, z, map, h);
}

template <typename S, bool WALLS>
__global__ void k_scatter27(S *dst, Geom g, int map, const float *__restrict__ f, int64_t n, int deviation) {
    int x, y, z;
    if (!node27(g, x, y, z)) return;
    const uint32_t self = ((uint32_t)z * g.ny + y) * g.nx + x;
    float h[3][3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float v = f[(size_t)q27_index(a, b, c) * n + self];
                h[a][b][c] = deviation ? v : v - rest_weight27_code(a, b, c);
            }
    scatter27<S, WALLS>(dst, g, x, y, z, map, h);
}

template <typename S, bool WALLS>
__global__ void k_gather27(const S *src, Geom g, int map, float *__restrict__ f, int64_t n, int deviation) {
    int x, y, z;
    if (!node27(g, x, y, z)) return;
    float h[3][3][3];
    const uint32_t self = state_load27<S, WALLS>(src, g, x, y, z, map, h);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                f[(size_t)q27_index(a, b, c) * n + self] =
                    deviation ? h[a][b][c] : h[a][b][c] + rest_weight27_code(a, b, c);
}

template <typename S, int FM, bool WALLS>
__global__ void k_macros27(const S *src, Geom g, int map, ForceArgs F, float *__restrict__ rho,
                           float *__restrict__ u, int64_t n) {
    int x, y, z;
    if (!node27(g, x, y, z)) return;
    float h[3][3][3];
    const uint32_t self = state_load27<S, WALLS>(src, g, x, y, z, map, h);
    float fx, fy, fz, jx, jy, jz;
    force27<FM>(F, g, z, self, fx, fy, fz);
    const float r = 1.0f + macros_dev27(h, fx, fy, fz, jx, jy, jz);
    if (rho) rho[self] = r;
    if (u) {
        u[self] = jx / r;
        u[n + self] = jy / r;
        u[2 * n + self] = jz / r;
    }
}

template <typename S, int FM, bool WALLS>
__global__ void k_moments27(const S *src, Geom g, int map, ForceArgs F, long long *partials) {
    long long q[4] = {0ll, 0ll, 0ll, 0ll};
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(s % g.nx);
        const int64_t t = s / g.nx;
        const int y = (int)(t % g.ny), z = (int)(t / g.ny);
        float h[3][3][3];
        state_load27<S, WALLS>(src, g, x, y, z, map, h);
        float fx, fy, fz, jx, jy, jz;
        force27<FM>(F, g, z, (uint32_t)s, fx, fy, fz);
        const float drho = macros_dev27(h, fx, fy, fz, jx, jy, jz);
        q[0] += to_fixed(drho); q[1] += to_fixed(jx); q[2] += to_fixed(jy); q[3] += to_fixed(jz);
    }
    block_sum_fixed<4>(q, partials + (size_t)blockIdx.x * 4);
}

cudaError_t launch_init27(int storage, const Launch &L, void *dst, const float *rho, const float *u, int64_t n,
                          const ForceArgs &F) {
    CLBM_Q27_STATE(storage, CLBM_Q27_FM(F.mode, {
        if (L.g.walls) k_init27<S, FM, true><<<L.grid, L.block, 0, L.stream>>>((S *)dst, L.g, L.map, rho, u, n, F);
        else k_init27<S, FM, false><<<L.grid, L.block, 0, L.stream>>>((S *)dst, L.g, L.map, rho, u, n, F);
    }))
    return cudaGetLastError();
}

cudaError_t launch_scatter27(int storage, const Launch &L, void *dst, const float *f, int64_t n, int deviation) {
    CLBM_Q27_STATE(storage, {
        if (L.g.walls) k_scatter27<S, true><<<L.grid, L.block, 0, L.stream>>>((S *)dst, L.g, L.map, f, n, deviation);
        else k_scatter27<S, false><<<L.grid, L.block, 0, L.stream>>>((S *)dst, L.g, L.map, f, n, deviation);
    })
    return cudaGetLastError();
}

cudaError_t launch_gather27(int storage, const Launch &L, const void *src, float *f, int64_t n, int deviation) {
    CLBM_Q27_STATE(storage, {
        if (L.g.walls) k_gather27<S, true><<<L.grid, L.block, 0, L.stream>>>((const S *)src, L.g, L.map, f, n, deviation);
        else k_gather27<S, false><<<L.grid, L.block, 0, L.stream>>>((const S *)src, L.g, L.map, f, n, deviation);
    })
    return cudaGetLastError();
}

cudaError_t launch_macros27(int storage, const Launch &L, const void *src, const ForceArgs &F, float *rho, float *u,
                            int64_t n) {
    CLBM_Q27_STATE(storage, CLBM_Q27_FM(F.mode, {
        if (L.g.walls) k_macros27<S, FM, true><<<L.grid, L.block, 0, L.stream>>>((const S *)src, L.g, L.map, F, rho, u, n);
        else k_macros27<S, FM, false><<<L.grid, L.block, 0, L.stream>>>((const S *)src, L.g, L.map, F, rho, u, n);
    }))
    return cudaGetLastError();
}

cudaError_t launch_moments27(int storage, const Launch &L, const void *src, const ForceArgs &F, long long *partials,
                             int nblocks, double *out) {
    CLBM_Q27_STATE(storage, CLBM_Q27_FM(F.mode, {
        if (L.g.walls) k_moments27<S, FM, true><<<nblocks, 256, 0, L.stream>>>((const S *)src, L.g, L.map, F, partials);
        else k_moments27<S, FM, false><<<nblocks, 256, 0, L.stream>>>((const S *)src, L.g, L.map, F, partials);
    }))
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_fixed_final4(partials, nblocks, out, (double)L.g.nx * L.g.ny * L.g.nz, L.stream);
}

}  // namespace clbm
