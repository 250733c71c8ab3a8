// step27.cu -- D3Q27 kernels: the fused pull stream-and-collide step
// (collision in d3q27.cuh) and the state kernels around it (initial
// equilibrium, import / export of post-streaming populations, Eq. 9 read-out,
// fixed-point conservation sums). Same layout and conventions as the D3Q19
// kernels: structure of arrays, 27 arrays of `stride` elements, deviations
// from the rest weights in the storage format S.
#include "block_reduce.cuh"
#include "d3q27.cuh"
#include "kernels.cuh"

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
            for (int c = 0; c < 3; ++c) h[a][b][c] = Codec<S>::load(src + (size_t)pop[a][b][c] * g.stride + off[a][b][c]);
    return ((uint32_t)z * g.ny + y) * g.nx + x;
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
                h[a][b][c] = Codec<S>::load_plain(src + (size_t)pop[a][b][c] * g.stride + off[a][b][c]);
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

template <typename S, int FM, bool WALLS>
__global__ void __launch_bounds__(256, 4) k_step27(const S *__restrict__ src, S *__restrict__ dst, Geom g, Rates27 r,
                                                ForceArgs F, int *__restrict__ flag, uint32_t key) {
    int x, y, z;
    if (!node27(g, x, y, z)) return;
    float h[3][3][3];
    const uint32_t self = pull27<S, WALLS>(src, g, x, y, z, h);
    float fx, fy, fz;
    force27<FM>(F, g, z, self, fx, fy, fz);
    const float drho = collide27(h, fx, fy, fz, r);
    if (!(fabsf(drho) < 0.9f)) *flag = 1;
    float f[kQ27];
    flatten27(h, f);
    store_node<S, kQ27>(dst + self, g.stride, f, self, key);
}

// In-place (AA) pattern, as k_step_aa in step_kernels.cuh: the even kind
// reads the node's natural slots and writes population (a,b,c) to the
// opposite slot at the node; the odd kind reads the swapped pull slots and
// writes population (a,b,c) to the slot the opposite direction was read from.
// A node writes exactly the slots it read; a slot is read once, by the thread
// that later overwrites it, so loads may take the read-only path. The odd
// kind stages the 18 populations with e_x != 0 in shared memory so that the
// thread whose own x is the destination stores them (aligned warp stores);
// values whose destination leaves the block row, wraps around a periodic x
// face or bounces back are stored directly.
template <typename S, int FM, bool WALLS, bool ODD>
__global__ void __launch_bounds__(256, 3) k_step27_aa(S *f, Geom g, Rates27 r, ForceArgs F, int *__restrict__ flag,
                                                   uint32_t key) {
    int x, y, z;
    const bool active = node27(g, x, y, z);
    if (!ODD && !active) return;
    const uint32_t self = ((uint32_t)z * g.ny + y) * g.nx + x;
    const int tx = threadIdx.x, bx = blockDim.x;
    const int tid = tx + bx * threadIdx.y;
    __shared__ S stage[ODD ? 18 : 1][ODD ? 256 : 1];
    if (active) {
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
                for (int c = 0; c < 3; ++c)
                    h[a][b][c] = Codec<S>::load(f + (size_t)pop[a][b][c] * g.stride + off[a][b][c]);
        float fx, fy, fz;
        force27<FM>(F, g, z, self, fx, fy, fz);
        const float drho = collide27(h, fx, fy, fz, r);
        if (!(fabsf(drho) < 0.9f)) *flag = 1;
        if (ODD) {
            // recompute the slots from coordinates the compiler must treat as new,
            // so that 27 offsets do not stay live through the collision
            int xs = x, ys = y, zs = z;
            asm volatile("" : "+r"(xs), "+r"(ys), "+r"(zs));
            pull_sources27<WALLS, true>(g, xs, ys, zs, off, pop);
        }
        // destination of population q27_index(a,b,c): the slot read for the opposite code
        float v[kQ27];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int c = 0; c < 3; ++c) v[q27_index(a, b, c)] = h[a][b][c];
        S e[kQ27];
        encode_each<S, kQ27>(v, self, key, e);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int p = q27_index(a, b, c);
                    const int oa = a ? 3 - a : 0, ob = b ? 3 - b : 0, oc = c ? 3 - c : 0;
                    S *dst = f + (size_t)pop[oa][ob][oc] * g.stride + off[oa][ob][oc];
                    if (!ODD || a == 0) {
                        *dst = e[p];
                    } else {
                        const int ex = e_of(a);
                        stage[ODD ? (a - 1) * 9 + b * 3 + c : 0][ODD ? tid : 0] = e[p];
                        const bool handed = pop[oa][ob][oc] == p && x + ex >= 0 && x + ex < g.nx &&
                                            tx + ex >= 0 && tx + ex < bx;
                        if (!handed) *dst = e[p];
                    }
                }
    }
    if (ODD) {
        __syncthreads();
        if (active) {
            const bool wy = WALLS && (g.walls & 2u), wz = WALLS && (g.walls & 4u);
            const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
            const int zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;
#pragma unroll
            for (int a = 1; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const int ex = e_of(a), ey = e_of(b), ez = e_of(c);
                        // the source x - e_x of this row sends population (a,b,c) to x
                        const bool row_bb = (wy && ((ey == 1 && y == g.ny - 1) || (ey == -1 && y == 0))) ||
                                            (wz && ((ez == 1 && z == g.nz - 1) || (ez == -1 && z == 0)));
                        if (x - ex >= 0 && x - ex < g.nx && tx - ex >= 0 && tx - ex < bx && !row_bb) {
                            const int yd = ey == 0 ? y : (ey > 0 ? yp : ym), zd = ez == 0 ? z : (ez > 0 ? zp : zm);
                            const uint32_t dst = ((uint32_t)zd * g.ny + yd) * g.nx + x;
                            f[(size_t)q27_index(a, b, c) * g.stride + dst] =
                                stage[ODD ? (a - 1) * 9 + b * 3 + c : 0][ODD ? tid - ex : 0];
                        }
                    }
        }
    }
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
            for (int c = 0; c < 3; ++c) dst[(size_t)pop[a][b][c] * g.stride + off[a][b][c]] = Codec<S>::from_f(h[a][b][c]);
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

cudaError_t launch_step27(int storage, const Launch &L, const void *src, void *dst, const Rates27 &r,
                          const ForceArgs &F, int *flag, uint32_t key) {
    CLBM_Q27_STORE(storage, CLBM_Q27_FM(F.mode, {
        if (L.g.walls)
            k_step27<S, FM, true><<<L.grid, L.block, 0, L.stream>>>((const S *)src, (S *)dst, L.g, r, F, flag, key);
        else
            k_step27<S, FM, false><<<L.grid, L.block, 0, L.stream>>>((const S *)src, (S *)dst, L.g, r, F, flag, key);
    }))
    return cudaGetLastError();
}

cudaError_t launch_step27_aa(int storage, const Launch &L, void *f, const Rates27 &r, const ForceArgs &F, int *flag,
                             uint32_t key, bool odd) {
    CLBM_Q27_STORE(storage, CLBM_Q27_FM(F.mode, {
        if (!odd)
            k_step27_aa<S, FM, false, false><<<L.grid, L.block, 0, L.stream>>>((S *)f, L.g, r, F, flag, key);
        else if (L.g.walls)
            k_step27_aa<S, FM, true, true><<<L.grid, L.block, 0, L.stream>>>((S *)f, L.g, r, F, flag, key);
        else
            k_step27_aa<S, FM, false, true><<<L.grid, L.block, 0, L.stream>>>((S *)f, L.g, r, F, flag, key);
    }))
    return cudaGetLastError();
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
