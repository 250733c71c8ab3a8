// aux.cu -- kernels around the step: initial equilibrium, state import/export
// in post-streaming form, Eq. 9 read-out and deterministic FP64 reductions.
#include "block_reduce.cuh"
#include "kernels.cuh"

namespace clbm {

template <int FM>
__device__ __forceinline__ void force_node(const ForceArgs &F, const Geom &g, int z, uint32_t self, float &fx,
                                           float &fy, float &fz) {
    if (FM == kForceUniform) {
        fx = F.fx; fy = F.fy; fz = F.fz;
    } else if (FM == kForceProfileZ) {
        fx = F.profile[z]; fy = F.profile[g.nz + z]; fz = F.profile[2 * g.nz + z];
    } else {
        fx = F.field[self]; fy = F.field[F.n + self]; fz = F.field[2 * F.n + self];
    }
    fx *= F.scale;
    fy *= F.scale;
    fz *= F.scale;
}

__device__ __forceinline__ bool node_of(const Geom &g, int &x, int &y, int &z, int z0 = 0) {
    x = blockIdx.x * blockDim.x + threadIdx.x;
    y = blockIdx.y * blockDim.y + threadIdx.y;
    z = z0 + (int)blockIdx.z;
    return x < g.nx && y < g.ny;
}

// Slots of the post-streaming populations of node (x,y,z) in a state buffer.
// map 0: A/B pattern, the pull map; 1: in-place (AA) pattern after an even
// number of steps, natural order at the node; 2: AA after an odd number of
// steps, the swapped pull map of the odd step (step.cu); 3: the pull map of a
// z-slab, through its halo planes across halo faces.
template <bool WALLS>
__device__ __forceinline__ void state_slots(const Geom &g, int x, int y, int z, int map, uint32_t (&off)[kQ],
                                            int (&pop)[kQ]) {
    if (map == 3) {
        pull_sources<WALLS, false, true>(g, x, y, z, off, pop);
    } else if (map == 1) {
        const uint32_t self = ((uint32_t)z * g.ny + y) * g.nx + x;
#pragma unroll
        for (int i = 0; i < kQ; ++i) { off[i] = self; pop[i] = i; }
    } else if (map == 2) {
        pull_sources<WALLS, true>(g, x, y, z, off, pop);
    } else {
        pull_sources<WALLS>(g, x, y, z, off, pop);
    }
}

// Write a post-streaming state h (deviations) of node (x,y,z) where the next
// step will find it.
template <typename S, bool WALLS>
__device__ __forceinline__ void scatter_node(S *dst, const Geom &g, int x, int y, int z, int map,
                                             const float (&h)[kQ]) {
    uint32_t off[kQ];
    int pop[kQ];
    state_slots<WALLS>(g, x, y, z, map, off, pop);
#pragma unroll
    for (int i = 0; i < kQ; ++i) dst[CLBM_IDX(g, (size_t)pop[i] * g.stride + off[i])] = Codec<S>::from_f(h[i]);
}

template <typename S, bool WALLS>
__device__ __forceinline__ uint32_t pull_node(const S *src, const Geom &g, int x, int y, int z, int map,
                                              float (&h)[kQ]) {
    uint32_t off[kQ];
    int pop[kQ];
    state_slots<WALLS>(g, x, y, z, map, off, pop);
#pragma unroll
    for (int i = 0; i < kQ; ++i) h[i] = Codec<S>::load_plain(src + CLBM_IDX(g, (size_t)pop[i] * g.stride + off[i]));
    return ((uint32_t)z * g.ny + y) * g.nx + x;
}

template <typename S, bool WALLS>
__global__ void k_scatter(S *dst, Geom g, int map, const float *__restrict__ f, int64_t n, int deviation) {
    int x, y, z;
    if (!node_of(g, x, y, z)) return;
    const uint32_t self = ((uint32_t)z * g.ny + y) * g.nx + x;
    float h[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const float v = f[(size_t)i * n + self];
        h[i] = deviation ? v : v - rest_weight(i);
    }
    scatter_node<S, WALLS>(dst, g, x, y, z, map, h);
}

template <typename S, int FM, bool WALLS>
__global__ void k_init_eq(S *dst, Geom g, int map, const float *__restrict__ rho, const float *__restrict__ u,
                          int64_t n, ForceArgs F, int z0) {
    int x, y, z;
    if (!node_of(g, x, y, z, z0)) return;
    const uint32_t self = ((uint32_t)z * g.ny + y) * g.nx + x;
    const float r = rho ? rho[self] : 1.0f;
    float fx, fy, fz;
    force_node<FM>(F, g, z, self, fx, fy, fz);
    const float half_inv = 0.5f / r;
    const float ux = (u ? u[self] : 0.0f) - fx * half_inv;
    const float uy = (u ? u[n + self] : 0.0f) - fy * half_inv;
    const float uz = (u ? u[2 * n + self] : 0.0f) - fz * half_inv;
    float h[kQ];
    equilibrium_dev(r, ux, uy, uz, h);
    scatter_node<S, WALLS>(dst, g, x, y, z, map, h);
}

template <typename S, bool WALLS>
__global__ void k_gather(const S *src, Geom g, int map, float *__restrict__ f, int64_t n, int deviation) {
    int x, y, z;
    if (!node_of(g, x, y, z)) return;
    float h[kQ];
    const uint32_t self = pull_node<S, WALLS>(src, g, x, y, z, map, h);
#pragma unroll
    for (int i = 0; i < kQ; ++i) f[(size_t)i * n + self] = deviation ? h[i] : h[i] + rest_weight(i);
}

template <typename S, int FM, bool WALLS>
__global__ void k_macros(const S *src, Geom g, int map, ForceArgs F, float *__restrict__ rho,
                         float *__restrict__ u, int64_t n, int z0) {
    int x, y, z;
    if (!node_of(g, x, y, z, z0)) return;
    float h[kQ];
    const uint32_t self = pull_node<S, WALLS>(src, g, x, y, z, map, h);
    float fx, fy, fz, jx, jy, jz;
    force_node<FM>(F, g, z, self, fx, fy, fz);
    const float drho = macros_dev(h, fx, fy, fz, jx, jy, jz);
    const float r = 1.0f + drho;
    if (rho) rho[self] = r;
    if (u) {
        u[self] = jx / r;
        u[n + self] = jy / r;
        u[2 * n + self] = jz / r;
    }
}

// ---- deterministic FP64 reductions: fixed grid, grid-stride loop, block
// sums (block_reduce.cuh) into per-block partials, one final block.
template <int K>
__global__ void k_reduce_final(const double *partials, int nblocks, double *out, double add0) {
    double v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] += partials[(size_t)b * K + k];
    __shared__ double tmp[K];
    block_sum_store<K>(v, tmp);
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) out[k] = tmp[k] + (k == 0 ? add0 : 0.0);
}

// Fixed-point totals of nblocks partials (one block), as FP64 (+ add0 on the first).
__global__ void k_fixed_final4(const long long *partials, int nblocks, double *out, double add0) {
    long long q[4] = {0ll, 0ll, 0ll, 0ll};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < 4; ++k) q[k] += partials[(size_t)b * 4 + k];
    __shared__ long long tmp[4];
    block_sum_fixed<4>(q, tmp);
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) out[k] = (double)tmp[k] * kFixUnit + (k == 0 ? add0 : 0.0);
}

template <typename S, int FM, bool WALLS>
__global__ void k_reduce_moments(const S *src, Geom g, int map, ForceArgs F, long long *partials) {
    long long q[4] = {0ll, 0ll, 0ll, 0ll};
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(s % g.nx);
        const int64_t t = s / g.nx;
        const int y = (int)(t % g.ny), z = (int)(t / g.ny);
        float h[kQ];
        const uint32_t self = pull_node<S, WALLS>(src, g, x, y, z, map, h);
        float fx, fy, fz, jx, jy, jz;
        force_node<FM>(F, g, z, self, fx, fy, fz);
        const float drho = macros_dev(h, fx, fy, fz, jx, jy, jz);
        q[0] += to_fixed(drho); q[1] += to_fixed(jx); q[2] += to_fixed(jy); q[3] += to_fixed(jz);
    }
    block_sum_fixed<4>(q, partials + (size_t)blockIdx.x * 4);
}

__global__ void k_reduce_pair(const float *__restrict__ a, const float *__restrict__ b, int64_t n,
                              double *partials) {
    double v[3] = {0.0, 0.0, 0.0};
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const double av = a[s], bv = b ? (double)b[s] : 0.0;
        const double d = av - bv;
        v[0] += d * d; v[1] += bv * bv; v[2] += av * bv;
    }
    block_sum_store<3>(v, partials + (size_t)blockIdx.x * 3);
}

// ---- dispatch helpers
// Stochastic formats share the bits of FP16 / BF16; state import and
// initialisation round them to nearest.
#define CLBM_DISPATCH_STORAGE(storage, ...)                                 \
    switch (storage) {                                                      \
        case 0: { using S = float; __VA_ARGS__; } break;                    \
        case 1: case 3: { using S = __half; __VA_ARGS__; } break;           \
        default: { using S = __nv_bfloat16; __VA_ARGS__; } break;           \
    }

template <typename S, bool W>
static void scatter_t(const Launch &L, void *dst, const float *f, int64_t n, int dev) {
    k_scatter<S, W><<<L.grid, L.block, 0, L.stream>>>((S *)dst, L.g, L.map, f, n, dev);
}

cudaError_t launch_scatter(int storage, const Launch &L, void *dst, const float *f, int64_t n, int deviation) {
    CLBM_DISPATCH_STORAGE(storage, {
        if (L.g.walls) scatter_t<S, true>(L, dst, f, n, deviation);
        else scatter_t<S, false>(L, dst, f, n, deviation);
    })
    return cudaGetLastError();
}

// The planes L.z0 .. L.z0 + L.nplanes - 1 of the init and read-out kernels
// (all planes when nplanes < 0): the launch's grid and first plane.
static dim3 plane_grid(const Launch &L, int &z0) {
    dim3 grid = L.grid;
    z0 = 0;
    if (L.nplanes >= 0) {
        grid.z = (unsigned)L.nplanes;
        z0 = L.z0;
    }
    return grid;
}

template <typename S, int FM>
static void init_t(const Launch &L, void *dst, const float *rho, const float *u, int64_t n, const ForceArgs &F) {
    int z0;
    const dim3 grid = plane_grid(L, z0);
    if (grid.z == 0) return;
    if (L.g.walls) k_init_eq<S, FM, true><<<grid, L.block, 0, L.stream>>>((S *)dst, L.g, L.map, rho, u, n, F, z0);
    else k_init_eq<S, FM, false><<<grid, L.block, 0, L.stream>>>((S *)dst, L.g, L.map, rho, u, n, F, z0);
}

cudaError_t launch_init_eq(int storage, const Launch &L, void *dst, const float *rho, const float *u, int64_t n,
                           const ForceArgs &F) {
    CLBM_DISPATCH_STORAGE(storage, {
        switch (F.mode) {
            case kForceUniform: init_t<S, kForceUniform>(L, dst, rho, u, n, F); break;
            case kForceProfileZ: init_t<S, kForceProfileZ>(L, dst, rho, u, n, F); break;
            default: init_t<S, kForceField>(L, dst, rho, u, n, F); break;
        }
    })
    return cudaGetLastError();
}

cudaError_t launch_gather(int storage, const Launch &L, const void *src, float *f, int64_t n, int deviation) {
    CLBM_DISPATCH_STORAGE(storage, {
        if (L.g.walls) k_gather<S, true><<<L.grid, L.block, 0, L.stream>>>((const S *)src, L.g, L.map, f, n, deviation);
        else k_gather<S, false><<<L.grid, L.block, 0, L.stream>>>((const S *)src, L.g, L.map, f, n, deviation);
    })
    return cudaGetLastError();
}

template <typename S, int FM>
static void macros_t(const Launch &L, const void *src, const ForceArgs &F, float *rho, float *u, int64_t n) {
    int z0;
    const dim3 grid = plane_grid(L, z0);
    if (grid.z == 0) return;
    if (L.g.walls)
        k_macros<S, FM, true><<<grid, L.block, 0, L.stream>>>((const S *)src, L.g, L.map, F, rho, u, n, z0);
    else
        k_macros<S, FM, false><<<grid, L.block, 0, L.stream>>>((const S *)src, L.g, L.map, F, rho, u, n, z0);
}

cudaError_t launch_macros(int storage, const Launch &L, const void *src, const ForceArgs &F, float *rho, float *u,
                          int64_t n) {
    CLBM_DISPATCH_STORAGE(storage, {
        switch (F.mode) {
            case kForceUniform: macros_t<S, kForceUniform>(L, src, F, rho, u, n); break;
            case kForceProfileZ: macros_t<S, kForceProfileZ>(L, src, F, rho, u, n); break;
            default: macros_t<S, kForceField>(L, src, F, rho, u, n); break;
        }
    })
    return cudaGetLastError();
}

template <typename S, int FM>
static void moments_t(const Launch &L, const void *src, const ForceArgs &F, long long *partials, int nb) {
    if (L.g.walls) k_reduce_moments<S, FM, true><<<nb, 256, 0, L.stream>>>((const S *)src, L.g, L.map, F, partials);
    else k_reduce_moments<S, FM, false><<<nb, 256, 0, L.stream>>>((const S *)src, L.g, L.map, F, partials);
}

cudaError_t launch_reduce_moments(int storage, const Launch &L, const void *src, const ForceArgs &F,
                                  long long *partials, int nblocks, double *out) {
    CLBM_DISPATCH_STORAGE(storage, {
        switch (F.mode) {
            case kForceUniform: moments_t<S, kForceUniform>(L, src, F, partials, nblocks); break;
            case kForceProfileZ: moments_t<S, kForceProfileZ>(L, src, F, partials, nblocks); break;
            default: moments_t<S, kForceField>(L, src, F, partials, nblocks); break;
        }
    })
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const double n = (double)L.g.nx * L.g.ny * L.g.nz;
    k_fixed_final4<<<1, 256, 0, L.stream>>>(partials, nblocks, out, n);
    return cudaGetLastError();
}

cudaError_t launch_fixed_final4(const long long *partials, int nblocks, double *out, double add0,
                                cudaStream_t stream) {
    k_fixed_final4<<<1, 256, 0, stream>>>(partials, nblocks, out, add0);
    return cudaGetLastError();
}

cudaError_t launch_reduce_pair(const float *a, const float *b, int64_t n, double *partials, int nblocks,
                               double *out, cudaStream_t stream) {
    k_reduce_pair<<<nblocks, 256, 0, stream>>>(a, b, n, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_final<3><<<1, 256, 0, stream>>>(partials, nblocks, out, 0.0);
    return cudaGetLastError();
}

}  // namespace clbm
