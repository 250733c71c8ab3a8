// step_diag.cu -- the fused step kernel with in-kernel conservation sums, for
// jobs that read mass and momentum back after every step.
//
// Same per-node work as k_step (pull, collide, store). In addition every
// block sums the Eq. 9 density deviation and momentum of the state it pulls
// (the state before the step): FP32 warp sums by shuffles, then the warps'
// results and all later levels in FP64. FP64 issues at a small fraction of
// the FP32 rate on this GPU, so it is kept off the per-node path. Block
// partials are added by a two-level deterministic FP64 reduction.
#include "block_reduce.cuh"
#include "kernels.cuh"

namespace clbm {

template <int FM>
__device__ __forceinline__ void force_diag(const ForceArgs &F, const Geom &g, int z, uint32_t self, float &fx,
                                           float &fy, float &fz) {
    if (FM == kForceUniform) {
        fx = F.fx; fy = F.fy; fz = F.fz;
    } else if (FM == kForceProfileZ) {
        fx = __ldg(F.profile + z); fy = __ldg(F.profile + g.nz + z); fz = __ldg(F.profile + 2 * g.nz + z);
    } else {
        fx = __ldg(F.field + self); fy = __ldg(F.field + F.n + self); fz = __ldg(F.field + 2 * F.n + self);
    }
}

template <typename S, int FM, bool WALLS>
__global__ void __launch_bounds__(512) k_step_diag(const S *__restrict__ src, S *__restrict__ dst, Geom g, Rates r,
                                                   ForceArgs F, int *__restrict__ flag,
                                                   double *__restrict__ partials) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (x < g.nx && y < g.ny) {
        uint32_t off[kQ];
        int pop[kQ];
        pull_sources<WALLS>(g, x, y, z, off, pop);
        float h[kQ];
#pragma unroll
        for (int i = 0; i < kQ; ++i) h[i] = Codec<S>::load(src + (size_t)pop[i] * g.stride + off[i]);
        float fx, fy, fz;
        force_diag<FM>(F, g, z, off[0], fx, fy, fz);
        float3 j;
        const float drho = collide(h, fx, fy, fz, r, &j);
        if (!(fabsf(drho) < 0.9f)) *flag = 1;
        S *d = dst + off[0];
#pragma unroll
        for (int i = 0; i < kQ; ++i) d[(size_t)i * g.stride] = Codec<S>::from_f(h[i]);
        v[0] = drho; v[1] = j.x; v[2] = j.y; v[3] = j.z;
    }
    const size_t b = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    block_sum_f32_store<4>(v, partials + 4 * b);
}

template <typename S, int FM>
static cudaError_t diag_walls(const Launch &L, const void *src, void *dst, const Rates &r, const ForceArgs &F,
                              int *flag, double *partials) {
    if (L.g.walls)
        k_step_diag<S, FM, true><<<L.grid, L.block, 0, L.stream>>>((const S *)src, (S *)dst, L.g, r, F, flag,
                                                                   partials);
    else
        k_step_diag<S, FM, false><<<L.grid, L.block, 0, L.stream>>>((const S *)src, (S *)dst, L.g, r, F, flag,
                                                                    partials);
    return cudaGetLastError();
}

template <typename S>
static cudaError_t diag_force(const Launch &L, const void *src, void *dst, const Rates &r, const ForceArgs &F,
                              int *flag, double *partials) {
    switch (F.mode) {
        case kForceUniform: return diag_walls<S, kForceUniform>(L, src, dst, r, F, flag, partials);
        case kForceProfileZ: return diag_walls<S, kForceProfileZ>(L, src, dst, r, F, flag, partials);
        default: return diag_walls<S, kForceField>(L, src, dst, r, F, flag, partials);
    }
}

cudaError_t launch_step_diag(int storage, const Launch &L, const void *src, void *dst, const Rates &r,
                             const ForceArgs &F, int *flag, double *partials) {
    switch (storage) {
        case 0: return diag_force<float>(L, src, dst, r, F, flag, partials);
        case 1: return diag_force<__half>(L, src, dst, r, F, flag, partials);
        default: return diag_force<__nv_bfloat16>(L, src, dst, r, F, flag, partials);
    }
}

// Sum nblocks partials of 4 doubles: blocks of the first pass each add a
// fixed contiguous chunk (FP64), the second pass adds the chunk sums.
__global__ void k_sum_partials4(const double *__restrict__ partials, int64_t nblocks, int64_t chunk,
                                double *__restrict__ mid) {
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    const int64_t lo = (int64_t)blockIdx.x * chunk, hi = min(nblocks, lo + chunk);
    for (int64_t b = lo + threadIdx.x; b < hi; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] += partials[4 * b + k];
    block_sum_store<4>(v, mid + 4 * (size_t)blockIdx.x);
}

cudaError_t launch_sum_partials4(const double *partials, int64_t nblocks, double *mid, int mid_blocks, double *out,
                                 double add0, cudaStream_t stream) {
    const int64_t chunk = (nblocks + mid_blocks - 1) / mid_blocks;
    k_sum_partials4<<<mid_blocks, 256, 0, stream>>>(partials, nblocks, chunk, mid);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_reduce_final4(mid, mid_blocks, out, add0, stream);
}

}  // namespace clbm
