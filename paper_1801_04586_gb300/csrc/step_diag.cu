// step_diag.cu -- the fused step kernel with in-kernel conservation sums, for
// jobs that read mass and momentum back after every step.
//
// Same per-node work as k_step (pull, collide, store). In addition every
// warp sums the Eq. 9 density deviation and momentum of the state it pulls
// (the state before the step) as exact fixed-point integers (block_reduce.cuh),
// so the totals equal clbm_reduce_moments' bit for bit. Lane 0 of each warp
// writes its 4 sums (32 bytes per 32 nodes): no block barrier holds the
// warps of a block together. The warp partials are added by a two-level
// integer reduction; only the final totals become FP64.
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
    fx *= F.scale;
    fy *= F.scale;
    fz *= F.scale;
}

template <typename S, int FM, bool WALLS>
__global__ void __launch_bounds__(512) k_step_diag(const S *__restrict__ src, S *__restrict__ dst, Geom g, Rates r,
                                                   ForceArgs F, int *__restrict__ flag,
                                                   long long *__restrict__ partials, uint32_t key) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    long long q[4] = {0ll, 0ll, 0ll, 0ll};
    if (x < g.nx && y < g.ny) {  // no early return: every lane joins the warp sums
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
        store_node<S>(dst + off[0], g.stride, h, off[0], key);
        q[0] = to_fixed(drho); q[1] = to_fixed(j.x); q[2] = to_fixed(j.y); q[3] = to_fixed(j.z);
    }
    // blockDim.x is a multiple of 32, so a warp is 32 threads of one row
    const size_t b = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const unsigned wpb = (blockDim.x * blockDim.y) >> 5;
    const unsigned w = (threadIdx.x + blockDim.x * threadIdx.y) >> 5;
    long long s[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) s[k] = warp_sum_fixed(q[k]);
    if ((threadIdx.x & 31) == 0) {
        long long *d = partials + 4 * (b * wpb + w);
#pragma unroll
        for (int k = 0; k < 4; ++k) d[k] = s[k];
    }
}

template <typename S, int FM>
static cudaError_t diag_walls(const Launch &L, const void *src, void *dst, const Rates &r, const ForceArgs &F,
                              int *flag, long long *partials, uint32_t key) {
    if (L.g.walls)
        k_step_diag<S, FM, true><<<L.grid, L.block, 0, L.stream>>>((const S *)src, (S *)dst, L.g, r, F, flag,
                                                                   partials, key);
    else
        k_step_diag<S, FM, false><<<L.grid, L.block, 0, L.stream>>>((const S *)src, (S *)dst, L.g, r, F, flag,
                                                                    partials, key);
    return cudaGetLastError();
}

template <typename S>
static cudaError_t diag_force(const Launch &L, const void *src, void *dst, const Rates &r, const ForceArgs &F,
                              int *flag, long long *partials, uint32_t key) {
    switch (F.mode) {
        case kForceUniform: return diag_walls<S, kForceUniform>(L, src, dst, r, F, flag, partials, key);
        case kForceProfileZ: return diag_walls<S, kForceProfileZ>(L, src, dst, r, F, flag, partials, key);
        default: return diag_walls<S, kForceField>(L, src, dst, r, F, flag, partials, key);
    }
}

cudaError_t launch_step_diag(int storage, const Launch &L, const void *src, void *dst, const Rates &r,
                             const ForceArgs &F, int *flag, long long *partials, uint32_t key) {
    switch (storage) {
        case 0: return diag_force<float>(L, src, dst, r, F, flag, partials, key);
        case 1: return diag_force<__half>(L, src, dst, r, F, flag, partials, key);
        case 2: return diag_force<__nv_bfloat16>(L, src, dst, r, F, flag, partials, key);
        case 3: return diag_force<HalfSR>(L, src, dst, r, F, flag, partials, key);
        default: return diag_force<BF16SR>(L, src, dst, r, F, flag, partials, key);
    }
}

// Sum nblocks fixed-point partials of 4 values: each block of the first pass
// adds a contiguous chunk, the second pass adds the chunk sums and writes the
// FP64 totals (plus add0 on the first).
__global__ void k_sum_partials4(const long long *__restrict__ partials, int64_t nblocks, int64_t chunk,
                                long long *__restrict__ mid) {
    long long q[4] = {0ll, 0ll, 0ll, 0ll};
    const int64_t lo = (int64_t)blockIdx.x * chunk, hi = min(nblocks, lo + chunk);
    for (int64_t b = lo + threadIdx.x; b < hi; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < 4; ++k) q[k] += partials[4 * b + k];
    block_sum_fixed<4>(q, mid + 4 * (size_t)blockIdx.x);
}

cudaError_t launch_sum_partials4(const long long *partials, int64_t nblocks, long long *mid, int mid_blocks,
                                 double *out, double add0, cudaStream_t stream) {
    const int64_t chunk = (nblocks + mid_blocks - 1) / mid_blocks;
    k_sum_partials4<<<mid_blocks, 256, 0, stream>>>(partials, nblocks, chunk, mid);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_fixed_final4(mid, mid_blocks, out, add0, stream);
}

}  // namespace clbm
