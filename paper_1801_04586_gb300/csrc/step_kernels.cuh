// step_kernels.cuh -- the D3Q19 step kernels, templated on the collision.
//
// k_step: the fused pull stream-and-collide kernel (one launch per time step).
// Per node (x, y, z): gather the 19 post-collision populations of the previous
// step from the neighbours x - e_i (Eq. 8; periodic wrap or halfway
// bounce-back), collide them and store the 19 post-collision values at the
// node itself. Loads use the read-only path so that the +-1 x-shifted reads of
// neighbouring threads share L1 sectors; stores are coalesced and aligned. One
// thread per node, x fastest, so each warp touches 19 contiguous 128-byte
// segments per direction.
//
// k_step_aa: the same update on one buffer in place (AA pattern).
//
// The collision is a policy C with
//   static float run(float (&h)[19], float Fx, float Fy, float Fz, const Rates &r)
// that collides the deviations h in place and returns rho - 1 (Eq. 9): the
// cascaded collision of the paper (step.cu), or the SRT and non-orthogonal
// MRT comparison models (models.cuh; step_srt.cu, step_mrt.cu).
#pragma once

#include "kernels.cuh"

namespace clbm {

template <int FM>
__device__ __forceinline__ void force_at(const ForceArgs &F, const Geom &g, int z, uint32_t self, float &fx,
                                         float &fy, float &fz) {
    if (FM == kForceUniform) {
        fx = F.fx; fy = F.fy; fz = F.fz;
    } else if (FM == kForceProfileZ) {
        fx = __ldg(F.profile + z);
        fy = __ldg(F.profile + g.nz + z);
        fz = __ldg(F.profile + 2 * g.nz + z);
    } else {
        fx = __ldg(F.field + self);
        fy = __ldg(F.field + F.n + self);
        fz = __ldg(F.field + 2 * F.n + self);
    }
    fx *= F.scale;
    fy *= F.scale;
    fz *= F.scale;
}

}  // namespace clbm

#include "step_tma.cuh"

namespace clbm {

template <typename C, typename S, int FM, bool WALLS>
__global__ void __launch_bounds__(512) k_step(const S *__restrict__ src, S *__restrict__ dst, Geom g, Rates r,
                                              ForceArgs F, int *__restrict__ flag, uint32_t key) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    uint32_t off[kQ];
    int pop[kQ];
    pull_sources<WALLS>(g, x, y, z, off, pop);
    float h[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) h[i] = Codec<S>::load(src + CLBM_IDX(g, (size_t)pop[i] * g.stride + off[i]));
    float fx, fy, fz;
    force_at<FM>(F, g, z, off[0], fx, fy, fz);
    const float drho = C::template run<sizeof(S) == 2>(h, fx, fy, fz, r);
    if (!(fabsf(drho) < 0.9f)) *flag = 1;
    // the node's slots off[0] + i * stride, i < kQ, lie below the last one's bound
    store_node<S>(dst + CLBM_SLOTS(g, off[0], (kQ - 1) * g.stride), g.stride, h, off[0], key);
}

// In-place (AA) pattern: one population array set, two step kinds that
// alternate. Same collision, same bytes per node update, half the memory.
//   even step: the slots hold the post-streaming f(x) in natural order; read
//              population i at (i, x), write post-collision population i to
//              (ibar, x), the slot the next odd step pulls it from.
//   odd step:  read population i at (ibar, x - e_i), or at (i, x) when x - e_i
//              lies beyond a wall (halfway bounce-back); write post-collision
//              population i where the next even step reads f_i(x + e_i):
//              (i, x + e_i), or (ibar, x) when x + e_i lies beyond a wall.
// In both kinds a node writes exactly the slots it read, and no other node
// touches them, so the update is race-free in place. Loads may take the
// read-only path: a slot is read once, by the thread that later overwrites
// it, and never after a write within the launch.
template <typename C, typename S, int FM, bool WALLS, bool ODD>
__global__ void __launch_bounds__(512, sizeof(S) == 2 ? 2 : 0) k_step_aa(S *f, Geom g, Rates r, ForceArgs F, int *__restrict__ flag,
                                                 uint32_t key) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const uint32_t self = ((uint32_t)z * g.ny + y) * g.nx + x;
    float h[kQ];
    if (ODD) {
        uint32_t off[kQ];
        int pop[kQ];
        pull_sources<WALLS, true>(g, x, y, z, off, pop);
#pragma unroll
        for (int i = 0; i < kQ; ++i) h[i] = Codec<S>::load(f + CLBM_IDX(g, (size_t)pop[i] * g.stride + off[i]));
        float fx, fy, fz;
        force_at<FM>(F, g, z, self, fx, fy, fz);
        const float drho = C::template run<sizeof(S) == 2>(h, fx, fy, fz, r);
        if (!(fabsf(drho) < 0.9f)) *flag = 1;
        // The slots read for the opposite directions are the push targets of
        // Eq. 8. They are recomputed from coordinates the compiler must treat
        // as new and as depending on the collision's outputs, so that 19
        // offsets do not stay live through the collision.
        int xs = x, ys = y, zs = z;
        asm volatile("" : "+r"(xs), "+r"(ys), "+r"(zs) : "f"(h[0]), "f"(h[kQ - 1]));
        push_targets<WALLS>(g, xs, ys, zs, off, pop);
        store_each<S, kQ>(h, self, key, [&](int i) { return f + CLBM_IDX(g, (size_t)pop[i] * g.stride + off[i]); });
    } else {
#pragma unroll
        for (int i = 0; i < kQ; ++i) h[i] = Codec<S>::load(f + CLBM_IDX(g, (size_t)i * g.stride + self));
        float fx, fy, fz;
        force_at<FM>(F, g, z, self, fx, fy, fz);
        const float drho = C::template run<sizeof(S) == 2>(h, fx, fy, fz, r);
        if (!(fabsf(drho) < 0.9f)) *flag = 1;
        store_each<S, kQ>(h, self, key, [&](int i) { return f + CLBM_IDX(g, (size_t)opposite(i) * g.stride + self); });
    }
}

template <typename C, typename S, int FM>
static cudaError_t step_walls_t(const Launch &L, const void *src, void *dst, const Rates &r, const ForceArgs &F,
                                int *flag, uint32_t key) {
    if constexpr (sizeof(S) == 2) {  // 16-bit storage: rows staged in shared memory where they apply
        cudaError_t e = cudaSuccess;
        if (L.staged && launch_step_tma<19, C, S, FM>(L, src, dst, r, F, flag, key, e)) return e;
    }
    if (L.g.walls)
        k_step<C, S, FM, true><<<L.grid, L.block, 0, L.stream>>>((const S *)src, (S *)dst, L.g, r, F, flag, key);
    else
        k_step<C, S, FM, false><<<L.grid, L.block, 0, L.stream>>>((const S *)src, (S *)dst, L.g, r, F, flag, key);
    return cudaGetLastError();
}

template <typename C, typename S>
static cudaError_t step_force_t(const Launch &L, const void *src, void *dst, const Rates &r, const ForceArgs &F,
                                int *flag, uint32_t key) {
    switch (F.mode) {
        case kForceUniform: return step_walls_t<C, S, kForceUniform>(L, src, dst, r, F, flag, key);
        case kForceProfileZ: return step_walls_t<C, S, kForceProfileZ>(L, src, dst, r, F, flag, key);
        default: return step_walls_t<C, S, kForceField>(L, src, dst, r, F, flag, key);
    }
}

// One A/B step (one node per thread) with collision C, any storage format.
template <typename C>
cudaError_t launch_step_with(int storage, const Launch &L, const void *src, void *dst, const Rates &r,
                             const ForceArgs &F, int *flag, uint32_t key) {
    switch (storage) {
        case 0: return step_force_t<C, float>(L, src, dst, r, F, flag, key);
        case 1: return step_force_t<C, __half>(L, src, dst, r, F, flag, key);
        case 2: return step_force_t<C, __nv_bfloat16>(L, src, dst, r, F, flag, key);
        case 3: return step_force_t<C, HalfSR>(L, src, dst, r, F, flag, key);
        default: return step_force_t<C, BF16SR>(L, src, dst, r, F, flag, key);
    }
}

template <typename C, typename S, int FM>
static cudaError_t step_aa_walls_t(const Launch &L, void *f, const Rates &r, const ForceArgs &F, int *flag,
                                   uint32_t key, bool odd) {
    if (!odd)
        k_step_aa<C, S, FM, false, false><<<L.grid, L.block, 0, L.stream>>>((S *)f, L.g, r, F, flag, key);
    else if (L.g.walls)
        k_step_aa<C, S, FM, true, true><<<L.grid, L.block, 0, L.stream>>>((S *)f, L.g, r, F, flag, key);
    else
        k_step_aa<C, S, FM, false, true><<<L.grid, L.block, 0, L.stream>>>((S *)f, L.g, r, F, flag, key);
    return cudaGetLastError();
}

template <typename C, typename S>
static cudaError_t step_aa_force_t(const Launch &L, void *f, const Rates &r, const ForceArgs &F, int *flag,
                                   uint32_t key, bool odd) {
    switch (F.mode) {
        case kForceUniform: return step_aa_walls_t<C, S, kForceUniform>(L, f, r, F, flag, key, odd);
        case kForceProfileZ: return step_aa_walls_t<C, S, kForceProfileZ>(L, f, r, F, flag, key, odd);
        default: return step_aa_walls_t<C, S, kForceField>(L, f, r, F, flag, key, odd);
    }
}

// One in-place (AA) step with collision C, any storage format.
template <typename C>
cudaError_t launch_step_aa_with(int storage, const Launch &L, void *f, const Rates &r, const ForceArgs &F,
                                int *flag, uint32_t key, bool odd) {
    switch (storage) {
        case 0: return step_aa_force_t<C, float>(L, f, r, F, flag, key, odd);
        case 1: return step_aa_force_t<C, __half>(L, f, r, F, flag, key, odd);
        case 2: return step_aa_force_t<C, __nv_bfloat16>(L, f, r, F, flag, key, odd);
        case 3: return step_aa_force_t<C, HalfSR>(L, f, r, F, flag, key, odd);
        default: return step_aa_force_t<C, BF16SR>(L, f, r, F, flag, key, odd);
    }
}

}  // namespace clbm
