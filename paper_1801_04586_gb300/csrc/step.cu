// step.cu -- the cascaded collision's step kernels (Eqs. 5, 7, 9 with A3, A5,
// A6; collision in d3q19.cuh, kernels in step_kernels.cuh), plus the form
// with two nodes per thread on the FP32x2 instructions.
#include "cascaded.cuh"
#include "step_kernels.cuh"

namespace clbm {

// Two nodes per thread: x and x + blockDim.x of a 2 * blockDim.x segment of a
// row, collided together with the FP32x2 instructions (f2 in d3q19.cuh), which
// halves the arithmetic issue slots per node. Each node's loads and stores stay
// warp-coalesced. At a row tail the second lane repeats the first node and is
// not stored.
template <typename S, int FM, bool WALLS>
__global__ void __launch_bounds__(256) k_step2(const S *__restrict__ src, S *__restrict__ dst, Geom g, Rates r,
                                               ForceArgs F, int *__restrict__ flag, uint32_t key) {
    const int x0 = blockIdx.x * (2 * blockDim.x) + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x0 >= g.nx || y >= g.ny) return;
    const int x1 = x0 + blockDim.x;
    const bool has1 = x1 < g.nx;
    const int xb = has1 ? x1 : x0;
    uint32_t oa[kQ], ob[kQ];
    int pa[kQ], pb[kQ];
    pull_sources<WALLS>(g, x0, y, z, oa, pa);
    pull_sources<WALLS>(g, xb, y, z, ob, pb);
    f2 h[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i)
        h[i] = mk2(Codec<S>::load(src + (size_t)pa[i] * g.stride + oa[i]),
                   Codec<S>::load(src + (size_t)pb[i] * g.stride + ob[i]));
    float fxa, fya, fza, fxb, fyb, fzb;
    force_at<FM>(F, g, z, oa[0], fxa, fya, fza);
    force_at<FM>(F, g, z, ob[0], fxb, fyb, fzb);
    const f2 drho = collide<sizeof(S) == 2>(h, mk2(fxa, fxb), mk2(fya, fyb), mk2(fza, fzb), r);
    if (!(fabsf(drho.v.x) < 0.9f) || !(fabsf(drho.v.y) < 0.9f)) *flag = 1;
    float ha[kQ], hb[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        ha[i] = h[i].v.x;
        hb[i] = h[i].v.y;
    }
    store_node<S>(dst + oa[0], g.stride, ha, oa[0], key);
    if (has1) store_node<S>(dst + ob[0], g.stride, hb, ob[0], key);
}

template <typename S, int FM>
static cudaError_t step2_walls(const Launch &L, const void *src, void *dst, const Rates &r, const ForceArgs &F,
                               int *flag, uint32_t key) {
    if (L.g.walls)
        k_step2<S, FM, true><<<L.grid, L.block, 0, L.stream>>>((const S *)src, (S *)dst, L.g, r, F, flag, key);
    else
        k_step2<S, FM, false><<<L.grid, L.block, 0, L.stream>>>((const S *)src, (S *)dst, L.g, r, F, flag, key);
    return cudaGetLastError();
}

template <typename S>
static cudaError_t step2_force(const Launch &L, const void *src, void *dst, const Rates &r, const ForceArgs &F,
                               int *flag, uint32_t key) {
    switch (F.mode) {
        case kForceUniform: return step2_walls<S, kForceUniform>(L, src, dst, r, F, flag, key);
        case kForceProfileZ: return step2_walls<S, kForceProfileZ>(L, src, dst, r, F, flag, key);
        default: return step2_walls<S, kForceField>(L, src, dst, r, F, flag, key);
    }
}

cudaError_t launch_step(int storage, const Launch &L, const void *src, void *dst, const Rates &r,
                        const ForceArgs &F, int *flag, uint32_t key) {
    if (!L.packed) return launch_step_with<Cascaded>(storage, L, src, dst, r, F, flag, key);
    switch (storage) {
        case 0: return step2_force<float>(L, src, dst, r, F, flag, key);
        case 1: return step2_force<__half>(L, src, dst, r, F, flag, key);
        case 2: return step2_force<__nv_bfloat16>(L, src, dst, r, F, flag, key);
        case 3: return step2_force<HalfSR>(L, src, dst, r, F, flag, key);
        default: return step2_force<BF16SR>(L, src, dst, r, F, flag, key);
    }
}

bool step_staged(const Geom &g, size_t elem, const void *src, int q, int force_mode) {
    return step_staged_for(g, elem, src, q, force_mode);
}

cudaError_t launch_step_aa(int storage, const Launch &L, void *f, const Rates &r, const ForceArgs &F, int *flag,
                           uint32_t key, bool odd) {
    cudaError_t e = cudaSuccess;
    if (L.staged && launch_step_aa_staged(storage, L, f, r, F, flag, key, odd, e)) return e;
    return launch_step_aa_with<Cascaded>(storage, L, f, r, F, flag, key, odd);
}

}  // namespace clbm
