// step_slab_kernels.cuh -- the cascaded step on a z-slab with halo faces
// (Eq. 8 across the slab faces; Geom::slab): the one-node-per-thread slab
// kernel and the launcher that picks it or the staged node-pair step
// (step_tma.cuh with its SLAB tiles). Included by step_slab.cu only.
#pragma once

#include <type_traits>

#include "step_kernels.cuh"

namespace clbm {

// The step on a z-slab of a larger lattice (Eq. 8 across the slab's halo
// faces, see Geom::slab): the same update as k_step for the planes
// z = z0, z0 + zs, ... (blockIdx.z counts them), pulling the populations that
// cross a halo face from the halo planes of src, and also writing the node's
// outgoing populations across a halo face into the send planes of dst for the
// neighbour. The dither of stochastic rounding takes the global node index
// (node0 + local index), so a slab stores exactly what the undivided lattice
// stores.
template <typename C, typename S, int FM, bool WALLS>
__global__ void __launch_bounds__(512) k_step_slab(const S *__restrict__ src, S *__restrict__ dst, Geom g, Rates r,
                                                   ForceArgs F, int *__restrict__ flag, uint32_t key, int z0, int zs) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = z0 + (int)blockIdx.z * zs;
    if (x >= g.nx || y >= g.ny) return;
    uint32_t off[kQ];
    int pop[kQ];
    pull_sources<WALLS, false, true>(g, x, y, z, off, pop);
    float h[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) h[i] = Codec<S>::load(src + CLBM_IDX(g, (size_t)pop[i] * g.stride + off[i]));
    const uint32_t plane = (uint32_t)g.nx * (uint32_t)g.ny;
    const uint32_t ps = (uint32_t)y * (uint32_t)g.nx + (uint32_t)x;
    const uint32_t self = (uint32_t)z * plane + ps;
    float fx, fy, fz;
    force_at<FM>(F, g, z, self, fx, fy, fz);
    const float drho = C::template run<sizeof(S) == 2>(h, fx, fy, fz, r);
    if (!(fabsf(drho) < 0.9f)) *flag = 1;
    S e[kQ];
    encode_each<S, kQ>(h, self + g.node0, key, e);
#pragma unroll
    for (int i = 0; i < kQ; ++i) dst[CLBM_IDX(g, (size_t)i * g.stride + self)] = e[i];
    const size_t send = (size_t)kQ * g.stride;
    if ((g.slab & 1u) && z == 0)
#pragma unroll
        for (int k = 0; k < 5; ++k) dst[CLBM_IDX(g, send + (size_t)(10 + k) * plane + ps)] = e[zminus_pop(k)];
    if ((g.slab & 2u) && z == g.nz - 1)
#pragma unroll
        for (int k = 0; k < 5; ++k) dst[CLBM_IDX(g, send + (size_t)(15 + k) * plane + ps)] = e[zplus_pop(k)];
}

template <typename C, typename S, int FM>
static cudaError_t step_slab_walls_t(const Launch &L, const void *src, void *dst, const Rates &r,
                                     const ForceArgs &F, int *flag, uint32_t key, int z0, int zs, int nplanes) {
    if (nplanes <= 0) return cudaSuccess;
    dim3 grid = L.grid;
    grid.z = (unsigned)nplanes;
    if (L.g.walls)
        k_step_slab<C, S, FM, true><<<grid, L.block, 0, L.stream>>>((const S *)src, (S *)dst, L.g, r, F, flag, key,
                                                                    z0, zs);
    else
        k_step_slab<C, S, FM, false><<<grid, L.block, 0, L.stream>>>((const S *)src, (S *)dst, L.g, r, F, flag, key,
                                                                     z0, zs);
    return cudaGetLastError();
}

// One z-slab step (or a part of it: the planes z0, z0 + zs, ..., nplanes of
// them) with collision C, any storage format. 16-bit storage takes the staged
// step where it applies: its copies read the halo planes across halo faces,
// and its launches over the first and last planes (SEND) also write the send
// planes. A whole-slab step is those two planes, then the rest, so that the
// interior runs the kernel without the send stores. Otherwise one node per
// thread.
template <typename C>
cudaError_t launch_step_slab_with(int storage, const Launch &L, const void *src, void *dst, const Rates &r,
                                  const ForceArgs &F, int *flag, uint32_t key, int z0, int zs, int nplanes) {
    auto by_force = [&](auto tag) -> cudaError_t {
        using S = decltype(tag);
        auto one_node = [&](int a, int b, int n) -> cudaError_t {
            switch (F.mode) {
                case kForceUniform:
                    return step_slab_walls_t<C, S, kForceUniform>(L, src, dst, r, F, flag, key, a, b, n);
                case kForceProfileZ:
                    return step_slab_walls_t<C, S, kForceProfileZ>(L, src, dst, r, F, flag, key, a, b, n);
                default:
                    return step_slab_walls_t<C, S, kForceField>(L, src, dst, r, F, flag, key, a, b, n);
            }
        };
        if constexpr (sizeof(S) == 2) {
            if (L.staged && nplanes > 0) {
                // the planes a, a + b, ... (n of them) staged; false: not launched (the staged step does not apply)
                auto staged = [&](auto send, int a, int b, int n, cudaError_t &e) -> bool {
                    constexpr int SD = decltype(send)::value ? kTileSlabSend : kTileSlab;
                    Launch Ls = L;
                    Ls.z0 = a;
                    Ls.zs = b;
                    Ls.nplanes = n;
                    switch (F.mode) {
                        case kForceUniform:
                            return launch_step_tma<19, C, S, kForceUniform, SD>(Ls, src, dst, r, F, flag, key, e);
                        case kForceProfileZ:
                            return launch_step_tma<19, C, S, kForceProfileZ, SD>(Ls, src, dst, r, F, flag, key,
                                                                                        e);
                        default:
                            return launch_step_tma<19, C, S, kForceField, SD>(Ls, src, dst, r, F, flag, key, e);
                    }
                };
                const int nz = L.g.nz;
                cudaError_t e = cudaSuccess;
                if (z0 == 0 && zs == 1 && nplanes == nz && nz > 2) {
                    if (staged(std::true_type{}, 0, nz - 1, 2, e)) {
                        if (e != cudaSuccess) return e;
                        if (staged(std::false_type{}, 1, 1, nz - 2, e)) return e;
                        return one_node(1, 1, nz - 2);
                    }
                } else {
                    bool ends = false;  // whether the set holds the first or last plane
                    for (int k = 0; k < nplanes; ++k) ends = ends || z0 + k * zs == 0 || z0 + k * zs == nz - 1;
                    if (ends ? staged(std::true_type{}, z0, zs, nplanes, e)
                             : staged(std::false_type{}, z0, zs, nplanes, e))
                        return e;
                }
            }
        }
        return one_node(z0, zs, nplanes);
    };
    switch (storage) {
        case 0: return by_force(float{});
        case 1: return by_force(__half{});
        case 2: return by_force(__nv_bfloat16{});
        case 3: return by_force(HalfSR{});
        default: return by_force(BF16SR{});
    }
}

}  // namespace clbm
