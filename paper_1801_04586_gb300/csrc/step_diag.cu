// step_diag.cu -- the fused step kernel with in-kernel conservation sums, for
// jobs that read mass and momentum back after every step.
//
// Same per-node work as k_step (pull, collide, store), for kDiagZ nodes per
// thread along z. In addition every warp sums the Eq. 9 density deviation and
// momentum of the state it pulls (the state before the step) as exact
// fixed-point integers (block_reduce.cuh), so the totals equal
// clbm_reduce_moments' bit for bit. Each thread adds the fixed-point parts of
// its nodes in registers; then two warp reductions per quantity and lane 0's
// four 64-bit integer atomics into one of kDiagSlots accumulator slots cover
// 32 x kDiagZ nodes. Integer addition is exact and order-independent, so the
// totals do not depend on scheduling, and no block barrier holds the warps of
// a block together. (With one node per thread the reductions and atomics
// cost 6 % of the step at 256^3; with four they are lost in the memory time.) The slots come in two sets used by alternate steps:
// block 0 of each step first drains the set the previous step filled (adds
// the slots, writes the FP64 totals, clears the set), so no separate launch
// sits between steps. k_drain4 drains the last step's set.
#include "block_reduce.cuh"
#include "kernels.cuh"

namespace clbm {

// Totals of a slot set as FP64 (plus add0 on the first) to out[0..3], then
// the set is cleared. Every thread of the block calls it.
__device__ __forceinline__ void drain_slots(unsigned long long *acc, double *out, double add0) {
    const int nt = blockDim.x * blockDim.y;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    long long q[4] = {0ll, 0ll, 0ll, 0ll};
    for (int s = tid; s < kDiagSlots; s += nt)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            q[k] += (long long)acc[4 * s + k];
            acc[4 * s + k] = 0ull;
        }
    __shared__ long long tot[4];
    block_sum_fixed<4>(q, tot);
    __syncthreads();
    if (tid == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) out[k] = (double)tot[k] * kFixUnit + (k == 0 ? add0 : 0.0);
}

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

// Nodes per thread along z. The per-thread part sums stay in 32 bits:
// kDiagZ x 32 high parts below 2^22 sum below 2^29.
constexpr int kDiagZ = 4;

template <typename S, int FM, bool WALLS>
__global__ void __launch_bounds__(512, 2) k_step_diag(const S *__restrict__ src, S *__restrict__ dst, Geom g,
                                                      Rates r, ForceArgs F, int *__restrict__ flag,
                                                      unsigned long long *__restrict__ acc,
                                                      unsigned long long *__restrict__ acc_prev, double *out_prev,
                                                      double add0, uint32_t key, int zb, int ze) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z0 = zb + blockIdx.z * kDiagZ;
    if (acc_prev && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0) drain_slots(acc_prev, out_prev, add0);
    int hi[4] = {0, 0, 0, 0}, lo[4] = {0, 0, 0, 0};  // fixed-point parts of the sums (to_fixed_parts)
    if (x < g.nx && y < g.ny) {  // no early return: every lane joins the warp sums
#pragma unroll 1
        for (int z = z0; z < z0 + kDiagZ && z < ze; ++z) {
            uint32_t off[kQ];
            int pop[kQ];
            pull_sources<WALLS>(g, x, y, z, off, pop);
            float h[kQ];
#pragma unroll
            for (int i = 0; i < kQ; ++i) h[i] = Codec<S>::load(src + (size_t)pop[i] * g.stride + off[i]);
            float fx, fy, fz;
            force_diag<FM>(F, g, z, off[0], fx, fy, fz);
            float3 j;
            const float drho = collide<sizeof(S) == 2>(h, fx, fy, fz, r, &j);
            if (!(fabsf(drho) < 0.9f)) *flag = 1;
            store_node<S>(dst + off[0], g.stride, h, off[0], key);
            const float q[4] = {drho, j.x, j.y, j.z};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                int a, b;
                to_fixed_parts(q[k], a, b);
                hi[k] += a;
                lo[k] += b;
            }
        }
    }
    // blockDim.x is a multiple of 32, so a warp is 32 threads of one row
    const size_t b = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const unsigned wpb = (blockDim.x * blockDim.y) >> 5;
    const unsigned w = (threadIdx.x + blockDim.x * threadIdx.y) >> 5;
    long long s[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        s[k] = (long long)__reduce_add_sync(0xffffffffu, hi[k]) * 1048576ll +
               (long long)__reduce_add_sync(0xffffffffu, lo[k]);
    if ((threadIdx.x & 31) == 0) {
        unsigned long long *d = acc + 4 * ((b * wpb + w) & (kDiagSlots - 1));
#pragma unroll
        for (int k = 0; k < 4; ++k) atomicAdd(d + k, (unsigned long long)s[k]);  // two's complement: signed sum
    }
}

template <typename S, int FM>
static cudaError_t diag_walls(const Launch &L, const void *src, void *dst, const Rates &r, const ForceArgs &F,
                              int *flag, const DiagSums &d, uint32_t key) {
    // the planes z0 .. z0 + nplanes - 1 (all planes if nplanes < 0)
    const int zb = L.nplanes < 0 ? 0 : L.z0;
    const int np = L.nplanes < 0 ? L.g.nz : L.nplanes;
    if (L.zs != 1 || zb < 0 || np < 1 || zb + np > L.g.nz) return cudaErrorInvalidValue;
    const dim3 grid(L.grid.x, L.grid.y, (np + kDiagZ - 1) / kDiagZ);
    if (L.g.walls)
        k_step_diag<S, FM, true><<<grid, L.block, 0, L.stream>>>((const S *)src, (S *)dst, L.g, r, F, flag, d.acc,
                                                                 d.acc_prev, d.out_prev, d.add0, key, zb, zb + np);
    else
        k_step_diag<S, FM, false><<<grid, L.block, 0, L.stream>>>((const S *)src, (S *)dst, L.g, r, F, flag, d.acc,
                                                                  d.acc_prev, d.out_prev, d.add0, key, zb, zb + np);
    return cudaGetLastError();
}

template <typename S>
static cudaError_t diag_force(const Launch &L, const void *src, void *dst, const Rates &r, const ForceArgs &F,
                              int *flag, const DiagSums &d, uint32_t key) {
    switch (F.mode) {
        case kForceUniform: return diag_walls<S, kForceUniform>(L, src, dst, r, F, flag, d, key);
        case kForceProfileZ: return diag_walls<S, kForceProfileZ>(L, src, dst, r, F, flag, d, key);
        default: return diag_walls<S, kForceField>(L, src, dst, r, F, flag, d, key);
    }
}

cudaError_t launch_step_diag(int storage, const Launch &L, const void *src, void *dst, const Rates &r,
                             const ForceArgs &F, int *flag, const DiagSums &d, uint32_t key) {
    switch (storage) {
        case 0: return diag_force<float>(L, src, dst, r, F, flag, d, key);
        case 1: return diag_force<__half>(L, src, dst, r, F, flag, d, key);
        case 2: return diag_force<__nv_bfloat16>(L, src, dst, r, F, flag, d, key);
        case 3: return diag_force<HalfSR>(L, src, dst, r, F, flag, d, key);
        default: return diag_force<BF16SR>(L, src, dst, r, F, flag, d, key);
    }
}

// Drain one slot set (the last step's). One block.
__global__ void k_drain4(unsigned long long *acc, double *out, double add0) { drain_slots(acc, out, add0); }

cudaError_t launch_drain4(unsigned long long *acc, double *out, double add0, cudaStream_t stream) {
    k_drain4<<<1, 1024, 0, stream>>>(acc, out, add0);
    return cudaGetLastError();
}

}  // namespace clbm
