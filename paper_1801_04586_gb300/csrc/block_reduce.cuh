// block_reduce.cuh -- deterministic FP64 block sums (warp shuffles, then one
// warp over the per-warp results). Every thread of the block must call it.
#pragma once

namespace clbm {

// Sums v over the block and writes the K totals to dst[0..K-1] (thread 0's
// warp writes). Blocks of at most 1024 threads.
template <int K>
__device__ __forceinline__ void block_sum_store(double (&v)[K], double *dst) {
    __shared__ double sm[32][K];
#pragma unroll
    for (int k = 0; k < K; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) sm[warp][k] = v[k];
    __syncthreads();
    if (warp == 0) {
        const int nw = (nthreads + 31) >> 5;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double t = lane < nw ? sm[lane][k] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) dst[k] = t;
        }
    }
}

// Fixed-point conservation sums. Each FP32 value is rounded to a multiple of
// 2^-36 and held as a 64-bit integer, so the sums are exact, independent of
// the order of addition and need no FP64 arithmetic (which issues at a small
// fraction of the FP32 rate on this GPU). Values must stay below 2^27 in
// magnitude and a sum of up to 2^24 values below 1 fits with room to spare;
// a state that breaks this has already tripped the instability flag.
constexpr double kFixScale = 68719476736.0;          // 2^36
constexpr double kFixUnit = 1.0 / 68719476736.0;     // 2^-36

__device__ __forceinline__ long long to_fixed(float v) { return __float2ll_rn(v * 68719476736.0f); }

// Warp sum of fixed-point values, exact, with two 32-bit warp reductions
// (redux.sync) instead of 64-bit shuffles: v is split into its low 20 bits
// (non-negative) and the rest (arithmetic shift). Exact while every |v| <
// 2^46 (|value| < 2^10): then 32 high parts sum below 2^31 and 32 low parts
// below 2^25. All 32 lanes must call it.
__device__ __forceinline__ long long warp_sum_fixed(long long v) {
    const int lo = (int)(v & 0xfffffll);
    const int hi = (int)(v >> 20);
    const int slo = __reduce_add_sync(0xffffffffu, lo);
    const int shi = __reduce_add_sync(0xffffffffu, hi);
    return (long long)shi * 1048576ll + (long long)slo;
}

// Block sum of fixed-point values q; thread 0's warp writes the K totals to
// dst[0..K-1]. Every thread of the block calls it.
template <int K>
__device__ __forceinline__ void block_sum_fixed(long long (&q)[K], long long *dst) {
    __shared__ long long sm[32][K];
#pragma unroll
    for (int k = 0; k < K; ++k)
        for (int o = 16; o > 0; o >>= 1) q[k] += __shfl_down_sync(0xffffffffu, q[k], o);
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) sm[warp][k] = q[k];
    __syncthreads();
    if (warp == 0) {
        const int nw = (nthreads + 31) >> 5;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            long long t = lane < nw ? sm[lane][k] : 0ll;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) dst[k] = t;
        }
    }
}

}  // namespace clbm
