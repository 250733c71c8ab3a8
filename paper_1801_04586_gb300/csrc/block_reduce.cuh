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

// Sums FP32 values v over the block: FP32 within each warp (shuffles), FP64
// across the warps. Writes the K totals to dst[0..K-1]. Every thread calls it.
template <int K>
__device__ __forceinline__ void block_sum_f32_store(float (&v)[K], double *dst) {
    __shared__ double sm[32][K];
#pragma unroll
    for (int k = 0; k < K; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) sm[warp][k] = (double)v[k];
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

}  // namespace clbm
