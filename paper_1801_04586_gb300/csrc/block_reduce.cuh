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
// 2^-36 and held as an integer, so the sums are exact, independent of the
// order of addition and need no FP64 arithmetic (which issues at a small
// fraction of the FP32 rate on this GPU). The rounding is done with FP32
// additions only (no 64-bit conversion): v * 2^36 rounded to nearest even is
// returned as hi * 2^20 + lo with hi = round(v * 2^16) and lo = round((v *
// 2^16 - hi) * 2^20), both taken from the mantissa of a sum with 1.5 * 2^23.
// Exact for |v| < 2^6; density deviations and momenta of any state that has
// not tripped the instability flag are far below that. A sum of up to 2^24
// values below 1 fits in 64 bits with room to spare.
constexpr double kFixScale = 68719476736.0;          // 2^36
constexpr double kFixUnit = 1.0 / 68719476736.0;     // 2^-36

__device__ __forceinline__ void to_fixed_parts(float v, int &hi, int &lo) {
    constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23: the ulp of the sum is 1
    const float t = fmaf(v, 65536.0f, kMagic);          // 1.5 * 2^23 + round(v * 2^16)
    const float r = fmaf(v, 65536.0f, -(t - kMagic));   // v * 2^16 - round(v * 2^16), exact, |r| <= 1/2
    const float l = fmaf(r, 1048576.0f, kMagic);        // 1.5 * 2^23 + round(r * 2^20)
    hi = __float_as_int(t) - __float_as_int(kMagic);
    lo = __float_as_int(l) - __float_as_int(kMagic);
}

__device__ __forceinline__ long long to_fixed(float v) {
    int hi, lo;
    to_fixed_parts(v, hi, lo);
    return (long long)hi * 1048576ll + (long long)lo;
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
