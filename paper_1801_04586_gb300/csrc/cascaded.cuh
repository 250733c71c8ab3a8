// cascaded.cuh -- the paper's cascaded collision with the consistent forcing
// scheme (Eqs. 5 and 7 with A3, A5, A6; collide in d3q19.cuh) as the
// collision policy of the step kernels (step.cu, step_slab.cu).
#pragma once

#include "d3q19.cuh"

namespace clbm {

struct Cascaded {
    static constexpr bool kPairs = true;  // also runs on f2 (two nodes at once): the staged step pairs nodes
    template <bool FR = false, typename T>
    static __device__ __forceinline__ T run(T (&h)[kQ], T Fx, T Fy, T Fz, const Rates &r) {
        return collide<FR>(h, Fx, Fy, Fz, r);
    }
};

}  // namespace clbm
