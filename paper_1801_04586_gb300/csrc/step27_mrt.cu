// step27_mrt.cu -- D3Q27 step kernels of the non-orthogonal MRT comparison model
// (models27.cuh) on the layout, streaming and storage formats of the cascaded
// step.
#include "models27.cuh"
#include "step27_kernels.cuh"

namespace clbm {

struct Mrt27 {
    template <bool FR = false>
    static __device__ __forceinline__ float run(float (&h)[3][3][3], float Fx, float Fy, float Fz,
                                                const Rates27 &r) {
        return collide_mrt27<FR>(h, Fx, Fy, Fz, r);
    }
};

cudaError_t launch_step27_mrt(int storage, const Launch &L, const void *src, void *dst, const Rates27 &r,
                               const ForceArgs &F, int *flag, uint32_t key) {
    return launch_step27_with<Mrt27>(storage, L, src, dst, r, F, flag, key);
}

cudaError_t launch_step27_aa_mrt(int storage, const Launch &L, void *f, const Rates27 &r, const ForceArgs &F,
                                  int *flag, uint32_t key, bool odd) {
    return launch_step27_aa_with<Mrt27>(storage, L, f, r, F, flag, key, odd);
}

}  // namespace clbm
