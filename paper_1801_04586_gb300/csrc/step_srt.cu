// step_srt.cu -- step kernels of the SRT-LBM comparison model (models.cuh)
// on the layout, streaming and storage formats of the cascaded step.
#include "models.cuh"
#include "step_kernels.cuh"

namespace clbm {

struct Srt {
    static constexpr bool kPairs = false;  // one node at a time (float only)
    template <bool FR = false>
    static __device__ __forceinline__ float run(float (&h)[kQ], float Fx, float Fy, float Fz, const Rates &r) {
        return collide_srt<FR>(h, Fx, Fy, Fz, r);
    }
};

cudaError_t launch_step_srt(int storage, const Launch &L, const void *src, void *dst, const Rates &r,
                            const ForceArgs &F, int *flag, uint32_t key) {
    return launch_step_with<Srt>(storage, L, src, dst, r, F, flag, key);
}

cudaError_t launch_step_aa_srt(int storage, const Launch &L, void *f, const Rates &r, const ForceArgs &F, int *flag,
                               uint32_t key, bool odd) {
    return launch_step_aa_with<Srt>(storage, L, f, r, F, flag, key, odd);
}

}  // namespace clbm
