// step_slab.cu -- the cascaded step on a z-slab with halo faces (Eq. 8
// across the slab faces): the staged node-pair step for 16-bit storage, the
// one-node kernel otherwise (step_slab_kernels.cuh, step_tma.cuh). Its own
// translation unit, so that the slab instantiations build beside step.cu.
#include "cascaded.cuh"
#include "step_slab_kernels.cuh"

namespace clbm {

cudaError_t launch_step_slab(int storage, const Launch &L, const void *src, void *dst, const Rates &r,
                             const ForceArgs &F, int *flag, uint32_t key, int z0, int zs, int nplanes) {
    return launch_step_slab_with<Cascaded>(storage, L, src, dst, r, F, flag, key, z0, zs, nplanes);
}

}  // namespace clbm
