// step_aa.cu -- the cascaded collision's in-place (AA) step with 16-bit
// storage, staged in shared memory by bulk copies and collided two adjacent
// nodes per thread (step_tma.cuh, modes kTileAAEven / kTileAAOdd). The even
// kind copies each tile's own rows and stores every population into the
// opposite slot of its node; the odd kind copies the opposite populations'
// rows shifted as the pull and stores to the push targets of Eq. 8. Both read
// and write exactly the slots of their own nodes, as the one-node kernel
// k_step_aa does, and store the same bits.
#include <type_traits>

#include "cascaded.cuh"
#include "step_kernels.cuh"

namespace clbm {

bool launch_step_aa_staged(int storage, const Launch &L, void *f, const Rates &r, const ForceArgs &F, int *flag,
                           uint32_t key, bool odd, cudaError_t &err) {
    auto by_type = [&](auto tag) -> bool {
        using S = decltype(tag);
        auto kind = [&](auto mode) -> bool {
            constexpr int M = decltype(mode)::value;
            switch (F.mode) {
                case kForceUniform:
                    return launch_step_tma<19, Cascaded, S, kForceUniform, M>(L, f, f, r, F, flag, key, err);
                case kForceProfileZ:
                    return launch_step_tma<19, Cascaded, S, kForceProfileZ, M>(L, f, f, r, F, flag, key, err);
                default:
                    return launch_step_tma<19, Cascaded, S, kForceField, M>(L, f, f, r, F, flag, key, err);
            }
        };
        return odd ? kind(std::integral_constant<int, kTileAAOdd>{}) : kind(std::integral_constant<int, kTileAAEven>{});
    };
    switch (storage) {
        case 1: return by_type(__half{});
        case 2: return by_type(__nv_bfloat16{});
        case 3: return by_type(HalfSR{});
        case 4: return by_type(BF16SR{});
        default: return false;  // FP32 stays on k_step_aa
    }
}

}  // namespace clbm
