// kernels.cuh -- launch interface between the C ABI (capi.cu) and the kernel
// translation units. Plain structs only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "d3q19.cuh"

namespace clbm {

enum ForceMode : int { kForceUniform = 0, kForceProfileZ = 1, kForceField = 2 };

struct ForceArgs {
    int mode;
    float fx, fy, fz;        // uniform
    const float *profile;    // 3 x nz
    const float *field;      // 3 x N
    int64_t n;               // N, component stride of `field`
    float scale;             // time factor e^{-gamma t} of the step (1 for a static force)
};

struct Launch {
    Geom g;
    dim3 block, grid;  // grid of the one-node-per-thread kernels
    cudaStream_t stream;
    bool packed;       // launch_step: two nodes per thread (grid.x halved)
    bool staged;       // launch_step (A/B) and launch_step_aa (16-bit, cascaded): rows staged by bulk copies
                       // where they apply (step_tma.cuh)
    int map;           // state kernels: slots of the post-streaming state (0 A/B pull map,
                       // 1 in-place pattern after even steps, 2 after odd steps, 3 the A/B pull
                       // map of a z-slab with halo faces)
    long long wait_cycles = 0;  // staged step: bound of a wait for a tile's copies (0: kWaitCycles)
    bool drop_first_tile = false;  // staged step, failure injection: tile 0's copies are not issued
    int z0 = 0, zs = 1, nplanes = -1;  // staged and fused-sums steps, init, read-out: the planes z0, z0 + zs, ...
                                       // (nplanes of them; -1: all)
};

// storage: 0 = f32, 1 = f16, 2 = bf16, 3 = f16 stochastic, 4 = bf16 stochastic
// (CLBM_STORAGE_*). key: per-step dither key (stochastic formats).
cudaError_t launch_step(int storage, const Launch &L, const void *src, void *dst, const Rates &r,
                        const ForceArgs &F, int *flag, uint32_t key);
// The cascaded step on a z-slab (Geom::slab halo faces): the planes z0,
// z0 + zs, ... (nplanes of them) from src into dst (step.cu).
cudaError_t launch_step_slab(int storage, const Launch &L, const void *src, void *dst, const Rates &r,
                             const ForceArgs &F, int *flag, uint32_t key, int z0, int zs, int nplanes);
// Whether an A/B step of a q-population lattice from a state buffer at src
// (elem bytes per value) with force mode force_mode runs the shared-memory
// staged kernel (step_tma.cuh) when the launch asks for it.
bool step_staged(const Geom &g, size_t elem, const void *src, int q, int force_mode);
// In-place (AA) pattern: one step on the single population array f; odd
// selects the odd step kind (step.cu).
cudaError_t launch_step_aa(int storage, const Launch &L, void *f, const Rates &r, const ForceArgs &F, int *flag,
                           uint32_t key, bool odd);
// The cascaded in-place step with 16-bit storage staged in node pairs, if it
// applies (step_aa.cu); false: nothing launched.
bool launch_step_aa_staged(int storage, const Launch &L, void *f, const Rates &r, const ForceArgs &F, int *flag,
                           uint32_t key, bool odd, cudaError_t &err);
// The comparison collision models (models.cuh): SRT-LBM and non-orthogonal
// MRT, A/B and in-place forms (step_srt.cu, step_mrt.cu).
cudaError_t launch_step_srt(int storage, const Launch &L, const void *src, void *dst, const Rates &r,
                            const ForceArgs &F, int *flag, uint32_t key);
cudaError_t launch_step_mrt(int storage, const Launch &L, const void *src, void *dst, const Rates &r,
                            const ForceArgs &F, int *flag, uint32_t key);
cudaError_t launch_step_aa_srt(int storage, const Launch &L, void *f, const Rates &r, const ForceArgs &F, int *flag,
                               uint32_t key, bool odd);
cudaError_t launch_step_aa_mrt(int storage, const Launch &L, void *f, const Rates &r, const ForceArgs &F, int *flag,
                               uint32_t key, bool odd);
// Fused step + fixed-point conservation sums of the pulled state into the
// kDiagSlots x 4 accumulators acc (zero on entry). If acc_prev is not null,
// the launch first drains that set (the previous step's) into out_prev[0..3]
// (FP64 totals, add0 added to the first) and clears it. launch_drain4 drains a set on its own (step_diag.cu).
// With L.nplanes >= 0 it steps the planes L.z0 .. L.z0 + L.nplanes - 1 only
// (L.zs = 1); the launches of one step's plane ranges add into the same set.
constexpr int kDiagSlots = 1024;
struct DiagSums {
    unsigned long long *acc;
    unsigned long long *acc_prev;
    double *out_prev;
    double add0;
};
cudaError_t launch_step_diag(int storage, const Launch &L, const void *src, void *dst, const Rates &r,
                             const ForceArgs &F, int *flag, const DiagSums &d, uint32_t key);
cudaError_t launch_drain4(unsigned long long *acc, double *out, double add0, cudaStream_t stream);
cudaError_t launch_fixed_final4(const long long *partials, int nblocks, double *out, double add0,
                                cudaStream_t stream);
cudaError_t launch_scatter(int storage, const Launch &L, void *dst, const float *f, int64_t n, int deviation);
cudaError_t launch_init_eq(int storage, const Launch &L, void *dst, const float *rho, const float *u, int64_t n,
                           const ForceArgs &F);
cudaError_t launch_gather(int storage, const Launch &L, const void *src, float *f, int64_t n, int deviation);
cudaError_t launch_macros(int storage, const Launch &L, const void *src, const ForceArgs &F, float *rho, float *u,
                          int64_t n);
cudaError_t launch_reduce_moments(int storage, const Launch &L, const void *src, const ForceArgs &F,
                                  long long *partials, int nblocks, double *out);
cudaError_t launch_adjoint_step(int storage, const Launch &L, const void *state, const float *lam_next, float *lam,
                                float *gF, const Rates &r, const ForceArgs &F, int64_t n);
cudaError_t launch_adjoint_seed(int storage, const Launch &L, const void *state, const float *gu, float *lam,
                                float *gF, const ForceArgs &F, int64_t n);
cudaError_t launch_reduce_pair(const float *a, const float *b, int64_t n, double *partials, int nblocks,
                               double *out, cudaStream_t stream);

// D3Q27 (step27.cu); Rates27 in d3q27.cuh.
struct Rates27;
cudaError_t launch_step27(int storage, const Launch &L, const void *src, void *dst, const Rates27 &r,
                          const ForceArgs &F, int *flag, uint32_t key);
cudaError_t launch_init27(int storage, const Launch &L, void *dst, const float *rho, const float *u, int64_t n,
                          const ForceArgs &F);
cudaError_t launch_scatter27(int storage, const Launch &L, void *dst, const float *f, int64_t n, int deviation);
cudaError_t launch_gather27(int storage, const Launch &L, const void *src, float *f, int64_t n, int deviation);
cudaError_t launch_macros27(int storage, const Launch &L, const void *src, const ForceArgs &F, float *rho, float *u,
                            int64_t n);
cudaError_t launch_step27_aa(int storage, const Launch &L, void *f, const Rates27 &r, const ForceArgs &F, int *flag,
                             uint32_t key, bool odd);
// The comparison models on D3Q27 (models27.cuh; step27_srt.cu, step27_mrt.cu).
cudaError_t launch_step27_srt(int storage, const Launch &L, const void *src, void *dst, const Rates27 &r,
                              const ForceArgs &F, int *flag, uint32_t key);
cudaError_t launch_step27_mrt(int storage, const Launch &L, const void *src, void *dst, const Rates27 &r,
                              const ForceArgs &F, int *flag, uint32_t key);
cudaError_t launch_step27_aa_srt(int storage, const Launch &L, void *f, const Rates27 &r, const ForceArgs &F,
                                 int *flag, uint32_t key, bool odd);
cudaError_t launch_step27_aa_mrt(int storage, const Launch &L, void *f, const Rates27 &r, const ForceArgs &F,
                                 int *flag, uint32_t key, bool odd);
cudaError_t launch_moments27(int storage, const Launch &L, const void *src, const ForceArgs &F, long long *partials,
                             int nblocks, double *out);

// Record `msg` as the calling thread's last error (clbm_last_error) and return code.
int set_error(int code, const char *msg);

// NVTX range for the span of one entry point (shown by profilers that
// record NVTX; a no-op otherwise), in the "clbm" domain.
struct Range {
    explicit Range(const char *name);
    ~Range();
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

}  // namespace clbm
