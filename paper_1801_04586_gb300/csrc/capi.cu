// capi.cu -- the extern "C" boundary declared in include/clbm.h: context
// lifetime, argument validation, A/B buffer bookkeeping and launches.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "../../include/clbm.h"
#include "d3q27.cuh"
#include "kernels.cuh"

using namespace clbm;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *where) {
    return fail(CLBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

size_t elem_size(int storage) { return storage == CLBM_STORAGE_F32 ? 4 : 2; }

constexpr int kReduceBlocks = 4 * 152;  // fixed reduction grid: deterministic sums

struct StateHeader {
    char magic[8];
    int32_t version, nx, ny, nz, walls, storage, q, pattern;
    int64_t stride, steps_done, bytes;
};

}  // namespace

int clbm::set_error(int code, const char *msg) { return fail(code, msg); }

namespace {
nvtxDomainHandle_t nvtx_domain() {
    static nvtxDomainHandle_t d = nvtxDomainCreateA("clbm");
    return d;
}
}  // namespace

clbm::Range::Range(const char *name) {
    nvtxEventAttributes_t a = {};
    a.version = NVTX_VERSION;
    a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
    a.messageType = NVTX_MESSAGE_TYPE_ASCII;
    a.message.ascii = name;
    nvtxDomainRangePushEx(nvtx_domain(), &a);
}

clbm::Range::~Range() { nvtxDomainRangePop(nvtx_domain()); }

// clbm_run_host moves its host input and output in this many plane chunks, so
// that each chunk's initialisation or read-out runs beside the next copy.
constexpr int kIoChunks = 8;

struct clbm_ctx {
    clbm_params p;
    Geom g;
    int64_t n;
    size_t elem;
    void *buf[2];
    int cur;
    cudaStream_t stream;
    Rates rates;
    double s2;
    ForceArgs force;
    int *d_flag;
    double *d_partials;
    float *d_io;               // clbm_run_host scratch (first use): 4 x N floats, then
    double *d_mom;             //   kMomRing x 4 doubles of per-step sums and
    unsigned long long *d_acc; //   2 sets of kDiagSlots x 4 fixed-point accumulators (kept zero between steps)
    cudaStream_t copy_stream;  // clbm_run_host: per-step sums copied back beside the steps (first use)
    cudaEvent_t ev_step, ev_copy;
    int64_t steps_done;
    double gamma;         // force decay rate (clbm_set_force_decay)
    bool packed;          // step kernel with two nodes per thread (FP32x2 arithmetic)
    bool staged;          // steps with rows staged in shared memory by bulk copies (variant 0; see clbm_create)
    int q;                // 19 (Appendix A) or 27 (Sec. II)
    bool aa;              // in-place (AA) pattern: one population buffer, step kind by parity
    int model;            // CLBM_MODEL_*
    Rates27 rates27;
    dim3 block;
    cudaStream_t cap_stream;   // private stream for graph capture (first use)
    cudaGraphExec_t graph;     // kGraphSteps steps from phase 0; null until built, dropped when the force changes
    bool slab_pending;         // z-slab: CLBM_SLAB_FACES done, CLBM_SLAB_INTERIOR not yet
    cudaStream_t io_stream;    // clbm_run_host: host copies in plane chunks beside init / read-out (first use)
    cudaEvent_t io_ev[kIoChunks];
};

namespace {

// Elements of one state buffer: the Q population arrays, then for a z-slab
// its halo planes (kSlabPlanes of nx * ny values, see d3q19.cuh).
size_t state_elems(const clbm_ctx *c) {
    size_t e = (size_t)c->q * c->g.stride;
    if (c->g.slab) e += (size_t)kSlabPlanes * c->g.nx * c->g.ny;
    return e;
}

size_t state_bytes(const clbm_ctx *c) { return state_elems(c) * c->elem; }

// The force in use at the context's current time step.
ForceArgs force_at_zero(const clbm_ctx *c) {
    ForceArgs F = c->force;
    F.scale = 1.0f;
    return F;
}

ForceArgs force_at(const clbm_ctx *c, int64_t step) {
    ForceArgs F = c->force;
    F.scale = c->gamma == 0.0 ? 1.0f : (float)std::exp(-c->gamma * (double)step);
    return F;
}

ForceArgs force_now(const clbm_ctx *c) { return force_at(c, c->steps_done); }

// clbm_run_host's fused path: the totals of step t land in slot t % kMomRing
// and are copied back on a second stream while the next steps run; every
// kMomSync steps the step stream waits for the copies issued kMomSync steps
// earlier, so no slot is overwritten before its copy (kMomRing >= 2 kMomSync).
constexpr int kMomRing = 64;
constexpr int kMomSync = 32;
static_assert(kMomRing >= 2 * kMomSync, "slot reuse needs two sync periods");

// Steps replayed from one captured CUDA graph (even, so a replay ends in the
// phase it started from).
constexpr int kGraphSteps = 16;

void drop_graph(clbm_ctx *c) {
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
}

Launch launch_of(const clbm_ctx *c) {
    Launch L;
    L.g = c->g;
    L.block = c->block;
    L.grid = dim3((c->g.nx + c->block.x - 1) / c->block.x, (c->g.ny + c->block.y - 1) / c->block.y, c->g.nz);
    L.stream = c->stream;
    L.packed = false;
    L.staged = c->staged;
    // A/B: the pull map (through the halo planes for a z-slab); AA: natural
    // slots after an even number of steps, the odd step's swapped pull map
    // after an odd number.
    L.map = c->aa ? ((c->steps_done & 1) ? 2 : 1) : (c->g.slab ? 3 : 0);
    L.wait_cycles = c->p.wait_cycles;
    L.drop_first_tile = c->p.inject == CLBM_INJECT_DROP_COPY;
    return L;
}

// The step launch: two nodes per thread when the context's variant says so.
Launch step_launch_of(const clbm_ctx *c) {
    Launch L = launch_of(c);
    if (c->packed) {
        L.packed = true;
        L.grid.x = (c->g.nx + 2 * c->block.x - 1) / (2 * c->block.x);
    }
    return L;
}

bool rate_ok(double s) { return std::isfinite(s) && s > 0.0 && s < 2.0; }

// One D3Q19 step of the context's collision model and pattern.
cudaError_t step19(const clbm_ctx *c, const Launch &L, const void *src, void *dst, const ForceArgs &F,
                   uint32_t key) {
    switch (c->model) {
        case CLBM_MODEL_SRT: return launch_step_srt(c->p.storage, L, src, dst, c->rates, F, c->d_flag, key);
        case CLBM_MODEL_MRT: return launch_step_mrt(c->p.storage, L, src, dst, c->rates, F, c->d_flag, key);
        default: return launch_step(c->p.storage, L, src, dst, c->rates, F, c->d_flag, key);
    }
}

cudaError_t step27(const clbm_ctx *c, const Launch &L, const void *src, void *dst, const ForceArgs &F,
                   uint32_t key) {
    switch (c->model) {
        case CLBM_MODEL_SRT: return launch_step27_srt(c->p.storage, L, src, dst, c->rates27, F, c->d_flag, key);
        case CLBM_MODEL_MRT: return launch_step27_mrt(c->p.storage, L, src, dst, c->rates27, F, c->d_flag, key);
        default: return launch_step27(c->p.storage, L, src, dst, c->rates27, F, c->d_flag, key);
    }
}

cudaError_t step27_aa(const clbm_ctx *c, const Launch &L, void *f, const ForceArgs &F, uint32_t key, bool odd) {
    switch (c->model) {
        case CLBM_MODEL_SRT: return launch_step27_aa_srt(c->p.storage, L, f, c->rates27, F, c->d_flag, key, odd);
        case CLBM_MODEL_MRT: return launch_step27_aa_mrt(c->p.storage, L, f, c->rates27, F, c->d_flag, key, odd);
        default: return launch_step27_aa(c->p.storage, L, f, c->rates27, F, c->d_flag, key, odd);
    }
}

cudaError_t step19_aa(const clbm_ctx *c, const Launch &L, void *f, const ForceArgs &F, uint32_t key, bool odd) {
    switch (c->model) {
        case CLBM_MODEL_SRT: return launch_step_aa_srt(c->p.storage, L, f, c->rates, F, c->d_flag, key, odd);
        case CLBM_MODEL_MRT: return launch_step_aa_mrt(c->p.storage, L, f, c->rates, F, c->d_flag, key, odd);
        default: return launch_step_aa(c->p.storage, L, f, c->rates, F, c->d_flag, key, odd);
    }
}

// One time step `step` of the context's lattice, pattern and model, from
// buffer cur (A/B) or in place (AA), launched with L.
cudaError_t one_step(const clbm_ctx *c, const Launch &L, int cur, int64_t step) {
    const ForceArgs F = force_at(c, step);
    const uint32_t key = step_key(step);
    if (c->aa) {
        const bool odd = (step & 1) != 0;
        return c->q == 27 ? step27_aa(c, L, c->buf[0], F, key, odd) : step19_aa(c, L, c->buf[0], F, key, odd);
    }
    if (c->g.slab)
        return launch_step_slab(c->p.storage, L, c->buf[cur], c->buf[cur ^ 1], c->rates, F, c->d_flag, key, 0, 1,
                                c->g.nz);
    return c->q == 27 ? step27(c, L, c->buf[cur], c->buf[cur ^ 1], F, key)
                      : step19(c, L, c->buf[cur], c->buf[cur ^ 1], F, key);
}

// Capture kGraphSteps steps starting from phase 0 (A/B: from buffer 0; AA: an
// even step) on a private stream. Only for launches whose arguments do not
// change from step to step: a static force and no stochastic dither key.
int ensure_graph(clbm_ctx *c) {
    if (c->graph) return CLBM_OK;
    Range range("clbm_step: graph capture");
    cudaError_t e = cudaSuccess;
    if (!c->cap_stream && (e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        c->cap_stream = nullptr;
        return cuda_fail(e, "clbm_step: capture stream");
    }
    Launch L = step_launch_of(c);
    L.stream = c->cap_stream;
    cudaGraph_t g = nullptr;
    if ((e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(e, "clbm_step: begin capture");
    for (int k = 0; k < kGraphSteps && e == cudaSuccess; ++k) e = one_step(c, L, k & 1, k);
    cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->graph = nullptr;
        cudaGetLastError();
        return cuda_fail(e, "clbm_step: graph capture");
    }
    return CLBM_OK;
}

}  // namespace

extern "C" {

const char *clbm_status_string(int status) {
    switch (status) {
        case CLBM_OK: return "ok";
        case CLBM_ERR_ARG: return "invalid argument";
        case CLBM_ERR_OOM: return "device out of memory";
        case CLBM_ERR_CUDA: return "CUDA error";
        case CLBM_ERR_UNSTABLE: return "unstable: density out of range or non-finite";
        case CLBM_ERR_STATE: return "invalid state";
        case CLBM_ERR_TIMEOUT: return "timeout: a staged copy did not complete";
        case CLBM_ERR_BOUNDS: return "bounds: a kernel derived an out-of-range index";
        default: return "unknown status";
    }
}

const char *clbm_last_error(void) { return g_last_error.c_str(); }

int clbm_create(const clbm_params *p, void *stream, clbm_ctx **out) {
    if (!p || !out) return fail(CLBM_ERR_ARG, "clbm_create: null pointer");
    *out = nullptr;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->nx > 65535 || p->ny > 65535 || p->nz > 65535)
        return fail(CLBM_ERR_ARG, "clbm_create: each extent must be in [1, 65535]");
    const int64_t n = (int64_t)p->nx * p->ny * p->nz;
    if (n > ((int64_t)1 << 31) - 1) return fail(CLBM_ERR_ARG, "clbm_create: more than 2^31-1 nodes");
    if (p->walls & ~7u) return fail(CLBM_ERR_ARG, "clbm_create: unknown wall bits");
    if (!(std::isfinite(p->nu) && p->nu > 0.0)) return fail(CLBM_ERR_ARG, "clbm_create: nu must be > 0");
    const double s2 = 1.0 / (3.0 * p->nu + 0.5);
    if (!rate_ok(s2) || !rate_ok(p->s2b) || !rate_ok(p->s3) || !rate_ok(p->s4))
        return fail(CLBM_ERR_ARG, "clbm_create: relaxation rates must lie in (0, 2)");
    if (p->storage < CLBM_STORAGE_F32 || p->storage > CLBM_STORAGE_BF16_SR)
        return fail(CLBM_ERR_ARG, "clbm_create: unknown storage format");
    if (p->variant < 0 || p->variant > 2) return fail(CLBM_ERR_ARG, "clbm_create: variant must be 0, 1 or 2");
    if (p->lattice != 0 && p->lattice != 19 && p->lattice != 27)
        return fail(CLBM_ERR_ARG, "clbm_create: lattice must be 19 or 27");
    const int q = p->lattice == 27 ? 27 : 19;
    auto or1 = [](double s) { return s == 0.0 ? 1.0 : s; };
    const double s3b = or1(p->s3b), s4b = or1(p->s4b), s5 = or1(p->s5), s6 = or1(p->s6);
    if (q == 27 && (!rate_ok(s3b) || !rate_ok(s4b) || !rate_ok(s5) || !rate_ok(s6)))
        return fail(CLBM_ERR_ARG, "clbm_create: relaxation rates must lie in (0, 2)");
    if (q == 27 && p->variant == 2)
        return fail(CLBM_ERR_ARG, "clbm_create: the two-nodes-per-thread form is D3Q19 only");
    if (p->pattern != CLBM_PATTERN_AB && p->pattern != CLBM_PATTERN_AA)
        return fail(CLBM_ERR_ARG, "clbm_create: pattern must be CLBM_PATTERN_AB or CLBM_PATTERN_AA");
    if (p->pattern == CLBM_PATTERN_AA && p->variant == 2)
        return fail(CLBM_ERR_ARG, "clbm_create: the in-place pattern runs one node per thread (variant 0 or 1)");
    if (p->model < CLBM_MODEL_CASCADED || p->model > CLBM_MODEL_MRT || p->reserved != 0 || p->reserved2 != 0)
        return fail(CLBM_ERR_ARG, "clbm_create: model must be CLBM_MODEL_CASCADED, _SRT or _MRT (reserved 0)");
    if (p->slab & ~(CLBM_SLAB_LO | CLBM_SLAB_HI)) return fail(CLBM_ERR_ARG, "clbm_create: unknown slab bits");
    if (p->wait_cycles < 0) return fail(CLBM_ERR_ARG, "clbm_create: wait_cycles must be >= 0");
    if (p->inject != 0 && p->inject != CLBM_INJECT_DROP_COPY)
        return fail(CLBM_ERR_ARG, "clbm_create: inject must be 0 or CLBM_INJECT_DROP_COPY");
    if (p->slab && (q != 19 || p->model != CLBM_MODEL_CASCADED || p->pattern != CLBM_PATTERN_AB || p->variant == 2))
        return fail(CLBM_ERR_ARG,
                    "clbm_create: z-slabs are D3Q19, cascaded, A/B pattern, one node per thread (variant 0 or 1)");
    if (p->z0 < 0 || (!p->slab && p->z0 != 0))
        return fail(CLBM_ERR_ARG, "clbm_create: z0 must be >= 0, and 0 unless slab is set");
    if (p->slab && ((int64_t)p->z0 + p->nz) * p->nx * p->ny > ((int64_t)1 << 31) - 1)
        return fail(CLBM_ERR_ARG, "clbm_create: the slab's global node indices exceed 2^31-1");
    if (p->slab && (int64_t)kSlabPlanes * p->nx * p->ny > ((int64_t)1 << 31) - 1)
        return fail(CLBM_ERR_ARG, "clbm_create: the slab's halo planes exceed 2^31-1 values");
    if (p->model != CLBM_MODEL_CASCADED && p->variant == 2)
        return fail(CLBM_ERR_ARG, "clbm_create: the SRT and MRT models run one node per thread");
    int bx = p->block_x, by = p->block_y;
    if (bx == 0) bx = p->nx >= 128 ? 128 : ((p->nx + 31) / 32) * 32;
    if (by == 0) by = std::max(1, std::min(p->ny, 256 / bx));
    if (bx < 32 || bx % 32 != 0 || by < 1 || bx * by > 512)
        return fail(CLBM_ERR_ARG, "clbm_create: block_x must be a multiple of 32 and block_x*block_y <= 512");
    if ((p->ny + by - 1) / by > 65535) return fail(CLBM_ERR_ARG, "clbm_create: ny / block_y exceeds grid limit");
    if (q == 27 && bx * by > 256) return fail(CLBM_ERR_ARG, "clbm_create: D3Q27 blocks hold at most 256 threads");

    clbm_ctx *c = new (std::nothrow) clbm_ctx();
    if (!c) return fail(CLBM_ERR_OOM, "clbm_create: host allocation failed");
    c->p = *p;
    c->n = n;
    c->elem = elem_size(p->storage);
    c->g.nx = p->nx; c->g.ny = p->ny; c->g.nz = p->nz;
    c->g.walls = p->walls;
    c->g.stride = (n + 63) / 64 * 64;  // every population array starts 256-byte aligned (f32)
    c->g.slab = (uint32_t)p->slab;
    c->g.node0 = (uint32_t)((int64_t)p->z0 * p->nx * p->ny);
    c->stream = (cudaStream_t)stream;
    c->s2 = s2;
    c->rates.om2 = (float)(1.0 - s2);
    c->rates.cb = (float)((p->s2b - s2) / 3.0);
    c->rates.om3 = (float)(1.0 - p->s3);
    c->rates.c3 = (float)((1.0 - 0.5 * p->s3) / 3.0);
    c->rates.om4 = (float)(1.0 - p->s4);
    c->force.mode = kForceUniform;
    c->force.fx = c->force.fy = c->force.fz = 0.0f;
    c->force.profile = nullptr;
    c->force.field = nullptr;
    c->force.n = n;
    c->force.scale = 1.0f;
    c->gamma = 0.0;
    c->q = q;
    c->packed = q == 19 && p->variant == 2;
    // staged: A/B steps, and the cascaded D3Q19 in-place step (node pairs)
    c->staged = p->variant == 0 &&
                (p->pattern != CLBM_PATTERN_AA || (q == 19 && p->model == CLBM_MODEL_CASCADED));
    c->aa = p->pattern == CLBM_PATTERN_AA;
    c->model = p->model;
    c->rates27.om2 = c->rates.om2;
    c->rates27.cb = c->rates.cb;
    c->rates27.om3 = c->rates.om3;
    c->rates27.c3 = c->rates.c3;
    c->rates27.om3b = (float)(1.0 - s3b);
    c->rates27.om4 = c->rates.om4;
    c->rates27.om4b = (float)(1.0 - s4b);
    c->rates27.om5 = (float)(1.0 - s5);
    c->rates27.c5 = (float)((1.0 - 0.5 * s5) / 9.0);
    c->rates27.om6 = (float)(1.0 - s6);
    c->block = dim3(bx, by, 1);
    c->cur = 0;
    c->steps_done = 0;
    const size_t bytes = (state_bytes(c) + 255) / 256 * 256;  // both buffers 256-byte aligned
    const size_t nbuf = c->aa ? 1 : 2;
    cudaError_t e = cudaMalloc(&c->buf[0], nbuf * bytes);
    if (e != cudaSuccess) {
        delete c;
        cudaGetLastError();
        return fail(CLBM_ERR_OOM, std::string("clbm_create: cudaMalloc: ") + cudaGetErrorString(e));
    }
    c->buf[1] = c->aa ? c->buf[0] : (char *)c->buf[0] + bytes;
    e = cudaMalloc(&c->d_flag, 256 + sizeof(double) * 4 * kReduceBlocks);
    if (e != cudaSuccess) {
        cudaFree(c->buf[0]);
        delete c;
        cudaGetLastError();
        return fail(CLBM_ERR_OOM, std::string("clbm_create: cudaMalloc: ") + cudaGetErrorString(e));
    }
    c->d_partials = (double *)((char *)c->d_flag + 256);
#ifdef CLBM_BOUNDS_CHECK
    c->g.bc = (BoundsRecord *)((char *)c->d_flag + 64);  // the flag block's bytes 64-79
    c->g.bc_limit = state_elems(c);
#endif
    // rest state: zero deviations in every buffer (zero bits are zero in all formats)
    if ((e = cudaMemsetAsync(c->buf[0], 0, nbuf * bytes, c->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(c->d_flag, 0, 128, c->stream)) != cudaSuccess) {
        cudaFree(c->d_flag);
        cudaFree(c->buf[0]);
        delete c;
        return cuda_fail(e, "clbm_create");
    }
    *out = c;
    return CLBM_OK;
}

int clbm_destroy(clbm_ctx *c) {
    if (!c) return CLBM_OK;
    cudaStreamSynchronize(c->stream);
    drop_graph(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
        cudaEventDestroy(c->ev_step);
        cudaEventDestroy(c->ev_copy);
    }
    if (c->io_stream) {
        cudaStreamSynchronize(c->io_stream);
        cudaStreamDestroy(c->io_stream);
        for (int k = 0; k < kIoChunks; ++k) cudaEventDestroy(c->io_ev[k]);
    }
    cudaFree(c->buf[0]);
    cudaFree(c->d_flag);
    if (c->d_io) cudaFree(c->d_io);
    delete c;
    return CLBM_OK;
}

int clbm_get_info(const clbm_ctx *c, clbm_info *info) {
    if (!c || !info) return fail(CLBM_ERR_ARG, "clbm_get_info: null pointer");
    info->n_nodes = c->n;
    info->pop_stride = c->g.stride;
    info->state_bytes = (int64_t)state_bytes(c);
    info->steps_done = c->steps_done;
    info->storage = c->p.storage;
    info->block_x = (int32_t)c->block.x;
    info->block_y = (int32_t)c->block.y;
    info->s2 = c->s2;
    info->nodes_per_thread = c->packed ? 2 : 1;
    info->q = c->q;
    info->pattern = c->aa ? CLBM_PATTERN_AA : CLBM_PATTERN_AB;
    info->buffers = c->aa ? 1 : 2;
    info->model = c->model;
    info->staged = c->staged && step_staged(c->g, c->elem, c->buf[0], c->q, c->force.mode) ? 1 : 0;
    info->slab = (int32_t)c->g.slab;
    info->face_bytes = c->g.slab ? (int64_t)5 * c->g.nx * c->g.ny * (int64_t)c->elem : 0;
    return CLBM_OK;
}

int clbm_set_force_uniform(clbm_ctx *c, double fx, double fy, double fz) {
    if (!c) return fail(CLBM_ERR_ARG, "clbm_set_force_uniform: null context");
    if (!(std::isfinite(fx) && std::isfinite(fy) && std::isfinite(fz)))
        return fail(CLBM_ERR_ARG, "clbm_set_force_uniform: non-finite force");
    c->force.mode = kForceUniform;
    c->force.fx = (float)fx; c->force.fy = (float)fy; c->force.fz = (float)fz;
    drop_graph(c);
    return CLBM_OK;
}

int clbm_set_force_profile_z(clbm_ctx *c, const float *F) {
    if (!c || !F) return fail(CLBM_ERR_ARG, "clbm_set_force_profile_z: null pointer");
    c->force.mode = kForceProfileZ;
    c->force.profile = F;
    drop_graph(c);
    return CLBM_OK;
}

int clbm_set_force_field(clbm_ctx *c, const float *F) {
    if (!c || !F) return fail(CLBM_ERR_ARG, "clbm_set_force_field: null pointer");
    c->force.mode = kForceField;
    c->force.field = F;
    drop_graph(c);
    return CLBM_OK;
}

int clbm_set_force_decay(clbm_ctx *c, double gamma) {
    if (!c) return fail(CLBM_ERR_ARG, "clbm_set_force_decay: null context");
    if (!std::isfinite(gamma)) return fail(CLBM_ERR_ARG, "clbm_set_force_decay: non-finite rate");
    c->gamma = gamma;
    drop_graph(c);
    return CLBM_OK;
}

int clbm_init_equilibrium(clbm_ctx *c, const float *rho, const float *u) {
    if (!c) return fail(CLBM_ERR_ARG, "clbm_init_equilibrium: null context");
    if (c->slab_pending) return fail(CLBM_ERR_STATE, "clbm_init_equilibrium: a split slab step is pending");
    c->steps_done = 0;  // before launch_of: the in-place pattern starts in natural order
    cudaError_t e = c->q == 27
        ? launch_init27(c->p.storage, launch_of(c), c->buf[c->cur], rho, u, c->n, force_at_zero(c))
        : launch_init_eq(c->p.storage, launch_of(c), c->buf[c->cur], rho, u, c->n, force_at_zero(c));
    if (e != cudaSuccess) return cuda_fail(e, "clbm_init_equilibrium");
    return CLBM_OK;
}

int clbm_step(clbm_ctx *c, int64_t nsteps) {
    if (!c) return fail(CLBM_ERR_ARG, "clbm_step: null context");
    if (nsteps < 0) return fail(CLBM_ERR_ARG, "clbm_step: nsteps < 0");
    if (c->g.slab && (nsteps > 1 || c->slab_pending))
        return fail(CLBM_ERR_STATE, "clbm_step: a z-slab takes one step per call (faces are exchanged between steps)");
    Range range("clbm_step");
    const Launch L = step_launch_of(c);
    auto advance = [&]() -> int {
        cudaError_t e = one_step(c, L, c->cur, c->steps_done);
        if (e != cudaSuccess) return cuda_fail(e, "clbm_step");
        if (!c->aa) c->cur ^= 1;
        ++c->steps_done;
        return CLBM_OK;
    };
    int64_t t = 0;
    // Long runs with static launch arguments replay a captured graph of
    // kGraphSteps steps: one launch call per 16 steps instead of 16.
    const bool stochastic = c->p.storage == CLBM_STORAGE_F16_SR || c->p.storage == CLBM_STORAGE_BF16_SR;
    if (!stochastic && c->gamma == 0.0 && nsteps >= 2 * kGraphSteps && !c->g.slab) {
        const int phase = c->aa ? (int)(c->steps_done & 1) : c->cur;
        if (phase != 0) {
            int rc = advance();
            if (rc != CLBM_OK) return rc;
            ++t;
        }
        int rc = ensure_graph(c);
        if (rc != CLBM_OK) return rc;
        for (; t + kGraphSteps <= nsteps; t += kGraphSteps) {
            cudaError_t e = cudaGraphLaunch(c->graph, c->stream);
            if (e != cudaSuccess) return cuda_fail(e, "clbm_step: graph launch");
            c->steps_done += kGraphSteps;
        }
    }
    for (; t < nsteps; ++t) {
        int rc = advance();
        if (rc != CLBM_OK) return rc;
    }
    return CLBM_OK;
}

int clbm_get_macros(clbm_ctx *c, float *rho, float *u) {
    if (!c) return fail(CLBM_ERR_ARG, "clbm_get_macros: null context");
    if (!rho && !u) return CLBM_OK;
    cudaError_t e = c->q == 27 ? launch_macros27(c->p.storage, launch_of(c), c->buf[c->cur], force_now(c), rho, u, c->n)
                               : launch_macros(c->p.storage, launch_of(c), c->buf[c->cur], force_now(c), rho, u, c->n);
    if (e != cudaSuccess) return cuda_fail(e, "clbm_get_macros");
    return CLBM_OK;
}

int clbm_get_populations(clbm_ctx *c, float *f, int deviation) {
    if (!c || !f) return fail(CLBM_ERR_ARG, "clbm_get_populations: null pointer");
    cudaError_t e = c->q == 27 ? launch_gather27(c->p.storage, launch_of(c), c->buf[c->cur], f, c->n, deviation)
                               : launch_gather(c->p.storage, launch_of(c), c->buf[c->cur], f, c->n, deviation);
    if (e != cudaSuccess) return cuda_fail(e, "clbm_get_populations");
    return CLBM_OK;
}

int clbm_set_populations(clbm_ctx *c, const float *f, int deviation) {
    if (!c || !f) return fail(CLBM_ERR_ARG, "clbm_set_populations: null pointer");
    if (c->slab_pending) return fail(CLBM_ERR_STATE, "clbm_set_populations: a split slab step is pending");
    c->steps_done = 0;  // before launch_of: the in-place pattern restarts in natural order
    cudaError_t e = c->q == 27 ? launch_scatter27(c->p.storage, launch_of(c), c->buf[c->cur], f, c->n, deviation)
                               : launch_scatter(c->p.storage, launch_of(c), c->buf[c->cur], f, c->n, deviation);
    if (e != cudaSuccess) return cuda_fail(e, "clbm_set_populations");
    return CLBM_OK;
}

int clbm_reduce_moments(clbm_ctx *c, double *out) {
    if (!c || !out) return fail(CLBM_ERR_ARG, "clbm_reduce_moments: null pointer");
    cudaError_t e = c->q == 27 ? launch_moments27(c->p.storage, launch_of(c), c->buf[c->cur], force_now(c),
                                                  (long long *)c->d_partials, kReduceBlocks, out)
                               : launch_reduce_moments(c->p.storage, launch_of(c), c->buf[c->cur], force_now(c),
                                                       (long long *)c->d_partials, kReduceBlocks, out);
    if (e != cudaSuccess) return cuda_fail(e, "clbm_reduce_moments");
    return CLBM_OK;
}

int clbm_reduce_pair(clbm_ctx *c, const float *a, const float *b, int64_t n, double *out) {
    if (!c || !out || n < 0 || (!a && n > 0)) return fail(CLBM_ERR_ARG, "clbm_reduce_pair: bad argument");
    cudaError_t e = launch_reduce_pair(a, b, n, c->d_partials, kReduceBlocks, out, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "clbm_reduce_pair");
    return CLBM_OK;
}

int clbm_check(clbm_ctx *c, int clear) {
    if (!c) return fail(CLBM_ERR_ARG, "clbm_check: null context");
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
#ifdef CLBM_BOUNDS_CHECK
    BoundsRecord rec = {0ull, 0ull};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&rec, c->g.bc, sizeof(rec), cudaMemcpyDeviceToHost, c->stream);
#endif
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "clbm_check");
    if (clear) {
        e = cudaMemsetAsync(c->d_flag, 0, 128, c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "clbm_check");
    }
#ifdef CLBM_BOUNDS_CHECK
    if (rec.count) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "clbm_check: %llu out-of-range indices; the first: kind %llu, index %llu",
                      rec.count, rec.first >> 56, rec.first & 0x00ffffffffffffffull);
        return fail(CLBM_ERR_BOUNDS, msg);
    }
#endif
    if (h & 2)
        return fail(CLBM_ERR_TIMEOUT, "clbm_check: a staged step's bulk copy did not complete; the state is invalid");
    if (h) return fail(CLBM_ERR_UNSTABLE, "clbm_check: a node's density left (0.1, 1.9) or became non-finite");
    return CLBM_OK;
}

int clbm_export_state(clbm_ctx *c, void *dst) {
    if (!c || !dst) return fail(CLBM_ERR_ARG, "clbm_export_state: null pointer");
    const size_t bytes = state_bytes(c);
    cudaError_t e = cudaMemcpyAsync(dst, c->buf[c->cur], bytes, cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "clbm_export_state");
    return CLBM_OK;
}

int clbm_import_state(clbm_ctx *c, const void *src, int64_t set_steps) {
    if (!c || !src) return fail(CLBM_ERR_ARG, "clbm_import_state: null pointer");
    if (c->slab_pending) return fail(CLBM_ERR_STATE, "clbm_import_state: a split slab step is pending");
    const size_t bytes = state_bytes(c);
    cudaError_t e = cudaMemcpyAsync(c->buf[c->cur], src, bytes, cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "clbm_import_state");
    if (set_steps >= 0) c->steps_done = set_steps;
    return CLBM_OK;
}

int clbm_save_state(clbm_ctx *c, void *host, size_t *bytes) {
    if (!c || !bytes) return fail(CLBM_ERR_ARG, "clbm_save_state: null pointer");
    const size_t raw = state_bytes(c);
    const size_t need = sizeof(StateHeader) + raw;
    if (!host) {
        *bytes = need;
        return CLBM_OK;
    }
    if (*bytes < need) return fail(CLBM_ERR_ARG, "clbm_save_state: buffer too small");
    StateHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, "CLBMLBM", 8);
    h.version = 2;
    h.nx = c->g.nx; h.ny = c->g.ny; h.nz = c->g.nz;
    h.walls = (int32_t)c->g.walls;
    h.storage = c->p.storage;
    h.q = c->q;
    h.pattern = c->aa ? CLBM_PATTERN_AA : CLBM_PATTERN_AB;
    h.stride = c->g.stride;
    h.steps_done = c->steps_done;
    h.bytes = (int64_t)raw;
    std::memcpy(host, &h, sizeof(h));
    cudaError_t e = cudaMemcpyAsync((char *)host + sizeof(h), c->buf[c->cur], raw, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "clbm_save_state");
    *bytes = need;
    return CLBM_OK;
}

int clbm_load_state(clbm_ctx *c, const void *host, size_t bytes) {
    if (!c || !host) return fail(CLBM_ERR_ARG, "clbm_load_state: null pointer");
    if (bytes < sizeof(StateHeader)) return fail(CLBM_ERR_ARG, "clbm_load_state: buffer too small");
    if (c->slab_pending) return fail(CLBM_ERR_STATE, "clbm_load_state: a split slab step is pending");
    StateHeader h;
    std::memcpy(&h, host, sizeof(h));
    const size_t raw = state_bytes(c);
    if (std::memcmp(h.magic, "CLBMLBM", 8) != 0 || h.version != 2)
        return fail(CLBM_ERR_ARG, "clbm_load_state: not a state buffer");
    if (h.nx != c->g.nx || h.ny != c->g.ny || h.nz != c->g.nz || h.walls != (int32_t)c->g.walls ||
        h.storage != c->p.storage || h.q != c->q || h.pattern != (c->aa ? CLBM_PATTERN_AA : CLBM_PATTERN_AB) ||
        h.stride != c->g.stride || h.bytes != (int64_t)raw ||
        bytes < sizeof(h) + raw)
        return fail(CLBM_ERR_ARG, "clbm_load_state: geometry, storage or size mismatch");
    cudaError_t e =
        cudaMemcpyAsync(c->buf[c->cur], (const char *)host + sizeof(h), raw, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "clbm_load_state");
    c->steps_done = h.steps_done;
    return CLBM_OK;
}

int clbm_step_raw(clbm_ctx *c, const void *src, void *dst) {
    if (!c || !src || !dst) return fail(CLBM_ERR_ARG, "clbm_step_raw: null pointer");
    if (c->q != 19) return fail(CLBM_ERR_ARG, "clbm_step_raw: D3Q19 only");
    if (c->aa) return fail(CLBM_ERR_ARG, "clbm_step_raw: A/B pattern only");
    if (c->model != CLBM_MODEL_CASCADED) return fail(CLBM_ERR_ARG, "clbm_step_raw: cascaded model only");
    if (c->gamma != 0.0) return fail(CLBM_ERR_STATE, "clbm_step_raw: needs a static force (decay 0)");
    const size_t bytes = state_bytes(c);
    if ((const char *)src < (const char *)dst + bytes && (const char *)dst < (const char *)src + bytes)
        return fail(CLBM_ERR_ARG, "clbm_step_raw: src and dst overlap");
    // a z-slab: every plane through the halo map, dst's send planes written (the caller exchanges them)
    cudaError_t e = c->g.slab ? launch_step_slab(c->p.storage, launch_of(c), src, dst, c->rates, c->force, c->d_flag,
                                                 step_key(0), 0, 1, c->g.nz)
                              : launch_step(c->p.storage, step_launch_of(c), src, dst, c->rates, c->force, c->d_flag,
                                            step_key(0));
    if (e != cudaSuccess) return cuda_fail(e, "clbm_step_raw");
    return CLBM_OK;
}

int clbm_adjoint_seed(clbm_ctx *c, const void *state, const float *gu, float *lam, float *gF) {
    if (!c || !gu || !lam || !gF) return fail(CLBM_ERR_ARG, "clbm_adjoint_seed: null pointer");
    if (c->q != 19) return fail(CLBM_ERR_ARG, "clbm_adjoint_seed: D3Q19 only");
    if (c->aa) return fail(CLBM_ERR_ARG, "clbm_adjoint_seed: A/B pattern only");
    if (c->model != CLBM_MODEL_CASCADED) return fail(CLBM_ERR_ARG, "clbm_adjoint_seed: cascaded model only");
    if (c->p.storage != CLBM_STORAGE_F32) return fail(CLBM_ERR_ARG, "clbm_adjoint_seed: FP32 storage only");
    if (c->gamma != 0.0) return fail(CLBM_ERR_STATE, "clbm_adjoint_seed: needs a static force (decay 0)");
    cudaError_t e = launch_adjoint_seed(c->p.storage, launch_of(c), state ? state : c->buf[c->cur], gu, lam, gF,
                                        c->force, c->n);
    if (e != cudaSuccess) return cuda_fail(e, "clbm_adjoint_seed");
    return CLBM_OK;
}

int clbm_adjoint_step(clbm_ctx *c, const void *state, const float *lam_next, float *lam, float *gF) {
    if (!c || !state || !lam_next || !lam || !gF) return fail(CLBM_ERR_ARG, "clbm_adjoint_step: null pointer");
    if (c->q != 19) return fail(CLBM_ERR_ARG, "clbm_adjoint_step: D3Q19 only");
    if (c->aa) return fail(CLBM_ERR_ARG, "clbm_adjoint_step: A/B pattern only");
    if (c->model != CLBM_MODEL_CASCADED) return fail(CLBM_ERR_ARG, "clbm_adjoint_step: cascaded model only");
    if (c->p.storage != CLBM_STORAGE_F32) return fail(CLBM_ERR_ARG, "clbm_adjoint_step: FP32 storage only");
    if (c->gamma != 0.0) return fail(CLBM_ERR_STATE, "clbm_adjoint_step: needs a static force (decay 0)");
    if (lam == lam_next) return fail(CLBM_ERR_ARG, "clbm_adjoint_step: lam aliases lam_next");
    cudaError_t e =
        launch_adjoint_step(c->p.storage, launch_of(c), state, lam_next, lam, gF, c->rates, c->force, c->n);
    if (e != cudaSuccess) return cuda_fail(e, "clbm_adjoint_step");
    return CLBM_OK;
}

int clbm_adjoint_segment(clbm_ctx *c, const void *ckpt, void *tape, int64_t k, float *lam, float *lam_tmp,
                         float *gF) {
    if (!c || !ckpt || !lam || !lam_tmp || !gF || k < 1 || (k > 1 && !tape) || lam == lam_tmp)
        return fail(CLBM_ERR_ARG, "clbm_adjoint_segment: bad argument");
    if (c->q != 19) return fail(CLBM_ERR_ARG, "clbm_adjoint_segment: D3Q19 only");
    if (c->g.slab)
        return fail(CLBM_ERR_STATE, "clbm_adjoint_segment: not for z-slabs (its recomputed steps need face exchanges)");
    if (c->aa) return fail(CLBM_ERR_ARG, "clbm_adjoint_segment: A/B pattern only");
    if (c->model != CLBM_MODEL_CASCADED) return fail(CLBM_ERR_ARG, "clbm_adjoint_segment: cascaded model only");
    Range range("clbm_adjoint_segment");
    if (c->p.storage != CLBM_STORAGE_F32) return fail(CLBM_ERR_ARG, "clbm_adjoint_segment: FP32 storage only");
    if (c->gamma != 0.0) return fail(CLBM_ERR_STATE, "clbm_adjoint_segment: needs a static force (decay 0)");
    const Launch L = launch_of(c);
    const size_t sb = (size_t)c->q * c->g.stride * c->elem;
    auto state = [&](int64_t j) -> const void * { return j == 0 ? ckpt : (const char *)tape + (j - 1) * sb; };
    cudaError_t e = cudaSuccess;
    for (int64_t j = 1; j < k && e == cudaSuccess; ++j)
        e = launch_step(c->p.storage, L, state(j - 1), (char *)tape + (j - 1) * sb, c->rates, c->force, c->d_flag,
                        step_key(0));
    float *in = lam, *out = lam_tmp;
    for (int64_t j = k - 1; j >= 0 && e == cudaSuccess; --j) {
        e = launch_adjoint_step(c->p.storage, L, state(j), in, out, gF, c->rates, c->force, c->n);
        float *t = in; in = out; out = t;
    }
    if (e == cudaSuccess && in != lam)
        e = cudaMemcpyAsync(lam, in, sizeof(float) * kQ * (size_t)c->n, cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "clbm_adjoint_segment");
    return CLBM_OK;
}

int clbm_run_host(clbm_ctx *c, const float *rho_h, const float *u_h, int64_t nsteps, float *rho_out,
                  float *u_out, double *moments_h) {
    if (!c) return fail(CLBM_ERR_ARG, "clbm_run_host: null context");
    Range range("clbm_run_host");
    if (nsteps < 0) return fail(CLBM_ERR_ARG, "clbm_run_host: nsteps < 0");
    if (c->g.slab) return fail(CLBM_ERR_STATE, "clbm_run_host: not for z-slabs (faces are exchanged between steps)");
    const Launch L = launch_of(c);
    cudaError_t e;
    if (!c->d_io) {
        const size_t io = (sizeof(float) * 4 * (size_t)c->n + 255) / 256 * 256;
        const size_t acc = sizeof(unsigned long long) * 2 * 4 * kDiagSlots;
        const size_t mom = sizeof(double) * 4 * kMomRing;
        const size_t bytes = io + mom + acc;
        void *p = nullptr;
        if ((e = cudaMalloc(&p, bytes)) != cudaSuccess) {
            c->d_io = nullptr;
            cudaGetLastError();
            return fail(CLBM_ERR_OOM, "clbm_run_host: cudaMalloc failed");
        }
        c->d_io = (float *)p;
        c->d_mom = (double *)((char *)p + io);
        c->d_acc = (unsigned long long *)((char *)p + io + mom);
        if ((e = cudaMemsetAsync(c->d_acc, 0, acc, c->stream)) != cudaSuccess)
            return cuda_fail(e, "clbm_run_host: clear accumulators");
    }
    float *d_rho = c->d_io, *d_u = c->d_io + c->n;
    const size_t nb = sizeof(float) * (size_t)c->n;
    // D3Q19: the host input travels in plane chunks on io_stream, and each chunk's
    // initialisation runs on the step stream once it has landed (a node's
    // initialisation reads only its own rho, u); the same for the read-out below.
    const bool chunked = c->q == 19;
    if (chunked && !c->io_stream) {
        cudaStream_t s = nullptr;
        if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "clbm_run_host: io stream");
        for (int k = 0; k < kIoChunks; ++k) {
            if ((e = cudaEventCreateWithFlags(&c->io_ev[k], cudaEventDisableTiming)) != cudaSuccess) {
                for (int j = 0; j < k; ++j) cudaEventDestroy(c->io_ev[j]);
                cudaStreamDestroy(s);
                return cuda_fail(e, "clbm_run_host: io events");
            }
        }
        c->io_stream = s;
    }
    const int64_t plane = (int64_t)c->g.nx * c->g.ny;
    const int nch = std::min(c->g.nz, kIoChunks);
    auto chunk = [&](int k, int64_t &z0, int64_t &z1) {
        z0 = (int64_t)c->g.nz * k / nch;
        z1 = (int64_t)c->g.nz * (k + 1) / nch;
    };
    int rc = CLBM_OK;
    const bool fused = c->q == 19 && !c->aa && c->model == CLBM_MODEL_CASCADED;
    // With per-step sums the steps are the fused kernel, which also steps a range
    // of planes. Then the first two steps run chunk by chunk as the input lands: a
    // node's step pulls exactly the slots its own initialisation scattered to, so
    // chunk k takes step 0 right after its initialisation. Step 1 of chunk k pulls
    // from step 0 of chunks k - 1, k and k + 1, so it follows step 0 of chunk
    // k + 1 (the two end chunks, neighbours across a periodic z, after the last).
    // The last step runs chunk by chunk too. A node's read-out pulls from the
    // neighbouring planes, so chunk k is read out and copied back once chunks
    // k - 1, k and k + 1 are stepped (the two end chunks after the last).
    const bool diag = fused && moments_h && nsteps > 0;
    const bool first_split = chunked && diag;
    const bool second_split = first_split && nsteps >= 3 && nch >= 3;
    const bool last_split = chunked && diag && nsteps > 1 && (rho_out || u_out);
    if (fused && moments_h && !c->copy_stream) {
        cudaStream_t cs = nullptr;
        cudaEvent_t e1 = nullptr, e2 = nullptr;
        if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&e1, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&e2, cudaEventDisableTiming)) != cudaSuccess) {
            if (cs) cudaStreamDestroy(cs);
            if (e1) cudaEventDestroy(e1);
            return cuda_fail(e, "clbm_run_host: copy stream");
        }
        c->copy_stream = cs;
        c->ev_step = e1;
        c->ev_copy = e2;
    }
    if (diag && (e = cudaMemsetAsync(c->d_acc, 0, sizeof(unsigned long long) * 2 * 4 * kDiagSlots, c->stream)) !=
                    cudaSuccess)
        return cuda_fail(e, "clbm_run_host: clear accumulators");
    const double add0 = (double)c->n;
    auto slot = [c](int64_t t) { return c->d_mom + 4 * (t % kMomRing); };
    // The fused step t of the job (or one plane range of it): it pulls buffer
    // cur0 ^ (t & 1), which holds state t, and the exact sums of that state go
    // to slot set t % 2. With drain_prev it first drains set (t - 1) % 2 into
    // the totals of state t - 1 (the first launch of a step whose predecessor
    // is complete).
    const int cur0 = c->cur;
    auto diag_step = [&](int64_t t, const Launch &Ls, bool drain_prev) {
        const int cur = cur0 ^ (int)(t & 1);
        DiagSums d;
        d.acc = c->d_acc + (t & 1) * 4 * kDiagSlots;
        d.acc_prev = t > 0 && drain_prev ? c->d_acc + ((t - 1) & 1) * 4 * kDiagSlots : nullptr;
        d.out_prev = t > 0 && drain_prev ? slot(t - 1) : nullptr;
        d.add0 = add0;
        return launch_step_diag(c->p.storage, Ls, c->buf[cur], c->buf[cur ^ 1], c->rates, force_at(c, t), c->d_flag,
                                d, step_key(t));
    };
    // chunk k's planes, with the state map of the current step count
    auto plane_chunk = [&](int k) {
        int64_t z0, z1;
        chunk(k, z0, z1);
        Launch Lk = launch_of(c);
        Lk.z0 = (int)z0;
        Lk.nplanes = (int)(z1 - z0);
        return Lk;
    };
    // Every kMomSync steps the step stream waits for the sum copies issued
    // kMomSync steps earlier, before their slots are reused.
    auto mom_sync = [&]() {
        cudaError_t r = cudaStreamWaitEvent(c->stream, c->ev_copy, 0);
        if (r == cudaSuccess) r = cudaEventRecord(c->ev_copy, c->copy_stream);
        return r;
    };
    // Chunk k's read-out of buffer b (force F), then its copies back on io_stream.
    auto read_out = [&](int k, const void *b, const ForceArgs &F) {
        const Launch Lk = plane_chunk(k);
        const int64_t off = (int64_t)Lk.z0 * plane;
        const size_t bytes = sizeof(float) * (size_t)((int64_t)Lk.nplanes * plane);
        cudaError_t r = launch_macros(c->p.storage, Lk, b, F, rho_out ? d_rho : nullptr, u_out ? d_u : nullptr, c->n);
        if (r == cudaSuccess) r = cudaEventRecord(c->io_ev[k], c->stream);
        if (r == cudaSuccess) r = cudaStreamWaitEvent(c->io_stream, c->io_ev[k], 0);
        if (r == cudaSuccess && rho_out)
            r = cudaMemcpyAsync(rho_out + off, d_rho + off, bytes, cudaMemcpyDeviceToHost, c->io_stream);
        for (int a = 0; a < 3 && u_out && r == cudaSuccess; ++a)
            r = cudaMemcpyAsync(u_out + a * c->n + off, d_u + a * c->n + off, bytes, cudaMemcpyDeviceToHost,
                                c->io_stream);
        return r;
    };
    if (first_split && (e = mom_sync()) != cudaSuccess) return cuda_fail(e, "clbm_run_host: copy sync");
    if (chunked) {
        if (c->slab_pending) return fail(CLBM_ERR_STATE, "clbm_run_host: a split slab step is pending");
        c->steps_done = 0;  // as clbm_init_equilibrium
        const ForceArgs F0 = force_at_zero(c);
        // d_io may still be read by the step stream (an earlier job's read-out)
        if ((e = cudaEventRecord(c->io_ev[0], c->stream)) == cudaSuccess)
            e = cudaStreamWaitEvent(c->io_stream, c->io_ev[0], 0);
        for (int k = 0; k < nch && e == cudaSuccess; ++k) {
            const Launch Lk = plane_chunk(k);
            const int64_t off = (int64_t)Lk.z0 * plane;
            const size_t bytes = sizeof(float) * (size_t)((int64_t)Lk.nplanes * plane);
            if (rho_h) e = cudaMemcpyAsync(d_rho + off, rho_h + off, bytes, cudaMemcpyHostToDevice, c->io_stream);
            for (int a = 0; a < 3 && u_h && e == cudaSuccess; ++a)
                e = cudaMemcpyAsync(d_u + a * c->n + off, u_h + a * c->n + off, bytes, cudaMemcpyHostToDevice,
                                    c->io_stream);
            if (e == cudaSuccess) e = cudaEventRecord(c->io_ev[k], c->io_stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->io_ev[k], 0);
            if (e == cudaSuccess)
                e = launch_init_eq(c->p.storage, Lk, c->buf[c->cur], rho_h ? d_rho : nullptr, u_h ? d_u : nullptr,
                                   c->n, F0);
            if (e == cudaSuccess && first_split) e = diag_step(0, Lk, false);
            if (e == cudaSuccess && second_split && k >= 2) e = diag_step(1, plane_chunk(k - 1), false);
        }
        if (e == cudaSuccess && second_split) {
            // step 0 is complete: its totals, then step 1 of the two end chunks
            e = launch_drain4(c->d_acc, slot(0), add0, c->stream);
            if (e == cudaSuccess) e = diag_step(1, plane_chunk(0), false);
            if (e == cudaSuccess) e = diag_step(1, plane_chunk(nch - 1), false);
        }
        if (e != cudaSuccess) return cuda_fail(e, "clbm_run_host: chunked copy and initialisation");
    } else {
        if (rho_h && (e = cudaMemcpyAsync(d_rho, rho_h, nb, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
            return cuda_fail(e, "clbm_run_host: copy rho");
        if (u_h && (e = cudaMemcpyAsync(d_u, u_h, 3 * nb, cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
            return cuda_fail(e, "clbm_run_host: copy u");
        rc = clbm_init_equilibrium(c, rho_h ? d_rho : nullptr, u_h ? d_u : nullptr);
        if (rc != CLBM_OK) return rc;
    }
    for (int64_t t = 0; t < nsteps && !fused; ++t) {
        // D3Q27 and the in-place pattern: the sums of state t, then a plain step
        if (moments_h) {
            if ((rc = clbm_reduce_moments(c, c->d_mom)) != CLBM_OK) return rc;
            e = cudaMemcpyAsync(moments_h + 4 * t, c->d_mom, sizeof(double) * 4, cudaMemcpyDeviceToHost, c->stream);
            if (e != cudaSuccess) return cuda_fail(e, "clbm_run_host: moments");
        }
        if ((rc = clbm_step(c, 1)) != CLBM_OK) return rc;
    }
    // The sums of step t - 1 land in ring slot (t - 1) % kMomRing during step t
    // and are copied back on copy_stream after it, beside the following
    // steps. (Writing them from the kernel straight into pinned host memory
    // made every step's kernel wait for that write: 9 us per step; a copy on
    // the step stream held each next step for 5 us.)
    for (int64_t t = 0; t < nsteps && fused; ++t) {
        if (moments_h) {
            if (t % kMomSync == 0 && !(t == 0 && first_split) && (e = mom_sync()) != cudaSuccess)
                return cuda_fail(e, "clbm_run_host: copy sync");
            e = cudaSuccess;
            if (t == nsteps - 1 && last_split) {
                // chunk by chunk; chunk k - 1 is read out (state t + 1, its force) once chunk k is stepped
                const ForceArgs F1 = force_at(c, c->steps_done + 1);
                for (int k = 0; k < nch && e == cudaSuccess; ++k) {
                    e = diag_step(t, plane_chunk(k), k == 0);
                    if (e == cudaSuccess && nch >= 3 && k >= 2) e = read_out(k - 1, c->buf[c->cur ^ 1], F1);
                }
                for (int k = 0; k < nch && e == cudaSuccess; ++k)
                    if (nch < 3 || k == 0 || k == nch - 1) e = read_out(k, c->buf[c->cur ^ 1], F1);
            } else if (!(t == 0 && first_split) && !(t == 1 && second_split)) {  // split steps ran as the input landed
                e = diag_step(t, L, true);
            }
            if (e == cudaSuccess && t == nsteps - 1)  // the last step's set
                e = launch_drain4(c->d_acc + (t & 1) * 4 * kDiagSlots, slot(t), add0, c->stream);
            if (e == cudaSuccess) e = cudaEventRecord(c->ev_step, c->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(c->copy_stream, c->ev_step, 0);
            if (e == cudaSuccess && t > 0)
                e = cudaMemcpyAsync(moments_h + 4 * (t - 1), slot(t - 1), sizeof(double) * 4, cudaMemcpyDeviceToHost,
                                    c->copy_stream);
            if (e == cudaSuccess && t == nsteps - 1)
                e = cudaMemcpyAsync(moments_h + 4 * t, slot(t), sizeof(double) * 4, cudaMemcpyDeviceToHost,
                                    c->copy_stream);
            if (e == cudaSuccess && t == nsteps - 1) {  // the step stream reuses slot 0 below
                e = cudaEventRecord(c->ev_copy, c->copy_stream);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, c->ev_copy, 0);
            }
        } else {
            e = step19(c, step_launch_of(c), c->buf[c->cur], c->buf[c->cur ^ 1], force_now(c),
                       step_key(c->steps_done));
        }
        if (e != cudaSuccess) return cuda_fail(e, "clbm_run_host: step");
        c->cur ^= 1;
        ++c->steps_done;
    }
    if (chunked && (rho_out || u_out)) {
        // each chunk's read-out, then its copies back on io_stream beside the next chunk's read-out
        const ForceArgs F1 = force_now(c);
        for (int k = 0; k < nch && !last_split && e == cudaSuccess; ++k) e = read_out(k, c->buf[c->cur], F1);
        if (e != cudaSuccess) return cuda_fail(e, "clbm_run_host: chunked read-out and copies back");
    } else {
        if ((rho_out || u_out) &&
            (rc = clbm_get_macros(c, rho_out ? d_rho : nullptr, u_out ? d_u : nullptr)) != CLBM_OK)
            return rc;
        if (rho_out && (e = cudaMemcpyAsync(rho_out, d_rho, nb, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
            return cuda_fail(e, "clbm_run_host: copy rho back");
        if (u_out && (e = cudaMemcpyAsync(u_out, d_u, 3 * nb, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
            return cuda_fail(e, "clbm_run_host: copy u back");
    }
    // the sums of the final state, on the step stream beside the copies back
    if (moments_h) {
        if ((rc = clbm_reduce_moments(c, c->d_mom)) != CLBM_OK) return rc;
        e = cudaMemcpyAsync(moments_h + 4 * nsteps, c->d_mom, sizeof(double) * 4, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "clbm_run_host: moments");
    }
    if (chunked && (rho_out || u_out)) {
        // the step stream ends after the copies (its synchronisation below covers them)
        if ((e = cudaEventRecord(c->io_ev[0], c->io_stream)) == cudaSuccess)
            e = cudaStreamWaitEvent(c->stream, c->io_ev[0], 0);
        if (e != cudaSuccess) return cuda_fail(e, "clbm_run_host: copies back");
    }
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(e, "clbm_run_host");
    if (moments_h)
        for (int64_t t = 0; t <= nsteps; ++t)
            if (!std::isfinite(moments_h[4 * t])) return fail(CLBM_ERR_UNSTABLE, "clbm_run_host: non-finite mass");
    return clbm_check(c, 0);
}

int clbm_slab_step(clbm_ctx *c, int part) {
    if (!c) return fail(CLBM_ERR_ARG, "clbm_slab_step: null context");
    if (!c->g.slab) return fail(CLBM_ERR_ARG, "clbm_slab_step: not a z-slab context");
    if (part != CLBM_SLAB_ALL && part != CLBM_SLAB_FACES && part != CLBM_SLAB_INTERIOR)
        return fail(CLBM_ERR_ARG, "clbm_slab_step: unknown part");
    if ((part == CLBM_SLAB_INTERIOR) != c->slab_pending)
        return fail(CLBM_ERR_STATE, part == CLBM_SLAB_INTERIOR
                                        ? "clbm_slab_step: CLBM_SLAB_INTERIOR needs CLBM_SLAB_FACES first"
                                        : "clbm_slab_step: a split step is pending (CLBM_SLAB_INTERIOR)");
    Range range("clbm_slab_step");
    const Launch L = launch_of(c);
    const ForceArgs F = force_now(c);
    const uint32_t key = step_key(c->steps_done);
    const int nz = c->g.nz;
    const void *src = c->buf[c->cur];
    void *dst = c->buf[c->cur ^ 1];
    cudaError_t e = cudaSuccess;
    if (part == CLBM_SLAB_ALL)
        e = launch_step_slab(c->p.storage, L, src, dst, c->rates, F, c->d_flag, key, 0, 1, nz);
    else if (part == CLBM_SLAB_FACES)  // planes 0 and nz - 1 (one plane if nz == 1)
        e = launch_step_slab(c->p.storage, L, src, dst, c->rates, F, c->d_flag, key, 0, nz > 1 ? nz - 1 : 1,
                             nz > 1 ? 2 : 1);
    else
        e = launch_step_slab(c->p.storage, L, src, dst, c->rates, F, c->d_flag, key, 1, 1, nz - 2);
    if (e != cudaSuccess) return cuda_fail(e, "clbm_slab_step");
    if (part == CLBM_SLAB_FACES) {
        c->slab_pending = true;
    } else {
        c->slab_pending = false;
        c->cur ^= 1;
        ++c->steps_done;
    }
    return CLBM_OK;
}

int clbm_slab_faces(clbm_ctx *c, void **send, void **recv, int64_t *face_bytes) {
    if (!c) return fail(CLBM_ERR_ARG, "clbm_slab_faces: null context");
    if (!c->g.slab) return fail(CLBM_ERR_ARG, "clbm_slab_faces: not a z-slab context");
    const size_t plane = (size_t)c->g.nx * c->g.ny;
    char *halo = (char *)c->buf[c->cur ^ (c->slab_pending ? 1 : 0)] + (size_t)c->q * c->g.stride * c->elem;
    if (recv) *recv = halo;
    if (send) *send = halo + 10 * plane * c->elem;
    if (face_bytes) *face_bytes = (int64_t)(5 * plane * c->elem);
    return CLBM_OK;
}

}  // extern "C"
