// batch.cu -- many independent lattices of uneven sizes and parameters stepped
// by one launch per time step.
//
// Every domain is a complete D3Q19 lattice (its own extents, walls, relaxation
// rates and uniform body force) with the per-node update of the single-lattice
// kernel (pull, Eqs. 5, 7, 8, 9 in deviation form; see d3q19.cuh). The
// domains' populations share two A/B allocations, domain after domain, each in
// the single-lattice layout. A host-built work list cuts every domain into
// tiles of T consecutive nodes in its linear index (T = threads per block),
// so every lane has a node whatever the domain's extents, a warp reads
// contiguous memory, and only a domain's last tile is partial. A grid of
// (SMs x resident blocks) walks the list with a stride: one launch covers all
// domains. Steps are replayed from a captured CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/clbm.h"
#include "kernels.cuh"

using namespace clbm;

namespace clbm {

// Does the pull of node (x, y, z) meet a wall (a node on a wall face)?
__device__ __forceinline__ bool on_wall_face(const Geom &g, int x, int y, int z) {
    return ((g.walls & 1u) && (x == 0 || x == g.nx - 1)) || ((g.walls & 2u) && (y == 0 || y == g.ny - 1)) ||
           ((g.walls & 4u) && (z == 0 || z == g.nz - 1));
}

// Load the 19 populations arriving at (x, y, z) (pull map of Eq. 8). With
// walls, a warp none of whose nodes lies on a wall face takes the periodic
// map, whose array indices are constants; only warps that touch a wall face
// evaluate the bounce-back substitutions. Returns the node's offset. (On the
// single-lattice step the two code paths measured 2 % slower than the
// bounce-back map alone; on the batched step, whose domains all have walls,
// 1 % faster.)
template <typename S, bool WALLS>
__device__ __forceinline__ uint32_t pull_load(const S *__restrict__ src, const Geom &g, int x, int y, int z,
                                              float (&h)[kQ]) {
    uint32_t off[kQ];
    int pop[kQ];
    if (WALLS && __any_sync(__activemask(), on_wall_face(g, x, y, z))) {
        pull_sources<true>(g, x, y, z, off, pop);
#pragma unroll
        for (int i = 0; i < kQ; ++i) h[i] = Codec<S>::load(src + (size_t)pop[i] * g.stride + off[i]);
    } else {
        pull_sources<false>(g, x, y, z, off, pop);
#pragma unroll
        for (int i = 0; i < kQ; ++i) h[i] = Codec<S>::load(src + (size_t)i * g.stride + off[i]);
    }
    return off[0];
}

struct DomainDesc {
    Geom g;
    Rates r;
    float fx, fy, fz;
    float inv_nx, inv_ny;  // 1/nx, 1/ny (FP32) for the tile coordinate decode
    int64_t offset;        // element offset of the domain's 19 x stride block in A and in B
};

// SMEM: the domain table is staged in shared memory once per launch (the
// usual case); otherwise it is read through the read-only cache. The next
// tile's entry is fetched while the current tile is processed.
template <typename S, bool SMEM>
__global__ void __launch_bounds__(512) k_batch_step(const S *__restrict__ A, S *__restrict__ B,
                                                    const DomainDesc *__restrict__ doms, int ndom,
                                                    const int4 *__restrict__ tiles, int ntiles,
                                                    int *__restrict__ flag) {
    extern __shared__ DomainDesc sdom[];
    if (SMEM) {
        for (int i = threadIdx.x; i < ndom; i += blockDim.x) sdom[i] = doms[i];
        __syncthreads();
    }
    int t = blockIdx.x;
    if (t >= ntiles) return;
    int4 tile = __ldg(tiles + t);  // (domain, x, y, z) of the tile's first node
    for (; t < ntiles; t += gridDim.x) {
        const int tn = t + gridDim.x;
        const int4 next = tn < ntiles ? __ldg(tiles + tn) : tile;
        const DomainDesc *D = SMEM ? sdom + tile.x : doms + tile.x;
        const Geom g = D->g;
        // node tile_start + threadIdx.x: carry x into y and y into z. The
        // quotients are below 2^17, so floor((v + 0.5) * (1/n)) in FP32 is exact.
        const int xt = tile.y + (int)threadIdx.x;
        const int cy = (int)(((float)xt + 0.5f) * D->inv_nx);
        const int yt = tile.z + cy;
        const int cz = (int)(((float)yt + 0.5f) * D->inv_ny);
        const int x = xt - cy * g.nx, y = yt - cz * g.ny, z = tile.w + cz;
        if (z < g.nz) {
            const S *src = A + D->offset;
            S *dst = B + D->offset;
            float h[kQ];
            const uint32_t self = pull_load<S, true>(src, g, x, y, z, h);
            const float drho = collide<sizeof(S) == 2>(h, D->fx, D->fy, D->fz, D->r);
            if (!(fabsf(drho) < 0.9f)) *flag = 1;
            store_node<S>(dst + self, g.stride, h, self, 0u);
        }
        tile = next;
    }
}

// The in-place (AA) pattern over the batch: every domain's one population
// array, even and odd step kinds as k_step_aa (step_kernels.cuh): the even
// kind reads a node's own slots and writes population i into the slot of
// ibar; the odd kind reads (ibar, x - e_i), or (i, x) across a wall, and writes
// population i to (i, x + e_i), or (ibar, x) across a wall. The same tiles,
// domain table and collision as k_batch_step, so the batch stores the bits of
// the A/B batch and of each domain stepped alone.
template <typename S, bool SMEM, bool ODD>
__global__ void __launch_bounds__(512) k_batch_step_aa(S *A, const DomainDesc *__restrict__ doms, int ndom,
                                                       const int4 *__restrict__ tiles, int ntiles,
                                                       int *__restrict__ flag) {
    extern __shared__ DomainDesc sdom[];
    if (SMEM) {
        for (int i = threadIdx.x; i < ndom; i += blockDim.x) sdom[i] = doms[i];
        __syncthreads();
    }
    int t = blockIdx.x;
    if (t >= ntiles) return;
    int4 tile = __ldg(tiles + t);
    for (; t < ntiles; t += gridDim.x) {
        const int tn = t + gridDim.x;
        const int4 next = tn < ntiles ? __ldg(tiles + tn) : tile;
        const DomainDesc *D = SMEM ? sdom + tile.x : doms + tile.x;
        const Geom g = D->g;
        const int xt = tile.y + (int)threadIdx.x;
        const int cy = (int)(((float)xt + 0.5f) * D->inv_nx);
        const int yt = tile.z + cy;
        const int cz = (int)(((float)yt + 0.5f) * D->inv_ny);
        const int x = xt - cy * g.nx, y = yt - cz * g.ny, z = tile.w + cz;
        if (z < g.nz) {
            S *f = A + D->offset;
            const uint32_t self = ((uint32_t)z * g.ny + y) * g.nx + x;
            float h[kQ];
            if (ODD) {
                uint32_t off[kQ];
                int pop[kQ];
                pull_sources<true, true>(g, x, y, z, off, pop);
#pragma unroll
                for (int i = 0; i < kQ; ++i) h[i] = Codec<S>::load(f + CLBM_IDX(g, (size_t)pop[i] * g.stride + off[i]));
                const float drho = collide<sizeof(S) == 2>(h, D->fx, D->fy, D->fz, D->r);
                if (!(fabsf(drho) < 0.9f)) *flag = 1;
                // the push targets from coordinates the compiler must treat as new (as in k_step_aa)
                int xs = x, ys = y, zs = z;
                asm volatile("" : "+r"(xs), "+r"(ys), "+r"(zs) : "f"(h[0]), "f"(h[kQ - 1]));
                push_targets<true>(g, xs, ys, zs, off, pop);
                store_each<S, kQ>(h, self, 0u,
                                  [&](int i) { return f + CLBM_IDX(g, (size_t)pop[i] * g.stride + off[i]); });
            } else {
#pragma unroll
                for (int i = 0; i < kQ; ++i) h[i] = Codec<S>::load(f + CLBM_IDX(g, (size_t)i * g.stride + self));
                const float drho = collide<sizeof(S) == 2>(h, D->fx, D->fy, D->fz, D->r);
                if (!(fabsf(drho) < 0.9f)) *flag = 1;
                store_each<S, kQ>(h, self, 0u,
                                  [&](int i) { return f + CLBM_IDX(g, (size_t)opposite(i) * g.stride + self); });
            }
        }
        tile = next;
    }
}

constexpr int kSmemDomains = 512;  // domain tables up to this size are staged in shared memory

template <typename S>
static cudaError_t batch_launch_t(const void *A, void *B, const DomainDesc *doms, int ndom, const int4 *tiles,
                                  int ntiles, int grid, dim3 block, int *flag, cudaStream_t s) {
    if (ndom <= kSmemDomains)
        k_batch_step<S, true><<<grid, block, sizeof(DomainDesc) * ndom, s>>>((const S *)A, (S *)B, doms, ndom, tiles,
                                                                            ntiles, flag);
    else
        k_batch_step<S, false><<<grid, block, 0, s>>>((const S *)A, (S *)B, doms, ndom, tiles, ntiles, flag);
    return cudaGetLastError();
}

template <typename S>
static cudaError_t batch_launch_aa_t(void *A, const DomainDesc *doms, int ndom, const int4 *tiles, int ntiles,
                                     int grid, dim3 block, int *flag, cudaStream_t s, bool odd) {
    const size_t sm = ndom <= kSmemDomains ? sizeof(DomainDesc) * ndom : 0;
    if (ndom <= kSmemDomains) {
        if (odd) k_batch_step_aa<S, true, true><<<grid, block, sm, s>>>((S *)A, doms, ndom, tiles, ntiles, flag);
        else k_batch_step_aa<S, true, false><<<grid, block, sm, s>>>((S *)A, doms, ndom, tiles, ntiles, flag);
    } else {
        if (odd) k_batch_step_aa<S, false, true><<<grid, block, 0, s>>>((S *)A, doms, ndom, tiles, ntiles, flag);
        else k_batch_step_aa<S, false, false><<<grid, block, 0, s>>>((S *)A, doms, ndom, tiles, ntiles, flag);
    }
    return cudaGetLastError();
}

static cudaError_t batch_launch_aa(int storage, void *A, const DomainDesc *doms, int ndom, const int4 *tiles,
                                   int ntiles, int grid, dim3 block, int *flag, cudaStream_t s, bool odd) {
    switch (storage) {
        case 0: return batch_launch_aa_t<float>(A, doms, ndom, tiles, ntiles, grid, block, flag, s, odd);
        case 1: return batch_launch_aa_t<__half>(A, doms, ndom, tiles, ntiles, grid, block, flag, s, odd);
        default: return batch_launch_aa_t<__nv_bfloat16>(A, doms, ndom, tiles, ntiles, grid, block, flag, s, odd);
    }
}

static cudaError_t batch_launch(int storage, const void *A, void *B, const DomainDesc *doms, int ndom,
                                const int4 *tiles, int ntiles, int grid, dim3 block, int *flag, cudaStream_t s) {
    switch (storage) {
        case 0: return batch_launch_t<float>(A, B, doms, ndom, tiles, ntiles, grid, block, flag, s);
        case 1: return batch_launch_t<__half>(A, B, doms, ndom, tiles, ntiles, grid, block, flag, s);
        default: return batch_launch_t<__nv_bfloat16>(A, B, doms, ndom, tiles, ntiles, grid, block, flag, s);
    }
}

template <typename S>
static int occupancy_t(int threads, int ndom) {
    int per_sm = 0;
    cudaError_t e;
    if (ndom <= kSmemDomains)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_step<S, true>, threads,
                                                          sizeof(DomainDesc) * ndom);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_step<S, false>, threads, 0);
    return (e == cudaSuccess && per_sm > 0) ? per_sm : 1;
}

static int batch_occupancy(int storage, int threads, int ndom) {
    switch (storage) {
        case 0: return occupancy_t<float>(threads, ndom);
        case 1: return occupancy_t<__half>(threads, ndom);
        default: return occupancy_t<__nv_bfloat16>(threads, ndom);
    }
}

}  // namespace clbm

struct clbm_batch {
    std::vector<clbm_domain> host;
    std::vector<DomainDesc> descs;
    int ndom;
    int storage;
    size_t elem;
    int64_t total_nodes, total_elems;
    void *buf[2];
    int cur;
    cudaStream_t stream, capture_stream;
    DomainDesc *d_descs;
    int4 *d_tiles;
    int ntiles, tiles_cap, grid;
    dim3 block;
    int *d_flag;
    cudaGraphExec_t graph;
    int graph_steps;
    int64_t steps_done;
    bool aa;  // in-place pattern: one buffer (buf[1] == buf[0]), step kind by the parity of steps_done
};

namespace {

int bfail(int code, const std::string &msg) { return clbm::set_error(code, msg.c_str()); }

int bcuda(cudaError_t e, const char *where) {
    return bfail(CLBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

Launch domain_launch(const clbm_batch *b, int d) {
    const Geom &g = b->descs[d].g;
    Launch L;
    L.g = g;
    const int bx = g.nx >= 128 ? 128 : ((g.nx + 31) / 32) * 32;
    const int by = std::max(1, std::min(g.ny, 256 / bx));
    L.block = dim3(bx, by, 1);
    L.grid = dim3((g.nx + bx - 1) / bx, (g.ny + by - 1) / by, g.nz);
    L.stream = b->stream;
    L.packed = false;
    L.staged = false;  // the per-domain schedule runs the one-node kernels
    // state maps: A/B pull map; in place, natural slots after an even number of steps, the odd map after an odd
    L.map = b->aa ? ((b->steps_done & 1) ? 2 : 1) : 0;
    return L;
}

ForceArgs domain_force(const clbm_batch *b, int d) {
    ForceArgs F;
    F.mode = kForceUniform;
    F.fx = b->descs[d].fx; F.fy = b->descs[d].fy; F.fz = b->descs[d].fz;
    F.profile = nullptr;
    F.field = nullptr;
    F.n = (int64_t)b->descs[d].g.nx * b->descs[d].g.ny * b->descs[d].g.nz;
    F.scale = 1.0f;
    return F;
}

void *domain_ptr(const clbm_batch *b, int which, int d) {
    return (char *)b->buf[which] + (size_t)b->descs[d].offset * b->elem;
}

// Build and upload the work list for T threads per block: tiles of T
// consecutive linear nodes, domain after domain.
int build_tiles(clbm_batch *b, int T) {
    std::vector<int4> tiles;
    for (int d = 0; d < b->ndom; ++d) {
        const Geom &g = b->descs[d].g;
        const int64_t n = (int64_t)g.nx * g.ny * g.nz;
        for (int64_t s0 = 0; s0 < n; s0 += T) {
            const int x = (int)(s0 % g.nx);
            const int64_t r = s0 / g.nx;
            tiles.push_back(make_int4(d, x, (int)(r % g.ny), (int)(r / g.ny)));
        }
    }
    if (tiles.size() > (size_t)INT32_MAX) return bfail(CLBM_ERR_ARG, "clbm_batch: too many tiles");
    if ((int)tiles.size() > b->tiles_cap) {
        if (b->d_tiles) cudaFree(b->d_tiles);
        b->d_tiles = nullptr;
        cudaError_t e = cudaMalloc(&b->d_tiles, tiles.size() * sizeof(int4));
        if (e != cudaSuccess) {
            b->tiles_cap = 0;
            cudaGetLastError();
            return bfail(CLBM_ERR_OOM, "clbm_batch: cudaMalloc of the work list failed");
        }
        b->tiles_cap = (int)tiles.size();
    }
    cudaError_t e = cudaMemcpyAsync(b->d_tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                    b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(e, "clbm_batch: work list upload");
    b->ntiles = (int)tiles.size();
    b->block = dim3(T, 1, 1);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->grid = std::max(1, std::min(b->ntiles, std::max(1, sms) * batch_occupancy(b->storage, T, b->ndom)));
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return CLBM_OK;
}

// One step of every domain: A/B from buffer `from`; in place, the odd kind when
// `from` is 1 (the parity of the step).
cudaError_t launch_all(clbm_batch *b, cudaStream_t s, int from) {
    if (b->aa)
        return batch_launch_aa(b->storage, b->buf[0], b->d_descs, b->ndom, b->d_tiles, b->ntiles, b->grid, b->block,
                               b->d_flag, s, from == 1);
    return batch_launch(b->storage, b->buf[from], b->buf[from ^ 1], b->d_descs, b->ndom, b->d_tiles, b->ntiles,
                        b->grid, b->block, b->d_flag, s);
}

// Capture graph_steps steps starting from buffer 0 (in place: from an even
// step); graph_steps is even, so the replay ends there again.
int ensure_graph(clbm_batch *b) {
    if (b->graph) return CLBM_OK;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bcuda(e, "clbm_batch: begin capture");
    for (int k = 0; k < b->graph_steps && e == cudaSuccess; ++k) e = launch_all(b, b->capture_stream, k & 1);
    cudaError_t e2 = cudaStreamEndCapture(b->capture_stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        return bcuda(e, "clbm_batch: graph capture");
    }
    return CLBM_OK;
}

}  // namespace

extern "C" {

int clbm_batch_create(const clbm_domain *doms, int32_t ndomains, int32_t storage, void *stream, clbm_batch **out) {
    return clbm_batch_create_pattern(doms, ndomains, storage, CLBM_PATTERN_AB, stream, out);
}

int clbm_batch_create_pattern(const clbm_domain *doms, int32_t ndomains, int32_t storage, int32_t pattern,
                              void *stream, clbm_batch **out) {
    if (!doms || !out || ndomains < 1) return bfail(CLBM_ERR_ARG, "clbm_batch_create: bad argument");
    *out = nullptr;
    if (pattern != CLBM_PATTERN_AB && pattern != CLBM_PATTERN_AA)
        return bfail(CLBM_ERR_ARG, "clbm_batch_create: pattern must be CLBM_PATTERN_AB or CLBM_PATTERN_AA");
    if (storage < CLBM_STORAGE_F32 || storage > CLBM_STORAGE_BF16)
        return bfail(CLBM_ERR_ARG, "clbm_batch_create: storage must be f32, f16 or bf16 (round to nearest)");
    clbm_batch *b = new (std::nothrow) clbm_batch();
    if (!b) return bfail(CLBM_ERR_OOM, "clbm_batch_create: host allocation failed");
    b->ndom = ndomains;
    b->storage = storage;
    b->aa = pattern == CLBM_PATTERN_AA;
    b->elem = storage == CLBM_STORAGE_F32 ? 4 : 2;
    b->stream = (cudaStream_t)stream;
    b->graph_steps = 16;
    int64_t off = 0, nodes = 0;
    for (int d = 0; d < ndomains; ++d) {
        const clbm_domain &p = doms[d];
        const double s2 = 1.0 / (3.0 * p.nu + 0.5);
        auto ok = [](double s) { return std::isfinite(s) && s > 0.0 && s < 2.0; };
        const int64_t n = (int64_t)p.nx * p.ny * p.nz;
        if (p.nx < 1 || p.ny < 1 || p.nz < 1 || p.nx > 65535 || p.ny > 65535 || p.nz > 65535 ||
            n > ((int64_t)1 << 31) - 1 || (p.walls & ~7u) || !(std::isfinite(p.nu) && p.nu > 0.0) || !ok(s2) ||
            !ok(p.s2b) || !ok(p.s3) || !ok(p.s4) || !std::isfinite(p.fx) || !std::isfinite(p.fy) ||
            !std::isfinite(p.fz)) {
            delete b;
            return bfail(CLBM_ERR_ARG, "clbm_batch_create: invalid domain " + std::to_string(d));
        }
        DomainDesc D;
        std::memset(&D, 0, sizeof(D));
        D.g.nx = p.nx; D.g.ny = p.ny; D.g.nz = p.nz;
        D.g.walls = p.walls;
        D.g.stride = (n + 63) / 64 * 64;
#ifdef CLBM_BOUNDS_CHECK
        D.g.bc_limit = (uint64_t)kQ * D.g.stride;  // the domain's own arrays (violations redirected, not recorded)
#endif
        D.r.om2 = (float)(1.0 - s2);
        D.r.cb = (float)((p.s2b - s2) / 3.0);
        D.r.om3 = (float)(1.0 - p.s3);
        D.r.c3 = (float)((1.0 - 0.5 * p.s3) / 3.0);
        D.r.om4 = (float)(1.0 - p.s4);
        D.fx = (float)p.fx; D.fy = (float)p.fy; D.fz = (float)p.fz;
        D.inv_nx = 1.0f / (float)p.nx;
        D.inv_ny = 1.0f / (float)p.ny;
        D.offset = off;
        off += (int64_t)kQ * D.g.stride;
        nodes += n;
        b->descs.push_back(D);
        b->host.push_back(p);
    }
    b->total_nodes = nodes;
    b->total_elems = off;
    const size_t nbuf = b->aa ? 1 : 2;
    cudaError_t e = cudaMalloc(&b->buf[0], nbuf * (size_t)off * b->elem);
    if (e != cudaSuccess) {
        delete b;
        cudaGetLastError();
        return bfail(CLBM_ERR_OOM, "clbm_batch_create: cudaMalloc of the populations failed");
    }
    b->buf[1] = b->aa ? b->buf[0] : (char *)b->buf[0] + (size_t)off * b->elem;
    if ((e = cudaMalloc(&b->d_descs, sizeof(DomainDesc) * ndomains + 256)) != cudaSuccess) {
        cudaFree(b->buf[0]);
        delete b;
        cudaGetLastError();
        return bfail(CLBM_ERR_OOM, "clbm_batch_create: cudaMalloc failed");
    }
    b->d_flag = (int *)((char *)b->d_descs + sizeof(DomainDesc) * ndomains);
    b->d_flag = (int *)(((uintptr_t)b->d_flag + 15) & ~(uintptr_t)15);
    if ((e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        cudaFree(b->d_descs);
        cudaFree(b->buf[0]);
        delete b;
        return bcuda(e, "clbm_batch_create: stream");
    }
    e = cudaMemcpyAsync(b->d_descs, b->descs.data(), sizeof(DomainDesc) * ndomains, cudaMemcpyHostToDevice,
                        b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_flag, 0, sizeof(int), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->buf[0], 0, nbuf * (size_t)off * b->elem, b->stream);
    int rc = e == cudaSuccess ? build_tiles(b, 256) : bcuda(e, "clbm_batch_create");
    if (rc != CLBM_OK) {
        clbm_batch_destroy(b);
        return rc;
    }
    *out = b;
    return CLBM_OK;
}

int clbm_batch_destroy(clbm_batch *b) {
    if (!b) return CLBM_OK;
    cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    if (b->d_tiles) cudaFree(b->d_tiles);
    if (b->d_descs) cudaFree(b->d_descs);
    if (b->buf[0]) cudaFree(b->buf[0]);
    delete b;
    return CLBM_OK;
}

int clbm_batch_get_info(const clbm_batch *b, clbm_batch_info *info) {
    if (!b || !info) return bfail(CLBM_ERR_ARG, "clbm_batch_get_info: null pointer");
    info->ndomains = b->ndom;
    info->total_nodes = b->total_nodes;
    info->state_bytes = (int64_t)b->total_elems * (int64_t)b->elem;
    info->ntiles = b->ntiles;
    info->grid = b->grid;
    info->threads = (int32_t)b->block.x;
    info->graph_steps = b->graph_steps;
    info->steps_done = b->steps_done;
    info->pattern = b->aa ? CLBM_PATTERN_AA : CLBM_PATTERN_AB;
    info->buffers = b->aa ? 1 : 2;
    return CLBM_OK;
}

int clbm_batch_set_tile(clbm_batch *b, int32_t threads) {
    if (!b || threads < 32 || threads % 32 != 0 || threads > 512)
        return bfail(CLBM_ERR_ARG, "clbm_batch_set_tile: threads must be a multiple of 32 in [32, 512]");
    return build_tiles(b, threads);
}

int clbm_batch_autotune(clbm_batch *b, int32_t trial_steps, int32_t *threads_out) {
    if (!b || trial_steps < 1) return bfail(CLBM_ERR_ARG, "clbm_batch_autotune: bad argument");
    static const int cand[] = {64, 128, 192, 256, 384, 512};
    // in place, a trial step overwrites the state: keep a copy and put it back after the trials
    void *saved = nullptr;
    const size_t sbytes = (size_t)b->total_elems * b->elem;
    if (b->aa) {
        cudaError_t e = cudaMalloc(&saved, sbytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return bfail(CLBM_ERR_OOM, "clbm_batch_autotune: no room for the copy of an in-place state");
        }
        if ((e = cudaMemcpyAsync(saved, b->buf[0], sbytes, cudaMemcpyDeviceToDevice, b->stream)) != cudaSuccess) {
            cudaFree(saved);
            return bcuda(e, "clbm_batch_autotune: save");
        }
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int bt = 256;
    int rc = CLBM_OK;
    for (int T : cand) {
        if ((rc = build_tiles(b, T)) != CLBM_OK) break;
        // A/B trials read the current buffer and write the other one: the state is unchanged. In place they
        // are steps of alternating kind from the current parity on the saved state, restored afterwards.
        int ph = b->aa ? (int)(b->steps_done & 1) : b->cur;
        auto trial = [&]() {
            cudaError_t r = launch_all(b, b->stream, ph);
            if (b->aa) ph ^= 1;
            return r;
        };
        cudaError_t e = trial();
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
        for (int k = 0; k < trial_steps && e == cudaSuccess; ++k) e = trial();
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            rc = bcuda(e, "clbm_batch_autotune");
            break;
        }
        if (ms < best) {
            best = ms;
            bt = T;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (saved) {
        cudaError_t e = cudaMemcpyAsync(b->buf[0], saved, sbytes, cudaMemcpyDeviceToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        cudaFree(saved);
        if (e != cudaSuccess && rc == CLBM_OK) rc = bcuda(e, "clbm_batch_autotune: restore");
    }
    if (rc != CLBM_OK) return rc;
    if ((rc = build_tiles(b, bt)) != CLBM_OK) return rc;
    if (threads_out) *threads_out = bt;
    return CLBM_OK;
}

int clbm_batch_init_equilibrium(clbm_batch *b) {
    if (!b) return bfail(CLBM_ERR_ARG, "clbm_batch_init_equilibrium: null pointer");
    b->steps_done = 0;  // before domain_launch: the in-place pattern starts in natural order
    for (int d = 0; d < b->ndom; ++d) {
        cudaError_t e = launch_init_eq(b->storage, domain_launch(b, d), domain_ptr(b, b->cur, d), nullptr, nullptr,
                                       domain_force(b, d).n, domain_force(b, d));
        if (e != cudaSuccess) return bcuda(e, "clbm_batch_init_equilibrium");
    }
    b->steps_done = 0;
    return CLBM_OK;
}

int clbm_batch_step(clbm_batch *b, int64_t nsteps, int32_t mode) {
    if (!b || nsteps < 0 || mode < 0 || mode > 2) return bfail(CLBM_ERR_ARG, "clbm_batch_step: bad argument");
    Range range("clbm_batch_step");
    cudaError_t e = cudaSuccess;
    int64_t t = 0;
    // the phase of the next step: the buffer (A/B) or the parity of the step (in place)
    auto phase = [&]() { return b->aa ? (int)((b->steps_done + t) & 1) : b->cur; };
    if (mode == CLBM_BATCH_GRAPH && nsteps >= b->graph_steps) {
        int rc = ensure_graph(b);
        if (rc != CLBM_OK) return rc;
        if (phase() == 1) {  // the graph starts from phase 0
            if ((e = launch_all(b, b->stream, 1)) != cudaSuccess) return bcuda(e, "clbm_batch_step");
            if (!b->aa) b->cur = 0;
            ++t;
        }
        for (; t + b->graph_steps <= nsteps; t += b->graph_steps)
            if ((e = cudaGraphLaunch(b->graph, b->stream)) != cudaSuccess) return bcuda(e, "clbm_batch_step: graph");
    }
    for (; t < nsteps; ++t) {
        if (mode == CLBM_BATCH_PER_DOMAIN) {
            const bool odd = phase() == 1;
            for (int d = 0; d < b->ndom && e == cudaSuccess; ++d) {
                Rates r = b->descs[d].r;
                if (b->aa)
                    e = launch_step_aa(b->storage, domain_launch(b, d), domain_ptr(b, 0, d), r, domain_force(b, d),
                                       b->d_flag, 0u, odd);
                else
                    e = launch_step(b->storage, domain_launch(b, d), domain_ptr(b, b->cur, d),
                                    domain_ptr(b, b->cur ^ 1, d), r, domain_force(b, d), b->d_flag, 0u);
            }
        } else {
            e = launch_all(b, b->stream, phase());
        }
        if (e != cudaSuccess) return bcuda(e, "clbm_batch_step");
        if (!b->aa) b->cur ^= 1;
    }
    b->steps_done += nsteps;
    return CLBM_OK;
}

int clbm_batch_get_macros(clbm_batch *b, int32_t d, float *rho, float *u) {
    if (!b || d < 0 || d >= b->ndom) return bfail(CLBM_ERR_ARG, "clbm_batch_get_macros: bad domain");
    if (!rho && !u) return CLBM_OK;
    cudaError_t e = launch_macros(b->storage, domain_launch(b, d), domain_ptr(b, b->cur, d), domain_force(b, d),
                                  rho, u, domain_force(b, d).n);
    if (e != cudaSuccess) return bcuda(e, "clbm_batch_get_macros");
    return CLBM_OK;
}

int clbm_batch_get_populations(clbm_batch *b, int32_t d, float *f, int deviation) {
    if (!b || !f || d < 0 || d >= b->ndom) return bfail(CLBM_ERR_ARG, "clbm_batch_get_populations: bad argument");
    cudaError_t e =
        launch_gather(b->storage, domain_launch(b, d), domain_ptr(b, b->cur, d), f, domain_force(b, d).n, deviation);
    if (e != cudaSuccess) return bcuda(e, "clbm_batch_get_populations");
    return CLBM_OK;
}

int clbm_batch_set_populations(clbm_batch *b, int32_t d, const float *f, int deviation) {
    if (!b || !f || d < 0 || d >= b->ndom) return bfail(CLBM_ERR_ARG, "clbm_batch_set_populations: bad argument");
    cudaError_t e = launch_scatter(b->storage, domain_launch(b, d), domain_ptr(b, b->cur, d), f,
                                   domain_force(b, d).n, deviation);
    if (e != cudaSuccess) return bcuda(e, "clbm_batch_set_populations");
    return CLBM_OK;
}

int clbm_batch_check(clbm_batch *b, int clear) {
    if (!b) return bfail(CLBM_ERR_ARG, "clbm_batch_check: null pointer");
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, b->d_flag, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess && clear) e = cudaMemsetAsync(b->d_flag, 0, sizeof(int), b->stream);
    if (e != cudaSuccess) return bcuda(e, "clbm_batch_check");
    if (h) return bfail(CLBM_ERR_UNSTABLE, "clbm_batch_check: a node's density left (0.1, 1.9) or became non-finite");
    return CLBM_OK;
}

}  // extern "C"
