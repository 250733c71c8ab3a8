// step_tma.cuh -- the A/B step for 16-bit storage (D3Q19 and D3Q27) with the
// pulled rows staged in shared memory by bulk asynchronous copies
// (cp.async.bulk: the TMA unit), templated on the collision like k_step.
//
// Why: k_step with 16-bit storage is bound by instruction issue, not DRAM:
// a node's 19 loads each need 64-bit address arithmetic (pull offsets with
// periodic wrap), and each load holds a register until its data arrive, so
// the warps alternate between waiting and computing. Here the TMA unit moves
// whole rows into shared memory a tile ahead of the threads, which read
// their values from shared memory at three addresses (x - 1, x, x + 1) plus
// constant offsets, collide and store exactly as k_step does: the results
// are bit-identical, with a fifth fewer instructions per node. FP32 storage
// stays on k_step, which already runs at the DRAM bound.
//
// Tile: `rows` consecutive x-rows (y0 .. y0 + rows - 1) of one z-plane, at
// most a pitch of nodes (TmaShape). Under the pull map of Eq. 8, population
// i of the tile's nodes comes from the same rows shifted by (-e_iy, -e_iz),
// each read at x - e_ix. The y/z shift is applied when copying (one or two
// contiguous runs of rows per population, two where the shift wraps around a
// periodic face); the x shift, with its periodic wrap, when reading shared
// memory. Every source row of every population is copied once per step, so
// the DRAM traffic is the algorithmic 2 x Q values per node.
//
// Walls (halfway bounce-back): a source row beyond a wall face is not
// copied; the nodes that would pull from it, and the nodes at an x wall, read
// their own opposite population from global memory instead.
//
// Pipeline: a persistent grid; block b walks tiles b, b + gridDim.x, ... with
// a few shared buffers (TmaShape) and one mbarrier each. A warp arms a
// buffer's barrier with the tile's byte count and issues its copies (lane i:
// population i). Every warp waits on the barrier of its next tile, computes
// its nodes and counts itself done with the buffer; the last warp to finish
// refills the buffer with the tile as many tiles ahead as there are buffers.
// There is no block barrier in the loop, so warps drift apart by up to that
// many tiles instead of waiting for the slowest. Every wait is bounded (the
// context's bound, kWaitCycles by default); on expiry the block sets bit 1 of
// the flag (reported as CLBM_ERR_TIMEOUT), its warps leave the loop, and one
// thread waits, bounded by kWaitCycles, for the copies still in flight before
// the block ends, so no copy lands in shared memory the block no longer owns.
#pragma once

#include <atomic>
#include <numeric>

#include "d3q27.cuh"
#include "kernels.cuh"

namespace clbm {

// Launch shapes: threads per block, resident blocks per SM (registers and
// shared memory are sized for them), shared buffers per block (at most 7),
// and the tile pitch: the most nodes of a tile, and the element pitch of a
// population's rows in a buffer.
template <int THREADS, int BLOCKS, int STAGES, int PITCH, bool PAIRS = false>
struct TmaShape {
    static constexpr int threads = THREADS, blocks = BLOCKS, stages = STAGES, pitch = PITCH;
    static constexpr bool pairs = PAIRS;  // each thread collides two adjacent nodes at once (FP32x2)
};
// D3Q19: two blocks of 512 threads take two nodes each of a 1024-node tile; a
// buffer of 19 populations of 16-bit values is 38 KB.
using TmaShape19 = TmaShape<512, 2, 2, 1024>;
// D3Q19 with walls: the bounce-back reads need more than the 64 registers of
// that shape (it spills 8-28 bytes); three blocks of 256 threads at up to 85
// registers take three nodes each of a 768-node tile (FP16 y/z-walled 256^3:
// 56.8k against 52.9k MLUPS). Rows above 768 nodes, and a force field, whose
// rows do not fit three blocks' buffers, take TmaShape19.
using TmaShape19W = TmaShape<256, 3, 2, 768>;
// D3Q19, two adjacent nodes per thread collided together on the FP32x2
// instructions (collisions that provide the f2 form): twice the live values,
// so two blocks of 256 threads (up to 128 registers) take two pairs each of a
// 1024-node tile.
using TmaShape19P = TmaShape<256, 2, 2, 1024, true>;
constexpr long long kWaitCycles = 4000000000ll;  // default bound of one barrier wait, about 2 s at 2 GHz

// What a staged launch computes (a compile-time mode).
enum TileMode : int {
    kTilePull = 0,      // A/B step: population i's rows shifted by e_i (the pull of Eq. 8), results to slot i
    kTileSlab = 1,      // the same on a z-slab: rows across a halo face come from its receive planes
    kTileSlabSend = 2,  // ... over a slab's first / last plane, which also writes the send planes
    kTileAAEven = 3,    // in-place even step: the node's own slots, results to the opposite slots
    kTileAAOdd = 4,     // in-place odd step: the opposite slots' rows shifted by e_i, results pushed by e_i
};
template <int M>
constexpr bool tile_slab() { return M == kTileSlab || M == kTileSlabSend; }

struct TilePlan {
    int rows;       // x-rows per tile
    int tiles_y;    // tiles per z-plane
    int ntiles;     // tiles_y * the number of planes stepped
    int z0, zs;     // the planes stepped: z0, z0 + zs, ... (all planes: 0, 1)
    int dz, dy;     // a block's step of gridDim.x tiles as (planes, tiles) : gridDim.x = dz tiles_y + dy
    uint32_t rdiv;  // ceil(2^32 / nx): the row of tile node n is umulhi(n, rdiv), exact for n, nx <= 1024
    long long wait; // bound of a thread's wait for a tile's copies, in SM clock cycles
    int drop_tile;  // failure injection: this tile's barrier is armed but its copies are not issued (-1: none)
};

// D3Q27: the collision wants about 115 registers, so 256 threads per block
// take four nodes each of a 1024-node tile (0.60 of roofline at 256^3 FP16;
// 512 threads at 64 registers spilled 60-150 bytes and measured 0.51, 384
// threads at 80 registers 0.59, one block of 512 threads with 4 buffers 0.52).
using TmaShape27 = TmaShape<256, 2, 2, 1024>;

// Bytes of one buffer: Q x pitch stored values, then the force on the tile's
// nodes: for a field its three components (3 x pitch floats), for a z-profile
// the tile plane's three values.
template <typename S, int FM, int Q, typename SH>
__host__ __device__ constexpr size_t stage_bytes() {
    return (size_t)Q * SH::pitch * sizeof(S) +
           (FM == kForceField ? 3 * SH::pitch * sizeof(float) : (FM == kForceProfileZ ? 16 : 0));
}

// Shared memory of one block: the barriers, then the buffers.
template <typename S, int FM, int Q, typename SH>
constexpr size_t tile_smem_bytes() {
    return 128 + SH::stages * stage_bytes<S, FM, Q, SH>();
}

// Whether the resident blocks fit the 228 KB of shared memory of an SM (1 KB
// of each block's share is reserved).
template <typename S, int FM, int Q, typename SH>
constexpr bool tile_fits() {
    return SH::blocks * (tile_smem_bytes<S, FM, Q, SH>() + 1024) <= 228 * 1024;
}

// Whether the staged step applies, and its plan for a grid of `grid` blocks
// (0: eligibility only) and tile pitch tn. The copies need 16-byte aligned
// rows (nx x elem and stride x elem multiples of 16, src 16-byte aligned) and
// a row must fit a tile.
inline bool tile_plan(const Geom &g, size_t elem, const void *src, int grid, int tn, TilePlan &p, int z0 = 0,
                      int zs = 1, int nplanes = -1) {
    if (elem != 2) return false;  // FP32 steps stay on k_step, which already runs at the DRAM bound
    if (g.nx > tn || ((size_t)g.nx * elem) % 16 != 0 || ((size_t)g.stride * elem) % 16 != 0 ||
        ((uintptr_t)src & 15u) != 0)
        return false;
    const int64_t n = (int64_t)g.nx * g.ny * g.nz;
    if (n >= (int64_t(1) << 31)) return false;
    p.rows = g.ny < tn / g.nx ? g.ny : tn / g.nx;
    p.tiles_y = (g.ny + p.rows - 1) / p.rows;
    p.ntiles = p.tiles_y * (nplanes < 0 ? g.nz : nplanes);
    p.z0 = z0;
    p.zs = zs;
    p.dz = grid / p.tiles_y;
    p.dy = grid - p.dz * p.tiles_y;
    p.rdiv = 0xffffffffu / (uint32_t)g.nx + 1u;
    p.wait = kWaitCycles;
    p.drop_tile = -1;
    return true;
}

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Make the initialised barriers and the generic-proxy use of the buffers
// visible to the asynchronous proxy (the bulk copies).
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for the phase of `parity` to complete; false after about `bound` cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long bound) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > bound) return false;
    return true;
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// e_iy + 1 and e_iz + 1 of population i (in the order of Eq. A1 for D3Q19, of
// Eq. 1 for D3Q27) in two bits each.
template <int Q>
__host__ __device__ constexpr uint64_t pack_shift(int axis) {
    uint64_t t = 0;
    if (Q == 19) {
        for (int i = 0; i < kQ; ++i) t |= (uint64_t)((axis == 1 ? ey19(i) : ez19(i)) + 1) << (2 * i);
    } else {
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                for (int c = 0; c < 3; ++c)
                    t |= (uint64_t)((axis == 1 ? e_of(b) : e_of(c)) + 1) << (2 * q27_index(a, b, c));
    }
    return t;
}

// Arm `bar` with the tile's byte count and copy its source rows into the
// buffer `stage`: population i's rows land at element i * pitch, slot row r
// at r * nx; after the populations, the force: for a field, component c of
// the tile's own rows at float c * pitch (bulk copies), for a z-profile the
// plane's three values (plain shared stores). Called by all 32
// lanes of one warp; lane i < Q handles population i, lanes Q to Q + 2 the
// force components.
// With drop (failure injection, from the host) the barrier is armed with the
// tile's byte count but no copy is issued, so no wait on it can complete.
// Slab modes: the tiles cover the planes z0, z0 + zs, ... of a z-slab, and
// rows across a halo face come from that face's receive plane. In-place
// modes: the even step copies the tile's own rows of population i, the odd
// step the rows of the opposite population, shifted as the pull.
template <typename S, int FM, bool WALLS, int Q, typename SH, int MODE>
__device__ __forceinline__ void issue_tile(const S *src, const ForceArgs &F, const Geom &g, const TilePlan &p,
                                           int t, unsigned char *stage, uint64_t *bar, int lane, bool drop = false) {
    constexpr bool SLAB = tile_slab<MODE>();
    static_assert(MODE < kTileAAEven || Q == kQ, "in-place modes: D3Q19");
    const int zi = t / p.tiles_y;
    const int z = SLAB ? p.z0 + zi * p.zs : zi;
    const int y0 = (t - zi * p.tiles_y) * p.rows;
    const int rows = min(p.rows, g.ny - y0);
    int src_a = 0, slot_a = 0, n_a = 0, src_b = 0, slot_b = 0, n_b = 0, zs = 0;
    int halo = -1;  // z-slab: the halo plane the rows come from (across a halo face), else -1
    if (lane < Q) {
        constexpr uint64_t kEy = pack_shift<Q>(1), kEz = pack_shift<Q>(2);
        const int ey = MODE == kTileAAEven ? 0 : (int)((kEy >> (2 * lane)) & 3u) - 1;
        const int ez = MODE == kTileAAEven ? 0 : (int)((kEz >> (2 * lane)) & 3u) - 1;
        const bool wy = WALLS && (g.walls & 2u), wz = WALLS && (g.walls & 4u);
        zs = z - ez;
        bool plane = true;
        if (zs < 0 || zs >= g.nz) {
            if (SLAB && zs < 0 && (g.slab & 1u)) halo = zface_index(lane);          // the lower neighbour's face
            else if (SLAB && zs >= g.nz && (g.slab & 2u)) halo = 5 + zface_index(lane);  // the upper one's
            else if (wz) plane = false;         // beyond a z wall: bounce-back, read from global
            else zs = zs < 0 ? zs + g.nz : zs - g.nz;
        }
        if (plane) {
            const int start = y0 - ey;
            if (start < 0) {                    // first slot row from row ny - 1 (periodic) or none (wall)
                if (!wy) { src_a = g.ny - 1; slot_a = 0; n_a = 1; }
                src_b = 0; slot_b = 1; n_b = rows - 1;
            } else if (start + rows > g.ny) {   // last slot row from row 0 (periodic) or none (wall)
                src_a = start; slot_a = 0; n_a = g.ny - start;
                if (!wy) { src_b = 0; slot_b = g.ny - start; n_b = rows - (g.ny - start); }
            } else {
                src_a = start; slot_a = 0; n_a = rows;
            }
        }
    }
    const bool force_lane = FM == kForceField && lane >= Q && lane < Q + 3;
    const uint32_t row_bytes = (uint32_t)g.nx * (uint32_t)sizeof(S);
    const uint32_t bytes = force_lane ? (uint32_t)rows * (uint32_t)g.nx * 4u : (uint32_t)(n_a + n_b) * row_bytes;
    const uint32_t total = __reduce_add_sync(0xffffffffu, bytes);
    if (FM == kForceProfileZ && lane >= Q && lane < Q + 3) {
        // the plane's force: a plain shared store, published to the waiting warps by the arrive below
        float *fdst = reinterpret_cast<float *>(stage + (size_t)Q * SH::pitch * sizeof(S));
        fdst[lane - Q] = __ldg(F.profile + (size_t)(lane - Q) * g.nz + z);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive_expect_tx(bar, total);
    __syncwarp();
    if (drop) return;
    if (lane < Q) {
        const int slot = MODE == kTileAAOdd ? opposite(lane) : lane;  // the population array the rows come from
        const size_t pop = SLAB && halo >= 0 ? (size_t)kQ * g.stride + (size_t)halo * g.ny * g.nx
                                             : (size_t)slot * g.stride + (size_t)zs * g.ny * g.nx;
        S *dst = reinterpret_cast<S *>(stage) + lane * SH::pitch;
        if (n_a > 0) {
            size_t from = pop + (size_t)src_a * g.nx, to = (size_t)slot_a * g.nx;
            if (!CLBM_RANGE_OK(g, from, (size_t)n_a * g.nx, g.bc_limit) ||
                !CLBM_RANGE_OK(g, to, (size_t)n_a * g.nx, SH::pitch))
                from = to = 0;  // bounds-checked build: recorded, the copy redirected in bounds
            bulk_copy_g2s(dst + to, src + from, (uint32_t)n_a * row_bytes, bar);
        }
        if (n_b > 0) {
            size_t from = pop + (size_t)src_b * g.nx, to = (size_t)slot_b * g.nx;
            if (!CLBM_RANGE_OK(g, from, (size_t)n_b * g.nx, g.bc_limit) ||
                !CLBM_RANGE_OK(g, to, (size_t)n_b * g.nx, SH::pitch))
                from = to = 0;
            bulk_copy_g2s(dst + to, src + from, (uint32_t)n_b * row_bytes, bar);
        }
    } else if (force_lane) {
        const int c = lane - Q;
        float *dst = reinterpret_cast<float *>(stage + (size_t)Q * SH::pitch * sizeof(S)) + c * SH::pitch;
        size_t from = (size_t)c * F.n + ((size_t)z * g.ny + y0) * g.nx;
        if (!CLBM_RANGE_OK(g, from, (size_t)rows * g.nx, 3 * (size_t)F.n)) from = 0;
        bulk_copy_g2s(dst, F.field + from, bytes, bar);
    }
}

// Collide and store the nodes of the tile of rows y0 .. y0 + rows - 1 of
// plane z from its staged rows.
template <typename C, typename S, int FM, bool WALLS, int Q, typename SH, typename R>
__device__ __forceinline__ void compute_tile(const S *__restrict__ src, S *__restrict__ dst, const Geom &g,
                                             const R &r, const ForceArgs &F, int *flag, uint32_t key,
                                             const TilePlan &p, int z, int y0, const unsigned char *buf,
                                             float tfx, float tfy, float tfz) {
    const S *stage = reinterpret_cast<const S *>(buf);
    const float *fst = reinterpret_cast<const float *>(buf + (size_t)Q * SH::pitch * sizeof(S));
    constexpr int TN = SH::pitch;
    const int rows = min(p.rows, g.ny - y0);
    const uint32_t nx = (uint32_t)g.nx;
    const uint32_t tile = (uint32_t)rows * nx;
    const uint32_t base = ((uint32_t)z * (uint32_t)g.ny + (uint32_t)y0) * nx;
    for (uint32_t n = threadIdx.x; n < tile; n += SH::threads) {
        const uint32_t rr = __umulhi(n, p.rdiv);
        const uint32_t x = n - rr * nx;
        const uint32_t self = base + n;
        // slots of x - 1 and x + 1 in the node's staged row, periodic in x
        const uint32_t sm = x == 0 ? n + nx - 1u : n - 1u;
        const uint32_t sp = x == nx - 1u ? n + 1u - nx : n + 1u;
        bool xl = false, xh = false, yl = false, yh = false, zl = false, zh = false, any = false;
        if (WALLS) {
            const int y = y0 + (int)rr;
            const bool wx = g.walls & 1u, wy = g.walls & 2u, wz = g.walls & 4u;
            xl = wx && x == 0; xh = wx && x == nx - 1u;
            yl = wy && y == 0; yh = wy && y == g.ny - 1;
            zl = wz && z == 0; zh = wz && z == g.nz - 1;
            // nodes next to a wall are few: the warps without one skip the bounce-back reads
            any = __any_sync(__activemask(), xl || xh || yl || yh || zl || zh);
        }
        float fx = tfx, fy = tfy, fz = tfz;
        if (FM == kForceField) {  // the staged field, scaled as force_at does
            fx = fst[n] * F.scale;
            fy = fst[TN + n] * F.scale;
            fz = fst[2 * TN + n] * F.scale;
        } else if (FM == kForceProfileZ) {
            fx = fst[0] * F.scale;
            fy = fst[1] * F.scale;
            fz = fst[2] * F.scale;
        }
        if constexpr (Q == 19) {
            float h[kQ];
#pragma unroll
            for (int i = 0; i < kQ; ++i) {
                const uint32_t j = ex19(i) > 0 ? sm : (ex19(i) < 0 ? sp : n);
                h[i] = Codec<S>::load_plain(stage + i * TN + CLBM_SIDX(g, j, tile));
            }
            if (WALLS && any) {
                const bool bb[kQ] = {false,
                                     xl, xh, yl, yh, zl, zh,
                                     xl || yl, xh || yl, xl || yh, xh || yh,
                                     xl || zl, xh || zl, xl || zh, xh || zh,
                                     yl || zl, yh || zl, yl || zh, yh || zh};
#pragma unroll
                for (int i = 1; i < kQ; ++i)
                    if (bb[i]) h[i] = Codec<S>::load(src + CLBM_IDX(g, (size_t)opposite(i) * g.stride + self));
            }
            const float drho = C::template run<sizeof(S) == 2>(h, fx, fy, fz, r);
            if (!(fabsf(drho) < 0.9f)) atomicOr(flag, 1);
            store_node<S>(dst + CLBM_SLOTS(g, self, (kQ - 1) * g.stride), g.stride, h, self, key);
        } else {  // D3Q27, the cube by velocity code (0: e = 0, 1: +1, 2: -1)
            float h[3][3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const uint32_t j = a == 1 ? sm : (a == 2 ? sp : n);
                        h[a][b][c] = Codec<S>::load_plain(stage + q27_index(a, b, c) * TN + CLBM_SIDX(g, j, tile));
                    }
            if (WALLS && any) {
                const bool bx[3] = {false, xl, xh}, by[3] = {false, yl, yh}, bz[3] = {false, zl, zh};
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b)
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            if (bx[a] || by[b] || bz[c]) {
                                const int o = q27_index(a ? 3 - a : 0, b ? 3 - b : 0, c ? 3 - c : 0);
                                h[a][b][c] = Codec<S>::load(src + CLBM_IDX(g, (size_t)o * g.stride + self));
                            }
            }
            const float drho = C::template run<sizeof(S) == 2>(h, fx, fy, fz, r);
            if (!(fabsf(drho) < 0.9f)) atomicOr(flag, 1);
            float f[kQ27];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b)
#pragma unroll
                    for (int c = 0; c < 3; ++c) f[q27_index(a, b, c)] = h[a][b][c];
            store_node<S, kQ27>(dst + CLBM_SLOTS(g, self, (kQ27 - 1) * g.stride), g.stride, f, self, key);
        }
    }
}

// Element o of population array `slot` of the 16-bit state f: the array's
// base first, then a 32-bit offset (bounds-checked builds check the index).
__device__ __forceinline__ unsigned short *pop_elem(unsigned short *f, const Geom &g, int slot, uint32_t o) {
#ifdef CLBM_BOUNDS_CHECK
    return f + CLBM_IDX(g, (size_t)slot * g.stride + o);
#else
    return (f + (size_t)slot * g.stride) + o;
#endif
}

// Stores of the in-place odd step for the node pair x, x + 1 (x even) of row
// y, plane z: population i of a node goes where the next even step reads it,
// (i, node + e_i) with periodic wrap, or (ibar, node) when node + e_i lies
// beyond a wall (Eq. 8 with halfway bounce-back). word(i) holds population i
// of both nodes, node x in the lower half. With e_x = 0 both targets are one
// aligned pair; otherwise they straddle a pair boundary and take two 16-bit
// stores.
template <typename S, bool WALLS, typename W>
__device__ __forceinline__ void push_pairs(S *f, const Geom &g, uint32_t x, uint32_t y, uint32_t z, uint32_t self,
                                           W word) {
    const uint32_t nx = (uint32_t)g.nx, ny = (uint32_t)g.ny, nz = (uint32_t)g.nz, plane = nx * ny;
    // steps to the next / previous row and plane, periodic
    const int32_t yp = y + 1u == ny ? -(int32_t)((ny - 1u) * nx) : (int32_t)nx;
    const int32_t ym = y == 0u ? (int32_t)((ny - 1u) * nx) : -(int32_t)nx;
    const int32_t zp = z + 1u == nz ? -(int32_t)((nz - 1u) * plane) : (int32_t)plane;
    const int32_t zm = z == 0u ? (int32_t)((nz - 1u) * plane) : -(int32_t)plane;
    const int32_t xm0 = x == 0u ? (int32_t)(nx - 1u) : -1;       // node x to x - 1
    const int32_t xp1 = x + 2u == nx ? -(int32_t)(nx - 1u) : 1;  // node x + 1 to x + 2
    bool xl0 = false, xh1 = false, yl = false, yh = false, zl = false, zh = false;
    if (WALLS) {  // leaving through a wall face: node x through x-, node x + 1 through x+
        const bool wx = g.walls & 1u, wy = g.walls & 2u, wz = g.walls & 4u;
        xl0 = wx && x == 0u;
        xh1 = wx && x + 2u == nx;
        yl = wy && y == 0u;
        yh = wy && y + 1u == ny;
        zl = wz && z == 0u;
        zh = wz && z + 1u == nz;
    }
    unsigned short *f16 = reinterpret_cast<unsigned short *>(f);
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const int ex = ex19(i), ey = ey19(i), ez = ez19(i);
        const uint32_t w = word(i);
        const int32_t dyz = (ey > 0 ? yp : ey < 0 ? ym : 0) + (ez > 0 ? zp : ez < 0 ? zm : 0);
        const bool byz = (ey > 0 && yh) || (ey < 0 && yl) || (ez > 0 && zh) || (ez < 0 && zl);
        const uint32_t o = (uint32_t)((int32_t)self + dyz);  // the pair's target in the shifted row
        if (ex == 0) {
            *reinterpret_cast<uint32_t *>(byz ? pop_elem(f16, g, opposite(i), self) : pop_elem(f16, g, i, o)) = w;
        } else {
            // targets relative to node x: e_x = +1: x + 1 and x + 2; e_x = -1: x - 1 and x
            const bool b0 = ex > 0 ? byz : (byz || xl0), b1 = ex > 0 ? (byz || xh1) : byz;
            const uint32_t o0 = o + (uint32_t)(ex > 0 ? 1 : xm0), o1 = o + (uint32_t)(ex > 0 ? 1 + xp1 : 0);
            *(b0 ? pop_elem(f16, g, opposite(i), self) : pop_elem(f16, g, i, o0)) = (unsigned short)(w & 0xffffu);
            *(b1 ? pop_elem(f16, g, opposite(i), self + 1u) : pop_elem(f16, g, i, o1)) = (unsigned short)(w >> 16);
        }
    }
}

// The D3Q19 tile two adjacent nodes at a time: nodes n and n + 1 (n even, so
// both in the same row: nx is even) are collided together in f2 lanes .x and
// .y. Populations with e_x = 0 take both staged values with one 32-bit shared
// load; each population's two results are converted by one pair conversion
// (the even node in the lower half) and stored with one 32-bit store. The
// collision of f2 rounds like the scalar 16-bit collision (f1), and the pair
// conversions like the single ones, so the stored bits equal compute_tile's.
// Slab modes: z walls only at faces that are not halo faces, and the dither
// hashes global pair indices; kTileSlabSend (a halo face's plane) also
// stores the outgoing pair words into the send planes. In-place modes (src
// and dst the one array): the even step reads the node's own slots and
// stores population i into slot ibar; the odd step bounces back from slot i
// and pushes population i to (i, x + e_i), or to (ibar, x) beyond a wall, as
// pair words where the two targets are adjacent (e_x = 0) and as two 16-bit
// stores otherwise.
template <typename C, typename S, int FM, bool WALLS, typename SH, int MODE, typename R>
__device__ __forceinline__ void compute_tile_pairs(const S *src, S *dst, const Geom &g, const R &r, const ForceArgs &F,
                                                   int *flag, uint32_t key, const TilePlan &p, int z, int y0,
                                                   const unsigned char *buf, float tfx, float tfy, float tfz) {
    constexpr bool SLAB = tile_slab<MODE>(), SEND = MODE == kTileSlabSend;
    const S *stage = reinterpret_cast<const S *>(buf);
    const float *fst = reinterpret_cast<const float *>(buf + (size_t)kQ * SH::pitch * sizeof(S));
    constexpr int TN = SH::pitch;
    const int rows = min(p.rows, g.ny - y0);
    const uint32_t nx = (uint32_t)g.nx;
    const uint32_t tile = (uint32_t)rows * nx;
    const uint32_t base = ((uint32_t)z * (uint32_t)g.ny + (uint32_t)y0) * nx;
    for (uint32_t n = 2u * threadIdx.x; n < tile; n += 2u * SH::threads) {
        const uint32_t rr = __umulhi(n, p.rdiv);
        const uint32_t x = n - rr * nx;  // even
        const uint32_t self = base + n;   // even: the pair's index is self / 2
        // staged slots of x - 1 for node n and of x + 2 for node n + 1, periodic in x
        const uint32_t sm0 = x == 0 ? n + nx - 1u : n - 1u;
        const uint32_t sp1 = x + 2u == nx ? n + 2u - nx : n + 2u;
        f2 h[kQ];
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            const S *row = stage + i * TN;
            if (ex19(i) == 0 || MODE == kTileAAEven) {
                // both slots n and n + 1 below tile: n below tile - 1
                const float2 v =
                    Codec<S>::unpack2(*reinterpret_cast<const uint32_t *>(row + CLBM_SIDX(g, n, tile - 1u)));
                h[i] = f2{v};
            } else if (ex19(i) > 0) {  // from x - 1
                h[i] = mk2(Codec<S>::load_plain(row + CLBM_SIDX(g, sm0, tile)),
                           Codec<S>::load_plain(row + CLBM_SIDX(g, n, tile)));
            } else {                   // from x + 1
                h[i] = mk2(Codec<S>::load_plain(row + CLBM_SIDX(g, n + 1u, tile)),
                           Codec<S>::load_plain(row + CLBM_SIDX(g, sp1, tile)));
            }
        }
        if (WALLS && MODE != kTileAAEven) {  // (the in-place even step reads only its own slots)
            const int y = y0 + (int)rr;
            const bool wx = g.walls & 1u, wy = g.walls & 2u, wz = g.walls & 4u;
            const bool yl = wy && y == 0, yh = wy && y == g.ny - 1;
            const bool zl = wz && z == 0 && !(SLAB && (g.slab & 1u));
            const bool zh = wz && z == g.nz - 1 && !(SLAB && (g.slab & 2u));
            const bool xl0 = wx && x == 0, xh1 = wx && x + 2u == nx;  // x wall of node n / node n + 1
            const bool any = __any_sync(__activemask(), xl0 || xh1 || yl || yh || zl || zh);
            if (any) {
                // node n (lane .x): no x+ wall unless nx == 1, impossible here (nx even)
                const bool bb0[kQ] = {false,
                                      xl0, false, yl, yh, zl, zh,
                                      xl0 || yl, yl, xl0 || yh, yh,
                                      xl0 || zl, zl, xl0 || zh, zh,
                                      yl || zl, yh || zl, yl || zh, yh || zh};
                // node n + 1 (lane .y): its x- neighbour is node n
                const bool bb1[kQ] = {false,
                                      false, xh1, yl, yh, zl, zh,
                                      yl, xh1 || yl, yh, xh1 || yh,
                                      zl, xh1 || zl, zh, xh1 || zh,
                                      yl || zl, yh || zl, yl || zh, yh || zh};
#pragma unroll
                for (int i = 1; i < kQ; ++i) {
                    // bounce-back: slot ibar of the node (A/B), slot i (in-place odd step)
                    const size_t b = (size_t)(MODE == kTileAAOdd ? i : opposite(i)) * g.stride + self;
                    if (bb0[i]) h[i].v.x = Codec<S>::load(src + CLBM_IDX(g, b));
                    if (bb1[i]) h[i].v.y = Codec<S>::load(src + CLBM_IDX(g, b + 1u));
                }
            }
        }
        f2 fx = mk2(tfx), fy = mk2(tfy), fz = mk2(tfz);
        if (FM == kForceField) {  // the staged field, scaled as force_at does
            const float2 a = *reinterpret_cast<const float2 *>(fst + n);
            const float2 b = *reinterpret_cast<const float2 *>(fst + TN + n);
            const float2 c = *reinterpret_cast<const float2 *>(fst + 2 * TN + n);
            fx = mk2(a.x * F.scale, a.y * F.scale);
            fy = mk2(b.x * F.scale, b.y * F.scale);
            fz = mk2(c.x * F.scale, c.y * F.scale);
        } else if (FM == kForceProfileZ) {
            fx = mk2(fst[0] * F.scale);
            fy = mk2(fst[1] * F.scale);
            fz = mk2(fst[2] * F.scale);
        }
        const f2 drho = C::template run<true>(h, fx, fy, fz, r);
        if (!(fabsf(drho.v.x) < 0.9f) || !(fabsf(drho.v.y) < 0.9f)) atomicOr(flag, 1);
        const uint32_t hb = Codec<S>::kStochastic ? pair_hash((SLAB ? self + g.node0 : self) >> 1, key) : 0u;
        auto word = [&](int i) -> uint32_t {  // population i of both nodes, the even node in the lower half
            if constexpr (Codec<S>::kStochastic)
                return Codec<S>::pair_sr(h[i].v.y, h[i].v.x, pop_bits(hb, i));
            else
                return Codec<S>::pair_rn(h[i].v.y, h[i].v.x);
        };
        if constexpr (MODE == kTileAAOdd) {
            push_pairs<S, WALLS>(dst, g, x, (uint32_t)(y0 + (int)rr), (uint32_t)z, self, word);
        } else if constexpr (MODE == kTileAAEven) {
            uint32_t *out = reinterpret_cast<uint32_t *>(dst + CLBM_SLOTS(g, self, (kQ - 1) * g.stride + 1u));
#pragma unroll
            for (int i = 0; i < kQ; ++i) out[(size_t)opposite(i) * (g.stride >> 1)] = word(i);
        } else if constexpr (!SEND) {
            uint32_t *out = reinterpret_cast<uint32_t *>(dst + CLBM_SLOTS(g, self, (kQ - 1) * g.stride + 1u));
#pragma unroll
            for (int i = 0; i < kQ; ++i) out[(size_t)i * (g.stride >> 1)] = word(i);
        } else {
            // the first / last plane also sends its outgoing face (send planes, see kSlabPlanes)
            uint32_t *out = reinterpret_cast<uint32_t *>(dst + CLBM_SLOTS(g, self, (kQ - 1) * g.stride + 1u));
            const uint32_t plane = nx * (uint32_t)g.ny, ps = self - (uint32_t)z * plane;
            const bool send_lo = (g.slab & 1u) && z == 0, send_hi = (g.slab & 2u) && z == g.nz - 1;
            const size_t send = (size_t)kQ * g.stride + ps;  // element offset of the node in send plane 0 (even)
#pragma unroll
            for (int i = 0; i < kQ; ++i) {
                const uint32_t w = word(i);
                out[(size_t)i * (g.stride >> 1)] = w;
                if (ez19(i) < 0 && send_lo)
                    *reinterpret_cast<uint32_t *>(dst + CLBM_IDX(g, send + (size_t)(10 + zface_index(i)) * plane)) = w;
                if (ez19(i) > 0 && send_hi)
                    *reinterpret_cast<uint32_t *>(dst + CLBM_IDX(g, send + (size_t)(15 + zface_index(i)) * plane)) = w;
            }
        }
    }
}

// MODE (TileMode): the A/B pull step, on a whole lattice or on a z-slab's
// planes z0, z0 + zs, ... (those two with the send-plane stores over its
// first and/or last plane), or one of the two in-place kinds (src == dst:
// every tile's copies and stores touch only its own nodes' slots).
template <typename C, typename S, int FM, bool WALLS, int Q, typename SH, int MODE, typename R>
__global__ void __launch_bounds__(SH::threads, SH::blocks)
    k_step_tma(const S *__restrict__ src, S *__restrict__ dst, Geom g, R r, ForceArgs F, int *__restrict__ flag,
               uint32_t key, TilePlan p) {
    constexpr bool SLAB = tile_slab<MODE>();
    static_assert(MODE == kTilePull || SH::pairs, "z-slabs and the in-place kinds take the node-pair tile");
    constexpr int kTmaStages = SH::stages;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);     // [stages]: copies of the buffer's tile arrived
    int *done = reinterpret_cast<int *>(smem + 64);         // [stages]: warps finished with the buffer's tile
    int *issued = reinterpret_cast<int *>(smem + 96);       // [stages]: tiles copied into the buffer so far
    volatile int *abort = reinterpret_cast<volatile int *>(smem + 124);
    unsigned char *buf = smem + 128;
    constexpr size_t SB = stage_bytes<S, FM, Q, SH>();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nwarps = blockDim.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kTmaStages; ++s) {
            mbar_init(&bar[s], 1);
            done[s] = 0;
            issued[s] = 0;
        }
        *abort = 0;
        fence_proxy_async();
    }
    __syncthreads();
    if (warp == 0)
        for (int k = 0; k < kTmaStages; ++k) {
            const int t = blockIdx.x + k * gridDim.x;
            if (t < p.ntiles) {
                const bool drop = t == p.drop_tile;
                issue_tile<S, FM, WALLS, Q, SH, MODE>(src, F, g, p, t, buf + k * SB, &bar[k], lane, drop);
                if (lane == 0 && !drop) issued[k] = 1;  // the drain waits only for copies actually issued
            }
        }
    // No block barrier inside the loop: each warp takes the tiles in order,
    // waiting only for their copies; the last warp to finish with a buffer
    // refills it with the tile kTmaStages ahead.
    int z = blockIdx.x / p.tiles_y, yt = blockIdx.x - z * p.tiles_y;  // tile t = z tiles_y + yt
    int k = 0;
    for (int t = blockIdx.x; t < p.ntiles; t += gridDim.x, ++k) {
        const int s = k % kTmaStages;
        float tfx = 0.0f, tfy = 0.0f, tfz = 0.0f;  // a uniform force (the others come staged)
        if (FM == kForceUniform) {
            tfx = F.fx * F.scale;
            tfy = F.fy * F.scale;
            tfz = F.fz * F.scale;
        }
        const bool ok = mbar_wait(&bar[s], (uint32_t)(k / kTmaStages) & 1u, p.wait);
        if (!ok || *abort) {
            if (!ok && lane == 0) {
                *abort = 1;
                atomicOr(flag, 2);
            }
            break;
        }
        // Only tiles with a node next to a wall take the wall code; the others run the periodic loop, which
        // the wall handling would otherwise slow on every tile (12-21 % for the node-pair loop).
        const int y0 = yt * p.rows;
        const int zp = SLAB ? p.z0 + z * p.zs : z;  // the tile's plane (z counts the planes stepped)
        const bool zlo = zp == 0 && !(SLAB && (g.slab & 1u)), zhi = zp == g.nz - 1 && !(SLAB && (g.slab & 2u));
        const bool wall_tile = WALLS && ((g.walls & 1u) || ((g.walls & 4u) && (zlo || zhi)) ||
                                         ((g.walls & 2u) && (y0 == 0 || y0 + p.rows >= g.ny)));
        if constexpr (SH::pairs) {
            const unsigned char *b = buf + s * SB;
            if (wall_tile)
                compute_tile_pairs<C, S, FM, true, SH, MODE>(src, dst, g, r, F, flag, key, p, zp, y0, b, tfx, tfy,
                                                             tfz);
            else
                compute_tile_pairs<C, S, FM, false, SH, MODE>(src, dst, g, r, F, flag, key, p, zp, y0, b, tfx, tfy,
                                                              tfz);
        } else {
            if (wall_tile)
                compute_tile<C, S, FM, true, Q, SH>(src, dst, g, r, F, flag, key, p, zp, y0, buf + s * SB, tfx, tfy,
                                                    tfz);
            else
                compute_tile<C, S, FM, false, Q, SH>(src, dst, g, r, F, flag, key, p, zp, y0, buf + s * SB, tfx, tfy,
                                                     tfz);
        }
        __syncwarp();
        int last = 0;
        if (lane == 0) {
            __threadfence_block();  // this warp's reads of the buffer precede the count
            last = atomicAdd(&done[s], 1) == nwarps - 1;
            if (last) done[s] = 0;
        }
        if (__shfl_sync(0xffffffffu, last, 0)) {
            const int tn = t + kTmaStages * gridDim.x;
            if (tn < p.ntiles) {
                fence_proxy_async();  // the buffer's reads by every warp precede the copies into it
                issue_tile<S, FM, WALLS, Q, SH, MODE>(src, F, g, p, tn, buf + s * SB, &bar[s], lane);
                if (lane == 0) ++issued[s];
            }
        }
        z += p.dz;
        yt += p.dy;
        if (yt >= p.tiles_y) {
            yt -= p.tiles_y;
            ++z;
        }
    }
    __syncthreads();
    if (*abort && threadIdx.x == 0) {
        // a copy did not arrive in time: before the block's shared memory is
        // released, wait (bounded) for the last copy issued into each buffer
        for (int s = 0; s < kTmaStages; ++s)
            if (issued[s] > 0) mbar_wait(&bar[s], (uint32_t)(issued[s] - 1) & 1u, kWaitCycles);
    }
}

// Launch the staged step in shape SH if it applies to this geometry, buffer
// and force; returns false (nothing launched) otherwise. MODE (TileMode):
// the slab modes step the planes L.z0, L.z0 + L.zs, ... (L.nplanes of them);
// the in-place modes take src == dst.
template <typename SH, bool WALLS, int Q, typename C, typename S, int FM, int MODE, typename R>
bool launch_step_tma_shape(const Launch &L, const void *src, void *dst, const R &r, const ForceArgs &F, int *flag,
                           uint32_t key, cudaError_t &err) {
    if constexpr (!tile_fits<S, FM, Q, SH>()) {
        return false;
    } else {
        constexpr bool SLAB = tile_slab<MODE>();
        TilePlan p;
        if (!tile_plan(L.g, sizeof(S), src, 0, SH::pitch, p, SLAB ? L.z0 : 0, SLAB ? L.zs : 1,
                       SLAB ? L.nplanes : -1))
            return false;
        if (FM == kForceField && ((((uintptr_t)F.field) & 15u) != 0 || (F.n & 3) != 0)) return false;
        int dev = 0, sms = 0;
        if ((err = cudaGetDevice(&dev)) != cudaSuccess) return true;
        if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return true;
        constexpr size_t smem = tile_smem_bytes<S, FM, Q, SH>();
        int grid = p.ntiles < SH::blocks * sms ? p.ntiles : SH::blocks * sms;
        // Block b takes the tiles b, b + grid, ...; with a grid sharing a factor with the tiles per plane a
        // block meets only some row positions, and the few blocks whose positions hold the y-wall rows take
        // all the slower wall tiles. A grid coprime to it spreads them evenly.
        if (WALLS && grid < p.ntiles)
            while (grid > 1 && std::gcd(grid, p.tiles_y) != 1) --grid;
        tile_plan(L.g, sizeof(S), src, grid, SH::pitch, p, SLAB ? L.z0 : 0, SLAB ? L.zs : 1, SLAB ? L.nplanes : -1);
        if (L.wait_cycles > 0) p.wait = L.wait_cycles;
        if (L.drop_first_tile) p.drop_tile = 0;
        auto kern = k_step_tma<C, S, FM, WALLS, Q, SH, MODE, R>;
        // the shared-memory opt-in, once per device for this kernel; host threads
        // may race to set it, which repeats a harmless call
        static std::atomic<int> opted_in[64] = {};
        if (dev < 0 || dev >= 64 || !opted_in[dev].load(std::memory_order_relaxed)) {
            if ((err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
                cudaSuccess)
                return true;
            if (dev >= 0 && dev < 64) opted_in[dev].store(1, std::memory_order_relaxed);
        }
        kern<<<grid, SH::threads, smem, L.stream>>>((const S *)src, (S *)dst, L.g, r, F, flag, key, p);
        err = cudaGetLastError();
        return true;
    }
}

// Launch the staged step (Q = 19 or 27 populations, rates R) if it applies;
// returns false (nothing launched) otherwise. Modes other than kTilePull:
// D3Q19 with a collision that has the node-pair form.
template <int Q, typename C, typename S, int FM, int MODE = kTilePull, typename R>
bool launch_step_tma(const Launch &L, const void *src, void *dst, const R &r, const ForceArgs &F, int *flag,
                     uint32_t key, cudaError_t &err) {
    if constexpr (Q == 27) {
        static_assert(MODE == kTilePull, "D3Q27: the A/B pull step");
        return L.g.walls ? launch_step_tma_shape<TmaShape27, true, Q, C, S, FM, MODE>(L, src, dst, r, F, flag, key, err)
                         : launch_step_tma_shape<TmaShape27, false, Q, C, S, FM, MODE>(L, src, dst, r, F, flag, key,
                                                                                      err);
    } else if constexpr (C::kPairs) {
        if constexpr (MODE == kTileAAEven)  // reads only its own slots: no wall code
            return launch_step_tma_shape<TmaShape19P, false, Q, C, S, FM, MODE>(L, src, dst, r, F, flag, key, err);
        else
            return L.g.walls
                       ? launch_step_tma_shape<TmaShape19P, true, Q, C, S, FM, MODE>(L, src, dst, r, F, flag, key, err)
                       : launch_step_tma_shape<TmaShape19P, false, Q, C, S, FM, MODE>(L, src, dst, r, F, flag, key,
                                                                                     err);
    } else {
        static_assert(MODE == kTilePull, "slabs and the in-place kinds: collisions with the node-pair form");
        if (!L.g.walls)
            return launch_step_tma_shape<TmaShape19, false, Q, C, S, FM, MODE>(L, src, dst, r, F, flag, key, err);
        return launch_step_tma_shape<TmaShape19W, true, Q, C, S, FM, MODE>(L, src, dst, r, F, flag, key, err) ||
               launch_step_tma_shape<TmaShape19, true, Q, C, S, FM, MODE>(L, src, dst, r, F, flag, key, err);
    }
}

// Whether a step of this context would run staged (for clbm_info).
inline bool step_staged_for(const Geom &g, size_t elem, const void *src, int q, int force_mode) {
    TilePlan p;
    if (!tile_plan(g, elem, src, 0, 1024, p)) return false;
    if (q == 27 && force_mode == kForceField) return tile_fits<__half, kForceField, 27, TmaShape27>();
    return true;
}

}  // namespace clbm
