// d3q19.cuh -- device-side D3Q19 cascaded-LBM node arithmetic for sm_103a.
//
// Method: Fei, Luo & Li, arXiv:1801.04586, Appendix A (D3Q19) with the GMRT
// collision of Sec. II.A (Eq. 5), the simplified central-moment set (Eq. A2),
// the block-diagonal S (Eq. A3), the continuous-Maxwellian equilibria (Eq. A5)
// and the consistent forcing terms (Eq. A6).
//
// Velocity order (Eq. A1): 0 rest; 1,2 = +-x; 3,4 = +-y; 5,6 = +-z;
// 7..10 = (+1,+1,0) (-1,+1,0) (+1,-1,0) (-1,-1,0); 11..14 = the same pattern
// in (x,z); 15..18 = the same pattern in (y,z).
//
// Arithmetic is done on deviations so that FP32 keeps its relative precision
// on the small quantities that carry the physics:
//   h_i = f_i - w_i                       (w = rest weights 1/3, 1/18, 1/36)
//   dT  = M h                             (raw-moment deviations, Eq. 4)
//   R   = M f - rho G(u)                  (non-equilibrium raw moments; rho G(u)
//                                          are the raw moments of the generalized
//                                          equilibrium, a product of the 1D moments
//                                          1, u, u^2 + c_s^2 per axis)
//   D   = N(u) R = T~ - T~eq              (non-equilibrium central moments)
//   D*  = (I - S) D + (I - S/2) C         (Eq. 5 minus T~eq on both sides)
//   h*  = M^-1 (N(-u) D* + rho G(u) - M w)
// which is Eq. 5 and Eq. 7 rearranged exactly. N(u) is applied as three
// per-axis binomial shifts (x, then y, then z), each acting on triplets
// (k0, k1, k2) of moments that differ only in that axis' exponent; N(-u)
// undoes them. M and M^-1 are written out from the plane structure of the
// velocity set (91 non-zeros of M^-1, Eq. 7).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "bounds.cuh"

namespace clbm {

constexpr int kQ = 19;
constexpr float kC = 1.0f / 3.0f;   // c_s^2
constexpr float kC2 = 1.0f / 9.0f;  // c_s^4

// Rest weights w_i (the u = 0 equilibrium at rho = 1).
__host__ __device__ constexpr float rest_weight(int i) {
    return i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
}

// Opposite direction (bounce-back partner): pairs (1,2) (3,4) (5,6), and in
// each diagonal plane group of four starting at b = 7, 11, 15: b+k <-> b+3-k.
__host__ __device__ constexpr int opposite(int i) {
    return i == 0 ? 0 : (i <= 6 ? ((i & 1) ? i + 1 : i - 1) : (2 * (7 + 4 * ((i - 7) / 4)) + 3 - i));
}

// Velocity components of the D3Q19 set in the order of Eq. A1.
__host__ __device__ constexpr int ex19(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int ey19(int i) {
    return (i == 3 || i == 7 || i == 8 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 9 || i == 10 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int ez19(int i) {
    return (i == 5 || i == 11 || i == 12 || i == 15 || i == 16) ? 1
         : (i == 6 || i == 13 || i == 14 || i == 17 || i == 18) ? -1 : 0;
}

// ---------------------------------------------------------------- storage
// Counter-based hash "lowbias32" (C. Wellons, hash-prospector, 2018): an
// invertible 32-bit mixer; used to draw the dither of stochastic rounding
// from (per-step key, node, direction), so results are reproducible and do not
// depend on the launch shape.
__host__ __device__ constexpr uint32_t lowbias32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Storage tags for stochastic rounding: same bits as __half / __nv_bfloat16.
struct HalfSR { __half v; };
struct BF16SR { __nv_bfloat16 v; };

// Codec<T>: load a stored deviation as FP32; store an FP32 deviation. Formats
// with kStochastic round with a random dither r (from_f_sr), the others to
// nearest even (from_f).
template <typename T> struct Codec;
template <> struct Codec<float> {
    static constexpr bool kStochastic = false;
    static __device__ __forceinline__ float load(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ float load_plain(const float *p) { return *p; }
    static __device__ __forceinline__ float from_f(float v) { return v; }
    static __device__ __forceinline__ float from_f_sr(float v, uint32_t) { return v; }
};
// 16-bit formats also convert a pair of FP32 values (hi, lo) in one
// instruction, the results in the upper and lower half of a word (pair_rn /
// pair_sr below), and widen a stored pair read as one word (unpack2: .x the
// lower half, the value at the lower address).
__device__ __forceinline__ uint32_t rn_pair_f16(float hi, float lo);
__device__ __forceinline__ uint32_t rn_pair_bf16(float hi, float lo);
__device__ __forceinline__ float2 unpack2_f16(uint32_t w) {
    __half2_raw raw;
    raw.x = (unsigned short)(w & 0xffffu);
    raw.y = (unsigned short)(w >> 16);
    return __half22float2(__half2(raw));
}
__device__ __forceinline__ float2 unpack2_bf16(uint32_t w) {
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
template <> struct Codec<__half> {
    static constexpr bool kStochastic = false;
    static __device__ __forceinline__ float load(const __half *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ float load_plain(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ __half from_f(float v) { return __float2half_rn(v); }
    static __device__ __forceinline__ __half from_f_sr(float v, uint32_t) { return __float2half_rn(v); }
    static __device__ __forceinline__ uint32_t pair_rn(float hi, float lo) { return rn_pair_f16(hi, lo); }
    static __device__ __forceinline__ float2 unpack2(uint32_t w) { return unpack2_f16(w); }
};
template <> struct Codec<__nv_bfloat16> {
    static constexpr bool kStochastic = false;
    static __device__ __forceinline__ float load(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ float load_plain(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ __nv_bfloat16 from_f(float v) { return __float2bfloat16_rn(v); }
    static __device__ __forceinline__ __nv_bfloat16 from_f_sr(float v, uint32_t) { return __float2bfloat16_rn(v); }
    static __device__ __forceinline__ uint32_t pair_rn(float hi, float lo) { return rn_pair_bf16(hi, lo); }
    static __device__ __forceinline__ float2 unpack2(uint32_t w) { return unpack2_bf16(w); }
};
// Stochastic rounding by the conversion instruction of sm_100-class GPUs,
// cvt.rs.{f16x2,bf16x2}.f32 d, a, b, rbits: it adds a random integer below one
// unit in the last place of the target to |x| (FP32 sign-magnitude bits) and
// truncates, so |x| rounds up with probability equal to the dropped fraction
// and the stored value is unbiased (also in the FP16 subnormal range). Of the
// 32 random bits, the lower half serves b (stored in the lower 16 bits of d),
// the upper half serves a (upper 16 bits); FP16 takes the low 13 bits of its
// half (the 13 bits it drops in its normal range), BF16 all 16.
// sr_pair(hi, lo, r): both values in one instruction; the 16-bit results in
// the upper and lower half of the returned word.
__device__ __forceinline__ uint32_t sr_pair_f16(float hi, float lo, uint32_t r) {
    uint32_t d;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
    return d;
}
__device__ __forceinline__ uint32_t sr_pair_bf16(float hi, float lo, uint32_t r) {
    uint32_t d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(r));
    return d;
}
// Round-to-nearest-even pair conversions (cvt.rn.{f16x2,bf16x2}.f32).
__device__ __forceinline__ uint32_t rn_pair_f16(float hi, float lo) {
    uint32_t d;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
__device__ __forceinline__ uint32_t rn_pair_bf16(float hi, float lo) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
// One value with the random half of r that its node's parity selects (odd:
// upper half, even: lower half), bit for bit what the pair conversion gives
// that node.
template <> struct Codec<HalfSR> {
    static constexpr bool kStochastic = true;
    static __device__ __forceinline__ float load(const HalfSR *p) { return __half2float(__ldg(&p->v)); }
    static __device__ __forceinline__ float load_plain(const HalfSR *p) { return __half2float(p->v); }
    static __device__ __forceinline__ HalfSR from_f(float v) { return HalfSR{__float2half_rn(v)}; }
    static __device__ __forceinline__ HalfSR from_f_sr(float v, uint32_t r, bool odd) {
        const uint32_t d = odd ? sr_pair_f16(v, 0.0f, r) >> 16 : sr_pair_f16(0.0f, v, r) & 0xffffu;
        __half_raw raw;
        raw.x = (unsigned short)d;
        return HalfSR{__half(raw)};
    }
    static __device__ __forceinline__ uint32_t pair_sr(float hi, float lo, uint32_t r) { return sr_pair_f16(hi, lo, r); }
    static __device__ __forceinline__ float2 unpack2(uint32_t w) { return unpack2_f16(w); }
};
template <> struct Codec<BF16SR> {
    static constexpr bool kStochastic = true;
    static __device__ __forceinline__ float load(const BF16SR *p) { return __bfloat162float(__ldg(&p->v)); }
    static __device__ __forceinline__ float load_plain(const BF16SR *p) { return __bfloat162float(p->v); }
    static __device__ __forceinline__ BF16SR from_f(float v) { return BF16SR{__float2bfloat16_rn(v)}; }
    static __device__ __forceinline__ BF16SR from_f_sr(float v, uint32_t r, bool odd) {
        const uint32_t d = odd ? sr_pair_bf16(v, 0.0f, r) >> 16 : sr_pair_bf16(0.0f, v, r) & 0xffffu;
        __nv_bfloat16_raw raw;
        raw.x = (unsigned short)d;
        return BF16SR{__nv_bfloat16(raw)};
    }
    static __device__ __forceinline__ uint32_t pair_sr(float hi, float lo, uint32_t r) {
        return sr_pair_bf16(hi, lo, r);
    }
    static __device__ __forceinline__ float2 unpack2(uint32_t w) { return unpack2_bf16(w); }
};

// Random bits of stochastic rounding for population i of the node pair
// p = node >> 1 (nodes 2p and 2p + 1, adjacent in x): 32 bits, the lower half
// for the even node and the upper half for the odd one, as the pair
// conversion takes them. The pair's hash is the full lowbias32 mix of (p,
// key); each population then takes one xorshift-multiply round of it offset
// by a Weyl step (the first round of the same mixer): a bijection of a
// uniform word, so every dither stays uniform. The bits depend on (key, node,
// i) alone, so every storage pattern and staging path stores the same values.
__device__ __forceinline__ uint32_t pair_hash(uint32_t pair, uint32_t key) { return lowbias32(pair ^ key); }
__device__ __forceinline__ uint32_t pop_bits(uint32_t base, int i) {
    uint32_t r = base + (uint32_t)i * 0x9e3779b9u;
    r ^= r >> 16;
    return r * 0x7feb352du;
}

// Encode the NQ post-collision deviations h (population order) of one node
// in the storage format. key: per-step random key (stochastic formats only).
template <typename S, int NQ>
__device__ __forceinline__ void encode_each(const float (&h)[NQ], uint32_t node, uint32_t key, S (&e)[NQ]) {
    if constexpr (Codec<S>::kStochastic) {
        const uint32_t base = pair_hash(node >> 1, key);
        const bool odd = node & 1u;
#pragma unroll
        for (int i = 0; i < NQ; ++i) e[i] = Codec<S>::from_f_sr(h[i], pop_bits(base, i), odd);
    } else {
#pragma unroll
        for (int i = 0; i < NQ; ++i) e[i] = Codec<S>::from_f(h[i]);
    }
}

// Store them: population i goes to addr(i).
template <typename S, int NQ, typename Addr>
__device__ __forceinline__ void store_each(const float (&h)[NQ], uint32_t node, uint32_t key, Addr addr) {
    S e[NQ];
    encode_each<S, NQ>(h, node, key, e);
#pragma unroll
    for (int i = 0; i < NQ; ++i) *addr(i) = e[i];
}

// Pull scheme: the node's own slots, population i in array i.
template <typename S, int NQ = 19>
__device__ __forceinline__ void store_node(S *d, int64_t stride, const float (&h)[NQ], uint32_t node, uint32_t key) {
    store_each<S, NQ>(h, node, key, [&](int i) { return d + (size_t)i * stride; });
}

// Per-step key of the stochastic dither.
__host__ __device__ constexpr uint32_t step_key(int64_t step) {
    return lowbias32((uint32_t)step * 0x9e3779b9u + 0x2545f491u);
}

// ---------------------------------------------------------------- geometry
struct Geom {
    int nx, ny, nz;
    uint32_t walls;     // bit 0: x walls, bit 1: y walls, bit 2: z walls
    int64_t stride;     // elements between population arrays
    // z-slab of a larger lattice: bit 0, the z- face takes the populations
    // crossing it from a halo plane set (the neighbour below); bit 1, the z+
    // face (the neighbour above). A halo face is neither periodic nor a wall.
    uint32_t slab = 0;
    uint32_t node0 = 0; // global linear index of the slab's first node (dither of stochastic rounding)
#ifdef CLBM_BOUNDS_CHECK
    BoundsRecord *bc = nullptr;  // violation record (bounds.cuh)
    uint64_t bc_limit = 0;       // elements of one state buffer
#endif
};

// Halo region of a z-slab's state buffer, after the Q population arrays (at
// element Q * stride), in planes of nx * ny values indexed y * nx + x:
//   planes 0-4:   received, e_z = +1 populations (Eq. A1 order 5, 11, 12, 15,
//                 16) of the plane below the slab, pulled across the z- face;
//   planes 5-9:   received, e_z = -1 populations (6, 13, 14, 17, 18) of the
//                 plane above, pulled across the z+ face;
//   planes 10-14: sent, the slab's own e_z = -1 populations of plane 0 (the
//                 lower neighbour's planes 5-9);
//   planes 15-19: sent, the slab's own e_z = +1 populations of plane nz - 1
//                 (the upper neighbour's planes 0-4).
constexpr int kSlabPlanes = 20;
__host__ __device__ constexpr int zface_index(int i) {
    return (i == 5 || i == 6) ? 0 : (i == 11 || i == 13) ? 1 : (i == 12 || i == 14) ? 2 : (i == 15 || i == 17) ? 3 : 4;
}
__host__ __device__ constexpr int zplus_pop(int k) { return k == 0 ? 5 : k == 1 ? 11 : k == 2 ? 12 : k == 3 ? 15 : 16; }
__host__ __device__ constexpr int zminus_pop(int k) { return k == 0 ? 6 : k == 1 ? 13 : k == 2 ? 14 : k == 3 ? 17 : 18; }

// Pull sources of the 19 populations arriving at node (x, y, z) (Eq. 8 read
// backwards): population i comes from (i, x - e_i) with periodic wrap, or,
// when x - e_i lies beyond a wall face, from (ibar, x) -- halfway bounce-back.
// pop[i] is the population array index and off[i] the node offset to read.
// The same map, used to write instead of read, turns a post-streaming state
// into the post-collision buffer a later pull reproduces it from.
// SWAP = true gives the same offsets with the opposite array index, (ibar,
// x - e_i) or (i, x): the slots of the in-place (AA) pattern's odd step, which
// reads population i there and writes post-collision population ibar there.
//
// SLAB = true: the z faces flagged in g.slab are halo faces. A population whose
// source lies across one (and is not bounced back at an x or y wall) is read
// from the halo region (pop = kQ, off = plane offset within it, see
// kSlabPlanes); z walls apply only to the faces that are not halo faces.
template <bool WALLS, bool SWAP = false, bool SLAB = false>
__device__ __forceinline__ void pull_sources(const Geom &g, int x, int y, int z,
                                             uint32_t (&off)[kQ], int (&pop)[kQ]) {
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    const uint32_t unx = (uint32_t)nx, uny = (uint32_t)ny;
    const uint32_t rc = ((uint32_t)z * uny + y) * unx;
    const uint32_t rym = ((uint32_t)z * uny + ym) * unx, ryp = ((uint32_t)z * uny + yp) * unx;
    const uint32_t rzm = ((uint32_t)zm * uny + y) * unx, rzp = ((uint32_t)zp * uny + y) * unx;
    const uint32_t rmm = ((uint32_t)zm * uny + ym) * unx, rpm = ((uint32_t)zm * uny + yp) * unx;
    const uint32_t rmp = ((uint32_t)zp * uny + ym) * unx, rpp = ((uint32_t)zp * uny + yp) * unx;
    const uint32_t self = rc + x;
    off[0] = self;
    off[1] = rc + xm;   off[2] = rc + xp;
    off[3] = rym + x;   off[4] = ryp + x;
    off[5] = rzm + x;   off[6] = rzp + x;
    off[7] = rym + xm;  off[8] = rym + xp;  off[9] = ryp + xm;  off[10] = ryp + xp;
    off[11] = rzm + xm; off[12] = rzm + xp; off[13] = rzp + xm; off[14] = rzp + xp;
    off[15] = rmm + x;  off[16] = rpm + x;  off[17] = rmp + x;  off[18] = rpp + x;
#pragma unroll
    for (int i = 0; i < kQ; ++i) pop[i] = SWAP ? opposite(i) : i;
    bool bbx[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) bbx[i] = false;
    if (WALLS) {
        const bool wx = g.walls & 1u, wy = g.walls & 2u, wz = g.walls & 4u;
        const bool xl = wx && x == 0, xh = wx && x == nx - 1;  // ex = +1 / -1 bounce
        const bool yl = wy && y == 0, yh = wy && y == ny - 1;
        const bool zl = wz && z == 0 && !(SLAB && (g.slab & 1u)), zh = wz && z == nz - 1 && !(SLAB && (g.slab & 2u));
        // ex, ey, ez of each direction decide which faces it can cross.
        const bool bb[kQ] = {false,
                             xl, xh, yl, yh, zl, zh,
                             xl || yl, xh || yl, xl || yh, xh || yh,
                             xl || zl, xh || zl, xl || zh, xh || zh,
                             yl || zl, yh || zl, yl || zh, yh || zh};
#pragma unroll
        for (int i = 1; i < kQ; ++i) {
            if (bb[i]) { pop[i] = SWAP ? i : opposite(i); off[i] = self; }
            bbx[i] = bb[i];
        }
    }
    if (SLAB) {
        // across a halo face: the neighbour's post-collision value, from the halo planes
        const uint32_t plane = unx * uny;
        if ((g.slab & 1u) && z == 0) {
#pragma unroll
            for (int i = 1; i < kQ; ++i)
                if (ez19(i) > 0 && !bbx[i]) {
                    pop[i] = kQ;
                    off[i] = (uint32_t)zface_index(i) * plane + (off[i] - (uint32_t)zm * plane);
                }
        }
        if ((g.slab & 2u) && z == nz - 1) {
#pragma unroll
            for (int i = 1; i < kQ; ++i)
                if (ez19(i) < 0 && !bbx[i]) {
                    pop[i] = kQ;
                    off[i] = (uint32_t)(5 + zface_index(i)) * plane + (off[i] - (uint32_t)zp * plane);
                }
        }
    }
}

// Targets of the 19 populations leaving node (x, y, z) under Eq. 8: (i, x + e_i)
// with periodic wrap, or (ibar, x) when x + e_i lies beyond a wall face. The
// adjoint gathers through this map; the in-place pattern's odd step writes
// through it.
template <bool WALLS>
__device__ __forceinline__ void push_targets(const Geom &g, int x, int y, int z, uint32_t (&off)[kQ],
                                             int (&pop)[kQ]) {
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    const uint32_t unx = (uint32_t)nx, uny = (uint32_t)ny;
    const uint32_t rc = ((uint32_t)z * uny + y) * unx;
    const uint32_t rym = ((uint32_t)z * uny + ym) * unx, ryp = ((uint32_t)z * uny + yp) * unx;
    const uint32_t rzm = ((uint32_t)zm * uny + y) * unx, rzp = ((uint32_t)zp * uny + y) * unx;
    const uint32_t rmm = ((uint32_t)zm * uny + ym) * unx, rpm = ((uint32_t)zm * uny + yp) * unx;
    const uint32_t rmp = ((uint32_t)zp * uny + ym) * unx, rpp = ((uint32_t)zp * uny + yp) * unx;
    const uint32_t self = rc + x;
    // destination x + e_i
    off[0] = self;
    off[1] = rc + xp;   off[2] = rc + xm;
    off[3] = ryp + x;   off[4] = rym + x;
    off[5] = rzp + x;   off[6] = rzm + x;
    off[7] = ryp + xp;  off[8] = ryp + xm;  off[9] = rym + xp;  off[10] = rym + xm;
    off[11] = rzp + xp; off[12] = rzp + xm; off[13] = rzm + xp; off[14] = rzm + xm;
    off[15] = rpp + x;  off[16] = rmp + x;  off[17] = rpm + x;  off[18] = rmm + x;
#pragma unroll
    for (int i = 0; i < kQ; ++i) pop[i] = i;
    if (WALLS) {
        const bool wx = g.walls & 1u, wy = g.walls & 2u, wz = g.walls & 4u;
        const bool xl = wx && x == 0, xh = wx && x == nx - 1;  // leaving through x- (ex = -1) / x+ (ex = +1)
        const bool yl = wy && y == 0, yh = wy && y == ny - 1;
        const bool zl = wz && z == 0, zh = wz && z == nz - 1;
        const bool bb[kQ] = {false,
                             xh, xl, yh, yl, zh, zl,
                             xh || yh, xl || yh, xh || yl, xl || yl,
                             xh || zh, xl || zh, xh || zl, xl || zl,
                             yh || zh, yl || zh, yh || zl, yl || zl};
#pragma unroll
        for (int i = 1; i < kQ; ++i) {
            if (bb[i]) { pop[i] = opposite(i); off[i] = self; }
        }
    }
}

// ---------------------------------------------------------------- collision
struct Rates {
    float om2;  // 1 - s2
    float cb;   // (s2b - s2)/3: trace coupling of the 3x3 block of Eq. A3
    float om3;  // 1 - s3
    float c3;   // (1 - s3/2) c_s^2: coefficient of F in the third-order terms (Eq. A6)
    float om4;  // 1 - s4
};

// One node's value with operators that round every operation on its own
// (__fadd_rn, __fsub_rn and __fmul_rn are never merged into fused
// multiply-adds; fused ones are written as fmaf). The collision of the 16-bit
// storage formats runs on it, so that it rounds exactly like the f2 form
// below, lane by lane: a step that collides two nodes at once with the FP32x2
// instructions then stores the same bits as one node per thread.
struct f1 {
    float v;
};
__device__ __forceinline__ f1 mk1(float a) { return f1{a}; }
__device__ __forceinline__ f1 operator+(f1 a, f1 b) { return f1{__fadd_rn(a.v, b.v)}; }
__device__ __forceinline__ f1 operator-(f1 a, f1 b) { return f1{__fsub_rn(a.v, b.v)}; }
__device__ __forceinline__ f1 operator-(f1 a) { return f1{-a.v}; }
__device__ __forceinline__ f1 operator*(f1 a, f1 b) { return f1{__fmul_rn(a.v, b.v)}; }
__device__ __forceinline__ f1 operator*(float s, f1 b) { return f1{__fmul_rn(s, b.v)}; }
__device__ __forceinline__ f1 operator*(f1 b, float s) { return f1{__fmul_rn(b.v, s)}; }
__device__ __forceinline__ f1 operator+(float s, f1 b) { return f1{__fadd_rn(s, b.v)}; }
__device__ __forceinline__ f1 operator+(f1 b, float s) { return f1{__fadd_rn(b.v, s)}; }
__device__ __forceinline__ f1 &operator*=(f1 &a, float s) { return a = a * s; }
__device__ __forceinline__ f1 fmaf(f1 a, f1 b, f1 c) { return f1{::fmaf(a.v, b.v, c.v)}; }
__device__ __forceinline__ f1 fmaf(float a, f1 b, f1 c) { return f1{::fmaf(a, b.v, c.v)}; }

// Two nodes' values packed for the FP32x2 instructions of sm_100-class GPUs
// (__fadd2_rn / __fmul2_rn / __ffma2_rn round each lane exactly like the
// scalar operation). The collision templates below run on float or on f2.
struct f2 {
    float2 v;
};
__device__ __forceinline__ f2 mk2(float a) { return f2{make_float2(a, a)}; }
__device__ __forceinline__ f2 mk2(float a, float b) { return f2{make_float2(a, b)}; }
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2{__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return f2{__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)}; }
__device__ __forceinline__ f2 operator-(f2 a) { return f2{make_float2(-a.v.x, -a.v.y)}; }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return f2{__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ f2 operator*(float s, f2 b) { return mk2(s) * b; }
__device__ __forceinline__ f2 operator*(f2 b, float s) { return b * mk2(s); }
__device__ __forceinline__ f2 operator+(float s, f2 b) { return mk2(s) + b; }
__device__ __forceinline__ f2 operator+(f2 b, float s) { return b + mk2(s); }
__device__ __forceinline__ f2 operator/(float s, f2 b) { return f2{make_float2(s / b.v.x, s / b.v.y)}; }
__device__ __forceinline__ f2 &operator*=(f2 &a, float s) { return a = a * s; }
using ::fmaf;
__device__ __forceinline__ f2 fmaf(f2 a, f2 b, f2 c) { return f2{__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ f2 fmaf(float a, f2 b, f2 c) { return fmaf(mk2(a), b, c); }

// 1/x for x near 1 (the density): the hardware reciprocal estimate
// (rcp.approx, relative error below 2^-23) refined by one Newton-Raphson
// step, e = 1 - x r, r' = r + r e, which leaves it within an ulp of the
// correctly rounded quotient in three instructions.
__device__ __forceinline__ float recip_nr(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    const float e = fmaf(-x, r, 1.0f);
    return fmaf(r, e, r);
}
__device__ __forceinline__ f2 recip_nr(f2 x) { return mk2(recip_nr(x.v.x), recip_nr(x.v.y)); }
__device__ __forceinline__ f1 recip_nr(f1 x) { return f1{recip_nr(x.v)}; }

// The collision's 1/rho: recip_nr when FR (16-bit storage, whose steps are
// bound by instruction issue: 3 to 6 % faster), the IEEE division otherwise
// (FP32 steps are bound by DRAM; there the shorter sequence let the compiler
// stretch live ranges, 58 -> 81 registers in the in-place odd step, and
// measured 1-4 % slower).
template <bool FR, typename T>
__device__ __forceinline__ T recip_of(T x) {
    if constexpr (FR)
        return recip_nr(x);
    else
        return 1.0f / x;
}

// Central shift of one triplet along an axis with velocity v (one factor of
// N(u)): (k0, k1, k2) -> (k0, k1 - v k0, k2 - 2 v k1 + v^2 k0).
template <typename T>
__device__ __forceinline__ void shift3(T k0, T &k1, T &k2, T v) {
    const T c1 = fmaf(-v, k0, k1);
    k2 = fmaf(-v, k1 + c1, k2);
    k1 = c1;
}
// Its inverse (one factor of N(-u)): (c0, c1, c2) -> (c0, c1 + v c0, c2 + 2 v c1 + v^2 c0).
template <typename T>
__device__ __forceinline__ void unshift3(T c0, T &c1, T &c2, T v) {
    const T k1 = fmaf(v, c0, c1);
    c2 = fmaf(v, c1 + k1, c2);
    c1 = k1;
}

// Raw-moment deviations dT = M h, named by exponents (Eq. A2 with k~002 as the
// tenth moment).
template <typename T>
struct MomentsT {
    T m000, m100, m010, m001, m110, m101, m011, m200, m020, m002;
    T m120, m102, m210, m201, m012, m021, m220, m202, m022;
};
using Moments = MomentsT<float>;

template <typename T>
__device__ __forceinline__ void raw_moments(const T (&h)[kQ], MomentsT<T> &k) {
    // xy plane (7..10): four moments ex^a ey^b with a, b in {1, 2}
    const T a = h[7] + h[8], b = h[9] + h[10], c = h[7] + h[9], d = h[8] + h[10];
    const T e = h[7] + h[10], f = h[8] + h[9];
    k.m220 = a + b; k.m210 = a - b; k.m120 = c - d; k.m110 = e - f;
    // xz plane (11..14)
    const T a2 = h[11] + h[12], b2 = h[13] + h[14], c2 = h[11] + h[13], d2 = h[12] + h[14];
    const T e2 = h[11] + h[14], f2 = h[12] + h[13];
    k.m202 = a2 + b2; k.m201 = a2 - b2; k.m102 = c2 - d2; k.m101 = e2 - f2;
    // yz plane (15..18)
    const T a3 = h[15] + h[16], b3 = h[17] + h[18], c3 = h[15] + h[17], d3 = h[16] + h[18];
    const T e3 = h[15] + h[18], f3 = h[16] + h[17];
    k.m022 = a3 + b3; k.m021 = a3 - b3; k.m012 = c3 - d3; k.m011 = e3 - f3;
    // axes
    const T s12 = h[1] + h[2], s34 = h[3] + h[4], s56 = h[5] + h[6];
    k.m200 = s12 + k.m220 + k.m202;
    k.m020 = s34 + k.m220 + k.m022;
    k.m002 = s56 + k.m202 + k.m022;
    k.m100 = (h[1] - h[2]) + k.m120 + k.m102;
    k.m010 = (h[3] - h[4]) + k.m210 + k.m012;
    k.m001 = (h[5] - h[6]) + k.m201 + k.m021;
    k.m000 = h[0] + s12 + s34 + s56 + k.m220 + k.m202 + k.m022;
}

// Deviations of the generalized-equilibrium raw moments, rho G(u) - M w,
// for the 15 moments other than the ones with a zero/first-order closed form.
template <typename T>
struct EqDevT {
    T d110, d101, d011, d200, d020, d002, d120, d102, d210, d201, d012, d021, d220, d202, d022;
};
using EqDev = EqDevT<float>;

template <typename T>
__device__ __forceinline__ void eq_dev(T drho, T rho, T jx, T jy, T jz, T ux, T uy, T uz, EqDevT<T> &q) {
    const T X = ux * ux, Y = uy * uy, Z = uz * uz;
    q.d110 = jx * uy; q.d101 = jx * uz; q.d011 = jy * uz;
    q.d200 = fmaf(jx, ux, drho * kC); q.d020 = fmaf(jy, uy, drho * kC); q.d002 = fmaf(jz, uz, drho * kC);
    q.d120 = jx * (Y + kC); q.d102 = jx * (Z + kC);
    q.d210 = jy * (X + kC); q.d201 = jz * (X + kC);
    q.d012 = jy * (Z + kC); q.d021 = jz * (Y + kC);
    q.d220 = fmaf(rho, fmaf(X, Y, kC * (X + Y)), drho * kC2);
    q.d202 = fmaf(rho, fmaf(X, Z, kC * (X + Z)), drho * kC2);
    q.d022 = fmaf(rho, fmaf(Y, Z, kC * (Y + Z)), drho * kC2);
}

// The four populations of one diagonal plane from its moments (22, 21, 12,
// 11 in the plane's two axes): 1/4 ((m22 +- m21) +- (m12 +- m11)).
template <typename T>
__device__ __forceinline__ void plane_inverse(T m22, T m21, T m12, T m11, T &pp, T &pm, T &mp, T &mm) {
    const T a = 0.25f * (m22 + m21), c = 0.25f * (m22 - m21);
    const T b = m12 + m11, d = m12 - m11;
    pp = fmaf(0.25f, b, a);
    pm = fmaf(-0.25f, b, a);
    mp = fmaf(0.25f, d, c);
    mm = fmaf(-0.25f, d, c);
}

// h = M^-1 Q for raw-moment deviations Q (Eq. 7, M^-1 of Eq. A4).
template <typename T>
__device__ __forceinline__ void inverse_moments(const MomentsT<T> &q, T (&h)[kQ]) {
    // Each pair s (a + b), s (a - b) is taken as s a +- s b with s a exact, so
    // the results are the same bits with one multiply fewer per pair.
    plane_inverse(q.m220, q.m210, q.m120, q.m110, h[7], h[8], h[9], h[10]);
    plane_inverse(q.m202, q.m201, q.m102, q.m101, h[11], h[12], h[13], h[14]);
    plane_inverse(q.m022, q.m021, q.m012, q.m011, h[15], h[16], h[17], h[18]);
    const T px = q.m200 - q.m220 - q.m202, vx = q.m100 - q.m120 - q.m102;
    const T py = q.m020 - q.m220 - q.m022, vy = q.m010 - q.m210 - q.m012;
    const T pz = q.m002 - q.m202 - q.m022, vz = q.m001 - q.m201 - q.m021;
    const T px2 = 0.5f * px, py2 = 0.5f * py, pz2 = 0.5f * pz;
    h[1] = fmaf(0.5f, vx, px2); h[2] = fmaf(-0.5f, vx, px2);
    h[3] = fmaf(0.5f, vy, py2); h[4] = fmaf(-0.5f, vy, py2);
    h[5] = fmaf(0.5f, vz, pz2); h[6] = fmaf(-0.5f, vz, pz2);
    h[0] = q.m000 - (q.m200 + q.m020 + q.m002) + (q.m220 + q.m202 + q.m022);
}

// One collision (Steps 1-3 of Sec. II.B) on deviations h, in place.
// Returns drho = rho - 1 of the pre-collision state (Eq. 9); if j_out is not
// null it receives rho*u of Eq. 9 (momentum including F/2).
template <bool FR, typename T>
__device__ __forceinline__ T collide_t(T (&h)[kQ], T Fx, T Fy, T Fz, const Rates &r, float3 *j_out) {
    MomentsT<T> k;
    raw_moments(h, k);
    const T drho = k.m000;
    const T rho = 1.0f + drho;
    const T inv = recip_of<FR>(rho);
    const T jx = fmaf(0.5f, Fx, k.m100), jy = fmaf(0.5f, Fy, k.m010), jz = fmaf(0.5f, Fz, k.m001);
    const T ux = jx * inv, uy = jy * inv, uz = jz * inv;
    if constexpr (std::is_same<T, float>::value) {
        if (j_out) *j_out = make_float3(jx, jy, jz);
    } else if constexpr (std::is_same<T, f1>::value) {
        if (j_out) *j_out = make_float3(jx.v, jy.v, jz.v);
    }
    EqDevT<T> e;
    eq_dev(drho, rho, jx, jy, jz, ux, uy, uz, e);

    // non-equilibrium raw moments R = dT - (rho G - M w); R000 = 0, R100 = -Fx/2, ...
    const T hFx = 0.5f * Fx, hFy = 0.5f * Fy, hFz = 0.5f * Fz;
    T r110 = k.m110 - e.d110, r101 = k.m101 - e.d101, r011 = k.m011 - e.d011;
    T r200 = k.m200 - e.d200, r020 = k.m020 - e.d020, r002 = k.m002 - e.d002;
    T r120 = k.m120 - e.d120, r102 = k.m102 - e.d102, r210 = k.m210 - e.d210;
    T r201 = k.m201 - e.d201, r012 = k.m012 - e.d012, r021 = k.m021 - e.d021;
    T r220 = k.m220 - e.d220, r202 = k.m202 - e.d202, r022 = k.m022 - e.d022;

    // D = N(u) R: x shift on (000,100,200) (010,110,210) (001,101,201) (020,120,220) (002,102,202)
    r200 = fmaf(ux, Fx, r200);                 // R000 = 0, R100 = -Fx/2
    shift3(-hFy, r110, r210, ux);
    shift3(-hFz, r101, r201, ux);
    shift3(r020, r120, r220, ux);
    shift3(r002, r102, r202, ux);
    // y shift on (000,010,020) (100,110,120) (001,011,021) (200,210,220) (002,012,022)
    r020 = fmaf(uy, Fy, r020);
    shift3(-hFx, r110, r120, uy);
    shift3(-hFz, r011, r021, uy);
    shift3(r200, r210, r220, uy);
    shift3(r002, r012, r022, uy);
    // z shift on (000,001,002) (100,101,102) (010,011,012) (200,201,202) (020,021,022)
    r002 = fmaf(uz, Fz, r002);
    shift3(-hFx, r101, r102, uz);
    shift3(-hFy, r011, r012, uz);
    shift3(r200, r201, r202, uz);
    shift3(r020, r021, r022, uz);

    // Eq. 5 on non-equilibrium central moments: D* = (I - S) D + (I - S/2) C.
    // s0 = s1 = 1: D*000 = 0, D*100 = Fx/2, ...
    r110 *= r.om2; r101 *= r.om2; r011 *= r.om2;
    {
        const T tr = r.cb * (r200 + r020 + r002);
        r200 = fmaf(r.om2, r200, -tr);
        r020 = fmaf(r.om2, r020, -tr);
        r002 = fmaf(r.om2, r002, -tr);
    }
    r120 = fmaf(r.om3, r120, r.c3 * Fx);
    r102 = fmaf(r.om3, r102, r.c3 * Fx);
    r210 = fmaf(r.om3, r210, r.c3 * Fy);
    r201 = fmaf(r.om3, r201, r.c3 * Fz);
    r012 = fmaf(r.om3, r012, r.c3 * Fy);
    r021 = fmaf(r.om3, r021, r.c3 * Fz);
    r220 *= r.om4; r202 *= r.om4; r022 *= r.om4;

    // R* = N(-u) D*: undo z, then y, then x (D*000 = 0, D*100 = Fx/2, ...)
    r002 = fmaf(uz, Fz, r002);
    unshift3(hFx, r101, r102, uz);
    unshift3(hFy, r011, r012, uz);
    unshift3(r200, r201, r202, uz);
    unshift3(r020, r021, r022, uz);
    r020 = fmaf(uy, Fy, r020);
    unshift3(hFx, r110, r120, uy);
    unshift3(hFz, r011, r021, uy);
    unshift3(r200, r210, r220, uy);
    unshift3(r002, r012, r022, uy);
    r200 = fmaf(ux, Fx, r200);
    unshift3(hFy, r110, r210, ux);
    unshift3(hFz, r101, r201, ux);
    unshift3(r020, r120, r220, ux);
    unshift3(r002, r102, r202, ux);

    // Q = R* + (rho G(u) - M w); first order: R*100 = Fx/2, so Q100 = jx + Fx/2.
    MomentsT<T> q;
    q.m000 = drho;
    q.m100 = jx + hFx; q.m010 = jy + hFy; q.m001 = jz + hFz;
    q.m110 = r110 + e.d110; q.m101 = r101 + e.d101; q.m011 = r011 + e.d011;
    q.m200 = r200 + e.d200; q.m020 = r020 + e.d020; q.m002 = r002 + e.d002;
    q.m120 = r120 + e.d120; q.m102 = r102 + e.d102; q.m210 = r210 + e.d210;
    q.m201 = r201 + e.d201; q.m012 = r012 + e.d012; q.m021 = r021 + e.d021;
    q.m220 = r220 + e.d220; q.m202 = r202 + e.d202; q.m022 = r022 + e.d022;
    inverse_moments(q, h);
    return drho;
}

// The collision of one node (float) or two (f2). With FR (16-bit storage) a
// float node runs on f1, rounding every operation on its own, so that it
// matches the f2 form bit for bit; FP32 storage keeps the compiler's fused
// multiply-adds.
template <bool FR = false, typename T>
__device__ __forceinline__ T collide(T (&h)[kQ], T Fx, T Fy, T Fz, const Rates &r, float3 *j_out = nullptr) {
    if constexpr (FR && std::is_same<T, float>::value) {
        f1 g[kQ];
#pragma unroll
        for (int i = 0; i < kQ; ++i) g[i].v = h[i];
        const f1 drho = collide_t<FR>(g, f1{Fx}, f1{Fy}, f1{Fz}, r, j_out);
#pragma unroll
        for (int i = 0; i < kQ; ++i) h[i] = g[i].v;
        return drho.v;
    } else {
        return collide_t<FR>(h, Fx, Fy, Fz, r, j_out);
    }
}

// Deviations of the generalized local equilibrium at (rho, u):
// h = M^-1 (rho G(u) - M w).
template <typename T>
__device__ __forceinline__ void equilibrium_dev(T rho, T ux, T uy, T uz, T (&h)[kQ]) {
    const T drho = rho - 1.0f;
    const T jx = rho * ux, jy = rho * uy, jz = rho * uz;
    EqDevT<T> e;
    eq_dev(drho, rho, jx, jy, jz, ux, uy, uz, e);
    MomentsT<T> q;
    q.m000 = drho; q.m100 = jx; q.m010 = jy; q.m001 = jz;
    q.m110 = e.d110; q.m101 = e.d101; q.m011 = e.d011;
    q.m200 = e.d200; q.m020 = e.d020; q.m002 = e.d002;
    q.m120 = e.d120; q.m102 = e.d102; q.m210 = e.d210; q.m201 = e.d201;
    q.m012 = e.d012; q.m021 = e.d021;
    q.m220 = e.d220; q.m202 = e.d202; q.m022 = e.d022;
    inverse_moments(q, h);
}

// Eq. 9 on deviations: returns drho and writes rho*u (momentum incl. F/2).
template <typename T>
__device__ __forceinline__ T macros_dev(const T (&h)[kQ], T Fx, T Fy, T Fz, T &jx, T &jy, T &jz) {
    MomentsT<T> k;
    raw_moments(h, k);
    jx = fmaf(0.5f, Fx, k.m100);
    jy = fmaf(0.5f, Fy, k.m010);
    jz = fmaf(0.5f, Fz, k.m001);
    return k.m000;
}

}  // namespace clbm
