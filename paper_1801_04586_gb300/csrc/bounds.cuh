// bounds.cuh -- index checks of the bounds-checked debug build.
//
// Built with -DCLBM_BOUNDS_CHECK (libclbm_bc.so), every element index that a
// step or state kernel derives from the pull map of Eq. 8, the push map of the
// in-place pattern or a staged tile is checked before the access: state
// buffer indices against the buffer's extent (Geom::bc_limit elements: the Q
// population arrays plus a z-slab's halo planes), shared-memory indices of a
// staged tile against the tile pitch, and the rows a bulk copy moves against
// both. A violation is counted in the context's record (Geom::bc: the count
// and the first offending index, tagged with the kind of access), and the
// access is redirected to element 0 of the same buffer, so nothing outside the
// buffers is touched; clbm_check then reports CLBM_ERR_BOUNDS. In the normal
// build the macros are the bare index and the record does not exist.
#pragma once

#include <stdint.h>

namespace clbm {

// Kinds of checked access (the top byte of BoundsRecord::first).
enum BoundsKind : unsigned {
    kBcGlobal = 1,  // a state-buffer element of a step or state kernel
    kBcShared = 2,  // a staged tile's element in shared memory
    kBcCopy = 3,    // the rows of a bulk copy (source or destination)
};

struct BoundsRecord {
    unsigned long long count;  // violations since the last clbm_check(clear)
    unsigned long long first;  // kind << 56 | index of the first one
};

#ifdef CLBM_BOUNDS_CHECK
__device__ __forceinline__ void bc_record(BoundsRecord *rec, uint64_t idx, unsigned kind) {
    if (rec && atomicAdd(&rec->count, 1ull) == 0ull)
        rec->first = ((unsigned long long)kind << 56) | (idx & 0x00ffffffffffffffull);
}
__device__ __forceinline__ uint64_t bc_check(BoundsRecord *rec, uint64_t idx, uint64_t limit, unsigned kind) {
    if (idx < limit) return idx;
    bc_record(rec, idx, kind);
    return 0;
}
__device__ __forceinline__ bool bc_range(BoundsRecord *rec, uint64_t first, uint64_t count, uint64_t limit) {
    if (first + count <= limit) return true;
    bc_record(rec, first + count - 1u, kBcCopy);
    return false;
}
__device__ __forceinline__ uint64_t bc_slots(BoundsRecord *rec, uint64_t base, uint64_t last, uint64_t limit) {
    if (base + last < limit) return base;
    bc_record(rec, base + last, kBcGlobal);
    return 0;
}
// A state-buffer index of geometry g.
#define CLBM_IDX(g, idx) ::clbm::bc_check((g).bc, (uint64_t)(idx), (g).bc_limit, ::clbm::kBcGlobal)
// A shared-memory element index below `limit`.
#define CLBM_SIDX(g, idx, limit) ::clbm::bc_check((g).bc, (uint64_t)(idx), (uint64_t)(limit), ::clbm::kBcShared)
// The first slot of a node whose slots run from base to base + last: base if
// base + last is a state-buffer index of g, else 0 (recorded).
#define CLBM_SLOTS(g, base, last) ::clbm::bc_slots((g).bc, (uint64_t)(base), (uint64_t)(last), (g).bc_limit)
// Whether the elements [first, first + count) lie below limit (a bulk copy); records if not.
#define CLBM_RANGE_OK(g, first, count, limit) \
    ::clbm::bc_range((g).bc, (uint64_t)(first), (uint64_t)(count), (uint64_t)(limit))
#else
#define CLBM_IDX(g, idx) (idx)
#define CLBM_SIDX(g, idx, limit) (idx)
#define CLBM_SLOTS(g, base, last) (base)
#define CLBM_RANGE_OK(g, first, count, limit) true
#endif

}  // namespace clbm
