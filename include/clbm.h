/*
 * clbm.h -- C ABI of the GB300 (sm_103a) cascaded lattice Boltzmann
 * library: the fused stream-and-collide step of Fei, Luo & Li,
 * "Three-dimensional cascaded lattice Boltzmann method: improved
 * implementation and consistent forcing scheme" (arXiv:1801.04586),
 * on D3Q19 (Appendix A) or D3Q27 (Sec. II.A-B, Eqs. 12-16), together with
 * the collisions the paper compares it with on the same lattices: SRT
 * (Sec. III.A, Table I) and the non-orthogonal MRT of Appendix B.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Return value: CLBM_OK (0) or a negative CLBM_ERR_* code. No C++ exception
 *   crosses this boundary. clbm_last_error() gives a message for the calling
 *   thread's most recent failure.
 * - Lattice: nx x ny x nz nodes, node index s = (z*ny + y)*nx + x (x fastest),
 *   N = nx*ny*nz. Node spacing and time step are 1 (lattice units, c_s^2 = 1/3).
 * - Population arrays exchanged with the caller are float32, structure of
 *   arrays, f[i*N + s] for the Q = 19 velocities in the order of Eq. A1 (or
 *   Q = 27 in the order of Eq. 1, see clbm_params.lattice). Vector
 *   fields are 3 x N (component-major: F[a*N + s]); scalar fields are N.
 * - Every pointer marked _dev is a CUDA device pointer owned by the caller; it
 *   must stay valid until the work that uses it has finished on the context's
 *   stream. Pointers marked _host are ordinary host memory.
 * - All GPU work is enqueued on the stream given to clbm_create; entry points
 *   return without synchronising unless they say otherwise.
 * - "State at step n" is the post-streaming distribution f(x, n) of Eq. 8;
 *   rho and u are always Eq. 9 on that state (with the +F/2 term).
 * - The library stores populations internally as deviations h = f - w_i from
 *   the rest weights w = {1/3, 1/18, 1/36} in the chosen storage format; this
 *   changes rounding only, not the method.
 */
#ifndef CLBM_H
#define CLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define CLBM_OK            0
#define CLBM_ERR_ARG      -1  /* invalid argument (null pointer, bad size, bad rate) */
#define CLBM_ERR_OOM      -2  /* device allocation failed */
#define CLBM_ERR_CUDA     -3  /* a CUDA runtime call or kernel launch failed */
#define CLBM_ERR_UNSTABLE -4  /* a node's density left (0.1, 1.9) or became non-finite */
#define CLBM_ERR_STATE    -5  /* call not valid in the context's current state */
#define CLBM_ERR_TIMEOUT  -6  /* a step kernel's wait for its staged copies gave up (clbm_params.wait_cycles); the state is invalid */
#define CLBM_ERR_BOUNDS   -7  /* bounds-checked build only: a kernel derived an out-of-range index (see clbm_check) */

/* ---- storage formats of the populations (deviations f - w_i) ---- */
#define CLBM_STORAGE_F32     0
#define CLBM_STORAGE_F16     1  /* IEEE binary16, round to nearest even */
#define CLBM_STORAGE_BF16    2  /* bfloat16, round to nearest even */
/* Stochastic rounding of the step's stores: the value rounds up with
 * probability equal to the dropped fraction of a unit in the last place, so
 * stored deviations are unbiased and per-step increments far below the
 * format's resolution are not lost. The dither comes from a counter-based hash
 * of (step, node, direction): runs are reproducible. Initialisation and
 * clbm_set_populations round to nearest. Not available in batches. */
#define CLBM_STORAGE_F16_SR  3
#define CLBM_STORAGE_BF16_SR 4

/* ---- storage patterns of the population state ---- */
/* Two buffers: each step pulls from one and writes the other (Eq. 8 read
 * backwards). */
#define CLBM_PATTERN_AB 0
/* One buffer updated in place, alternating two step kinds: even steps read
 * and write the node's own slots (writing population i into the slot of its
 * opposite), odd steps read from and write to the neighbours' slots. Each node
 * writes exactly the slots it read, so no other node races it. Same results,
 * same bytes per node update, half the memory. The raw layout of the state
 * depends on the parity of the step count: clbm_export_state and
 * clbm_import_state move raw layouts, so import into a context whose step
 * count has the same parity. Not available for the recomputation and adjoint
 * entry points or in batches. */
#define CLBM_PATTERN_AA 1

/* ---- collision models ---- */
/* The paper's method: the cascaded (central-moment) collision of Eq. 5 with
 * the consistent forcing scheme (Eqs. A5-A6 / 15-16). */
#define CLBM_MODEL_CASCADED 0
/* Comparison models the paper measures against, on the same layout,
 * streaming and storage formats, for both lattices (one node per thread;
 * not in batches, not for the adjoint entry points):
 * SRT-LBM (Sec. III.A): one rate s2 (from nu), the second-order discrete
 * equilibrium written out in Sec. II.B and Guo's forcing term. */
#define CLBM_MODEL_SRT      1
/* Non-orthogonal MRT-LBM (Appendix B): the raw moments of Eq. A4 (Eq. 14 for
 * D3Q27) relaxed with the S of Eq. A3 (Eq. 13: nu, s2b, s3, s4 and for D3Q27
 * s3b, s4b, s5, s6) towards M f_D, with the forcing moments M R_G of Guo's
 * term. */
#define CLBM_MODEL_MRT      2

/* ---- wall axes: both faces of the axis are halfway bounce-back walls ---- */
#define CLBM_WALL_X 1u
#define CLBM_WALL_Y 2u
#define CLBM_WALL_Z 4u

/* Lattice and relaxation parameters.
 * nu:  kinematic viscosity, s2 = 1/(3 nu + 1/2) (Sec. II.B after Eq. 13); it
 *      relaxes k~110, k~101, k~011 and the normal-stress differences.
 * s2b: rate of the trace k~200 + k~020 + k~002 (bulk viscosity
 *      xi = 2/3 (1/s2b - 1/2) c_s^2); s3: third-order moments (Eq. A3);
 *      s4: fourth-order moments. Each must lie in (0, 2).
 * s0 = s1 = 1 (Sec. III); the method's result does not depend on them.
 * walls: CLBM_WALL_* bits; an axis without a bit is periodic.
 * block_x, block_y: CUDA block shape of the step kernel (block_x a multiple
 *      of 32, block_x*block_y <= 512); 0 selects the built-in default.
 * variant: step kernel form. 0 (the default): A/B steps with 16-bit storage,
 *      and the cascaded D3Q19 in-place (AA) steps with 16-bit storage, stage
 *      the rows they read in shared memory with bulk asynchronous copies
 *      where the geometry allows (nx <= 1024, nx a multiple of 8; D3Q27 not
 *      with a force field), one node per thread otherwise; 1: always one node per thread,
 *      plain loads (block_x, block_y apply); 2: two nodes per thread (x and
 *      x + block_x), collided together with the FP32x2 instructions (D3Q19
 *      only; measured slower on GB300 for every storage format, kept as an
 *      option). Forms 0 and 1 give bit-identical results; form 2 the same up
 *      to the rounding of fused operations.
 * lattice: 19 (or 0): D3Q19 of Appendix A (Eqs. A1-A6); 27: D3Q27 of Sec. II
 *      (velocities Eq. 1, moments Eq. 12, S Eq. 13, T~eq Eq. 15, C Eq. 16).
 *      D3Q27 runs the one-node-per-thread form (blocks of at most 256
 *      threads); the recomputation/adjoint entry points and batches are D3Q19
 *      only. Population arrays then hold 27 x N floats in the order of Eq. 1.
 * s3b, s4b, s5, s6: the further D3Q27 rates of Eq. 13 (k~111; k~211, k~121,
 *      k~112; k~122, k~212, k~221; k~222); 0 selects 1. Ignored for D3Q19.
 * slab, z0: the context holds the z-slab z0 .. z0 + nz - 1 of a larger lattice
 *      that is split along z across contexts (the decomposition of the
 *      streaming step, Eq. 8, across the z faces; see clbm_slab_step). slab
 *      bit 0 (CLBM_SLAB_LO): across the z- face the populations with e_z = +1
 *      (Eq. A1: 5, 11, 12, 15, 16) come from the neighbour below; bit 1
 *      (CLBM_SLAB_HI): across the z+ face the populations with e_z = -1 (6, 13,
 *      14, 17, 18) come from the neighbour above. Such a halo face is neither
 *      periodic nor a wall; a z face without its bit follows `walls` (periodic
 *      within the slab, or a wall with CLBM_WALL_Z). z0 is the global index of
 *      the slab's first plane: it only feeds the dither of stochastic
 *      rounding, so that the slabs store exactly what one undivided lattice
 *      would. slab = 0 (the default) is an ordinary lattice. Slabs: D3Q19,
 *      cascaded model, A/B pattern, variant 0 (16-bit storage staged where it
 *      applies) or 1.
 * wait_cycles: bound, in SM clock cycles, of each wait of the staged step
 *      (variant 0, 16-bit storage) for the bulk copies of its next tile; 0
 *      selects 4e9 (about 2 s). A wait that runs out makes the kernel give up
 *      the step and return: every block first waits (bounded by 4e9 cycles)
 *      for the copies it has in flight, then sets the flag that clbm_check
 *      reports as CLBM_ERR_TIMEOUT; the state is then invalid. Tests make a
 *      wait run out on purpose with inject = CLBM_INJECT_DROP_COPY. */
typedef struct clbm_params {
    int32_t nx, ny, nz;
    uint32_t walls;
    double nu;
    double s2b, s3, s4;
    int32_t storage;
    int32_t block_x, block_y;
    int32_t variant;
    int32_t lattice;
    int32_t pattern;          /* CLBM_PATTERN_AB (0) or CLBM_PATTERN_AA */
    double s3b, s4b, s5, s6;
    int32_t model;            /* CLBM_MODEL_CASCADED (0), CLBM_MODEL_SRT or CLBM_MODEL_MRT */
    int32_t slab;             /* 0, or CLBM_SLAB_LO | CLBM_SLAB_HI halo faces of a z-slab */
    int32_t z0;               /* global index of a z-slab's first plane (0 otherwise) */
    int32_t reserved;         /* must be 0 */
    int64_t wait_cycles;      /* staged step's wait bound in SM clock cycles (0: the default, about 2 s) */
    int32_t inject;           /* failure injection for tests: 0, or CLBM_INJECT_DROP_COPY */
    int32_t reserved2;        /* must be 0 */
} clbm_params;

/* Failure injection (clbm_params.inject), decided on the host: the staged
 * step arms the barrier of its first tile with the tile's byte count but
 * issues none of that tile's copies, so the waits on it run out after
 * wait_cycles and the step ends with CLBM_ERR_TIMEOUT. Nothing faults: no copy
 * is lost in flight, every wait is bounded. For failure-detection tests. */
#define CLBM_INJECT_DROP_COPY 1

#define CLBM_SLAB_LO 1
#define CLBM_SLAB_HI 2

typedef struct clbm_info {
    int64_t n_nodes;          /* N */
    int64_t pop_stride;       /* elements between consecutive population arrays */
    int64_t state_bytes;      /* bytes of one population buffer (19 * pop_stride * elem) */
    int64_t steps_done;       /* time steps since init */
    int32_t storage;
    int32_t block_x, block_y; /* block shape in use */
    double s2;                /* 1/(3 nu + 1/2) */
    int32_t nodes_per_thread; /* of the step kernel: 1 or 2 */
    int32_t q;                /* 19 or 27 */
    int32_t pattern;          /* CLBM_PATTERN_AB or CLBM_PATTERN_AA */
    int32_t buffers;          /* population buffers held: 2 (A/B) or 1 (AA) */
    int32_t model;            /* CLBM_MODEL_* */
    int32_t staged;           /* 1: steps stage the pulled rows in shared memory (variant 0, see clbm_params) */
    int32_t slab;             /* halo faces of a z-slab (clbm_params.slab) */
    int64_t face_bytes;       /* z-slab: bytes of one face's 5 populations (5 x nx x ny values), else 0 */
} clbm_info;

typedef struct clbm_ctx clbm_ctx;

/* Create a lattice context: validates p, allocates the population buffers
 * of Q * N elements each on the current CUDA device (two for the A/B
 * pattern, one for the in-place pattern), and binds the context to `stream`
 * (a cudaStream_t; NULL = legacy default stream).
 * The populations are zero deviations (f = w, rest at rho = 1) until an init
 * call. *out receives the context (owned by the caller; free with
 * clbm_destroy). Errors: CLBM_ERR_ARG, CLBM_ERR_OOM, CLBM_ERR_CUDA. */
int clbm_create(const clbm_params *p, void *stream, clbm_ctx **out);

/* Release all device memory of the context (synchronises its stream). NULL is
 * accepted. */
int clbm_destroy(clbm_ctx *ctx);

/* Fill *info with the context's sizes, layout and launch choices (see
 * clbm_info). No GPU work. Errors: CLBM_ERR_ARG for a NULL argument. */
int clbm_get_info(const clbm_ctx *ctx, clbm_info *info);

/* Body force (Sec. II.A, Eqs. 5-6 and 9; a force density). Exactly one force
 * source is active; the latest call wins. Uniform: F is the same at every node
 * (F = 0 after create). Profile along z: F_dev holds 3 x nz floats,
 * F_a(z) at F_dev[a*nz + z]. Field: F_dev holds 3 x N floats. Profile and
 * field pointers are borrowed, not copied: they must stay valid and unchanged
 * while steps run. */
int clbm_set_force_uniform(clbm_ctx *ctx, double fx, double fy, double fz);
int clbm_set_force_profile_z(clbm_ctx *ctx, const float *F_dev);
int clbm_set_force_field(clbm_ctx *ctx, const float *F_dev);

/* Time dependence of the body force: the force in use at time step t (in
 * Eq. 9 on the state f(t) and in the collision that advances it) becomes
 * F e^{-gamma t}, where F is the force set by clbm_set_force_* and t the
 * context's steps_done. gamma = 0 (the default) keeps the force static. The
 * decaying Taylor-Green force of Sec. III.D has this form. Initialisation uses
 * t = 0. The recomputation and adjoint entry points require gamma = 0
 * (CLBM_ERR_STATE otherwise). */
int clbm_set_force_decay(clbm_ctx *ctx, double gamma);

/* Initial state: at every node the generalized local equilibrium (Sec. II.B
 * after Eq. 15, central moments of Eq. A5) at density rho and velocity
 * u' = u - F/(2 rho), so that Eq. 9 returns exactly the given rho and u.
 * rho_dev (N floats) may be NULL for rho = 1; u_dev (3 x N) may be NULL for
 * u = 0. Uses the force set at the time of the call. Resets steps_done. */
int clbm_init_equilibrium(clbm_ctx *ctx, const float *rho_dev, const float *u_dev);

/* Advance nsteps >= 0 time steps. Each step is one launch of the fused pull
 * kernel: for every node it gathers the post-collision populations of the
 * neighbours (Eq. 8, periodic wrap, or halfway bounce-back f_i <- f*_ibar at
 * a wall face), forms rho and u (Eq. 9), raw moments T = M f (Eq. A4),
 * central moments N(u) T (Eq. 4), relaxes them with S, T~eq and C
 * (Eqs. 5, A3, A5, A6), maps back with N(u)^-1 = N(-u) and M^-1 (Eq. 7) and
 * stores f*. Asynchronous. For nsteps >= 32 with a static force and a storage
 * format without stochastic rounding, the steps are replayed from a CUDA graph
 * of 16 launches captured on first use (bit-identical results; the graph is
 * dropped when the force changes). */
int clbm_step(clbm_ctx *ctx, int64_t nsteps);

/* Eq. 9 on the current state: rho_dev (N floats) and u_dev (3 x N floats);
 * either may be NULL. */
int clbm_get_macros(clbm_ctx *ctx, float *rho_dev, float *u_dev);

/* Copy the current post-streaming populations out (Q x N floats). With
 * deviation != 0 the values are f - w_i, else f. */
int clbm_get_populations(clbm_ctx *ctx, float *f_dev, int deviation);

/* Replace the current state by the given post-streaming populations
 * (Q x N floats, f - w_i if deviation != 0, else f). Values are rounded to
 * the storage format. Resets steps_done. */
int clbm_set_populations(clbm_ctx *ctx, const float *f_dev, int deviation);

/* FP64 conservation sums over the current state (Eq. 9): out_dev[0] = sum rho,
 * out_dev[1..3] = sum rho*u (including the F/2 term). out_dev: 4 doubles on
 * the device. Deterministic (fixed reduction order). */
int clbm_reduce_moments(clbm_ctx *ctx, double *out_dev);

/* FP64 reductions of two float arrays of n elements, for error norms and
 * finite-difference dot products: out_dev[0] = sum (a-b)^2, out_dev[1] =
 * sum b^2, out_dev[2] = sum a*b. b_dev may be NULL (treated as zeros).
 * Deterministic. Runs on the context's stream. */
int clbm_reduce_pair(clbm_ctx *ctx, const float *a_dev, const float *b_dev, int64_t n, double *out_dev);

/* Read the instability flag (synchronises the stream): CLBM_OK, or
 * CLBM_ERR_UNSTABLE if any step since the last clear saw a density outside
 * (0.1, 1.9) or a non-finite one, or CLBM_ERR_TIMEOUT if a staged step's
 * wait for its bulk copies gave up (the state is then invalid). In the
 * bounds-checked debug build (libclbm_bc.so, compiled with
 * -DCLBM_BOUNDS_CHECK) every index a step or state kernel derives from the
 * streaming maps or a staged tile is checked against its buffer; a violation
 * is redirected in bounds and recorded, and this call then returns
 * CLBM_ERR_BOUNDS with the count and the first offending index in its
 * message. clear != 0 resets the flag and the record. */
int clbm_check(clbm_ctx *ctx, int clear);

/* Raw state: the internal population buffer (clbm_info.state_bytes bytes).
 * Device-to-device copies on the context's stream, for checkpoints. Importing
 * does not change steps_done unless set_steps >= 0, which sets it. */
int clbm_export_state(clbm_ctx *ctx, void *dst_dev);
int clbm_import_state(clbm_ctx *ctx, const void *src_dev, int64_t set_steps);

/* Checkpoint to / restore from host memory: a small header (geometry,
 * storage, steps_done) plus the raw buffer. clbm_save_state with
 * host_buf == NULL writes the required size to *bytes. Both synchronise. A
 * restored context continues bit-identically. */
int clbm_save_state(clbm_ctx *ctx, void *host_buf, size_t *bytes);
int clbm_load_state(clbm_ctx *ctx, const void *host_buf, size_t bytes);

/* One user job with host buffers: copy rho_host (N floats, may be NULL) and
 * u_host (3 x N, may be NULL) to the device, initialise as
 * clbm_init_equilibrium, run nsteps steps, then copy Eq. 9 rho and u of the
 * final state back to rho_out_host / u_out_host (either may be NULL). If
 * moments_host is not NULL it receives 4 * (nsteps + 1) doubles: entry k
 * (k = 0..nsteps) holds the FP64 sums of clbm_reduce_moments for the state at
 * step k. With the cascaded collision, the A/B pattern and D3Q19 they are
 * formed inside step k+1's kernel from the state it pulls (exact fixed-point
 * warp sums, no extra pass over the populations), totalled by the next
 * step's launch and copied back on a second stream of the context while
 * the following steps run. Otherwise they come from one
 * clbm_reduce_moments pass before each step, copied back asynchronously.
 * The last comes from one reduction after the final step, beside the copies
 * back. With D3Q19 the host copies travel in up to 8 chunks of z-planes on a
 * second stream, each chunk initialised (and read out) as soon as it has
 * landed (been stepped). When the fused step with sums runs, it also steps the
 * first two steps chunk by chunk as the input lands, and the last step chunk by
 * chunk, each chunk read out and copied back as soon as it and its two
 * neighbouring chunks are stepped; the results are the same bit for bit. The call synchronises once, at the end, then returns
 * CLBM_ERR_UNSTABLE if any mass sum is non-finite or the instability flag is
 * set. Device scratch for the staging fields and partial sums is allocated
 * on first use and kept by the context. Host buffers should be pinned for
 * full copy speed and for the copies to overlap the steps. */
int clbm_run_host(clbm_ctx *ctx, const float *rho_host, const float *u_host, int64_t nsteps,
                  float *rho_out_host, float *u_out_host, double *moments_host);

/* ---- recomputation and adjoint (FP32 storage only; CLBM_ERR_ARG otherwise) ----
 *
 * A "raw state" is a device buffer of clbm_info.state_bytes bytes in the
 * context's internal layout (clbm_export_state); pulling it gives the
 * post-streaming state f^t. Adjoint arrays (lam, 19 x N floats) are in the
 * post-streaming layout f[i*N + s]: lam^t = dL/df^t.
 *
 * clbm_step_raw: one time step (as clbm_step) from src_dev into dst_dev with
 * the context's parameters and force; the context's own state and step count
 * are untouched. src_dev and dst_dev must not overlap.
 *
 * clbm_adjoint_seed: start the adjoint from a cotangent gu_dev (3 x N floats)
 * on the Eq. 9 velocity of the state in state_dev (NULL: the context's current
 * state): lam_i = sum_a gu_a (e_ia - u_a)/rho is written to lam_dev, and
 * gF_dev (3 x N) is SET to the direct term gu/(2 rho) of Eq. 9.
 *
 * clbm_adjoint_step: adjoint of the step f^{t+1} = P C(f^t, F) (Eqs. 5, 7, 8,
 * 9), with f^t the pull of state_dev: lam_dev = J_f^T lam*, where lam* is
 * lam_next_dev read at the slot each population streams into (periodic wrap,
 * or its opposite at its own node across a wall face; on a z-slab, across a
 * halo face, from lam_next_dev's receive planes, see the z-slab section),
 * and gF_dev +=
 * J_F^T lam* (dL/dF of a force field, accumulated). lam_dev must not alias
 * lam_next_dev. The force in use is the context's (any mode; for a uniform or
 * profile force gF is still per node). */
int clbm_step_raw(clbm_ctx *ctx, const void *src_dev, void *dst_dev);

/* Backward pass over one checkpointed segment of k >= 1 steps (Eqs. 5, 7, 8,
 * 9 reversed): recompute the segment's states 1..k-1 from its checkpoint
 * ckpt_dev (state 0, a raw state) into tape_dev ((k-1) * state_bytes bytes,
 * may be NULL when k == 1), then apply clbm_adjoint_step k times back to
 * front. On entry lam_dev holds the adjoint at the end of the segment; on
 * return it holds the adjoint at its start. lam_tmp_dev (19 x N floats) is
 * scratch; gF_dev accumulates dL/dF. One call replaces 2k - 1 launches issued
 * from the caller. */
int clbm_adjoint_segment(clbm_ctx *ctx, const void *ckpt_dev, void *tape_dev, int64_t k, float *lam_dev,
                         float *lam_tmp_dev, float *gF_dev);
int clbm_adjoint_seed(clbm_ctx *ctx, const void *state_dev, const float *gu_dev, float *lam_dev, float *gF_dev);
int clbm_adjoint_step(clbm_ctx *ctx, const void *state_dev, const float *lam_next_dev, float *lam_dev,
                      float *gF_dev);

/* ---- z-slab decomposition (clbm_params.slab) ----
 *
 * One lattice split along z into slabs, one context each (for example one
 * per GPU). The pull of Eq. 8 at a slab's first plane needs, for the 5
 * populations with e_z = +1, the post-collision values of the last plane of
 * the slab below; at its last plane, for the 5 with e_z = -1, those of the
 * first plane of the slab above. A slab context keeps these in halo planes
 * of its state and writes its own outgoing values to send planes, so one
 * time step of the whole lattice is: every slab steps, then every pair of
 * neighbours exchanges one face each way (5 x nx x ny values). The interior
 * update is the same kernel arithmetic as clbm_step; the slabs together give
 * bit for bit the state of one undivided lattice.
 *
 * Initialisation (clbm_init_equilibrium, clbm_set_populations) needs no
 * exchange: it fills the slab's halo planes from its own state. After every
 * step, before the next step or any read-out (clbm_get_macros,
 * clbm_get_populations, clbm_reduce_moments), the caller must move each
 * face: the first half of this slab's send planes (its first plane's e_z = -1
 * populations) into the second half of the lower neighbour's receive planes,
 * and the second half of the send planes (its last plane's e_z = +1
 * populations) into the first half of the upper neighbour's receive planes.
 * A slab with both halo faces may be its own neighbour (a periodic z axis on
 * one context). clbm_step on a slab context takes at most one step per call.
 * Slab contexts refuse clbm_run_host and clbm_adjoint_segment, whose inner
 * steps would need exchanges (CLBM_ERR_STATE).
 *
 * Recomputation and adjoint on slabs (the reverse-direction halo):
 * clbm_step_raw steps every plane of a raw state through the halo map and
 * writes dst's send planes; the caller moves dst's faces as above (the halo
 * planes of a raw state follow its q x pop_stride values: 10 receive, then 10
 * send planes of nx x ny values). The adjoint gathers lambda from the node
 * each population streams into, so at the slab's last plane the e_z = +1
 * populations need the upper neighbour's first-plane lambda, and at its first
 * plane the e_z = -1 populations the lower neighbour's last-plane lambda. The
 * adjoint arrays of a slab (lam_dev, lam_next_dev) therefore hold 19 x N
 * floats, then 10 receive planes (0-4 from the lower neighbour, populations
 * 6, 13, 14, 17, 18; 5-9 from the upper neighbour, populations 5, 11, 12,
 * 15, 16), then 10 send planes that clbm_adjoint_seed and clbm_adjoint_step
 * write (10-14: this slab's first-plane lambda of 5, 11, 12, 15, 16; 15-19:
 * its last-plane lambda of 6, 13, 14, 17, 18); each plane is nx x ny floats.
 * Before the next adjoint step the caller moves them like the population
 * faces: the first half of the send planes into the second half of the lower
 * neighbour's receive planes, the second half into the first half of the
 * upper neighbour's. The slabs' lambda and dL/dF then equal those of one
 * undivided lattice bit for bit. */
#define CLBM_SLAB_ALL      0  /* the whole step, then the state advances */
#define CLBM_SLAB_FACES    1  /* only the first and last planes (the send planes are then complete) */
#define CLBM_SLAB_INTERIOR 2  /* the other planes, then the state advances (after CLBM_SLAB_FACES) */

/* Enqueue one time step, or a part of it, on the context's stream. Splitting
 * the step lets the face exchange overlap the interior update: after
 * CLBM_SLAB_FACES the send planes are complete (once that work has run) and
 * the receive planes of the new state may be written while
 * CLBM_SLAB_INTERIOR runs. Errors: CLBM_ERR_ARG (not a slab context, unknown
 * part), CLBM_ERR_STATE (CLBM_SLAB_INTERIOR without CLBM_SLAB_FACES before
 * it, or another part while a split step is pending). */
int clbm_slab_step(clbm_ctx *ctx, int part);

/* Device addresses of the newest state's send and receive planes (the
 * state the latest step writes, even before CLBM_SLAB_INTERIOR finishes it).
 * Each is 10 planes of nx x ny values in the storage format (x fastest),
 * 2 * face_bytes bytes: send_dev first holds the slab's first plane's e_z = -1
 * populations (6, 13, 14, 17, 18) for the lower neighbour, then its last
 * plane's e_z = +1 populations (5, 11, 12, 15, 16) for the upper neighbour;
 * recv_dev first takes the lower neighbour's e_z = +1 face, then the upper
 * neighbour's e_z = -1 face. The addresses belong to the context and change
 * from step to step (the A/B buffers alternate): query them after each step.
 * Any output pointer may be NULL. Errors: CLBM_ERR_ARG (not a slab context). */
int clbm_slab_faces(clbm_ctx *ctx, void **send_dev, void **recv_dev, int64_t *face_bytes);

/* ---- FP64 pair reduction without a context or allocation ----
 *
 * Same sums as clbm_reduce_pair (out_dev[0] = sum (a-b)^2, out_dev[1] =
 * sum b^2, out_dev[2] = sum a*b over n floats; b_dev may be NULL), enqueued on
 * `stream` (a cudaStream_t, NULL = legacy default) of the current device. The
 * paper has no counterpart: this exists for callers that cannot allocate
 * device memory, because cudaMalloc/cudaFree can synchronise the device and
 * can fail with out-of-memory (for example a hook inside a running simulation,
 * or code beside a caching allocator that holds nearly all device memory).
 * It allocates nothing and needs no context: the per-block partial sums live
 * in a fixed 384 KiB __device__ array that every GPU loading the library holds
 * until exit. n may not exceed 134,217,728 (CLBM_ERR_ARG, with a message).
 * The first call on each device is its set-up: it looks up that array's
 * device address and caches it for the process. Under CUDA's lazy module
 * loading (the default since CUDA 12.2) that first call may also load the
 * library's device code, which allocates the array and the code and may
 * synchronise; make it once at set-up, before any stream capture. Later calls
 * allocate nothing. The cached address belongs to the device's primary
 * context: after cudaDeviceReset (or anything else that destroys that
 * context) later calls would use a stale address and must not be made.
 * All calls on a device share the array: calls that overlap on the GPU
 * (different streams, or other host threads) race and must be serialised by
 * the caller. The sums may differ from clbm_reduce_pair's in the last bits
 * (different block count). */
int clbm_reduce_pair_noalloc(const float *a_dev, const float *b_dev, int64_t n, double *out_dev, void *stream);

/* ---- many independent lattices in one launch per step ----
 *
 * A batch holds ndomains complete lattices, each with its own extents, walls,
 * rates (as clbm_params) and uniform body force, all in one storage format.
 * Each domain follows exactly the per-node update of clbm_step. The batch
 * steps all domains with one launch per time step: a grid of (SMs x resident
 * blocks) walks a work list of tiles, each `threads` consecutive nodes of one
 * domain in its linear index. The batch owns its population buffers. */
typedef struct clbm_domain {
    int32_t nx, ny, nz;
    uint32_t walls;
    double nu, s2b, s3, s4;
    double fx, fy, fz;
} clbm_domain;

typedef struct clbm_batch_info {
    int32_t ndomains;
    int32_t ntiles, grid, threads, graph_steps;
    int64_t total_nodes;
    int64_t state_bytes;   /* both buffers: 2 x state_bytes are allocated */
    int64_t steps_done;
    int32_t pattern;       /* CLBM_PATTERN_AB or CLBM_PATTERN_AA */
    int32_t buffers;       /* population buffers allocated: 2 (A/B) or 1 (in place) */
} clbm_batch_info;

/* Step modes of clbm_batch_step. */
#define CLBM_BATCH_GRAPH       0  /* one launch per step, replayed from a captured CUDA graph */
#define CLBM_BATCH_DIRECT      1  /* one launch per step, issued directly */
#define CLBM_BATCH_PER_DOMAIN  2  /* one clbm_step-style launch per domain per step (reference schedule) */

typedef struct clbm_batch clbm_batch;

/* Create: validates every domain as clbm_create does, allocates the A/B
 * population buffers of all domains and a work list for 256-thread tiles,
 * binds to `stream`. Populations start at rest (f = w). Errors: CLBM_ERR_ARG,
 * CLBM_ERR_OOM, CLBM_ERR_CUDA. */
int clbm_batch_create(const clbm_domain *domains, int32_t ndomains, int32_t storage, void *stream,
                      clbm_batch **out);
/* The same with a storage pattern: CLBM_PATTERN_AB (what clbm_batch_create
 * makes) or CLBM_PATTERN_AA, one population buffer per domain updated in
 * place by alternating even and odd steps (as clbm_params.pattern): half the
 * memory, the same bits. clbm_batch_autotune then keeps a temporary copy of
 * the state for its trials. */
int clbm_batch_create_pattern(const clbm_domain *domains, int32_t ndomains, int32_t storage, int32_t pattern,
                              void *stream, clbm_batch **out);
int clbm_batch_destroy(clbm_batch *b);
int clbm_batch_get_info(const clbm_batch *b, clbm_batch_info *info);
/* Rebuild the work list for another block size (threads per block and
 * nodes per tile: a multiple of 32 in [32, 512]). Synchronises the stream. */
int clbm_batch_set_tile(clbm_batch *b, int32_t threads);
/* Time trial_steps launches for each block size in {64, 128, 192, 256, 384,
 * 512} (trials read the current state and write the other buffer, so the
 * state is not changed), keep the fastest and report it. Synchronises. */
int clbm_batch_autotune(clbm_batch *b, int32_t trial_steps, int32_t *threads_out);
/* Every domain to the generalized equilibrium at rho = 1, u = 0 (u' = -F/2). */
int clbm_batch_init_equilibrium(clbm_batch *b);
/* Advance every domain by nsteps steps with the given CLBM_BATCH_* mode. The
 * graph mode captures graph_steps steps once (on a private stream) and replays
 * them; remaining steps are launched directly. */
int clbm_batch_step(clbm_batch *b, int64_t nsteps, int32_t mode);
/* Per-domain read-out and state, as clbm_get_macros / clbm_get_populations /
 * clbm_set_populations with the domain's N. */
int clbm_batch_get_macros(clbm_batch *b, int32_t domain, float *rho_dev, float *u_dev);
int clbm_batch_get_populations(clbm_batch *b, int32_t domain, float *f_dev, int deviation);
int clbm_batch_set_populations(clbm_batch *b, int32_t domain, const float *f_dev, int deviation);
/* Instability flag of the batch, as clbm_check. */
int clbm_batch_check(clbm_batch *b, int clear);

/* Text for a status code; clbm_last_error(): message of this thread's last
 * failure ("" if none). Both strings are owned by the library. */
const char *clbm_status_string(int status);
const char *clbm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CLBM_H */
