/*
 * clbm_oracle.c -- plain, slow FP64 CPU oracle for the D3Q19 cascaded lattice
 * Boltzmann method (CLBM) with the consistent forcing scheme of
 * Fei, Luo & Li, "Three-dimensional cascaded lattice Boltzmann method:
 * improved implementation and consistent forcing scheme" (arXiv:1801.04586).
 *
 * TEST INFRASTRUCTURE. This library exists to check the GPU path. Only the
 * test suite, the package smoke check and the benchmark's CPU-baseline leg may
 * load it. It shares no code, header, table or helper with the CUDA library.
 *
 * Built twice from this one source: ORACLE_Q = 19 (Appendix A, exported as
 * ora_*) and ORACLE_Q = 27 (Sec. II, the paper's main development, exported
 * as ora27_*). The lattice enters only through the tables below.
 *
 * What it computes (everything in double precision):
 *   - The velocities in the order of Eq. A1 (Eq. 1), the simplified
 *     central-moment set of Eq. A2 (Eq. 12), M built from its definition
 *     (Eq. 4), M^-1 by Gauss-Jordan.
 *   - Per node, the algorithm of Sec. II.B: Step 1 central moments straight
 *     from Eq. 2 (no M, no N); Step 2 the collision of Eq. 5 with the dense
 *     block-diagonal S of Eq. A3 (Eq. 13), T~eq of Eq. A5 (Eq. 15) and C of
 *     Eq. A6 (Eq. 16); Step 3
 *     T* = N(u)^-1 T~* by a dense solve and f* = M^-1 T*; Step 4 push streaming
 *     (Eq. 8) with periodic faces or halfway bounce-back walls, and Eq. 9.
 *   - An adjoint of one step: per-node Jacobians by complex-step
 *     differentiation of the same collision code, transposed, and the
 *     transposed streaming map.
 *   - The two comparison collision models the paper sets beside the cascaded
 *     one (model field of ora_lattice): the SRT-LBM with the discrete
 *     equilibrium of Sec. II.B and Guo's forcing term (Sec. III.A), and the
 *     non-orthogonal raw-moment MRT-LBM of Appendix B on the same M and S.
 *     The lattice weights they use are the generalized equilibrium at rest,
 *     rho = 1, u = 0.
 *
 * Readings of points the paper leaves open or prints garbled:
 *   - Eq. 2 prints (e_iy - u_z)^p as the third factor; read (e_iz - u_z)^p.
 *   - Eqs. A2 and 12 list k~020 twice; the tenth moment is k~002 (M row 9 is
 *     e_z^2 in both printed matrices).
 *   - S uses s_nu for k~110, k~101, k~011 and s_2 in the viscosity relation; we
 *     read s_nu = s_2 (the deviatoric eigenvalue of the 3x3 block is s_2).
 *   - Halfway bounce-back: a population whose streaming destination lies
 *     beyond a wall face (on any wall axis, so duct edge links included)
 *     returns to its own node in the opposite direction: f_ibar(x,t+1) =
 *     f*_i(x,t). Walls carry no velocity.
 *   - Time step dt = 1, so Eq. 9 carries +F/2; F is a force density.
 *   - Initial state: the generalized equilibrium with u' = u - F/(2 rho), so
 *     that Eq. 9 returns the prescribed u.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORACLE_Q
#define ORACLE_Q 19
#endif
#define Q ORACLE_Q
#define CS2 (1.0 / 3.0)

#if ORACLE_Q == 27
#define ORA(name) ora27_##name
/* Eq. 1 (D3Q27). */
static const int EV[Q][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, 1, 0}, {1, -1, 0}, {-1, -1, 0},
    {1, 0, 1}, {-1, 0, 1}, {1, 0, -1}, {-1, 0, -1},
    {0, 1, 1}, {0, -1, 1}, {0, 1, -1}, {0, -1, -1},
    {1, 1, 1}, {-1, 1, 1}, {1, -1, 1}, {-1, -1, 1},
    {1, 1, -1}, {-1, 1, -1}, {1, -1, -1}, {-1, -1, -1},
};
/* Eq. 12: exponents of the simplified central-moment set. */
static const int MOM[Q][3] = {
    {0, 0, 0},
    {1, 0, 0}, {0, 1, 0}, {0, 0, 1},
    {1, 1, 0}, {1, 0, 1}, {0, 1, 1},
    {2, 0, 0}, {0, 2, 0}, {0, 0, 2},
    {1, 2, 0}, {1, 0, 2}, {2, 1, 0}, {2, 0, 1}, {0, 1, 2}, {0, 2, 1},
    {1, 1, 1},
    {2, 2, 0}, {2, 0, 2}, {0, 2, 2},
    {2, 1, 1}, {1, 2, 1}, {1, 1, 2},
    {1, 2, 2}, {2, 1, 2}, {2, 2, 1},
    {2, 2, 2},
};
/* Eq. 15: T~eq_j = rho c_s^(2 p) with p = TEQ_POW[j], 0 where p < 0. */
static const int TEQ_POW[Q] = {0,  -1, -1, -1, -1, -1, -1, 1,  1,  1,  -1, -1, -1, -1,
                               -1, -1, -1, 2,  2,  2,  -1, -1, -1, -1, -1, -1, 3};
/* Eq. 16: C_j = F_a c_s^(2 p) with a = CF_AXIS[j] (-1: zero), p = CF_POW[j]. */
static const int CF_AXIS[Q] = {-1, 0,  1,  2,  -1, -1, -1, -1, -1, -1, 0, 0, 1, 2,
                               1,  2,  -1, -1, -1, -1, -1, -1, -1, 0,  1, 2, -1};
static const int CF_POW[Q] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 0, 0, 0, 0, 0, 0, 0, 2, 2, 2, 0};
#else
#define ORA(name) ora_##name
/* Eq. A1 (D3Q19): rest, +-x, +-y, +-z, xy, xz, yz diagonals. */
static const int EV[Q][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, 1, 0}, {1, -1, 0}, {-1, -1, 0},
    {1, 0, 1}, {-1, 0, 1}, {1, 0, -1}, {-1, 0, -1},
    {0, 1, 1}, {0, -1, 1}, {0, 1, -1}, {0, -1, -1},
};

/* Eq. A2: exponents (m,n,p) of the simplified central-moment set. */
static const int MOM[Q][3] = {
    {0, 0, 0},
    {1, 0, 0}, {0, 1, 0}, {0, 0, 1},
    {1, 1, 0}, {1, 0, 1}, {0, 1, 1},
    {2, 0, 0}, {0, 2, 0}, {0, 0, 2},
    {1, 2, 0}, {1, 0, 2}, {2, 1, 0}, {2, 0, 1}, {0, 1, 2}, {0, 2, 1},
    {2, 2, 0}, {2, 0, 2}, {0, 2, 2},
};
/* Eq. A5: T~eq_j = rho c_s^(2 p) with p = TEQ_POW[j], 0 where p < 0. */
static const int TEQ_POW[Q] = {0, -1, -1, -1, -1, -1, -1, 1, 1, 1, -1, -1, -1, -1, -1, -1, 2, 2, 2};
/* Eq. A6: C_j = F_a c_s^(2 p) with a = CF_AXIS[j] (-1: zero), p = CF_POW[j]. */
static const int CF_AXIS[Q] = {-1, 0, 1, 2, -1, -1, -1, -1, -1, -1, 0, 0, 1, 2, 1, 2, -1, -1, -1};
static const int CF_POW[Q] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 0, 0, 0};
#endif

typedef struct {
    int nx, ny, nz;
    int walls;          /* bit 0: x faces are walls, bit 1: y, bit 2: z */
    double s0, s1, s2, s2b, s3, s4;
    double s3b, s4b, s5, s6;  /* D3Q27 only (Eq. 13) */
    int model;          /* 0: cascaded (Sec. II); 1: SRT-LBM (rate s2); 2: non-orthogonal MRT (Appendix B) */
    int pad;
} ora_lattice;

static int binom(int n, int k)
{
    int r = 1;
    for (int i = 0; i < k; ++i) r = r * (n - i) / (i + 1);
    return r;
}

static int moment_index(int a, int b, int c)
{
    for (int j = 0; j < Q; ++j)
        if (MOM[j][0] == a && MOM[j][1] == b && MOM[j][2] == c) return j;
    abort(); /* the set of Eq. A2 is closed under lowering an exponent */
}

static int opposite(int i)
{
    for (int k = 0; k < Q; ++k)
        if (EV[k][0] == -EV[i][0] && EV[k][1] == -EV[i][1] && EV[k][2] == -EV[i][2]) return k;
    abort();
}

/* ---- node arithmetic, real and complex instantiations ---- */
#define REAL double
#define SFX(name) name##_r
#define RE(x) (x)
#include "oracle_node.inc"
#undef REAL
#undef SFX
#undef RE

#define REAL double complex
#define SFX(name) name##_c
#define RE(x) creal(x)
#include "oracle_node.inc"
#undef REAL
#undef SFX
#undef RE

/* ---- constant matrices ---- */

/* Eq. 4 with Eq. A2: M[j][i] = e_ix^m e_iy^n e_iz^p. */
static void build_M(double M[Q][Q])
{
    for (int j = 0; j < Q; ++j)
        for (int i = 0; i < Q; ++i)
            M[j][i] = ipow_r((double)EV[i][0], MOM[j][0]) * ipow_r((double)EV[i][1], MOM[j][1])
                    * ipow_r((double)EV[i][2], MOM[j][2]);
}

/* M^-1 by Gauss-Jordan elimination with partial pivoting. */
static void build_Minv(double Minv[Q][Q])
{
    double A[Q][2 * Q];
    double M[Q][Q];
    build_M(M);
    for (int r = 0; r < Q; ++r)
        for (int c = 0; c < 2 * Q; ++c) A[r][c] = c < Q ? M[r][c] : (c - Q == r ? 1.0 : 0.0);
    for (int col = 0; col < Q; ++col) {
        int piv = col;
        for (int r = col + 1; r < Q; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        for (int c = 0; c < 2 * Q; ++c) { double t = A[col][c]; A[col][c] = A[piv][c]; A[piv][c] = t; }
        double d = A[col][col];
        for (int c = 0; c < 2 * Q; ++c) A[col][c] /= d;
        for (int r = 0; r < Q; ++r) {
            if (r == col) continue;
            double fac = A[r][col];
            if (fac == 0.0) continue;
            for (int c = 0; c < 2 * Q; ++c) A[r][c] -= fac * A[col][c];
        }
    }
    for (int r = 0; r < Q; ++r)
        for (int c = 0; c < Q; ++c) Minv[r][c] = A[r][Q + c];
}

/* Eq. A3 (D3Q19) or Eq. 13 (D3Q27) with s_nu read as s_2,
 * s_+ = (s2b + 2 s2)/3, s_- = (s2b - s2)/3. */
static void build_S(const ora_lattice *L, double S[Q][Q])
{
    memset(S, 0, sizeof(double) * Q * Q);
    double sp = (L->s2b + 2.0 * L->s2) / 3.0, sm = (L->s2b - L->s2) / 3.0;
    S[0][0] = L->s0;
    for (int j = 1; j <= 3; ++j) S[j][j] = L->s1;
    for (int j = 4; j <= 6; ++j) S[j][j] = L->s2;
    for (int r = 7; r <= 9; ++r)
        for (int c = 7; c <= 9; ++c) S[r][c] = (r == c) ? sp : sm;
    for (int j = 10; j <= 15; ++j) S[j][j] = L->s3;
#if ORACLE_Q == 27
    S[16][16] = L->s3b;
    for (int j = 17; j <= 19; ++j) S[j][j] = L->s4;
    for (int j = 20; j <= 22; ++j) S[j][j] = L->s4b;
    for (int j = 23; j <= 25; ++j) S[j][j] = L->s5;
    S[26][26] = L->s6;
#else
    for (int j = 16; j <= 18; ++j) S[j][j] = L->s4;
#endif
}

static double g_M[Q][Q];
static double g_Minv[Q][Q];
static double g_w[Q];
static int g_ready = 0;

static void ensure_ready(void)
{
    if (!g_ready) {
        build_M(g_M);
        build_Minv(g_Minv);
        double u0[3] = {0.0, 0.0, 0.0};
        equilibrium_r(g_Minv, 1.0, u0, g_w);  /* lattice weights */
        g_ready = 1;
    }
}

/* One collision of the lattice's model. */
static void collide_model_r(const ora_lattice *L, const double S[Q][Q], const double f[Q], const double F[3],
                            double fs[Q])
{
    if (L->model == 1) collide_srt_r(L->s2, g_w, f, F, fs);
    else if (L->model == 2) collide_mrt_r(S, g_M, g_Minv, g_w, f, F, fs);
    else collide_r(S, g_Minv, f, F, fs);
}

static void collide_model_c(const ora_lattice *L, const double S[Q][Q], const double complex f[Q],
                            const double complex F[3], double complex fs[Q])
{
    if (L->model == 1) collide_srt_c(L->s2, g_w, f, F, fs);
    else if (L->model == 2) collide_mrt_c(S, g_M, g_Minv, g_w, f, F, fs);
    else collide_c(S, g_Minv, f, F, fs);
}

/* ---- exported: tables and matrices ---- */

void ORA(velocities)(int *e)
{
    for (int i = 0; i < Q; ++i)
        for (int a = 0; a < 3; ++a) e[3 * i + a] = EV[i][a];
}

void ORA(moment_exponents)(int *m)
{
    for (int j = 0; j < Q; ++j)
        for (int a = 0; a < 3; ++a) m[3 * j + a] = MOM[j][a];
}

void ORA(matrix_M)(double *out)
{
    double M[Q][Q];
    build_M(M);
    memcpy(out, M, sizeof(M));
}

void ORA(matrix_Minv)(double *out)
{
    ensure_ready();
    memcpy(out, g_Minv, sizeof(g_Minv));
}

void ORA(matrix_N)(const double *u, double *out)
{
    double N[Q][Q];
    shift_matrix_r(u, N);
    memcpy(out, N, sizeof(N));
}

void ORA(matrix_S)(const ora_lattice *L, double *out)
{
    double S[Q][Q];
    build_S(L, S);
    memcpy(out, S, sizeof(S));
}

void ORA(teq)(double rho, double *out) { teq_r(rho, out); }
void ORA(cforce)(const double *F, double *out) { cforce_r(F, out); }

void ORA(central_moments)(const double *f, const double *u, double *kt) { central_moments_r(f, u, kt); }

void ORA(macros_node)(const double *f, const double *F, double *rho, double *u) { macros_r(f, F, rho, u); }

void ORA(collide)(const ora_lattice *L, const double *f, const double *F, double *fs)
{
    ensure_ready();
    double S[Q][Q];
    build_S(L, S);
    collide_model_r(L, S, f, F, fs);
}

/* The discrete equilibrium of Sec. II.B and Guo's forcing term (Appendix B). */
void ORA(feq_discrete)(double rho, const double *u, double *feq)
{
    ensure_ready();
    feq_discrete_r(g_w, rho, u, feq);
}

void ORA(guo_force)(const double *u, const double *F, double *R)
{
    ensure_ready();
    guo_force_r(g_w, u, F, R);
}

void ORA(equilibrium)(double rho, const double *u, double *feq)
{
    ensure_ready();
    equilibrium_r(g_Minv, rho, u, feq);
}

/* ---- lattice operations. Arrays are SoA: a[i*N + node], node = (z*ny + y)*nx + x. ---- */

static long lattice_n(const ora_lattice *L) { return (long)L->nx * L->ny * L->nz; }

/* Destination of population i leaving node (x,y,z) under Eq. 8: returns the
 * destination node and writes the arriving direction (i itself, or its
 * opposite when the link leaves through a wall face: halfway bounce-back). */
static long push_target(const ora_lattice *L, int x, int y, int z, int i, int *dir)
{
    int n[3] = {L->nx, L->ny, L->nz};
    int c[3] = {x + EV[i][0], y + EV[i][1], z + EV[i][2]};
    int beyond_wall = 0;
    for (int a = 0; a < 3; ++a) {
        if (c[a] < 0 || c[a] >= n[a]) {
            if (L->walls & (1 << a)) beyond_wall = 1;
            else c[a] = (c[a] + n[a]) % n[a];
        }
    }
    if (beyond_wall) {
        *dir = opposite(i);
        return ((long)z * L->ny + y) * L->nx + x;
    }
    *dir = i;
    return ((long)c[2] * L->ny + c[1]) * L->nx + c[0];
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int ORA(num_threads)(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Initial state: generalized equilibrium at (rho, u - F/(2 rho)). */
int ORA(init)(const ora_lattice *L, const double *rho, const double *u, const double *F, double *f)
{
    ensure_ready();
    long N = lattice_n(L);
    for (long s = 0; s < N; ++s) {
        double r = rho ? rho[s] : 1.0;
        double up[3], feq[Q];
        for (int a = 0; a < 3; ++a) {
            double ua = u ? u[a * N + s] : 0.0;
            double Fa = F ? F[a * N + s] : 0.0;
            up[a] = ua - Fa / (2.0 * r);
        }
        equilibrium_r(g_Minv, r, up, feq);
        for (int i = 0; i < Q; ++i) f[i * N + s] = feq[i];
    }
    return 0;
}

/* nsteps full time steps (Steps 1-4), in place on f (post-streaming state),
 * with the force F(x) e^{-gamma t}, t = t0, t0 + 1, ... the time of each
 * collision (gamma = 0: a static force). */
int ORA(step_decay)(const ora_lattice *L, const double *F, double *f, int nsteps, int nthreads, double t0,
                   double gamma);

int ORA(step)(const ora_lattice *L, const double *F, double *f, int nsteps, int nthreads)
{
    return ORA(step_decay)(L, F, f, nsteps, nthreads, 0.0, 0.0);
}

int ORA(step_decay)(const ora_lattice *L, const double *F, double *f, int nsteps, int nthreads, double t0,
                   double gamma)
{
    ensure_ready();
    long N = lattice_n(L);
    double S[Q][Q];
    build_S(L, S);
    double *tmp = (double *)malloc(sizeof(double) * Q * N);
    if (!tmp) return -1;
    set_threads(nthreads);
    for (int t = 0; t < nsteps; ++t) {
        const double decay = gamma == 0.0 ? 1.0 : exp(-gamma * (t0 + t));
#pragma omp parallel for collapse(2) schedule(static)
        for (int z = 0; z < L->nz; ++z) {
            for (int y = 0; y < L->ny; ++y) {
                for (int x = 0; x < L->nx; ++x) {
                    long s = ((long)z * L->ny + y) * L->nx + x;
                    double fl[Q], Fl[3], fs[Q];
                    for (int i = 0; i < Q; ++i) fl[i] = f[i * N + s];
                    for (int a = 0; a < 3; ++a) Fl[a] = F ? F[a * N + s] * decay : 0.0;
                    collide_model_r(L, S, fl, Fl, fs);
                    for (int i = 0; i < Q; ++i) {
                        int d;
                        long t2 = push_target(L, x, y, z, i, &d);
                        tmp[d * N + t2] = fs[i];
                    }
                }
            }
        }
        memcpy(f, tmp, sizeof(double) * Q * N);
    }
    free(tmp);
    return 0;
}

/* Eq. 9 over the lattice. */
int ORA(macros)(const ora_lattice *L, const double *f, const double *F, double *rho, double *u)
{
    long N = lattice_n(L);
    for (long s = 0; s < N; ++s) {
        double fl[Q], Fl[3], r, ul[3];
        for (int i = 0; i < Q; ++i) fl[i] = f[i * N + s];
        for (int a = 0; a < 3; ++a) Fl[a] = F ? F[a * N + s] : 0.0;
        macros_r(fl, Fl, &r, ul);
        rho[s] = r;
        for (int a = 0; a < 3; ++a) u[a * N + s] = ul[a];
    }
    return 0;
}

/* One step for a list of nodes only, starting from the initial state that
 * ora_init would build from (rho, u, F): out[k*Q + i] = f_i(node_k, t = 1).
 * Lets a test check sampled nodes of a lattice too large for ora_step. */
int ORA(first_step_nodes)(const ora_lattice *L, const double *rho, const double *u, const double *F,
                         int nnodes, const long *nodes, double *out, int nthreads)
{
    ensure_ready();
    long N = lattice_n(L);
    double S[Q][Q];
    build_S(L, S);
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic)
    for (int k = 0; k < nnodes; ++k) {
        long s = nodes[k];
        int x = (int)(s % L->nx), y = (int)((s / L->nx) % L->ny), z = (int)(s / ((long)L->nx * L->ny));
        /* every (source node, direction) whose push lands on (s, i) */
        for (int src_i = 0; src_i < Q; ++src_i) {
            int n[3] = {L->nx, L->ny, L->nz};
            int c[3] = {x - EV[src_i][0], y - EV[src_i][1], z - EV[src_i][2]};
            /* candidate source (c, src_i) streaming along src_i; check it lands on (s, src_i) */
            int ok = 1;
            for (int a = 0; a < 3; ++a) {
                if (c[a] < 0 || c[a] >= n[a]) {
                    if (L->walls & (1 << a)) ok = 0;
                    else c[a] = (c[a] + n[a]) % n[a];
                }
            }
            long src;
            int take;
            if (ok) { src = ((long)c[2] * L->ny + c[1]) * L->nx + c[0]; take = src_i; }
            else { src = s; take = opposite(src_i); }
            double r = rho ? rho[src] : 1.0, up[3], Fl[3], feq[Q], fs[Q];
            for (int a = 0; a < 3; ++a) {
                Fl[a] = F ? F[a * N + src] : 0.0;
                up[a] = (u ? u[a * N + src] : 0.0) - Fl[a] / (2.0 * r);
            }
            equilibrium_r(g_Minv, r, up, feq);
            collide_model_r(L, S, feq, Fl, fs);
            int d;
            int sx = (int)(src % L->nx), sy = (int)((src / L->nx) % L->ny), sz = (int)(src / ((long)L->nx * L->ny));
            long dest = push_target(L, sx, sy, sz, take, &d);
            if (dest != s || d != src_i) abort();
            out[(long)k * Q + src_i] = fs[take];
        }
    }
    return 0;
}

/* ---- adjoint ---- */

#define HCS 1e-30

/* Jacobian of the node collision f* = C(f, F): J[i][k], k < 19 w.r.t. f_k,
 * k = 19..21 w.r.t. F_{k-19}, by complex-step differentiation. */
static void collide_jacobian(const ora_lattice *L, const double S[Q][Q], const double f[Q], const double F[3],
                             double J[Q][Q + 3])
{
    for (int k = 0; k < Q + 3; ++k) {
        double complex fc[Q], Fc[3], out[Q];
        for (int i = 0; i < Q; ++i) fc[i] = f[i];
        for (int a = 0; a < 3; ++a) Fc[a] = F[a];
        if (k < Q) fc[k] += HCS * I;
        else Fc[k - Q] += HCS * I;
        collide_model_c(L, S, fc, Fc, out);
        for (int i = 0; i < Q; ++i) J[i][k] = cimag(out[i]) / HCS;
    }
}

/* Adjoint of one step f^{t+1} = P C(f^t, F):
 *   lam*_i(x) = lam^{t+1} at the slot that (x, i) streams into (P transposed),
 *   lam^t(x)  = J_f(x)^T lam*(x),   gF(x) += J_F(x)^T lam*(x).
 * f_t is the post-streaming state at t; gF is accumulated (3N SoA). */
int ORA(adjoint_step)(const ora_lattice *L, const double *f_t, const double *F, const double *lam_next,
                     double *lam_t, double *gF, int nthreads)
{
    ensure_ready();
    long N = lattice_n(L);
    double S[Q][Q];
    build_S(L, S);
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < L->nz; ++z) {
        for (int y = 0; y < L->ny; ++y)
            for (int x = 0; x < L->nx; ++x) {
                long s = ((long)z * L->ny + y) * L->nx + x;
                double fl[Q], Fl[3], ls[Q], J[Q][Q + 3];
                for (int i = 0; i < Q; ++i) fl[i] = f_t[i * N + s];
                for (int a = 0; a < 3; ++a) Fl[a] = F ? F[a * N + s] : 0.0;
                for (int i = 0; i < Q; ++i) {
                    int d;
                    long t2 = push_target(L, x, y, z, i, &d);
                    ls[i] = lam_next[d * N + t2];
                }
                collide_jacobian(L, S, fl, Fl, J);
                for (int k = 0; k < Q; ++k) {
                    double acc = 0.0;
                    for (int i = 0; i < Q; ++i) acc += J[i][k] * ls[i];
                    lam_t[k * N + s] = acc;
                }
                if (gF)
                    for (int a = 0; a < 3; ++a) {
                        double acc = 0.0;
                        for (int i = 0; i < Q; ++i) acc += J[i][Q + a] * ls[i];
                        gF[a * N + s] += acc;
                    }
            }
    }
    return 0;
}

/* Seed of the adjoint from a cotangent g on the final velocity u(x,T) of Eq. 9:
 * lam^T_i(x) = sum_a g_a(x) du_a/df_i, gF_a(x) += g_a(x) du_a/dF_a. */
int ORA(adjoint_seed)(const ora_lattice *L, const double *f_T, const double *F, const double *g,
                     double *lam_T, double *gF)
{
    long N = lattice_n(L);
    for (long s = 0; s < N; ++s) {
        double ga[3];
        for (int a = 0; a < 3; ++a) ga[a] = g[a * N + s];
        for (int k = 0; k < Q + 3; ++k) {
            double complex fc[Q], Fc[3], rho, u[3];
            for (int i = 0; i < Q; ++i) fc[i] = f_T[i * N + s];
            for (int a = 0; a < 3; ++a) Fc[a] = F ? F[a * N + s] : 0.0;
            if (k < Q) fc[k] += HCS * I;
            else Fc[k - Q] += HCS * I;
            macros_c(fc, Fc, &rho, u);
            double acc = 0.0;
            for (int a = 0; a < 3; ++a) acc += ga[a] * cimag(u[a]) / HCS;
            if (k < Q) lam_T[k * N + s] = acc;
            else if (gF) gF[(k - Q) * N + s] += acc;
        }
    }
    return 0;
}
