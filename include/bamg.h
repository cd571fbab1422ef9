/*
 * bamg.h — C ABI of the GB300 Bootstrap AMG library for Markov chains.
 *
 * Computes the stationary vector x of an irreducible column-stochastic transition
 * matrix A (A x = x, x > 0, 1^T x = 1; Section 1, Eq. (1.1)) by solving B x = 0 with
 * B = I - A: a bootstrap setup (Section 1 steps 1-4; Algorithm 3, the multilevel
 * eigensolver, followed by the rebuild of all P_l, B_l, T_l) and flexible GMRES
 * preconditioned by a V(2,2) cycle (Section 4.2, Eq. (4.4)).
 *
 * Conventions for every entry point:
 *  - A is column stochastic and a_ij is the probability of the transition j -> i, so
 *    CSR row i lists the source states j.  Column indices of a row must be sorted
 *    ascending and unique.  Self-loops are allowed (B keeps them on its diagonal).
 *  - Integer index arrays are int32; floating arrays are FP64 unless a `dtype`
 *    argument says otherwise (BAMG_F64 = double, BAMG_F32 = float).
 *  - Pointers are device pointers unless the argument name starts with h_ or a flag
 *    says the buffer lives in host memory.  The caller owns every buffer it passes;
 *    the library never frees them and keeps no reference after the call returns.
 *  - Test-vector blocks are "row interleaved": X[i * ld + k] is vector k at state i;
 *    `ld` and `col0` must be multiples of 2 (FP64) or 4 (FP32) so rows load as
 *    16-byte vectors, and X must be 16-byte aligned.
 *  - Work is queued on `stream` (a cudaStream_t; NULL = the legacy default stream).
 *    Entry points that return sizes or statuses synchronise that stream first.
 *  - Every call returns BAMG_OK (0) or a negative code; bamg_last_error() returns a
 *    message for the calling thread's last failure.  No call is thread-safe on the
 *    same handle.
 */
#ifndef BAMG_H
#define BAMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    BAMG_OK = 0,
    BAMG_EINVAL = -1,    /* bad argument, size or layout */
    BAMG_ENOTSTOCH = -2, /* A not column stochastic (|colsum - 1| > 1e-12), a negative entry, or a_ii = 1 */
    BAMG_ECUDA = -3,     /* CUDA runtime error */
    BAMG_ENOMEM = -4,    /* device allocation failed */
    BAMG_ENOCONV = -5,   /* tolerance not reached within max_it iterations */
    BAMG_ETIMEOUT = -6,  /* a device-side loop hit its iteration cap */
    BAMG_ENUMERIC = -7,  /* NaN/Inf, or a singular coarsest factor */
    BAMG_ESIZE = -8,     /* output capacity too small; the needed size is returned */
    BAMG_EOVERFLOW = -9  /* a fixed per-row capacity was exceeded (neighbourhood search) */
};

enum { BAMG_F64 = 0, BAMG_F32 = 1 };
enum { BAMG_PREC_FP64 = 0, BAMG_PREC_MIXED = 1 };
enum { BAMG_COARSEN_GRID = 0, BAMG_COARSEN_CR = 1 };

/* Column-stochastic A.  `on_host` = 1: the three arrays are host memory and are
 * copied to the device inside the call; 0: device memory. */
typedef struct {
    int32_t n, nnz;
    const int32_t* row_ptr; /* n + 1 */
    const int32_t* col;     /* nnz */
    const double* val;      /* nnz */
    int32_t on_host;
} bamg_csr;

/* A device CSR matrix used by the step entry points; `val` has the call's dtype. */
typedef struct {
    int32_t n, nnz;
    const int32_t* row_ptr;
    const int32_t* col;
    const void* val;
} bamg_mat;

/* The MLP of the learned interpolation (opaque; bamg_model_create). */
typedef struct bamg_model bamg_model;

typedef struct {
    double omega;       /* omega-Jacobi damping (Section 3: 0.7) */
    int32_t nu_tv;      /* setup sweeps on the random test vectors */
    int32_t nu_ev;      /* sweeps on interpolated eigenvector approximations */
    int32_t nu_pre, nu_post; /* V(nu_pre, nu_post) cycle (Section 5.1: V(2,2)) */
    int32_t caliber;    /* c: max non-zeros per interpolation row (Section 3.2; 2) */
    int32_t z;          /* path length of the neighbourhoods, Eq. (3.5), 1..3 */
    int32_t mmax;       /* candidates kept per fine point, closest first (<= 16) */
    int32_t k_ev;       /* coarsest-level eigenvectors carried up (Section 5.1: 6) */
    int32_t coarse_max; /* stop coarsening at n_l <= coarse_max (<= 64) */
    int32_t gmres_m;    /* FGMRES restart length (<= 256) */
    int32_t max_it;     /* total FGMRES iteration cap */
    int32_t precision;  /* BAMG_PREC_FP64 or BAMG_PREC_MIXED (FP32 setup + V-cycle) */
    int32_t coarsen;    /* BAMG_COARSEN_GRID (needs grid_nx, grid_ny) or BAMG_COARSEN_CR */
    int32_t grid_nx, grid_ny; /* state (ix, iy) has index ix + iy * grid_nx */
    uint64_t seed;      /* counter-based random numbers (SplitMix64) */
    double tv_lo, tv_hi;/* initial test vectors uniform in [tv_lo, tv_hi) */
    double ev_change_tol;/* an eigenvector joins the test set if |dlambda|/|lambda| exceeds this */
    double ridge;       /* Tikhonov factor of the local LS systems, FP64 runs */
    double ridge32;     /* the same for FP32 (mixed) runs */
    double weight_floor;/* floor of ||B x||^2 in the LS weights */
    double cr_theta;    /* compatible relaxation threshold (Section 3.1: 0.85) */
    int32_t cr_nu;      /* CR sweeps per round (Section 3.1: 8) */
    int32_t cr_max_rounds;
    double cr_omega;
    void* stream;       /* cudaStream_t for all work of the handle */
    /* learned interpolation (no counterpart in the paper; see bamg_model_create) */
    int32_t interp;     /* BAMG_INTERP_LS (Algorithm 2) or BAMG_INTERP_LEARNED */
    int32_t learned_refit; /* learned rows: 1 = Eq. (3.6) weights over the MLP's choice, 0 = MLP weights */
    const bamg_model* model; /* the MLP for BAMG_INTERP_LEARNED (caller keeps ownership) */
    double learned_rho_max; /* > 0: fall back to least squares when the learned hierarchy's
                               V-cycle factor (bamg_vcycle_factor, 20 steps) exceeds this */
    int32_t device_loop;    /* 1 (default): between true-residual checks the Arnoldi steps run in a
                               device-side loop (a CUDA graph WHILE node, one host wait per check);
                               0: one graph launch and one host wait per step.  Same iterates. */
    /* setup cycling and restarts (Section 4.1; Section 5.1) */
    int32_t mle_restart;    /* 1 (default): after every FGMRES restart cycle that ends above tol, an MLE
                               restart: the iterate becomes the state-vector test vector of every level
                               (injected downwards) and all P_l, B_l, T_l and B_L^+ are rebuilt before
                               the next cycle ("alternate several times between the MLE and AMG-GMRES
                               iterations", Section 4.1); 0: plain restarts */
    int32_t setup_cycles;   /* MLE cycles in the setup before the final rebuild (1; the tables' V^2 = 2) */
    int32_t mu;             /* Algorithm 3's loop count: 1 = V-cycle setup, 2 = W-cycle setup */
    int32_t smoother;       /* V-cycle smoother: BAMG_SMOOTH_JACOBI (omega-Jacobi, Section 3; default) or
                               BAMG_SMOOTH_MCGS (multicolour Gauss-Seidel, Section 3's other relaxation:
                               colour c is an independent set of the states the earlier colours left in
                               the symmetrised graph of B_l; colours ascending before the coarse
                               correction, descending after it; the setup's relaxations stay Jacobi) */
    int32_t persistent;     /* 1: where the hierarchy qualifies (short-row grid levels, at most 24 levels,
                               the coarse tail within shared memory, no Gauss-Seidel smoother) and the
                               device supports it, the Arnoldi steps between true-residual checks run in
                               one cooperative launch with grid-wide barriers instead of a graph per step
                               (same iterates; a barrier wait that gives up returns BAMG_ETIMEOUT).
                               0 (default): the graph form, which measured faster (the grid barriers
                               between the step's phases cost more than graph kernel boundaries).
                               bamg_solve_batch with more than one worker always uses the graph form. */
    int32_t coarse_tail;    /* the coarse end of the V-cycle (Eq. (4.4) on the small levels) in one
                               launch per cycle: 0 (default) = every level from the first one with at
                               most 4096 rows on one cluster of 8 thread blocks (each block owns a slice
                               of every level's rows and sends its values to the others through
                               distributed shared memory; cluster barriers between the phases), where
                               the device supports clusters; 1 = every level from the first one with at
                               most 1024 rows in a single thread block.  One thread per row in the grid
                               kernels' order of operations: on hierarchies whose levels have fewer than
                               12 entries per row on average the iterates are the same bit for bit,
                               otherwise equal up to rounding. */
} bamg_opts;

enum { BAMG_SMOOTH_JACOBI = 0, BAMG_SMOOTH_MCGS = 1 };

enum { BAMG_INTERP_LS = 0, BAMG_INTERP_LEARNED = 1 };

typedef struct {
    int32_t status;
    int32_t iterations;   /* FGMRES iterations */
    int32_t restarts;
    int32_t true_checks;  /* true-residual evaluations */
    double residual_l1;   /* ||B x||_1 / ||x||_1 of the returned x */
    double setup_ms;      /* wall time of bamg_setup */
    double solve_ms;      /* wall time of this bamg_solve */
    int32_t host_waits;   /* host synchronisations on Arnoldi steps: one per step, or one per
                             estimate-triggered check where the steps loop on the device */
    int32_t mle_restarts; /* MLE restarts between restart cycles (bamg_opts.mle_restart) */
} bamg_stats;

typedef struct bamg_handle bamg_handle;

/* Fills *o with the paper's settings (Section 5.1) and the readings for the rest. */
int bamg_default_opts(bamg_opts* o);

/* Bootstrap setup (Section 1 steps 1-4; Algorithm 3 with mu = 1; rebuild).
 * A: the transition matrix (copied; the caller may free it on return).
 * r: number of random test vectors (1..24).  levels: maximum number of coarsenings.
 * On success *h owns all device memory of the hierarchy until bamg_free(*h).
 * Errors: EINVAL (sizes, r, options, grid dims), ENOTSTOCH, ENOMEM, ECUDA, ENUMERIC.
 * The setup returns without waiting for its last kernels: two errors found on the device
 * at its end, a neighbourhood search that overflowed (EOVERFLOW) and a singular coarsest
 * factor (ENUMERIC), are returned by the next call that uses the handle (bamg_solve,
 * bamg_parnoldi, bamg_vcycle_apply, the smoother and export calls). */
int bamg_setup(const bamg_csr* A, int r, int levels, const bamg_opts* o, bamg_handle** h);

enum { BAMG_X_GUESS = 1, BAMG_X_HOST = 2, BAMG_NORM_L2 = 4 };
/* Preconditioned flexible GMRES on B x = 0 (Section 4.2) until
 * ||B x||_1 / ||x||_1 <= tol, then x is scaled to 1^T x = 1.
 * x: n doubles, device memory unless flags has BAMG_X_HOST.  With BAMG_X_GUESS the
 * incoming x is the initial guess, otherwise the setup's state-vector approximation
 * (Section 4.1) is used.  With BAMG_NORM_L2 the stopping test is ||B x||_2 / ||x||_2 <= tol
 * (Section 5.1's criterion; st->residual_l1 still reports the l1 ratio).
 * st may be NULL.  Errors: ENOCONV (x holds the last iterate),
 * ENUMERIC, ECUDA; and EOVERFLOW or ENUMERIC left by bamg_setup (see there). */
int bamg_solve(bamg_handle* h, double* x, int flags, double tol, bamg_stats* st);

/* Batched form: sets up and solves nchains independent chains to ||B x||_1/||x||_1 <= tol
 * and frees them, with nworkers host threads (0: one per 4 chains, at most 16), each
 * driving its own non-blocking stream; chains are taken largest first from a shared
 * queue, so the small latency-bound kernels of several chains overlap on the GPU.
 * As[k], r[k], levels[k], opts[k] as for bamg_setup (opts[k].stream is ignored);
 * xs[k]: n_k doubles for the result, device memory unless flags has BAMG_X_HOST
 * (BAMG_X_GUESS is not accepted).  st (may be NULL) receives one entry per chain.
 * With more than one worker, opts[k].device_loop is taken as 0 (one graph launch per
 * Arnoldi step): conditional-node graphs in concurrent threads slowed the other threads'
 * setups more than the device-side loop saves.
 * Returns BAMG_OK if every chain succeeded, else the first failing chain's code (its
 * message in bamg_last_error); the other chains are still solved. */
int bamg_solve_batch(int nchains, const bamg_csr* As, const int* r, const int* levels, const bamg_opts* opts,
                     double* const* xs, int flags, double tol, int nworkers, bamg_stats* st);

/* The MLE as a stand-alone solver (Section 4.1; the "MLE" rows of Tables 1, 2 and 4):
 * MLE cycles (Algorithm 3 with loop count o->mu) from the random test vectors until the
 * state-vector approximation x = V_0[:, 0] meets ||B x||_1 / ||x||_1 <= tol (with
 * BAMG_NORM_L2 in flags: ||B x||_2 / ||x||_2 <= tol, Section 5.1's criterion) or
 * max_cycles cycles ran.  Algorithm 3 empties V_l at the start of a call; that is read as
 * holding on the first visit of level l only, so every later cycle relaxes V_l (nu_ev
 * shifted sweeps) on the way down and fits P_l to U_l and the selected V_l, and U_l is
 * relaxed on the first visit only.  x: n doubles (device memory, or host with
 * BAMG_X_HOST) receiving the last approximation with 1^T x = 1 (may be NULL).
 * st->iterations = cycles, st->residual_l1 = its l1 ratio.  h (may be NULL) receives the
 * hierarchy, rebuilt from the final test sets, for bamg_solve / bamg_parnoldi (the
 * "alternate MLE and AMG-GMRES" use); it is returned with ENOCONV too.
 * Errors: as bamg_setup, plus ENOCONV when max_cycles cycles did not reach tol. */
int bamg_mle_solve(const bamg_csr* A, int r, int levels, const bamg_opts* o, double tol, int max_cycles, int flags,
                   double* x, bamg_stats* st, bamg_handle** h);

/* Multigrid-preconditioned Arnoldi (Section 4.3): orthonormal v_1, v_2, ... of the Krylov
 * space of C B (C = the V(nu_pre, nu_post) cycle, left preconditioning) from y = the
 * setup's state-vector approximation (or x with BAMG_X_GUESS); the eigenvector eta of
 * H_k = V_k^T C B V_k for its eigenvalue closest to 0 (inverse iteration with shift 0 on
 * H_k: it converges when that eigenvalue is real and simple, as the eigenvalue 0 of C B
 * is); the Ritz vector V_k eta, whose true residual is tested after every step (l1 ratio,
 * or the 2-norm ratio with BAMG_NORM_L2).  The Gram-Schmidt process is the FGMRES one
 * (FP64, one reorthogonalisation); after min(gmres_m, 64) steps the process restarts from
 * the Ritz vector.  x receives the result with 1^T x = 1.  Errors: ENOCONV (x holds the
 * last Ritz vector), ENUMERIC, ECUDA. */
int bamg_parnoldi(bamg_handle* h, double* x, int flags, double tol, bamg_stats* st);

/* Frees the handle and its device memory.  NULL is allowed. */
void bamg_free(bamg_handle* h);

/* Message of the calling thread's last failed call ("" if none).  Static storage. */
const char* bamg_last_error(void);

/* Number of kernels this library has launched in the process (all threads; each
 * replayed Arnoldi step counts its kernels).  Bookkeeping, no passage of the paper. */
uint64_t bamg_launch_count(void);

/* Levels of the hierarchy: *nlevels, and per level the size and non-zeros of B_l into
 * h_n[], h_nnz[] (capacity 32 each, may be NULL); operator complexity sum nnz / nnz_0. */
int bamg_hierarchy_info(const bamg_handle* h, int* nlevels, int64_t* h_n, int64_t* h_nnz, double* opc);

enum {
    BAMG_EXPORT_B = 0,   /* CSR of B_l: h_dst = [row_ptr (n+1) int32 | col (nnz) int32 | val (nnz) double] */
    BAMG_EXPORT_T = 1,   /* T_l values on B_l's pattern (nnz doubles) */
    BAMG_EXPORT_P = 2,   /* P_l as ELL: [pcol (n*c) int32 | pcnt (n) int32 | pval (n*c) double] */
    BAMG_EXPORT_CF = 3,  /* cf (n bytes, 1 = coarse) */
    BAMG_EXPORT_X = 4,   /* test-vector block, n * ld doubles (ld via bamg_hierarchy_layout) */
    BAMG_EXPORT_PINV = 5,/* coarsest B_L^+ (n_L * n_L doubles, row-major) */
    BAMG_EXPORT_XINIT = 6,/* the setup's state-vector approximation (n_0 doubles) */
    BAMG_EXPORT_LAMBDA = 7 /* eigenvalue approximations of level l (nvec doubles) */
};
/* Copies one object of level l to host memory h_dst (converted to double).  Returns
 * ESIZE with *h_bytes = the needed size when cap_bytes is too small. */
int bamg_level_export(const bamg_handle* h, int level, int what, void* h_dst, int64_t cap_bytes, int64_t* h_bytes);

/* Layout of the test-vector block of level l: leading dimension, random vectors r,
 * eigenvector columns start (col0 of V) and count. */
int bamg_hierarchy_layout(const bamg_handle* h, int level, int* ld, int* r, int* v_col0, int* nvec);

/* ---------------------------------------------------------------------------------
 * Hierarchy import (checkpoint/resume): builds a handle from a given hierarchy, all
 * arrays in host memory, FP64.  Level l has B_l (CSR) and, for l < nlevels-1, P_l in
 * CSR (n_l x n_{l+1}, at most `caliber` entries per row); Q_l is derived from P_l as
 * in Section 4 (Q[I, i] = 1/|J_i|).  pinv is the coarsest B_L^+ (row-major), x_init the
 * initial guess.  Used to run the solve phase on a hierarchy built elsewhere.
 * --------------------------------------------------------------------------------- */
typedef struct {
    int32_t n, nnz;
    const int32_t* h_row_ptr; const int32_t* h_col; const double* h_val;  /* B_l */
    int32_t p_nnz;
    const int32_t* h_p_row_ptr; const int32_t* h_p_col; const double* h_p_val; /* P_l */
} bamg_level_in;
/* BAMG_EINVAL when nlevels is outside 1..30, the coarsest level has more than 64 states,
 * or a row of P has more than o->caliber entries; *h is untouched on failure. */
int bamg_import(int nlevels, const bamg_level_in* levels, const double* h_pinv, const double* h_x_init,
                const bamg_opts* o, bamg_handle** h);

/* z = C v: one V(nu_pre, nu_post) cycle of the handle's hierarchy on v (Eq. (4.4),
 * zero initial guess, B_L^+ on the coarsest level).  v, z: n_0 device doubles. */
int bamg_vcycle_apply(bamg_handle* h, const double* v, double* z);

/* Arithmetic of the handle's hierarchy and V-cycle: BAMG_F32 (mixed precision) or
 * BAMG_F64; BAMG_EINVAL for a NULL handle. */
int bamg_hierarchy_precision(const bamg_handle* h);

/* `sweeps` sweeps of the V-cycle smoother of Eq. (4.4), x <- x + omega D^{-1} (b - B_l x),
 * on level l of the handle's hierarchy: one kernel launch per sweep on the handle's
 * stream, asynchronous (no synchronisation; time it with events on that stream).
 * b, x, work: n_l device elements in the hierarchy's arithmetic (bamg_hierarchy_precision);
 * x is updated in place, work is scratch.  The V-cycle's own smoothing steps. */
int bamg_smooth_apply(bamg_handle* h, int level, int sweeps, const void* b, void* x, void* work);

/* ---------------------------------------------------------------------------------
 * Learned interpolation.  No counterpart in the paper: a 112-128-128-16 ReLU MLP maps the
 * features of a fine point (its candidates of Eq. (3.5): per slot [valid, path length / 3,
 * g_ij / g_jj, g_ij / sqrt(g_ii g_jj), -b_ij / b_ii, -b_ji / b_jj] with g_ab the LS-weighted
 * test-vector inner products of Section 3.2, then [m / 16, sum_{j!=i} |b_ij| / b_ii],
 * zero-padded) to 16 slot weights; the c slots of largest |y| form the row of P, with the
 * MLP's weights or the Eq. (3.6) minimiser over them (learned_refit).  It is trained on
 * the least-squares rows of Algorithm 2 (bamg_interp_dataset).  Products take bfloat16
 * inputs with FP32 sums; loss = (1/rows) sum over valid slots of (y - t)^2; Adam with
 * beta1 = 0.9, beta2 = 0.999, eps = 1e-8.  Parameters: one flat FP32 array
 * [W1 (128 x 112) | b1 | W2 (128 x 128) | b2 | W3 (16 x 128) | b3], W row-major (out x in).
 * All calls are synchronous with respect to the host except bamg_model_forward.
 * --------------------------------------------------------------------------------- */
enum { BAMG_MLP_F = 112, BAMG_MLP_H = 128, BAMG_MLP_S = 16 };
/* He-uniform weights W = (2u - 1) sqrt(6 / fan_in), u from SplitMix64 (seed, layer, index). */
int bamg_model_create(uint64_t seed, bamg_model** m);
/* frees the model (NULL allowed); a handle set up with it must not outlive it */
void bamg_model_free(bamg_model* m);
/* number of FP32 parameters of the MLP (112*128 + 128 + 128*128 + 128 + 128*16 + 16) */
int64_t bamg_model_param_count(void);
/* host FP32 parameters in (set; resets Adam) or out (get); count = bamg_model_param_count() */
int bamg_model_set(bamg_model* m, const float* h_params, int64_t count);
int bamg_model_get(const bamg_model* m, float* h_params, int64_t count);
/* d_out (rows x 16, FP32) = MLP(d_feat (rows x 112, FP32)); asynchronous on stream */
int bamg_model_forward(const bamg_model* m, const float* d_feat, int64_t rows, float* d_out, void* stream);
/* gradient of the loss over all rows (one batch) into h_grad (param_count floats, may be
 * NULL) and the loss into *h_loss; parameters unchanged */
int bamg_model_gradients(bamg_model* m, const float* d_feat, const float* d_target, int64_t rows, float* h_grad,
                         double* h_loss, void* stream);
/* epochs x (rows / batch) Adam steps over contiguous batches in row order; h_epoch_loss
 * (epochs doubles, may be NULL) = mean batch loss of each epoch */
int bamg_model_train(bamg_model* m, const float* d_feat, const float* d_target, int64_t rows, int epochs, int batch,
                     double lr, double* h_epoch_loss, void* stream);
/* Training data: runs the least-squares setup of A and writes, for every point of every
 * level of both passes, its features (d_feat, rows x 112) and its Algorithm 2 row on the
 * slots (d_target, rows x 16; coarse points and empty slots 0).  *h_rows = rows needed;
 * BAMG_ESIZE (nothing written beyond cap_rows) when cap_rows is smaller. */
int bamg_interp_dataset(const bamg_csr* A, int r, int levels, const bamg_opts* o, float* d_feat, float* d_target,
                        int64_t cap_rows, int64_t* h_rows);
/* rho of the stationary iteration x <- x - C B x: power iteration on the residual
 * propagator I - B C (mean removed, unit norm each step) from B x0, x0 in U[1, 2)
 * (SplitMix64 seed 7); geometric mean of the growth over the second half of iters. */
int bamg_vcycle_factor(bamg_handle* h, int iters, double* rho);
/* BAMG_INTERP_LS or BAMG_INTERP_LEARNED: the interpolation the hierarchy was built with
 * (LS after a fallback); *h_rho (may be NULL) = the factor measured for the fallback
 * decision, or 0 when none was measured. */
int bamg_hierarchy_interp(const bamg_handle* h, double* h_rho);

/* ---------------------------------------------------------------------------------
 * Step entry points: one step of the setup on caller buffers (device memory).
 * --------------------------------------------------------------------------------- */

/* Initial test vectors (Section 5.1: uniform positive random entries):
 * X[i*ld + col0 + k] = lo + (hi - lo) * u, u the (k * 2^40 + i + 1)-th SplitMix64 draw
 * (Steele, Lea, Flood 2014) of `seed`, k < ncols, computed in FP64 then rounded to dtype. */
int bamg_tv_init(int dtype, int n, int ncols, int ld, int col0, uint64_t seed, double lo, double hi,
                 void* X, void* stream);

/* nu omega-Jacobi sweeps (Section 3, Eq. (3.1), M = diag(B)/omega) on the columns
 * [col0, col0 + ncols) of X (col0 >= 0): X <- X - omega D^{-1} (B X).  With T_val and d_lambda
 * the sweeps solve (B - lambda_k T) x_k = 0 (Algorithm 3): D_k = diag(B) - lambda_k diag(T).
 * T_val: values of T on B's pattern (NULL: T = I); d_lambda: ncols FP64 shifts (NULL: 0).
 * work: scratch of n * ld elements of dtype.  B must store its diagonal. */
int bamg_relax(int dtype, const bamg_mat* B, const void* T_val, const double* d_lambda, int ncols, int ld,
               int col0, double omega, int nu, void* X, void* work, void* stream);

/* Launch shapes chosen by the sweep's autotuner.  On levels with more than four rows per
 * thread of the one-chunk grid, the first sweep of each key times the launch shapes (one
 * or two 16-byte chunks per thread; 1, 2 or 4 blocks per SM), which all write the same
 * bits, and keeps the fastest for the process (BAMG_AUTOTUNE=0 in the environment: the
 * fixed rule instead).  Writes up to max_rows rows of 7 int32 to h_rows (host memory):
 * element bytes, shift (0/1), entry batch, 16-byte chunks per row, floor(log2 n), chunks
 * per thread, blocks per SM.  Returns the number of rows written (>= 0). */
int bamg_autotune_report(int32_t* h_rows, int max_rows);

/* LS weights of Section 3.2: scales each active column k of [col0, col0+ncols) to unit
 * 2-norm and sets w_k = 1 / max(||B x_k||_2^2, floor), then divides the active weights by
 * their maximum; inactive columns (d_active[k] = 0, or d_active NULL = all active) get 0.
 * d_w: ncols doubles. */
int bamg_tv_weights(int dtype, const bamg_mat* B, int ncols, int ld, int col0, const uint8_t* d_active,
                    double floor, void* X, double* d_w, void* stream);

/* Same sweeps as bamg_relax, but the call allocates nothing: no paper counterpart;
 * it exists for callers that cannot let a library allocate device memory (a service
 * that reserves its whole device budget at start-up, a framework whose allocator owns
 * the device, a latency-critical loop where cudaMalloc/cudaFree would block).  The
 * second copy of the vector block and the diagonals live in one 8 MiB device array
 * compiled into the library, held by every device that loads it until the process
 * exits.  Requires n * (ld + 3) * sizeof(element) <= 8 MiB (each part rounded up to 256
 * bytes); larger problems return BAMG_EINVAL.  The first call on a device looks up the
 * array's device address with that device current (make that first call before any
 * stream capture).  All calls share the array and nothing in it needs to start at zero;
 * calls that overlap on the GPU, from any stream or thread, race on it.  Arguments and
 * results as for bamg_relax (col0 >= 0; ld at least one 16-byte chunk); the call
 * synchronises `stream` and returns after the work has completed on it. */
int bamg_relax_noalloc(int dtype, const bamg_mat* B, const void* T_val, const double* d_lambda, int ncols, int ld,
                       int col0, double omega, int nu, void* X, void* stream);

/* Full coarsening (Section 5.1): cf[i] = 1 on states with even ix and even iy;
 * cidx[i] = (ix/2) + (iy/2) * ((nx+1)/2) on coarse states, -1 on fine states. */
int bamg_coarsen_grid(int nx, int ny, uint8_t* cf, int32_t* cidx, void* stream);

/* Compatible-relaxation coarsening, Algorithm 1 (Section 3.1), on level `level` of the
 * seed's random streams: an independent set of G(B) to start, then rounds of nu
 * F-relaxation sweeps from U[1,2) starts adding an independent set of the slow points
 * while rho_f > theta.  Writes cf, cidx; *h_nc = coarse count, *h_rounds = rounds. */
int bamg_coarsen_cr(const bamg_mat* B, int level, uint64_t seed, double theta, int nu, double omega,
                    int max_rounds, uint8_t* cf, int32_t* cidx, int* h_nc, int* h_rounds, void* stream);

/* Least-squares interpolation rows (Section 3.2, Eq. (3.5), Eq. (3.6), Algorithm 2) for
 * every fine point: candidates are the coarse points within path length z in G(B),
 * ordered by (length, coarse index), at most mmax; greedy selection of up to c points,
 * each step minimising Eq. (3.6) with the weights d_w over the ncols columns of X
 * (from col 0).  Output P in ELL form: pcol[i*c + t] (coarse index), pval, pcnt[i];
 * coarse points get the unit row.  Rows are sorted by coarse index. */
int bamg_interp_ls(int dtype, const bamg_mat* B, const uint8_t* cf, const int32_t* cidx, const void* X,
                   int ncols, int ld, const double* d_w, int z, int mmax, int c, double ridge,
                   int32_t* pcol, void* pval, int32_t* pcnt, void* stream);

/* The LS kernel's candidates and features without Algorithm 2 (d_target == NULL), or with
 * it (d_target: the LS rows on the slots, and P written to pcol/pval/pcnt when these are
 * not NULL): d_feat rows x 112 and d_cand (rows x 16, -1 padded) may each be NULL. */
int bamg_interp_features(int dtype, const bamg_mat* B, const uint8_t* cf, const int32_t* cidx, const void* X, int ncols,
                         int ld, const double* d_w, int z, int mmax, int c, double ridge, float* d_feat,
                         float* d_target, int32_t* d_cand, void* stream);
/* Learned interpolation of one level (arguments as bamg_interp_ls, plus the model and
 * refit): P in ELL form (pcol/pval/pcnt). */
int bamg_interp_learned(int dtype, const bamg_mat* B, const uint8_t* cf, const int32_t* cidx, const void* X, int ncols,
                        int ld, const double* d_w, int z, int mmax, int c, double ridge, const bamg_model* m, int refit,
                        int32_t* pcol, void* pval, int32_t* pcnt, void* stream);

/* Petrov-Galerkin products B_c = Q B P and T_c = Q T P (Section 1 step 3; Algorithm 3)
 * with the averaging Q of Section 4 (Q[I,i] = 1/pcnt[i] for I in row i of P).
 * T_val: T on B's pattern (NULL: T = I); T_c is returned on B_c's pattern.
 * Output CSR with nc rows; cap = capacity of out_col/out_bv/out_tv.  *h_nnz = nnz(B_c);
 * returns ESIZE (nothing written) when cap < nnz(B_c). */
int bamg_galerkin(int dtype, const bamg_mat* B, const void* T_val, int nc, const int32_t* pcol,
                  const void* pval, const int32_t* pcnt, int c, int32_t* out_row_ptr, int32_t* out_col,
                  void* out_bv, void* out_tv, int64_t cap, int64_t* h_nnz, void* stream);

/* Coarsest level (Algorithm 3, first branch): eigenpairs of B_L x = lambda T_L x of
 * smallest |lambda| (dense n x n row-major FP64, n <= 64).  Complex pairs are returned
 * as two real columns (Re v, Im v) sharing Re lambda; at most k_ev + 1 columns.
 * d_lam[col], d_V (n x ncols, column-major, unit norm, <w, v> > 0 for w_i = i+1),
 * d_kind[col] (0 real, 1 real part, 2 imaginary part); *h_nvec = columns written.
 * dtype: arithmetic of the eigenvector refinement and of B_L^+ (BAMG_F64, or BAMG_F32 as
 * in the mixed-precision setup, whose V-cycle applies B_L^+ in FP32); the outputs are
 * FP64 either way.  The eigenvalue estimates that serve as shifts are FP32 in both.
 * The smallest eigenvalue is set to exactly 0.  With d_pinv != NULL also writes
 * B_L^+ (row-major), the minimal-norm inverse of Section 4.2. */
int bamg_coarse_eig(int dtype, int n, const double* d_B, const double* d_T, int k_ev, double* d_lam, double* d_V,
                    int32_t* d_kind, int* h_nvec, double* d_pinv, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* BAMG_H */
