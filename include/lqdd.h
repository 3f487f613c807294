/*
 * lqdd.h -- C ABI of the GB300 (sm_103a) odd-even Wilson-clover library.
 *
 * The library computes the finest-level, data-parallel part of DD-alpha-AMG
 * as described in arxiv 2407.08092: the odd-even (Schur-complement)
 * preconditioned Wilson-clover Dirac operator (Sec. 2.3, Sec. 2.4.5, Eq. 1-3),
 * the Richardson and GMRES smoothers built on it (Algorithms 2 and 4,
 * Sec. 2.4.5) and an odd-even (F)GMRES solve to a relative residual (Sec. 2.3).
 *
 * Conventions shared by every call
 * --------------------------------
 * Operator.  (D psi)(x) = C(x) psi(x) - 1/2 sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu)
 *                                      + (1 + g_mu) U_mu(x-mu)^+ psi(x-mu) ]
 *   C(x) = (4 + m0) + c_sw (i/4) sum_{mu,nu} sigma_mu_nu F_mu_nu(x), sigma_mu_nu =
 *   (i/2)[g_mu, g_nu], F_mu_nu = (Q_mu_nu - Q_mu_nu^+)/8 with Q the sum of the four
 *   plaquette leaves at x.  Chiral gamma basis: g_k = [[0,-i s_k],[i s_k,0]],
 *   g_4 = [[0,1],[1,0]], g_5 = diag(1,1,-1,-1); C(x) is two 6x6 blocks (spins
 *   {0,1} and {2,3}).  Space is periodic; hops across the time boundary are
 *   multiplied by lq_lattice.t_bc.
 * Lattice.  L = {Lx, Ly, Lz, Lt}, every extent even and >= 2.  Natural site
 *   order is lexicographic with x fastest: lex = x + Lx*(y + Ly*(z + Lz*t)).
 *   A site is even iff x+y+z+t is even (Sec. 2.4.5).
 * Fields (caller-owned DEVICE memory unless stated; complex double, i.e.
 *   interleaved re/im doubles, 16-byte aligned):
 *   gauge       U[V][4][3][3]   U[x][mu][a][b] = row a, column b of U_mu(x)
 *   full spinor psi[V][4][3]    spin, then colour
 *   half spinor psi[V/2][4][3]  the sites of one parity in lexicographic order
 *                               (entry i is the site with lex/2 == i)
 *   The library keeps its own internal copies in a checkerboarded,
 *   structure-of-arrays layout; that layout never crosses this boundary.
 * Streams.  Every call enqueues its work on the stream given to lq_create and
 *   returns without a device synchronisation, except where a call returns host
 *   scalars (lq_set_gauge, lq_estimate_norm, lq_norm2, lq_solve, lq_smooth with a
 *   GMRES smoother): those synchronise the stream before returning.
 * Errors.  Every call returns an lq_status; nothing aborts, traps or throws
 *   across this boundary.  lq_last_error() describes the most recent failure
 *   of a context.  A failed call leaves output buffers unspecified.
 * Tracing.  Every call that launches work opens an NVTX range named after the
 *   call (visible in profiler timelines; without a profiler it costs nothing).
 * Ownership.  The library owns the context, its internal field copies and
 *   the Krylov workspace (allocated on first use, sized by the restart
 *   length, freed by lq_destroy).  The caller owns every buffer it passes.
 */
#ifndef LQDD_H
#define LQDD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lq_ctx lq_ctx;
typedef struct lq_group lq_group;

typedef enum {
    LQ_OK = 0,
    LQ_ERR_ARG = 1,            /* invalid argument (null pointer, bad size, bad enum) */
    LQ_ERR_CUDA = 2,           /* a CUDA runtime call failed; see lq_last_error */
    LQ_ERR_OOM = 3,            /* device or pinned-host allocation failed */
    LQ_ERR_NOT_CONVERGED = 4,  /* tolerance not reached within max_restarts; x is the last iterate */
    LQ_ERR_BREAKDOWN = 5,      /* a clover block is not invertible (non-positive LDL pivot) */
    LQ_ERR_NAN = 6,            /* a NaN or Inf appeared in a residual or norm */
    LQ_ERR_STATE = 7,          /* call out of order (e.g. an operator before lq_set_gauge) */
    LQ_ERR_BOUNDS = 8          /* checked build only: a kernel's index check failed (lq_bounds_check) */
} lq_status;

/* LQ_BF16 stores spinors and 12-real links in BF16 (8 significand bits) and
 * computes in FP32 with the FP32 clover blocks: the low-precision storage of
 * the mixed-precision scheme.  It is offered for lq_apply (LQ_OP_SCHUR and
 * LQ_OP_SCHUR_DAG) and as the inner precision of the Richardson smoother. */
/* Arithmetic precisions.  LQ_DF64 is FP64-accurate "double-float" arithmetic:
 * each real is an unevaluated sum of two floats (about 48 significand bits)
 * combined with the error-free transformations of Knuth and Dekker, so it runs
 * on the FP32 units, which GB300 provides at 64 times its FP64 rate; it meets
 * the same 1e-12 parity bound as LQ_F64 with a float exponent range. */
typedef enum { LQ_F64 = 0, LQ_F32 = 1, LQ_DF64 = 2, LQ_BF16 = 3 } lq_prec;

typedef enum {
    LQ_OP_FULL = 0,      /* D on the full lattice: in, out are full spinors */
    LQ_OP_SCHUR = 1,     /* D_S = D_ee - D_eo D_oo^{-1} D_oe (Eq. 3): even half spinors */
    LQ_OP_SCHUR_DAG = 2, /* D_S^+ = g5 D_S g5: even half spinors */
    LQ_OP_EE = 3,        /* D_ee = C on even sites: even half spinors */
    LQ_OP_OO_INV = 4     /* D_oo^{-1} = C^{-1} on odd sites: odd half spinors */
} lq_op;

typedef enum { LQ_SOLVER_GMRES = 0, LQ_SOLVER_FGMRES = 1 } lq_solver_kind;
typedef enum { LQ_SMOOTH_NONE = 0, LQ_SMOOTH_RICHARDSON = 1, LQ_SMOOTH_GMRES = 2, LQ_SMOOTH_SAP = 3 } lq_smoother_kind;

typedef struct {
    int L[4];      /* Lx, Ly, Lz, Lt: even, >= 2 */
    int t_bc;      /* +1 periodic or -1 antiperiodic in time (fermion hops only) */
    double m0;     /* bare mass: the site diagonal is 4 + m0 */
    double csw;    /* clover coefficient c_sw (Table 5 lists the paper's value) */
} lq_lattice;

typedef struct {
    int solver;          /* lq_solver_kind.  GMRES(m) on D_S (Algorithm 2), or flexible GMRES(m)
                            in FP64 right-preconditioned by the smoother (the outer solver of
                            Sec. 2.3) */
    int prec;            /* lq_prec of the FP64-class steps: the plain GMRES solve (any lq_prec),
                            the FGMRES outer iteration (LQ_F64 or LQ_DF64), and prepare,
                            reconstruct and the true residual (LQ_F64 or LQ_DF64; LQ_F32 selects
                            LQ_F64 there) */
    double tol;          /* relative residual of the full system, ||b - D x|| <= tol ||b||: after the
                            reconstruction of Eq. 2 the odd residual vanishes and the even one is
                            b_hat_e - D_S x_e, so the Schur solve stops when
                            ||b_hat_e - D_S x_e|| <= tol ||b|| (recomputed, FP64-class) */
    int restart;         /* Krylov length m of each cycle, 1..256 */
    int max_restarts;    /* maximum number of cycles, >= 1 */
    int smoother;        /* lq_smoother_kind: preconditioner of FGMRES, or the method of lq_smooth */
    int smooth_n;        /* Richardson sweeps n, GMRES(n, m) cycles n, or SAP(n, m) iterations n */
    int smooth_m;        /* GMRES(n, m) cycle length m, 1..256, or SAP(n, m) Minimal Residual steps m */
    double omega;        /* Richardson weight omega = delta / |lambda_max(D_S)| (Algorithm 4) */
    double smooth_tol;   /* GMRES smoother: also stop once its relative residual <= smooth_tol
                            (0 runs exactly n cycles of m steps) */
    int inner_prec;      /* lq_prec of the smoother / preconditioner (LQ_F32 for SAP) */
    int sap_block[4];    /* SAP: block extents (even, dividing the lattice, with an even number of
                            blocks or one along each direction, at most 256 sites); zeros select
                            4 along every direction that allows it */
} lq_solver_params;

typedef struct {
    int cycles;              /* restart cycles of the (outer) solver */
    int iters;               /* Arnoldi steps of the (outer) solver */
    long long inner_iters;   /* D_S applications inside smoother / preconditioner calls */
    double rel_resid;        /* ||b_hat_e - D_S x_e|| / ||b|| at exit (FP64 or df64): recomputed when
                                the solver ran out of cycles; when it stopped on its least-squares
                                estimate, the full residual below, which equals it after Eq. 2 */
    double rel_resid_true;   /* ||b - D x|| / ||b|| on the full lattice, FP64 */
    double time_ms;          /* host wall time of the call */
    double bytes;            /* algorithmic bytes of every kernel the call launched */
    long long launches;      /* kernels the call launched */
} lq_stats;

/* Create a context for one lattice on the current CUDA device.  `stream` is a
 * cudaStream_t (NULL: the legacy default stream).  *out receives the context.
 * LQ_ERR_ARG for an odd or < 2 extent, t_bc not +-1, non-finite m0 / c_sw, or
 * a volume of 2^31 sites or more (one FP64 spinor field would exceed HBM). */
lq_status lq_create(lq_ctx **out, const lq_lattice *lat, void *stream);

/* Release the context and all library-owned device and host memory. */
lq_status lq_destroy(lq_ctx *ctx);

/* Load a gauge field (device U[V][4][3][3], complex double, natural order) and
 * build from it, on the device: the internal df64 and FP32 link copies, the
 * clover term C(x) of every site (Sec. 2.3) and the inverse D_oo^{-1} of the odd
 * blocks (6x6 Hermitian blocks, Sec. 2.4.5), both in df64 and FP32.  The FP64
 * links and clover blocks (hi + lo of the df64 copies, about 48 significand
 * bits) and the BF16 links are rounded from these when an FP64 or BF16
 * operator (or lq_export_clover) first needs them after the call.
 * Links are expected to be SU(3); the FP32 and BF16 copies keep two rows and
 * rebuild the third as conj(r1 x r2).  The caller's U may be freed on return.
 * Synchronises; LQ_ERR_BREAKDOWN if a clover block has a non-positive pivot. */
lq_status lq_set_gauge(lq_ctx *ctx, const void *U);

/* out = op(in) in precision `prec` (lq_prec): the data are read as complex
 * double, converted to the internal layout of that precision, the operator is
 * applied there and the result converted back.  Field sizes per lq_op. */
lq_status lq_apply(lq_ctx *ctx, int op, int prec, const void *in, void *out);

/* Right factor of Eq. 2: bhat_e = b_e - D_eo D_oo^{-1} b_o.
 * b: full spinor; bhat_e: even half spinor.  FP64. */
lq_status lq_prepare(lq_ctx *ctx, const void *b, void *bhat_e);

/* Left factor of Eq. 2: x_o = D_oo^{-1} (b_o - D_oe x_e); writes the full x
 * (even part = x_e).  b, x: full spinors; x_e: even half spinor.  FP64. */
lq_status lq_reconstruct(lq_ctx *ctx, const void *b, const void *x_e, void *x);

/* Power iteration on D_S^+ D_S (Sec. 2.4.4: lambda_max "computed approximately
 * with a few iterations of power iteration"): v = v0/||v0||, then `iters` times
 * w = D_S^+ D_S v, lam = ||w||, v = w/lam; *out = sqrt(lam), an estimate of
 * ||D_S||_2 >= |lambda_max(D_S)| from below.  D_S^+ = g5 D_S g5.  v0: even half
 * spinor (device); the iteration runs in precision `prec` (lq_prec).
 * Synchronises every iteration. */
lq_status lq_estimate_norm(lq_ctx *ctx, int prec, int iters, const void *v0, double *out);

/* *out = ||v||^2 for a device field of n_sites sites x 12 complex doubles.
 * Deterministic two-stage FP64 reduction.  Synchronises. */
lq_status lq_norm2(lq_ctx *ctx, const void *v, long long n_sites, double *out);

/* The smoother e = M r, started from zero, run in params->inner_prec.
 * Richardson or GMRES: the odd-even smoother M_n of Sec. 2.4.5 / Fig. 1, i.e.
 * Eq. 2 with D_S^{-1} replaced by `smooth_n` Richardson sweeps (weight omega,
 * Algorithm 4) or by GMRES(smooth_n, smooth_m) (Algorithm 2).
 * SAP: SAP(smooth_n, smooth_m) on the full lattice (Algorithm 1): red then black
 * blocks of extents sap_block, each block solved by odd-even Minimal Residual
 * with smooth_m steps (FP32; one launch per colour, one CTA per block).  As the
 * FGMRES preconditioner of lq_solve, SAP is applied to (v_e, 0) and its even
 * half taken (the even-even block of D^{-1} is D_S^{-1}).
 * r, e: full spinors. */
lq_status lq_smooth(lq_ctx *ctx, const lq_solver_params *params, const void *r, void *e);

/* Solve D x = b by odd-even reduction (Eq. 2): prepare, solve the Schur system
 * with the method in params, reconstruct.  The Krylov solver stops once its
 * least-squares estimate of the residual reaches tol ||b||; convergence is then
 * decided on the full system's residual ||b - D x|| recomputed after the
 * reconstruction, and the solve resumes (within max_restarts cycles) if that
 * residual still exceeds the tolerance.  x holds the initial guess on entry
 * (its even half starts the iteration; pass zeros for none) and the solution on
 * exit.  b, x: full spinors.  stats may be NULL.  Synchronises.
 * LQ_ERR_NOT_CONVERGED still writes the last iterate and fills stats. */
lq_status lq_solve(lq_ctx *ctx, const lq_solver_params *params, const void *b, void *x,
                   lq_stats *stats);

/* Solve D x_r = b_r for n_rhs right-hand sides together (1..256), e.g. the 12
 * spin-colour point sources of a propagator.  Sec. 3.3 names multiple right-hand
 * sides as the cache-friendly extension: here every operator launch applies D_S
 * to all right-hand sides, reading each site's links and clover block once.
 * Method: odd-even reduction (Eq. 2) per right-hand side, then defect correction
 * in df64 -- R = b_hat - D_S x, stop when ||R_r|| <= tol ||b_r|| for every r --
 * whose corrections come from batched GMRES(m) in FP32 (Algorithm 2 per right-hand
 * side, Givens least squares on the device, one CUDA-graph replay per cycle) run to
 * a relative residual of smooth_tol or smooth_n cycles.
 *   params->prec must be LQ_DF64, inner_prec LQ_F32; restart = m (1..64);
 *   max_restarts = outer corrections; smooth_n, smooth_tol as above.
 *   b, x: n_rhs full spinors back to back ([n_rhs][V][4][3], device); x holds the
 *   initial guesses on entry.  stats: NULL or n_rhs entries (cycles = iters = outer
 *   corrections of that right-hand side, inner_iters = inner Arnoldi steps launched
 *   for it; time, bytes and launches are those of the whole call).  Synchronises.
 *   LQ_ERR_NOT_CONVERGED still writes every x_r and fills stats.
 * This is lq_solve_group on a one-member group that the context keeps. */
lq_status lq_solve_batch(lq_ctx *ctx, const lq_solver_params *params, int n_rhs, const void *b, void *x,
                         lq_stats *stats);

/* A group of contexts (lattices of any sizes, on one device) whose right-hand
 * sides are solved together by lq_solve_group.  The group does not own its
 * members: destroy the group before any of them.  `stream`: the cudaStream_t
 * of the group's calls (NULL: the legacy default stream).  Errors of group
 * calls are described by lq_last_error of the first member. */
lq_status lq_group_create(lq_group **out, lq_ctx *const *members, int n_members, void *stream);
lq_status lq_group_destroy(lq_group *grp);

/* Solve D_l x_{l,r} = b_{l,r} for every member l and each of its n_rhs[l]
 * right-hand sides (1..256 each, at most 1024 in total), with the method of
 * lq_solve_batch applied to all of them at once (Sec. 3.3 names multiple
 * right-hand sides as the cache-friendly extension; here they also span
 * lattices of different sizes): odd-even reduction (Eq. 2) per right-hand side;
 * df64 defect correction per member; corrections from one batched FP32
 * GMRES(m) (Algorithm 2 per system, Givens least squares on the device) whose
 * every operator launch is a single persistent grid walking a work table of
 * (lattice, site block, right-hand sides) tiles over all members, and whose
 * cycles replay captured CUDA graphs.  The first solve of a new layout (members'
 * n_rhs, restart) lays out the workspace and, unless disabled, autotunes the
 * tile shape, grid and BLAS blocking on the group's own buffers.
 *   params: as lq_solve_batch (prec LQ_DF64, inner_prec LQ_F32, restart 1..64).
 *   b[l], x[l]: device [n_rhs[l]][V_l][4][3] complex double; x holds initial
 *   guesses.  stats: NULL or sum(n_rhs) entries, member by member.
 * Synchronises.  LQ_ERR_NOT_CONVERGED still writes every x and fills stats. */
lq_status lq_solve_group(lq_group *grp, const lq_solver_params *params, const int *n_rhs, const void *const *b,
                         void *const *x, lq_stats *stats);

/* Autotuning of the group's launch shapes on (default) or off (fixed shapes:
 * 32 sites x 4 right-hand sides per tile, twice the resident blocks); drops the
 * current layout and captured graphs. */
lq_status lq_group_set_autotune(lq_group *grp, int on);

/* Pin the launch shape of the batched hop instead of autotuning it:
 * sites_per_tile 16, 32, 64 or 128 with rhs_per_thread 1 or 2 (each thread one
 * or two right-hand sides of one site), or sites_per_tile 32 or 64 with
 * rhs_per_thread 0 (the staged form: a tile's links and clover blocks are read
 * once into shared memory and applied to every right-hand side of its lattice);
 * grid_factor 1 or 2 (times the resident blocks, persistent) or 0 (one block
 * per tile).  The BLAS
 * blocking keeps its default.  Drops the current layout and captured graphs;
 * lq_group_set_autotune(grp, 1) returns to autotuning. */
lq_status lq_group_set_shape(lq_group *grp, int sites_per_tile, int rhs_per_thread, int grid_factor);

/* The launch shapes in use after a solve: sites per tile of the batched hop,
 * right-hand sides per thread (1 or 2; right-hand sides per tile =
 * rhs_per_thread * 128 / sites_per_tile; 0 for the staged form, whose tiles
 * cover every right-hand side), its grid, BLAS blocks per system,
 * and the measured times of the chosen hop pair and BLAS pair (0 if untuned).
 * LQ_ERR_STATE before the first solve.  Any pointer may be NULL. */
lq_status lq_group_tuning(lq_group *grp, int *sites_per_tile, int *rhs_per_thread, int *grid, int *blas_blocks,
                          double *hop_ms, double *blas_ms);

/* Gradient of the bilinear form b(U) = Re(Y^+ D(U) X) with respect to every
 * link, for given full spinors X and Y (no paper counterpart: the operator is
 * the Wilson-clover D of Sec. 2.3, differentiated through its hopping term and
 * through the plaquette leaves of its clover term).
 *   G: device complex double [V][4][3][3] in the layout of the gauge field;
 *   G = coef * (db/dRe U + i db/dIm U), so that db = Re sum conj(G) dU.
 * Computed in df64 (FP64-accurate).  Needs lq_set_gauge.  Enqueued on the
 * context's stream; does not synchronise. */
lq_status lq_force(lq_ctx *ctx, const void *X, const void *Y, double coef, void *G);

/* The pseudofermion action S = phi^+ (D^+ D)^{-1} phi of the gauge field set
 * by lq_set_gauge (no paper counterpart).  With D^+ = g5 D g5:
 * Y = D^{-+} phi = g5 D^{-1} g5 phi and X = D^{-1} Y = (D^+ D)^{-1} phi by two
 * lq_solve calls with `params` (initial guesses zero), and S = ||Y||^2.
 *   phi: device full spinor; X, Y: device full spinors written by the call (the
 *   inputs lq_force needs for dS/dU = -2 grad_U Re(Y^+ D X)); S: host double;
 *   stats: NULL or two entries (the two solves).
 * Synchronises.  LQ_ERR_NOT_CONVERGED still writes X, Y and S from the last
 * iterates. */
lq_status lq_fermion_action(lq_ctx *ctx, const lq_solver_params *params, const void *phi, void *X, void *Y,
                            double *S, lq_stats *stats);

/* lq_fermion_action followed by lq_force(X, Y, -2): S and its gradient
 * G = dS/dU ([V][4][3][3] as in lq_force), with X and Y in library-owned
 * workspace.  Synchronises; LQ_ERR_NOT_CONVERGED as above. */
lq_status lq_fermion_force(lq_ctx *ctx, const lq_solver_params *params, const void *phi, double *S, void *G,
                           lq_stats *stats);

/* Copy the clover blocks out for inspection: which = 0 gives C(x), which = 1
 * gives C(x)^{-1} (odd sites only; even entries are zero).  out: device
 * complex double [V][2][6][6], natural site order, block 0 = spins {0,1},
 * block 1 = spins {2,3}, index (spin%2)*3 + colour. */
lq_status lq_export_clover(lq_ctx *ctx, int which, void *out);

/* Kernel classes of the per-class device timing. */
typedef enum {
    LQ_K_HOP_K1_F64 = 0, /* K1: t_o = D_oo^{-1} D_oe x_e, FP64 */
    LQ_K_HOP_K1_F32,     /* K1, FP32 */
    LQ_K_HOP_K2_F64,     /* K2: y_e = D_ee x_e - D_eo t_o (and its fused Richardson form), FP64 */
    LQ_K_HOP_K2_F32,     /* K2, FP32 */
    LQ_K_HOP_OTHER,      /* full-lattice D, prepare, reconstruct, clover apply */
    LQ_K_CLOVER,         /* clover assembly from the field strengths, inverse (df64 and FP32), export */
    LQ_K_LAYOUT,         /* natural <-> internal layout, precision conversion, gamma5 */
    LQ_K_DOT_F64, LQ_K_DOT_F32,    /* multi-dot products */
    LQ_K_AXPY_F64, LQ_K_AXPY_F32,  /* axpby / multi-axpy */
    LQ_K_NORM,           /* norms */
    LQ_K_FINISH,         /* second stage of the deterministic reductions, and the small kernels
                            that move solver scalars between host and device */
    LQ_K_COPY,           /* field copies (a kernel) and memsets (not kernels) */
    LQ_K_HOP_K1_DF64, LQ_K_HOP_K2_DF64,   /* K1, K2 in df64 */
    LQ_K_DOT_DF64, LQ_K_AXPY_DF64,        /* BLAS-1 in df64 */
    LQ_K_CLOVER_FIELD,   /* field strengths F_munu of the six planes from the leaves (df64) */
    LQ_K_FORCE,          /* fermion force: clover insertion and per-link gradient (df64) */
    LQ_K_SAP,            /* SAP block solves (FP32) */
    LQ_K_HOP_K1_BF16, LQ_K_HOP_K2_BF16,   /* K1, K2 (and the fused Richardson form) with BF16 storage */
    LQ_K_COUNT
} lq_kernel_class;

/* Start (on != 0, clearing earlier records) or stop recording a pair of CUDA
 * events on the context's stream around every launch. */
lq_status lq_profile(lq_ctx *ctx, int on);

/* Totals of the records of one kernel class since lq_profile(ctx, 1): launches,
 * summed device time in milliseconds, algorithmic bytes and algorithmic flops
 * (FP64-equivalent flops for df64 kernels).  Synchronises.  Any output pointer
 * may be NULL. */
lq_status lq_profile_read(lq_ctx *ctx, int cls, long long *launches, double *ms, double *bytes, double *flops);

/* A static name for a kernel class ("" when out of range). */
const char *lq_kernel_class_name(int cls);

/* Counters since the context was created: kernels launched and their
 * algorithmic bytes.  Either pointer may be NULL. */
lq_status lq_counters(lq_ctx *ctx, long long *launches, double *bytes);

/* Largest field lq_norm2_noalloc accepts, in sites (12 complex doubles each):
 * 4096 partial sums of 8192 complex values each, divided by 12. */
#define LQ_NORM2_NOALLOC_MAX_SITES 2796202LL

/* The paper has no counterpart of this call: it serves callers that cannot
 * allocate device memory (for example code that works inside a fixed memory
 * budget handed out by another framework, where a cudaMalloc could fail or
 * synchronise the device at the wrong moment).  It computes the same value as
 * lq_norm2 -- *out = ||v||^2 for a device field of n_sites sites x 12 complex
 * doubles -- but needs no context and allocates nothing: its reduction scratch
 * is a static device array of 4096 doubles (32 KiB) inside the library, which
 * every GPU that loads the library keeps until the process exits.
 *   v:      device, n_sites x 12 complex doubles (may be NULL when n_sites == 0)
 *   out:    device pointer to ONE double, written on `stream`
 *   stream: cudaStream_t (NULL: the legacy default stream)
 * The call only enqueues work and does not synchronise.  The first call on a
 * device looks up the scratch array's device address for that device (with it
 * current) and caches it.  With CUDA's lazy module loading (the default), that
 * first call may also load the library's module on the device, which allocates
 * the device's copy of the array and of the kernels' code: make the first call
 * on each device at set-up, outside any fixed memory budget, and before any
 * stream capture.  Later calls allocate nothing.
 * All calls share the one scratch array, which keeps the last call's partial
 * sums; each call writes every slot it reads, so nothing needs clearing, but
 * calls whose kernels overlap on the GPU (different streams, or different host
 * threads on one device) race on it and must be serialised by the caller.
 * Errors: LQ_ERR_ARG for a NULL pointer, n_sites < 0 or
 * n_sites > LQ_NORM2_NOALLOC_MAX_SITES (nothing is launched); LQ_ERR_CUDA if
 * the device, the scratch address or a launch fails, or if a launch error from
 * earlier work is pending on the calling thread (nothing is launched then, and
 * that error is left for its owner to read). */
lq_status lq_norm2_noalloc(const void *v, long long n_sites, double *out, void *stream);

/* The index checks of the checked build (no paper counterpart: a test aid).
 * A library compiled with -DLQ_BOUNDS (LQ_NVCC_EXTRA, or build(checked=True),
 * which writes liblqdd_checked.so) range-checks every computed neighbour,
 * site, block-local and layout-tile index inside its kernels against the
 * extent of the array it indexes.  A failed check does not trap: the kernel
 * counts it, remembers the code of the first one (the enum BoundsSite of the
 * internal header: 1 hop site, 2 hop neighbour, 3 df64 hop neighbour, 4
 * batched-hop neighbour, 5 SAP block-local, 6 SAP lattice, 7 clover/force
 * lexicographic, 8 layout) and uses index 0 instead, so the access stays in
 * bounds.  This call synchronises the current device, reads and clears those
 * flags and returns LQ_ERR_BOUNDS if any check failed since the last call,
 * else LQ_OK.  *checked = 1 in a checked build, 0 otherwise (where nothing is
 * checked and the call returns LQ_OK).  Any pointer may be NULL. */
lq_status lq_bounds_check(int *checked, unsigned long long *violations, int *first_code);

/* A static description of the last failure on this context ("" if none). */
const char *lq_last_error(lq_ctx *ctx);

/* A static name for a status code. */
const char *lq_status_string(lq_status s);

#ifdef __cplusplus
}
#endif

#endif /* LQDD_H */
