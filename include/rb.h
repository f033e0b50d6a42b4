/*
 * rb.h - C interface of librb: the online phase of the reduced-basis (RB)
 * iteration (Alg. 2) and RB-preconditioned conjugate gradients (Alg. 3) for
 * many-query parametrized SPD systems A(mu) x = f(mu) (eq. 1) with the affine
 * form A(mu) = sum_q Theta_q(mu) A_q, f(mu) = sum_r Phi_r(mu) f_r (eq. 12).
 *
 * Problem family.  -div(kappa grad u) = f on the unit square / cube with
 * u = 0 on the boundary, discretised by finite differences on m_d interior
 * nodes per direction (h_d = 1/(m_d+1), x fastest).  kappa = mu_p on block p
 * of a box partition, block of node i_d is floor(i_d * nb_d / m_d); a face
 * between two nodes carries (mu_p(i) + mu_p(j))/2, a face to the boundary
 * mu_p(i).  Theta_q(mu) = mu_q, Q = P = nb_x nb_y nb_z.
 * With coefficient fields (rb_problem.n_fields = Q > 0; the paper's Section 5
 * cases) the node coefficient is kappa(i) = sum_q mu_q F_q(i) with given node
 * values F_q and the same face rule, so A(mu) = sum_q mu_q A_q still holds.
 * Non-zero Dirichlet data enter as load terms (RB_LOAD_BOUNDARY): the face of
 * node i to boundary node j carries kappa(i), so g(j) moves to the right-hand
 * side as sum_q mu_q F_q(i) g(j) / h_d^2, one load term per field.
 *
 * Conventions for every call:
 *  - Vectors of a batch are [B][N_dof] doubles, query-major, x fastest.
 *  - Pointers named "host or device" may point to either; the library asks
 *    the CUDA runtime which one it is.  Host buffers are copied in and out
 *    inside the call.  Device buffers must be allocated on the current device.
 *  - Parameter vectors mu are always host memory, [B][n_mu] doubles.
 *  - Calls are ordered on opts->stream (NULL = legacy default stream) and are
 *    synchronous: they return after the per-query statistics are on the host.
 *  - A context is not reentrant: one call at a time per rb_ctx.
 *  - Errors: every call returns an rb_status; rb_last_error() gives the text
 *    of the last failure on that context.  Per-query outcomes go to
 *    stats[i].status; the call returns the worst of them.
 */
#ifndef RB_H
#define RB_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rb_ctx rb_ctx;
typedef struct rb_mlp rb_mlp;   /* learned warm-start network (rb_mlp_create) */

typedef enum {
    RB_OK = 0,
    RB_EINVAL = 1,      /* bad argument (dimensions, null pointer, non-finite mu) */
    RB_ENOMEM = 2,      /* device or host allocation failed */
    RB_EFORMAT = 3,     /* malformed or corrupted basis file */
    RB_ECUDA = 4,       /* a CUDA runtime call failed */
    RB_EBREAKDOWN = 5,  /* non-positive Cholesky pivot, p^T A p <= 0 or NaN */
    RB_ENOCONV = 6,     /* iteration budget spent before the tolerance was met */
    RB_ETIMEOUT = 7,    /* a device-side wait gave up */
    RB_EIO = 8          /* file could not be opened, read or written */
} rb_status;

/* One load term f_r of f(mu) = sum_r Phi_r(mu) f_r (eq. 12). */
enum { RB_LOAD_CONST = 0, RB_LOAD_GAUSS = 1, RB_LOAD_ARRAY = 2, RB_LOAD_BOUNDARY = 3 };
typedef struct {
    int kind;           /* RB_LOAD_CONST: f_r = 1; RB_LOAD_GAUSS: exp(-|x-c|^2/(2 sigma^2));
                           RB_LOAD_ARRAY: f_r(i) = values[i] ([N_dof]);
                           RB_LOAD_BOUNDARY: the lift of Dirichlet data g through field
                           `field`: f_r(i) = sum over the faces of node i to a boundary node j
                           of F_field(i) g(j) / h_d^2, with g = values on the grid extended by
                           the boundary layer ([m_z+2][m_y+2][m_x+2], x fastest; 2D:
                           [m_y+2][m_x+2]; only the boundary layer is read).  In a block
                           problem F_q is the indicator of block q. */
    int param;          /* -1: Phi_r = 1; otherwise Phi_r(mu) = mu[param] */
    double center[3];
    double sigma;
    int field;          /* RB_LOAD_BOUNDARY: q in 0..Q-1 */
    const double* values;   /* RB_LOAD_ARRAY / RB_LOAD_BOUNDARY: host memory, copied when a
                               context is created (NULL for the other kinds) */
} rb_load;

typedef struct {
    int dim;            /* 2 or 3 */
    int m[3];           /* interior nodes per direction; m[2] = 1 when dim = 2 */
    int nb[3];          /* blocks per direction; nb[2] = 1 when dim = 2; all 1 with fields */
    int n_loads;        /* R >= 1 */
    const rb_load* loads;
    int n_mu;           /* entries of one parameter vector (>= P and > every load param) */
    int n_fields;       /* 0: block coefficients; Q >= 1: coefficient fields, P = Q */
    const double* fields;   /* [Q][N_dof] node values F_q (host, copied when a context is created;
                               NULL when n_fields = 0).  On 3D grids whose rows hold a
                               multiple of 4 points field problems run the z-march tile kernels
                               (rb_opts.kernels = 0; they read kappa(mu) at the nodes), elsewhere
                               the generic stencil kernels. */
} rb_problem;

enum { RB_SMOOTH_NONE = 0, RB_SMOOTH_RBGS = 1, RB_SMOOTH_JACOBI = 2 };
enum { RB_PREC_FP64 = 0, RB_PREC_MIXED = 1 };
enum { RB_BETA_FR = 0, RB_BETA_PR = 1 };
enum { RB_X0_ZERO = 0, RB_X0_GIVEN = 1, RB_X0_RB = 2 };
enum { RB_GEMM_AUTO = 0, RB_GEMM_CUDA_CORES = 1, RB_GEMM_TENSOR = 2 };
enum { RB_STORE_F32 = 0, RB_STORE_BF16 = 1 };

typedef struct {
    double tol;         /* stop at ||f - A x|| / ||f|| < tol (true FP64 residual) */
    int max_iter;       /* iteration budget per query */
    int smoother;       /* RB_SMOOTH_*: S(A, b, y) of eq. 8 */
    int nu;             /* smoother sweeps per application */
    double omega;       /* Jacobi weight */
    int precision;      /* RB_PREC_FP64: all FP64; RB_PREC_MIXED: FP32 inner RBCG
                           with FP64 residual refinement (rb_pcg only) */
    int beta_form;      /* RB_BETA_FR (Alg. 3 as printed) or RB_BETA_PR */
    int x0_mode;        /* RB_X0_ZERO; RB_X0_GIVEN (x holds the start on entry); RB_X0_RB: start
                           from the RB approximation x_hat(mu) = W a_N(mu) of eq. 3 (Galerkin
                           coefficients of eq. 2 by FP64 Cholesky, lifted with the FP64 basis) -
                           the point the first step of Alg. 2 / Alg. 3 reaches; with a basis that
                           resolves the solution it saves the mixed solver its FP32 cycles */
    double inner_tol;   /* mixed: relative residual reduction of each FP32 solve */
    int max_outer;      /* mixed: maximum FP64 refinement steps */
    int gemm;           /* RB_GEMM_*: engine for the batched W^T R and W E products */
    int graph;          /* 1: replay the iteration body as a captured CUDA graph */
    int kernels;        /* stencil kernels on 2D grids whose rows hold a multiple of 128 points:
                           0: CG body and one smoother pass per sweep with rows staged in shared
                              memory by bulk asynchronous copies;
                           1: as 0, but all red-black sweeps fused in one pass (FP32 mixed path,
                              nu <= 6);
                           2: CG body and one smoother pass per sweep with rows held in registers;
                           3: as 0, but up to three red-black sweeps per pass over memory (FP32
                              mixed path with FP32 storage; other cases as 0);
                           4: as 3 with up to two sweeps per pass.
                           On 3D grids (RBCG): 0 marches the CG body, the red-black smoother and
                           the FP64 outer residual in z with planes prefetched into shared memory
                           by asynchronous tensor copies; 1 the smoother marching in z with direct
                           loads and the generic CG body (block coefficients only); 2 the generic
                           kernels.  Other grids take the generic kernels. */
    int store;          /* RB_STORE_*: storage of the preconditioner's intermediate vectors (the
                           prolongation W e_N and the smoother sweeps before the last one).
                           RB_STORE_BF16 halves their bytes; the arithmetic stays FP32 and the
                           preconditioned residual y is FP32.  It applies to the mixed solver with
                           the red-black smoother and kernels = 0 on 2D grids whose rows hold a
                           multiple of 128 points; elsewhere the storage is FP32. */
    int adaptive_n;     /* RBCG only (rb_pcg; rb_solve ignores it).  0: every preconditioner
                           application uses the whole basis.  k >= 1: the adaptive choice of N at the
                           end of Section 4.1: start with the first k basis vectors (W_k, nested in W_n)
                           and use one more after every iteration whose recurrence residual fell by
                           less than gamma, ||r_k|| / ||r_{k+1}|| < gamma, up to n. */
    double gamma;       /* ratio of that test (the paper suggests 10) */
    void* stream;       /* cudaStream_t or NULL */
} rb_opts;

typedef struct {
    int iters;          /* RBI: corrections applied; RBCG: matrix-vector products (inner ones in mixed mode) */
    int outer;          /* FP64 residual evaluations (refinement steps + final check) */
    int restarts;       /* residual replacements after a failed true-residual check */
    int status;         /* rb_status of this query */
    double rel_res;     /* final true ||f - A x|| / ||f|| in FP64 */
    int n_used;         /* basis vectors of the last preconditioner application (n unless adaptive) */
} rb_stats;

typedef struct {
    double truth_tol;   /* relative residual of the snapshot solves (default 1e-11) */
    int truth_max_iter; /* budget of one snapshot solve (default 200000) */
    int score;          /* 0: L1 norm of the coefficients in the snapshot basis; 1: literal RB coefficients */
    double drop_tol;    /* a snapshot whose Gram-Schmidt remainder is below drop_tol ||x|| is skipped */
} rb_build_opts;

/* Fill defaults: tol 1e-10, red-black Gauss-Seidel with nu = 1, FP64, PR beta,
 * zero start, inner_tol 1e-5, max_outer 12, automatic GEMM engine, graphs on,
 * staged kernels (kernels = 0), FP32 storage, fixed N (adaptive_n 0, gamma 10). */
void rb_default_opts(rb_opts* opts);
void rb_default_build_opts(rb_build_opts* opts);

/*
 * Online context from precomputed offline arrays (Section 2.3, eq. 12c).
 *   W   host, [N_dof][n] row-major: the orthonormal basis W_N;
 *   ANq host, [Q][n][n]: A_{N,q} = W^T A_q W;  fNr host, [R][n]: f_{N,r} = W^T f_r.
 *   n may be 0 (no basis: the RB correction is skipped).
 * max_batch fixes the device workspace: larger batches are run in waves.
 * All device memory of the context is allocated here; solves allocate nothing.
 * On failure *out is NULL and nothing is leaked.
 */
rb_status rb_offline_load_arrays(rb_ctx** out, const rb_problem* prob, int n,
                                 const double* W, const double* ANq, const double* fNr,
                                 int max_batch);

/* Offline greedy (Alg. 1 steps, snapshots solved on the device by RBCG with
 * W_{N-1} as in Alg. 4, in solve_opts->precision: FP64, or FP32 inner RBCG with
 * FP64 residual refinement, both to the FP64 relative residual truth_tol;
 * Gram-Schmidt twice; eq. 12c grown one row and column per step).  mu_train host [n_train][n_mu]; the first training vector is mu_1.
 * Produces a context with n = n_max basis vectors (fewer if the training set
 * runs out of independent snapshots). */
rb_status rb_offline_build(rb_ctx** out, const rb_problem* prob, int n_max, int n_train,
                           const double* mu_train, const rb_build_opts* bopts,
                           const rb_opts* solve_opts, int max_batch);

/* Multi-fidelity offline build (Section 4.2, last paragraph): the greedy of
 * rb_offline_build runs on the coarse problem (the fine problem's block
 * partition, loads and parameters on a coarser grid) and selects the
 * parameter sample S_N; the snapshots of S_N are then solved on the fine grid
 * (RBCG with W_{N-1}, as Alg. 4, in solve_opts->precision) and orthonormalised
 * in the selection order into the fine basis.  A fine snapshot that falls inside
 * the span of the previous ones is skipped.  RB_EINVAL when the two problems
 * differ in anything but the grid. */
rb_status rb_offline_build_mf(rb_ctx** out, const rb_problem* fine, const rb_problem* coarse, int n_max, int n_train,
                              const double* mu_train, const rb_build_opts* bopts, const rb_opts* solve_opts,
                              int max_batch);

/* Basis file (.rbb): header, W, A_{N,q}, f_{N,r}, snapshot factor R,
 * selected training indices, FNV-1a checksum.  Load fails with RB_EFORMAT on a
 * bad magic, size or checksum and RB_EIO when the file cannot be read. */
rb_status rb_save(const rb_ctx* ctx, const char* path);
rb_status rb_offline_load(rb_ctx** out, const char* path, int max_batch);

/* Sizes of a context: N_dof, basis size n, Q (= P), R, n_mu. Any pointer may be NULL. */
rb_status rb_info(const rb_ctx* ctx, long long* n_dof, int* n, int* Q, int* R, int* n_mu);

/* Copy the offline data back to host arrays laid out as in
 * rb_offline_load_arrays; Rsnap [n][n] (upper, X = W R; zero if unknown),
 * selected [n] (-1 if unknown).  Any pointer may be NULL. */
rb_status rb_get_basis(const rb_ctx* ctx, double* W, double* ANq, double* fNr,
                       double* Rsnap, int* selected);

/*
 * RB iteration, Alg. 2: x <- 0; repeat r = f - A x (stop when ||r|| < tol ||f||),
 * r_N = W^T r (eq. 5), A_N e_N = r_N (eq. 6, Cholesky), x += W e_N (eq. 7),
 * x = S(A, f, x) (eq. 8).  FP64 throughout.
 *   mu host [B][n_mu];  x host or device [B][N_dof], written with the solutions
 *   (read first when opts->x0_mode == RB_X0_GIVEN);  stats host [B] or NULL.
 */
rb_status rb_solve(rb_ctx* ctx, int B, const double* mu, double* x,
                   const rb_opts* opts, rb_stats* stats);

/*
 * RB-preconditioned CG, Alg. 3, preconditioner y = RBI(A, r, W, 1) from zero:
 * y = W A_N^{-1} W^T r then S(A, r, y).  opts->precision selects plain FP64 or
 * the mixed scheme (FP32 inner RBCG, TF32/FP32 projections, FP64 residual and
 * solution, iterative refinement to opts->tol).  Arguments as rb_solve.
 */
rb_status rb_pcg(rb_ctx* ctx, int B, const double* mu, double* x,
                 const rb_opts* opts, rb_stats* stats);

/*
 * Ragged batch: several problems, each with its own context (grid, basis and
 * workspace), solved by RBCG (Alg. 3, as rb_pcg) in one launch sequence.  Each
 * round enqueues the next steps of every unfinished context on that context's
 * own stream, so the kernels of the different grids run side by side on the
 * GPU, then polls them all.  ctxs [nctx] distinct contexts (nctx <= 16);
 * B [nctx] queries of each (0 .. max_batch of that context, one wave each);
 * mu [nctx] host [B[c]][n_mu]; x [nctx] device [B[c]][N_dof] of context c;
 * stats [nctx] host [B[c]] each, or stats NULL; opts as rb_pcg (opts->stream,
 * when set, is waited for first; the contexts then use their own streams).
 * Returns the worst status over all queries; errors of a context go to its
 * rb_last_error, argument errors before any context to rb_last_error(NULL).
 */
rb_status rb_pcg_ragged(rb_ctx* const* ctxs, int nctx, const int* B, const double* const* mu, double* const* x,
                        const rb_opts* opts, rb_stats* const* stats);

/* The two batched products of the RB preconditioner in FP32 storage, with the
 * engine of the mixed path: WtR[b] = W^T R[b] (eq. 5, as in Alg. 2 step 4) and
 * WE[b] = W E[b] (eq. 7, as in Alg. 2 step 6).  engine: RB_GEMM_CUDA_CORES
 * (FP32 FMA), RB_GEMM_TENSOR (tcgen05 with TF32 operands, FP32 accumulation;
 * RB_EINVAL where unavailable) or RB_GEMM_AUTO.  R host or device [B][N_dof]
 * float, WtR host [B][n] double; E host [B][n] float, WE host or device
 * [B][N_dof] float.  Either pair may be NULL.  B <= max_batch.  Uses the
 * context's workspace (overwrites solver state; not during a solve). */
rb_status rb_products(rb_ctx* ctx, int B, const float* R, double* WtR, const float* E, float* WE, int engine);

/* The RB preconditioner of Alg. 3 (steps 2 and 9): y_b = RBI(A(mu_b), r_b, W, 1)
 * from zero, i.e. y = W A_N^{-1} W^T r (eqs. 5-7) followed by opts->nu sweeps of
 * the smoother S(A, r, y) (eq. 8).  opts->precision selects FP64 (r, y double)
 * or the mixed inner precision (r, y float; TF32 or FP32 products, FP32
 * smoother); opts->kernels and opts->gemm select the kernels.  mu host
 * [B][n_mu]; r, y host or device [B][N_dof]; B <= max_batch.  Uses the
 * context's workspace (not during a solve).  RB_EBREAKDOWN if A_N(mu) is not SPD. */
rb_status rb_precondition(rb_ctx* ctx, int B, const double* mu, const void* r, void* y, const rb_opts* opts);

/* y = A(mu_b) x_b for every query b (eq. 1 operator, FP64).  x, y host or device
 * [B][N_dof]; stream as in rb_opts (may be NULL). */
rb_status rb_apply(rb_ctx* ctx, int B, const double* mu, const double* x, double* y,
                   void* stream);

/* Autotuner.  Times rb_pcg on the B sample queries (host mu; x host or device
 * [B][N_dof] scratch) and picks, by coordinate descent from *opts, the smoother
 * sweep count nu (1..6, then 2..9 once a smoother with several sweeps per pass is
 * chosen; the paper leaves the smoother's iteration count open, Section 3.1) for each storage of the preconditioner's intermediate vectors that
 * applies (rb_opts.store), the FP32 cycle reduction inner_tol (1e-4, 1e-5, 1e-6;
 * mixed only), the smoother kernels (rb_opts.kernels), the GEMM engine (mixed
 * only) and the start (zero or the RB approximation).  Only configurations under which every
 * sample query converges are eligible.  Writes the fastest into *opts and
 * summarises it in *res (may be NULL). */
typedef struct {
    int nu;
    double inner_tol;
    int gemm;
    double ms_per_solve;   /* of the chosen configuration on the sample */
    int trials;
    int kernels;
    int store;
    int x0_mode;           /* RB_X0_ZERO or RB_X0_RB (tried when opts->x0_mode is not RB_X0_GIVEN) */
} rb_tune_result;
rb_status rb_autotune(rb_ctx* ctx, int B, const double* mu, double* x, rb_opts* opts, rb_tune_result* res);

/* Per-kernel timing.  rb_profile(ctx, 1) clears the counters and from then on
 * brackets every kernel launch of rb_solve / rb_pcg with CUDA events on the
 * call's stream (the iteration body is then launched directly, not as a CUDA
 * graph); rb_profile(ctx, 0) stops.  rb_profile_read copies up to cap entries
 * (one per kernel kind that ran: launches and summed device milliseconds) and
 * sets *count to the number of kinds. */
typedef struct {
    char name[24];
    long long launches;
    double ms;
} rb_kernel_time;
rb_status rb_profile(rb_ctx* ctx, int enable);
rb_status rb_profile_read(const rb_ctx* ctx, rb_kernel_time* out, int cap, int* count);

/* Measured FMA rate of the current device: *flops_per_s = 2 x FMAs per second of a
 * launch that fills every SM with independent chains of dependent fused multiply-adds
 * (fp64 = 1: double, 0: float), timed with CUDA events on stream (NULL = legacy default
 * stream) after one warm-up launch of the same size; about 50-200 ms in all.  It is the
 * denominator of the roofline of a kernel bound by arithmetic rather than by memory (the
 * FP64 outer residual of the mixed solver).  Allocates and frees a few MB of device
 * memory; needs no context.  RB_EINVAL if flops_per_s is NULL. */
rb_status rb_fma_rate(int fp64, double* flops_per_s, void* stream);

/*
 * Starting vectors.  Alg. 2 and Alg. 3 start from x_0 = 0 but accept any x_0
 * (rb_opts.x0_mode = RB_X0_GIVEN).  rb_warm_start writes x_b = W c_b with
 *   net == NULL: c_b = a_N(mu_b), the Galerkin coefficients of eq. 2
 *                (A_N(mu) a = f_N(mu), eq. 12b, Cholesky in FP64), so x_b is
 *                the RB approximation x_hat(mu) of eq. 3;
 *   net != NULL: c_b = the network's prediction for mu_b (rb_mlp_predict);
 *                net must have n_in = n_mu and n_out = n of the context.
 * The lift W c runs on FP32 copies of W and c (relative error about 1e-7; the
 * solvers correct it).  mu host [B][n_mu] (diffusion coefficients > 0);
 * x host or device [B][N_dof], written; coef host or device [B][n], written
 * when not NULL.  Uses the context's workspace (not during a solve).
 * RB_EBREAKDOWN if A_N(mu_b) is not SPD for some b (its c_b and x_b are zero).
 */
rb_status rb_warm_start(rb_ctx* ctx, rb_mlp* net, int B, const double* mu, double* x, double* coef,
                        void* stream);

/*
 * Error basis of the learned warm start.  A start in span(W) is sent by the
 * first RB correction of Alg. 3 to about the same iterate (the paper's
 * analysis of Alg. 2 from any start in span(W)), so the learned start that can
 * gain leaves span(W): x_0 = x_hat(mu) + V z(mu), with x_hat = W a_N(mu) the RB
 * approximation of eq. 3 and V an orthonormal basis of the errors
 * e_s = x_s - x_hat(mu_s) of training solutions (the paper has no learned
 * component; this is an addition to its method).
 *
 * rb_error_basis: proper orthogonal decomposition of the errors of S training
 * solutions by the method of snapshots (Gram matrix E^T E in FP64 on the
 * device, its eigenpairs on the host): V = E Phi_m diag(lambda_m)^{-1/2}, m
 * modes kept in the context (FP64 and an FP32 copy, allocated here; a later
 * call replaces them).  mu host [S][n_mu] (diffusion coefficients > 0);
 * X host or device [S][N_dof] (solutions, e.g. from rb_pcg); 1 <= S <=
 * min(max_batch, 512); 1 <= m <= min(S, 64).  Z host or device [S][m] or
 * NULL: Z = V^T E (the targets of a network); sigma host [m] or NULL: the
 * singular values of E (a mode below 1e-12 of the largest is set to zero).
 * Uses the context's workspace (not during a solve).
 */
rb_status rb_error_basis(rb_ctx* ctx, int S, const double* mu, const double* X, int m, double* Z, double* sigma,
                         void* stream);

/* Z_b = V^T (x_b - x_hat(mu_b)) for B solutions (host or device [B][N_dof]) and
 * host mu [B][n_mu]; Z host or device [B][m].  FP32 products, FP64 sums.
 * RB_EINVAL without an error basis. */
rb_status rb_error_coefficients(rb_ctx* ctx, int B, const double* mu, const double* X, double* Z, void* stream);

/* x_b = x_hat(mu_b) + V z_b with z_b from the network (net != NULL: n_in = n_mu,
 * n_out = m) or given (z host or device [B][m], net == NULL; exactly one of the
 * two).  x host or device [B][N_dof], written; the lifts run on FP32 copies of
 * W and V (relative error about 1e-7; the solvers correct it).  A start for
 * rb_pcg with rb_opts.x0_mode = RB_X0_GIVEN. */
rb_status rb_warm_start_error(rb_ctx* ctx, rb_mlp* net, int B, const double* mu, double* x, const double* z,
                              void* stream);

/* Reduced coefficients c_b = W^T x_b of given vectors (eq. 5 applied to x
 * instead of r): with an orthonormal W, W c_b is the orthogonal projection of
 * x_b onto span(W).  FP32 products, FP64 sums over chunks of 32 points
 * (relative error about 1e-7).  x host or device [B][N_dof]; coef host or
 * device [B][n], written.  Uses the context's workspace (not during a solve). */
rb_status rb_coefficients(rb_ctx* ctx, int B, const double* x, double* coef, void* stream);

/*
 * Learned warm start: a network c(mu) predicting reduced coefficients (the
 * paper has no learned component; the network only supplies x_0 = W c(mu) to
 * rb_warm_start; the RB iterations then remove whatever error the prediction has).
 *   features   log mu_i for i < n_log (diffusion coefficients), mu_i for
 *              n_log <= i < n_in (load parameters), standardised by the
 *              per-column mean and population standard deviation (floored at
 *              1e-12) of the training set of the first fit / gradient call;
 *   layers     n_in -> hidden -> hidden -> n_out, GELU (z Phi(z), Phi the
 *              standard normal CDF) after both hidden layers, linear output;
 *   output     c = out_mean + out_scale * y, out_mean / out_scale the
 *              per-column statistics of the training targets;
 *   precision  weights used as BF16 (FP32 masters rounded to nearest even),
 *              biases and activations FP32, products accumulated in FP32;
 *   training   loss = sum (y - t)^2 / (S n_out) over standardised targets t,
 *              full batch, back-propagation, Adam (beta1 0.9, beta2 0.999,
 *              eps 1e-8) on the FP32 masters; the gradient treats the BF16
 *              rounding as the identity.
 * Flat parameter vector (doubles, this order): W1 [hidden][n_in], b1 [hidden],
 * W2 [hidden][hidden], b2 [hidden], W3 [n_out][hidden], b3 [n_out].
 * Errors of these calls are reported by rb_last_error(NULL).  A network is not
 * reentrant: one call at a time.
 */

/* n_in <= 32, hidden <= 128, n_out <= 128; params host [rb_mlp_num_params]
 * (initial values); max_samples bounds S of fit / gradient and the device
 * staging of predict.  All device memory of the network is allocated here. */
rb_status rb_mlp_create(rb_mlp** out, int n_in, int n_log, int hidden, int n_out, const double* params,
                        int max_samples);
int rb_mlp_num_params(const rb_mlp* net);   /* -1 for NULL */

/* steps (<= 65536) Adam steps with learning rate lr on the S training pairs:
 * mu host [S][n_in], Y host or device [S][n_out] (target coefficients).
 * loss host or device [steps] or NULL: the loss before each step.  The step
 * body is replayed as a CUDA graph; synchronous. */
rb_status rb_mlp_fit(rb_mlp* net, int S, const double* mu, const double* Y, int steps, double lr, double* loss,
                     void* stream);

/* Loss and gradient of the current parameters on S pairs (no update):
 * loss host or device [1], grad host or device [rb_mlp_num_params] (layout of
 * the parameter vector); either may be NULL. */
rb_status rb_mlp_gradient(rb_mlp* net, int S, const double* mu, const double* Y, double* loss, double* grad,
                          void* stream);

/* Y [B][n_out] (host or device) = c(mu_b) for mu host [B][n_in].  Needs the
 * standardisation of a fit or gradient call. */
rb_status rb_mlp_predict(rb_mlp* net, int B, const double* mu, double* Y, void* stream);

/* Read back the FP32 master parameters (as doubles, host [num_params]), the
 * standardisation (host [2 n_in + 2 n_out]: in_mean, in_scale, out_mean,
 * out_scale; zeros before the first fit) and the Adam step count.  Any pointer
 * may be NULL. */
rb_status rb_mlp_get(const rb_mlp* net, double* params, double* scaling, int* adam_steps);

void rb_mlp_free(rb_mlp* net);

/*
 * Relative residuals rel_res[b] = ||f(mu_b) - A(mu_b) x_b|| / ||f(mu_b)|| (FP64)
 * of a batch of device vectors, computed WITHOUT ALLOCATING device memory.
 * The paper has no counterpart: this is a service for callers that cannot call
 * cudaMalloc, such as code running under a framework whose caching allocator
 * holds the device memory, or latency-bound code that cannot accept the
 * device-wide synchronisation an allocation may cause.  It needs no rb_ctx.
 *   prob     the problem, checked as for rb_offline_load_arrays (RB_EINVAL);
 *            block coefficients and RB_LOAD_CONST / RB_LOAD_GAUSS loads only (field
 *            problems and array or boundary loads need a context: RB_EINVAL);
 *   mu       host [B][n_mu];   x  device [B][N_dof] of the current device
 *            (host memory and another device's memory are rejected, RB_EINVAL);
 *   rel_res  host [B], written; stream as in rb_opts (may be NULL).
 * Scratch: one static 1 MiB device array per GPU that loads the library, held
 * until the process exits.  It must hold B*n_mu + 2*B*ceil(N_dof/1024) + B
 * doubles (each part rounded up to 256 bytes); a larger batch is rejected with
 * RB_EINVAL and a message in rb_last_error(NULL).  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current and keeps it for that device's CUDA context; after a device reset the
 * next call looks it up again.  Make the first call on a device (and the first
 * after a reset) before any stream capture.  Every call shares
 * the array and overwrites what it reads, so calls that overlap on the GPU
 * (other threads or streams) race: serialise them.  Synchronous: returns after
 * rel_res is on the host.
 */
rb_status rb_residual_noalloc(const rb_problem* prob, int B, const double* mu, const double* x,
                              double* rel_res, void* stream);

/* Failure-path test hook.  Every kernel that waits on an asynchronous copy
 * bounds the wait (2 s by default): on expiry it raises a device error flag,
 * keeps its barriers matched, lets its copies land (bounded) and returns; the
 * call then returns RB_ETIMEOUT and the context stays usable.  This sets that
 * limit to limit_s seconds (0 < limit_s <= 2) and, when skip_stage >= 0, makes
 * the first CTA of the staged CG part-B kernel (2D grids whose rows hold a
 * multiple of 128 points) leave its stage number skip_stage unissued, so that
 * the wait on it runs out without any copy in flight.  rb_debug_wait(ctx, 2.0,
 * -1) restores the defaults.  The paper has no counterpart. */
rb_status rb_debug_wait(rb_ctx* ctx, double limit_s, long long skip_stage);

/* Text of the last error on ctx (or of the last failed context creation when
 * ctx is NULL).  Valid until the next call on that context. */
const char* rb_last_error(const rb_ctx* ctx);
const char* rb_status_string(rb_status s);

/* Release every device and host resource of the context.  NULL is a no-op. */
void rb_free(rb_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* RB_H */
