// Internal declarations shared by the librb translation units.
//
// Data layout in HBM (per context):
//   W64c  [nbp][N]   FP64 basis, column-major (basis vector k contiguous)
//   W32c  [nbp][N]   FP32 copy (K-major operand of the batched projection)
//   W32r  [N][nbp32] FP32 copy, row-major (K-major operand of the prolongation)
//   fr    [R][N]     FP64 load terms f_r (eq. 12)
//   batch vectors [B][N] per buffer, query-major, x fastest.  The search
//   direction is ping-ponged ([2][B][N]): the kernel that rebuilds it reads its
//   neighbours, which another CTA of the same launch may already have
//   rewritten.  The residual is updated in place (only point-wise reads).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rb.h"

namespace rbk {

constexpr int MAX_P = 64;        // blocks (affine terms)
constexpr int MAX_MU = 128;      // entries of one parameter vector
constexpr int MAX_LOADS = 8;
constexpr int MAX_N = 128;       // basis size
constexpr int THREADS = 256;     // CTA size of the streaming kernels
constexpr int TILE = 1024;       // points per flat tile (4 per thread)

// Geometry of the grid and of the block partition.
struct Geo {
    int dim, mx, my, mz;
    int nbx, nby, nbz, P;
    long long n;                 // N_dof
    double ihx2, ihy2, ihz2;     // 1/h_d^2
    const int* bx;               // block index along x of every node column, [mx]
    const int* by;               // [my]
    const int* bz;               // [mz]
    const int* rkey;             // [my] block rows of y-rows k-1, k, k+1 packed (0xFF: no row); rows
                                 // with equal keys have equal face coefficients in 2D
    int nf;                      // coefficient fields (0: block coefficients)
    const double* kf64;          // [nf][n] node values of the fields
    const float* kf32;           // the same in FP32
    const double* kap64;         // [Bmax][n] kappa(mu) = sum_q mu_q F_q at the nodes of each query slot
    const float* kap32;          // (3D field problems; filled when a wave starts)
};

// Per-query phase of the solver state machine.
enum Phase : int {
    PH_OUTER = 0,    // needs an FP64 residual f - A x (start, refinement step, final check)
    PH_PREC = 1,     // needs the RBI preconditioner y = RBI(A, r, W, 1)
    PH_ITER = 2,     // in the CG body (q = A p, alpha, updates)
    PH_DONE = 3
};

// Work lists (one per phase that a kernel consumes).
enum ListId : int { L_OUT = 0, L_PREC = 1, L_ITER = 2, N_LISTS = 3 };

struct QState {
    double fnorm;        // ||f(mu)||
    double target;       // absolute residual target of the current CG cycle
    double rho;          // r^T y of the current cycle
    double alpha, beta;
    double rnorm;        // last recurrence residual norm
    double rel_res;      // last true relative residual (FP64)
    int iters, outer, restarts, status;
    int phase;
    int start;           // 1: the next preconditioner output starts a CG cycle (beta = 0)
    int ppar;            // current half of the p ping-pong buffer
    int n_used;          // basis vectors of the next preconditioner application (adaptive N)
    int xzero;           // x is exactly zero (skip A x in the residual)
    int pad_;
};

// Everything a solver kernel needs; passed by value.
struct Params {
    Geo g;
    int B;                       // slots in this wave
    int Bmax;
    int n_mu;
    const double* mu;            // [B][n_mu]
    int R;
    const double* fr;            // [R][N]
    int load_param[MAX_LOADS];
    // basis
    int nb, nbp;                 // basis size and padded stride
    const double* W64c;
    const float* W32c;
    const double* L;             // [Bmax][nbp][nbp] A_N(mu)^{-1} (row-major, formed from the Cholesky factor);
                                 // with adaptive N the inverse factor X = L^{-1} + L^{-T} - diag(L^{-1})
    // vectors
    double* x64;                 // [B][N] FP64 iterate / solution
    void* r;                     // [B][N] of T (updated in place)
    void* p;                     // [2][B][N] of T
    void* y;                     // [B][N] of T
    void* ypro;                  // [B][N] of T
    void* tmp;                   // [B][N] of T (smoother ping-pong for nu >= 2)
    void* d;                     // [B][N] of T: inner iterate (aliases x64 in FP64 mode)
    void* e;                     // [B][lde] of T: reduced correction e_N (zero beyond nb)
    int lde;
    // reductions and lists
    QState* st;
    double* part;                // [B][max_tiles][4]
    int max_tiles;
    double* proj;                // [nsplit][B][nbp] partial W^T r
    int nsplit;
    unsigned* tick;              // [B] arrival counters
    int* lcnt;                   // [N_LISTS]
    int* lidx;                   // [N_LISTS][Bmax]
    int* ndone;                  // queries that reached PH_DONE
    int* done;                   // [Bmax] those queries in the order they finished (or null)
    int* err;                    // raised by a kernel whose bounded wait expired
    // options
    double tol, inner_tol;
    int max_iter, max_outer;
    int beta_form, smoother;
    double omega;
    int mixed;                   // 1: T = float inner with FP64 refinement
    int ybf16;                   // 1: the smoother's iterates (ypro, tmp) are stored as BF16
    int adaptive;                // 1: N grows per query (end of Section 4.1); QState.n_used
    double gamma;                // residual-ratio threshold of the growth test
    unsigned long long wait_ns;  // limit of every bounded wait on an asynchronous copy
    long long dbg_skip;          // test hook (rb_debug_wait): the staged CG part-B producer of CTA 0
                                 // leaves this stage unissued (-1: never)
};

// ----------------------------------------------------------------------------
// small device helpers

// (ix, iy, iz) of flat index i; N_dof < 2^31 is enforced at context creation
__device__ __forceinline__ void node_xyz(const Geo& g, long long i, int& ix, int& iy, int& iz) {
    const unsigned ii = (unsigned)i;
    const unsigned t = ii / (unsigned)g.mx;
    ix = (int)(ii - t * (unsigned)g.mx);
    iz = (int)(t / (unsigned)g.my);
    iy = (int)(t - (unsigned)iz * (unsigned)g.my);
}

// Face coefficients kappa_f / h^2 of one node (zero where the face is missing
// is NOT used: a missing neighbour has value 0, the face still counts in the
// diagonal with kappa = mu_p(i)).
template <typename T>
struct Coef {
    T kxm, kxp, kym, kyp, kzm, kzp, diag;
};

template <typename T>
__device__ __forceinline__ const T* field_values(const Geo& g);
template <>
__device__ __forceinline__ const double* field_values<double>(const Geo& g) { return g.kf64; }
template <>
__device__ __forceinline__ const float* field_values<float>(const Geo& g) { return g.kf32; }

// kappa(i) = sum_q mu_q F_q(i) of a problem with coefficient fields
template <typename T>
__device__ __forceinline__ T field_kappa(const Geo& g, const T* __restrict__ mus, long long i) {
    const T* F = field_values<T>(g);
    T k = T(0);
    for (int q = 0; q < g.nf; ++q) k += mus[q] * __ldg(F + (size_t)q * g.n + i);
    return k;
}

template <typename T>
__device__ __forceinline__ void node_coef(const Geo& g, const T* __restrict__ mus, int ix, int iy, int iz,
                                          Coef<T>& c) {
    if (g.nf > 0) {   // coefficient fields: the same face rule on kappa(i) = sum_q mu_q F_q(i)
        const T half = T(0.5);
        const T hx = (T)g.ihx2, hy = (T)g.ihy2, hz = (T)g.ihz2;
        const long long i = ix + (long long)g.mx * (iy + (long long)g.my * iz);
        const T m = field_kappa(g, mus, i);
        c.kxm = hx * (ix > 0 ? half * (m + field_kappa(g, mus, i - 1)) : m);
        c.kxp = hx * (ix < g.mx - 1 ? half * (m + field_kappa(g, mus, i + 1)) : m);
        c.kym = hy * (iy > 0 ? half * (m + field_kappa(g, mus, i - g.mx)) : m);
        c.kyp = hy * (iy < g.my - 1 ? half * (m + field_kappa(g, mus, i + g.mx)) : m);
        T dg = c.kxm + c.kxp + c.kym + c.kyp;
        if (g.dim == 3) {
            const long long pl = (long long)g.mx * g.my;
            c.kzm = hz * (iz > 0 ? half * (m + field_kappa(g, mus, i - pl)) : m);
            c.kzp = hz * (iz < g.mz - 1 ? half * (m + field_kappa(g, mus, i + pl)) : m);
            dg += c.kzm + c.kzp;
        } else {
            c.kzm = c.kzp = T(0);
        }
        c.diag = dg;
        return;
    }
    const int bxc = __ldg(g.bx + ix), byc = __ldg(g.by + iy), bzc = __ldg(g.bz + iz);
    const int pyz = g.nbx * (byc + g.nby * bzc);
    const T m = mus[bxc + pyz];
    const T half = T(0.5);
    const T hx = (T)g.ihx2, hy = (T)g.ihy2, hz = (T)g.ihz2;
    c.kxm = hx * (ix > 0 ? half * (m + mus[__ldg(g.bx + ix - 1) + pyz]) : m);
    c.kxp = hx * (ix < g.mx - 1 ? half * (m + mus[__ldg(g.bx + ix + 1) + pyz]) : m);
    const int pxz = bxc + g.nbx * g.nby * bzc;
    c.kym = hy * (iy > 0 ? half * (m + mus[pxz + g.nbx * __ldg(g.by + iy - 1)]) : m);
    c.kyp = hy * (iy < g.my - 1 ? half * (m + mus[pxz + g.nbx * __ldg(g.by + iy + 1)]) : m);
    T dg = c.kxm + c.kxp + c.kym + c.kyp;
    if (g.dim == 3) {
        const int pxy = bxc + g.nbx * byc;
        c.kzm = hz * (iz > 0 ? half * (m + mus[pxy + g.nbx * g.nby * __ldg(g.bz + iz - 1)]) : m);
        c.kzp = hz * (iz < g.mz - 1 ? half * (m + mus[pxy + g.nbx * g.nby * __ldg(g.bz + iz + 1)]) : m);
        dg += c.kzm + c.kzp;
    } else {
        c.kzm = c.kzp = T(0);
    }
    c.diag = dg;
}

// sum over the faces of node i of kappa_f/h^2 * v_j (v_j = 0 outside the grid)
template <typename T, typename Get>
__device__ __forceinline__ T offdiag_sum(const Geo& g, const Coef<T>& c, long long i, int ix, int iy, int iz,
                                         Get get) {
    T s = T(0);
    if (ix > 0) s += c.kxm * get(i - 1);
    if (ix < g.mx - 1) s += c.kxp * get(i + 1);
    if (iy > 0) s += c.kym * get(i - g.mx);
    if (iy < g.my - 1) s += c.kyp * get(i + g.mx);
    if (g.dim == 3) {
        const long long pl = (long long)g.mx * g.my;
        if (iz > 0) s += c.kzm * get(i - pl);
        if (iz < g.mz - 1) s += c.kzp * get(i + pl);
    }
    return s;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red /* >= 32 entries */) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    T s = T(0);
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : T(0);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;  // valid in thread 0
}

__device__ __forceinline__ void list_push(const Params& P, int list, int q) {
    const int pos = atomicAdd(P.lcnt + list, 1);
    P.lidx[list * P.Bmax + pos] = q;
}

__device__ __forceinline__ void mark_done(const Params& P, QState& s, int status) {
    s.phase = PH_DONE;
    s.status = status;
    const int pos = atomicAdd(P.ndone, 1);
    if (P.done) P.done[pos] = (int)(&s - P.st);
}

// Preconditioner finalizer: ry = r_{k+1}^T y_{k+1}, apy = (A p_k)^T y_{k+1}.
// Polak-Ribiere numerator y_{k+1}^T (r_{k+1} - r_k) = -alpha_k apy since
// r_{k+1} = r_k - alpha_k A p_k; Fletcher-Reeves uses ry (Alg. 3 step 10).
__device__ __forceinline__ void finalize_prec_state(const Params& P, int q, double ry, double apy) {
    QState& s = P.st[q];
    if (!(ry > 0.0)) { mark_done(P, s, RB_EBREAKDOWN); return; }
    if (s.start) {
        s.beta = 0.0;
        s.start = 0;
    } else {
        s.beta = (P.beta_form == RB_BETA_FR) ? ry / s.rho : -s.alpha * apy / s.rho;
    }
    s.rho = ry;
    s.phase = PH_ITER;
    list_push(P, L_ITER, q);
}

// Outer (true-residual) finalizer: rr = ||f - A x||^2 in FP64, ff = ||f||^2.
__device__ __forceinline__ void finalize_outer_state(const Params& P, int q, double rr, double ff) {
    QState& s = P.st[q];
    if (s.outer == 0) s.fnorm = sqrt(ff);
    const double prev = s.rel_res;
    s.outer += 1;
    const double rn = sqrt(rr);
    const double fn = s.fnorm > 0.0 ? s.fnorm : 1.0;
    s.rel_res = rn / fn;
    s.rnorm = rn;
    s.xzero = 0;
    if (!(rn == rn)) { mark_done(P, s, RB_EBREAKDOWN); return; }
    if (s.rel_res < P.tol) { mark_done(P, s, RB_OK); return; }
    if (s.iters >= P.max_iter || s.outer > P.max_outer) { mark_done(P, s, RB_ENOCONV); return; }
    // a full CG cycle that gained less than 10% on the true residual has hit
    // the rounding floor of the FP64 residual: stop instead of cycling
    if (s.outer > 2 && s.rel_res > 0.9 * prev) { mark_done(P, s, RB_ENOCONV); return; }
    if (s.outer > 1 && !P.mixed) s.restarts += 1;
    // mixed: each FP32 cycle reduces its own residual by inner_tol, but never
    // aims below half the outer tolerance (the FP64 step then finishes).
    // FP64: the first cycle stops at tol (Alg. 3 step 8); a restart after a
    // failed true-residual check aims at half of it.
    s.target = P.mixed ? fmax(P.inner_tol * rn, 0.5 * P.tol * fn) : (s.outer > 1 ? 0.5 : 1.0) * P.tol * fn;
    s.phase = PH_PREC;
    s.start = 1;
    list_push(P, L_PREC, q);
}

// CG part A finalizer: pap = p^T A p of the new direction; alpha = rho / pap (Alg. 3 step 5).
__device__ __forceinline__ void finalize_cg_a_state(const Params& P, int q, double pap) {
    QState& s = P.st[q];
    if (!(pap > 0.0)) {
        mark_done(P, s, RB_EBREAKDOWN);
        return;
    }
    s.alpha = s.rho / pap;
    s.ppar ^= 1;
}

// CG part B finalizer: rr = ||r_{k+1}||^2 of the recurrence residual (Alg. 3 step 8).
// Below the cycle's target (or out of iterations) the query goes to the outer
// residual check, else to the next preconditioner application.
__device__ __forceinline__ void finalize_cg_b_state(const Params& P, int q, double rr) {
    QState& s = P.st[q];
    const double rn = sqrt(rr);
    s.iters += 1;
    if (!(rn == rn)) {
        s.rnorm = rn;
        mark_done(P, s, RB_EBREAKDOWN);
        return;
    }
    if (rn < s.target || s.iters >= P.max_iter) {
        s.rnorm = rn;
        s.phase = PH_OUTER;
        list_push(P, L_OUT, q);
    } else {
        // adaptive N (end of Section 4.1): a residual that fell by less than gamma in this
        // iteration, ||r_k|| / ||r_{k+1}|| < gamma, adds one basis vector to the next application
        if (P.adaptive && s.n_used < P.nb && s.rnorm < P.gamma * rn) s.n_used += 1;
        s.rnorm = rn;
        s.phase = PH_PREC;
        list_push(P, L_PREC, q);
    }
}

// Thread 0 publishes a CTA's partial sums for (q, tile); returns true in every
// thread of the CTA that is the last to do so for q.  The caller then reduces
// the partials in a fixed order (deterministic) and resets tick[q].
__device__ __forceinline__ bool arrive(const Params& P, int q, int tile, int ntiles, const double* vals, int nv) {
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        double* dst = P.part + ((size_t)q * P.max_tiles + tile) * 4;
        for (int j = 0; j < nv; ++j) dst[j] = vals[j];
        __threadfence();
        const unsigned prev = atomicAdd(P.tick + q, 1u);
        s_last = (prev == (unsigned)ntiles - 1u);
    }
    __syncthreads();
    const bool last = s_last != 0;
    if (last) __threadfence();
    return last;
}

// Fixed-order sum of the partials of q; result in out[0..nv) of thread 0.
__device__ __forceinline__ void gather_partials(const Params& P, int q, int ntiles, int nv, double* out,
                                                double* red) {
    for (int j = 0; j < nv; ++j) {
        double s = 0.0;
        for (int t = threadIdx.x; t < ntiles; t += blockDim.x)
            s += __ldcg(P.part + ((size_t)q * P.max_tiles + t) * 4 + j);
        s = block_sum(s, red);
        if (threadIdx.x == 0) out[j] = s;
    }
}

// ----------------------------------------------------------------------------
// launch wrappers (defined in the .cu files)

struct Launch {
    int grid;          // persistent grid size of the streaming kernels
    cudaStream_t s;
};

template <typename T> void launch_outer_residual(const Params& P, const Launch& L);
void launch_outer_update(const Params& P, const Launch& L);
template <typename T> void launch_project(const Params& P, const Launch& L);
template <typename T> void launch_reduced_solve(const Params& P, const Launch& L);
template <typename T> void launch_prolong(const Params& P, const Launch& L, bool rbi_mode);
template <typename T> void launch_smoother(const Params& P, const Launch& L, int nu, bool rbi_mode);
// row-marching 2D variants (dim 2, mx a multiple of 128, mx <= 1024)
bool use_rowmarch(const Geo& g);
template <typename T> void launch2d_cg_a(const Params& P, const Launch& L);
template <typename T> void launch2d_cg_b(const Params& P, const Launch& L);
template <typename T> void launch2d_smooth(const Params& P, const Launch& L, int nu);
// FP64 outer residual with rows of x staged in shared memory by bulk asynchronous copies
bool use_staged_outer(const Geo& g);
template <typename TR> void launch2d_outer_residual_staged(const Params& P, const Launch& L);
// CG body with rows staged in shared memory by bulk asynchronous copies
bool use_staged_cg(const Geo& g);
template <typename T> void launch2d_cg_a_staged(const Params& P, const Launch& L);
template <typename T> void launch2d_cg_b_staged(const Params& P, const Launch& L);
// one sweep per launch with rows staged in shared memory by bulk asynchronous copies
bool use_tma_smoother(const Geo& g);
template <typename T> void launch2d_smooth_tma(const Params& P, const Launch& L, int nu);
// nu sweeps in passes of up to three, rows staged by bulk asynchronous copies (FP32, dim 2,
// rows of a multiple of 128 points)
bool use_multi_smoother(const Geo& g);
void launch2d_smooth_multi(const Params& P, const Launch& L, int nu, int max_nf);
// all nu sweeps in one pass (FP32, dim 2, mx even, nu <= 6)
bool use_fused_smoother(const Geo& g, int nu);
void launch2d_smooth_fused(const Params& P, const Launch& L, int nu);
int fused_tiles(const Geo& g, int nu);
// 3D kernels marching in z (PCG mode; tiles of 32 x 8 x 16): the red-black smoother with
// direct loads, and the smoother and CG body with planes prefetched by asynchronous copies
bool use_zmarch_smoother(const Geo& g);
template <typename T> void launch3d_smooth(const Params& P, const Launch& L, int nu);
template <typename T> void launch3d_smooth_staged(const Params& P, const Launch& L, int nu);
template <typename T> void launch3d_cg_a(const Params& P, const Launch& L);
template <typename T> void launch3d_cg_b(const Params& P, const Launch& L);
// 3D kernels marching in z over tiles of whole x-rows (rows of a multiple of 4 points, at most
// 256): 4 points per thread, planes staged by bulk row copies, one CTA barrier per plane
bool use_ztile(const Geo& g, bool fp64);
// the FP64 outer residual on the same tiles (x staged with its halo rows)
bool use_ztile_outer(const Geo& g);
template <typename TR>
bool launch3d_outer_tile(const Params& P, const Launch& L);
// (false: a tensor map could not be encoded; nothing was launched)
template <typename T> bool launch3d_cg_tile(const Params& P, const Launch& L, bool part_a);
template <typename T> bool launch3d_smooth_tile(const Params& P, const Launch& L, int nu);
template <typename T> void launch_cg_a(const Params& P, const Launch& L);
template <typename T> void launch_cg_b(const Params& P, const Launch& L);
void launch_rbi_residual(const Params& P, const Launch& L);
void launch_cholesky(const Params& P, cudaStream_t s, const double* ANq, int Q);
void launch_apply(const Geo& g, int B, int n_mu, const double* mu, const double* x, double* y, cudaStream_t s);
void launch_fill_loads(const Geo& g, int R, const int* kind, const double* center, const double* sigma,
                       double* fr, cudaStream_t s);

// offline-build helpers
void launch_project_cols(const Geo& g, int nb, const double* W64c, int nv, const double* V, double* out,
                         double* scratch, cudaStream_t s);                 // out[v][k] = W[:,k]^T V[v]
void launch_sub_cols(const Geo& g, int nb, const double* W64c, const double* c, double* v, cudaStream_t s);
void launch_scores(const Geo& g, int P, int R, const int* load_param, int n_mu, int nb, int nbp,
                   const double* ANq, const double* fNr, const double* Rsnap, int ntrain, const double* mu,
                   int literal, double* score, int* bad, cudaStream_t s);
double launch_norm(const Geo& g, const double* v, double* scratch, cudaStream_t s);

// starting vectors and reduced coefficients (rb_warm_start, rb_coefficients)
struct LoadMap {
    int param[MAX_LOADS];        // Phi_r(mu) = mu[param[r]], or 1 when param[r] < 0
};
void launch_galerkin(int nb, int Q, const double* ANq, int R, const LoadMap& lm, const double* fNr, int n_mu, int B,
                     const double* mu, double* coef, int* bad, cudaStream_t s);   // A_N(mu) a = f_N(mu)
void launch_lift(long long n, int nb, const float* W32c, int B, const double* coef, double* x, int grid,
                 cudaStream_t s);
void launch_lift64(long long n, int nb, const double* W64c, int B, const double* coef, double* x, int grid,
                   cudaStream_t s);                                                  // x_b = W c_b
int coef_splits(int B, int num_sms);
void launch_coefficients(long long n, int nb, const float* W32c, int B, const double* X, double* coef,
                         double* scratch, int num_sms, cudaStream_t s);            // c_b = W^T x_b

// error basis of the learned warm start (rb_errbasis.cu)
void launch_eb_errors(long long n, int nb, const double* W64c, int S, const double* a, const double* X, double* E,
                      int grid, cudaStream_t s);                                   // E = X - W a
size_t eb_gram_part_elems(int S);
void launch_eb_gram(long long n, int S, const double* E, double* part, double* G, int grid, cudaStream_t s);
void launch_eb_modes(long long n, int S, int m, const double* E, const double* C, double* V64, float* V32, int grid,
                     cudaStream_t s);                                              // V = E C
void launch_eb_lift_add(long long n, int m, const float* V32, int B, const double* z, double* x, int grid,
                        cudaStream_t s);                                           // x_b += V z_b
void jacobi_eigen(int S, std::vector<double>& A, std::vector<double>& lam, std::vector<double>& Phi);

// learned warm start (rb_mlp.cu)
int mlp_n_in(const rb_mlp* net);
int mlp_n_out(const rb_mlp* net);
bool mlp_ready(const rb_mlp* net);
rb_status mlp_predict_device(rb_mlp* net, int B, const double* d_mu, int ld_mu, double* d_out, cudaStream_t s);

int tiles_flat(long long n);
// kappa(mu_b) = sum_q mu_b,q F_q at every node of the first B query slots (g.kap64 / g.kap32)
void launch_field_kappa(const Geo& g, int B, int n_mu, const double* mu, cudaStream_t s);
int tiles_box(const Geo& g);

// Where a caller's buffer lives.  Device memory of another GPU is rejected by
// every call: a kernel of this device cannot read it without peer access.
enum PtrKind { PTR_HOST = 0, PTR_DEVICE = 1, PTR_OTHER_DEVICE = 2 };
PtrKind pointer_kind(const void* p);   // managed memory counts as PTR_DEVICE

// Checks of an rb_problem shared by every entry point that takes one (rb_api.cu).
rb_status validate_problem(const rb_problem* prob, std::string& why);

}  // namespace rbk
