// Stencil-side kernels of the online solvers.
//
// All streaming kernels are persistent: the grid is a multiple of the SM
// count and every CTA walks the work items (query, tile) of one device-side
// work list.  Per-query dot products are reduced deterministically: every
// CTA publishes its tile partial, and the CTA that arrives last for a query
// sums the partials in a fixed order and advances that query's state
// (the "finalizer"), pushing it onto the list of its next phase.
#include "rb_common.cuh"

namespace rbk {

int tiles_flat(long long n) { return (int)((n + TILE - 1) / TILE); }

// Smoother tile: 32 x 8 (2D) or 16 x 4 x 4 (3D) points, one per thread.
template <int DIM> struct Box;
template <> struct Box<2> { static constexpr int X = 32, Y = 8, Z = 1; };
template <> struct Box<3> { static constexpr int X = 16, Y = 4, Z = 4; };

int tiles_box(const Geo& g) {
    const int X = g.dim == 2 ? Box<2>::X : Box<3>::X;
    const int Y = g.dim == 2 ? Box<2>::Y : Box<3>::Y;
    const int Z = g.dim == 2 ? Box<2>::Z : Box<3>::Z;
    return ((g.mx + X - 1) / X) * ((g.my + Y - 1) / Y) * ((g.mz + Z - 1) / Z);
}

__device__ __forceinline__ int d_tiles_flat(long long n) { return (int)((n + TILE - 1) / TILE); }

template <typename T>
__device__ __forceinline__ T* vec(void* base, const Params& P, int q, int half_idx) {
    return reinterpret_cast<T*>(base) + ((size_t)q * 2 + half_idx) * (size_t)P.g.n;
}
template <typename T>
__device__ __forceinline__ T* vec1(void* base, const Params& P, int q) {
    return reinterpret_cast<T*>(base) + (size_t)q * (size_t)P.g.n;
}

template <typename T>
__device__ __forceinline__ void load_mu(const Params& P, int q, T* mus) {
    __syncthreads();
    if (threadIdx.x < P.n_mu) mus[threadIdx.x] = (T)P.mu[(size_t)q * P.n_mu + threadIdx.x];
    __syncthreads();
}

__device__ __forceinline__ double load_value(const Params& P, const double* mus, long long i) {
    double b = 0.0;
    for (int r = 0; r < P.R; ++r) {
        const int pr = P.load_param[r];
        const double phi = pr < 0 ? 1.0 : mus[pr];
        b += phi * __ldg(P.fr + (size_t)r * P.g.n + i);
    }
    return b;
}

// Block reduction of per-thread T partials, accumulated across warps in FP64.
template <typename T>
__device__ __forceinline__ double block_sum_d(T v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = (double)v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;
}

// ----------------------------------------------------------------------------
// outer residual r = f(mu) - A(mu) x  (FP64 arithmetic, stored as T)

template <typename T>
__global__ void __launch_bounds__(THREADS) k_outer_residual(Params P) {
    __shared__ double mus[MAX_MU];
    __shared__ double red[32];
    const int cnt = P.lcnt[L_OUT];
    const int ntiles = d_tiles_flat(P.g.n);
    const long long total = (long long)cnt * ntiles;
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        const int slot = (int)(w / ntiles), tile = (int)(w % ntiles);
        const int q = P.lidx[L_OUT * P.Bmax + slot];
        if (P.st[q].phase == PH_DONE) continue;
        load_mu(P, q, mus);
        const QState& s = P.st[q];
        const int xzero = s.xzero;
        T* rout = vec1<T>(P.r, P, q);
        const double* x = P.x64 + (size_t)q * P.g.n;
        double rr = 0.0, ff = 0.0;
#pragma unroll
        for (int j = 0; j < TILE / THREADS; ++j) {
            const long long i = (long long)tile * TILE + j * THREADS + threadIdx.x;
            if (i < P.g.n) {
                const double b = load_value(P, mus, i);
                double ax = 0.0;
                if (!xzero) {
                    int ix, iy, iz;
                    node_xyz(P.g, i, ix, iy, iz);
                    Coef<double> c;
                    node_coef(P.g, mus, ix, iy, iz, c);
                    ax = c.diag * x[i] - offdiag_sum(P.g, c, i, ix, iy, iz, [&](long long k) { return x[k]; });
                }
                const double rv = b - ax;
                rout[i] = (T)rv;
                rr += rv * rv;
                ff += b * b;
            }
        }
        double v[2];
        v[0] = block_sum_d(rr, red);
        v[1] = block_sum_d(ff, red);
        if (arrive(P, q, tile, ntiles, v, 2)) {
            double tot[2];
            gather_partials(P, q, ntiles, 2, tot, red);
            if (threadIdx.x == 0) {
                finalize_outer_state(P, q, tot[0], tot[1]);
                P.tick[q] = 0;
            }
        }
    }
}

// mixed refinement step: x64 += d, d = 0
__global__ void __launch_bounds__(THREADS) k_outer_update(Params P) {
    const int cnt = P.lcnt[L_OUT];
    const int ntiles = d_tiles_flat(P.g.n);
    const long long total = (long long)cnt * ntiles;
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        const int slot = (int)(w / ntiles), tile = (int)(w % ntiles);
        const int q = P.lidx[L_OUT * P.Bmax + slot];
        if (P.st[q].phase == PH_DONE) continue;
        float* d = vec1<float>(P.d, P, q);
        double* x = P.x64 + (size_t)q * P.g.n;
#pragma unroll
        for (int j = 0; j < TILE / THREADS; ++j) {
            const long long i = (long long)tile * TILE + j * THREADS + threadIdx.x;
            if (i < P.g.n) {
                x[i] += (double)d[i];
                d[i] = 0.0f;
            }
        }
    }
}

// ----------------------------------------------------------------------------
// CG body, part A: p_new = y + beta p_old, p_new^T A p_new  (Alg. 3 steps 11, 5)

template <typename T>
__global__ void __launch_bounds__(THREADS) k_cg_a(Params P) {
    __shared__ T mus[MAX_MU];
    __shared__ double red[32];
    const int cnt = P.lcnt[L_ITER];
    const int ntiles = d_tiles_flat(P.g.n);
    const long long total = (long long)cnt * ntiles;
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        const int slot = (int)(w / ntiles), tile = (int)(w % ntiles);
        const int q = P.lidx[L_ITER * P.Bmax + slot];
        const QState& s = P.st[q];
        if (s.phase != PH_ITER) continue;          // uniform across the CTA
        load_mu(P, q, mus);
        const T beta = (T)s.beta;
        const T* y = vec1<T>(P.y, P, q);
        const T* pold = vec<T>(P.p, P, q, s.ppar);
        T* pnew = vec<T>(P.p, P, q, s.ppar ^ 1);
        T acc = T(0);
        const bool use_old = beta != T(0);
        auto pv = [&](long long k) { return use_old ? y[k] + beta * pold[k] : y[k]; };
#pragma unroll
        for (int j = 0; j < TILE / THREADS; ++j) {
            const long long i = (long long)tile * TILE + j * THREADS + threadIdx.x;
            if (i < P.g.n) {
                int ix, iy, iz;
                node_xyz(P.g, i, ix, iy, iz);
                Coef<T> c;
                node_coef(P.g, mus, ix, iy, iz, c);
                const T pi = pv(i);
                const T api = c.diag * pi - offdiag_sum(P.g, c, i, ix, iy, iz, pv);
                pnew[i] = pi;
                acc += pi * api;
            }
        }
        double v = block_sum_d(acc, red);
        if (arrive(P, q, tile, ntiles, &v, 1)) {
            double tot;
            gather_partials(P, q, ntiles, 1, &tot, red);
            if (threadIdx.x == 0) {
                finalize_cg_a_state(P, q, tot);
                P.tick[q] = 0;
            }
        }
    }
}

// CG body, part B: d += alpha p, r_new = r_old - alpha A p, ||r_new||^2  (steps 6-8)

template <typename T>
__global__ void __launch_bounds__(THREADS) k_cg_b(Params P) {
    __shared__ T mus[MAX_MU];
    __shared__ double red[32];
    const int cnt = P.lcnt[L_ITER];
    const int ntiles = d_tiles_flat(P.g.n);
    const long long total = (long long)cnt * ntiles;
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        const int slot = (int)(w / ntiles), tile = (int)(w % ntiles);
        const int q = P.lidx[L_ITER * P.Bmax + slot];
        const QState& s = P.st[q];
        if (s.phase != PH_ITER) continue;
        load_mu(P, q, mus);
        const T alpha = (T)s.alpha;
        const T* p = vec<T>(P.p, P, q, s.ppar);
        T* rr = vec1<T>(P.r, P, q);
        T* d = P.mixed ? vec1<T>(P.d, P, q) : reinterpret_cast<T*>(P.x64 + (size_t)q * P.g.n);
        T acc = T(0);
#pragma unroll
        for (int j = 0; j < TILE / THREADS; ++j) {
            const long long i = (long long)tile * TILE + j * THREADS + threadIdx.x;
            if (i < P.g.n) {
                int ix, iy, iz;
                node_xyz(P.g, i, ix, iy, iz);
                Coef<T> c;
                node_coef(P.g, mus, ix, iy, iz, c);
                const T pi = p[i];
                const T api = c.diag * pi - offdiag_sum(P.g, c, i, ix, iy, iz, [&](long long k) { return p[k]; });
                d[i] += alpha * pi;
                const T rv = rr[i] - alpha * api;
                rr[i] = rv;
                acc += rv * rv;
            }
        }
        double v = block_sum_d(acc, red);
        if (arrive(P, q, tile, ntiles, &v, 1)) {
            double tot;
            gather_partials(P, q, ntiles, 1, &tot, red);
            if (threadIdx.x == 0) {
                finalize_cg_b_state(P, q, tot);
                P.tick[q] = 0;
            }
        }
    }
}

// ----------------------------------------------------------------------------
// Smoother z = S(A, b, y) of eq. 8, one sweep per launch.
//   RBGS: red points (colour 0) first, then black, each point
//         z_i = (b_i + sum_f kappa_f/h^2 z_j) / a_ii with the newest z.  One CTA
//         recomputes the red half-sweep on its tile plus a one-node halo in
//         shared memory, then does the black half-sweep on the tile: no CTA
//         ever reads a value written by another CTA of the same launch.
//   JACOBI: z = y + omega (b - A y) / D.    NONE: z = y.
// Mode PCG: b = r (current half), output y, last sweep adds r^T y and
//           r_old^T y and runs the beta finalizer.
// Mode RBI: b = f(mu) in FP64, output x (last sweep) and no dot products.

enum { SM_NONE = 0, SM_RBGS = 1, SM_JACOBI = 2 };

template <typename T, int DIM, int KIND, bool RBI, bool LAST>
__global__ void __launch_bounds__(THREADS) k_smooth(Params P, const T* __restrict__ src_base, T* dst_base) {
    using BX = Box<DIM>;
    constexpr int EX = BX::X + 2, EY = BX::Y + 2, EZ = DIM == 3 ? BX::Z + 2 : 1;
    constexpr int NEXT = EX * EY * EZ;
    __shared__ T mus[MAX_MU];
    __shared__ double musd[MAX_MU];
    __shared__ T red_ext[NEXT];
    __shared__ double red[32];
    const Geo& g = P.g;
    const int ntx = (g.mx + BX::X - 1) / BX::X, nty = (g.my + BX::Y - 1) / BX::Y;
    const int ntz = (g.mz + BX::Z - 1) / BX::Z;
    const int ntiles = ntx * nty * ntz;
    const int cnt = P.lcnt[L_PREC];
    const long long total = (long long)cnt * ntiles;
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        const int slot = (int)(w / ntiles), tile = (int)(w % ntiles);
        const int q = P.lidx[L_PREC * P.Bmax + slot];
        const QState& s = P.st[q];
        __syncthreads();
        if (threadIdx.x < P.n_mu) {
            mus[threadIdx.x] = (T)P.mu[(size_t)q * P.n_mu + threadIdx.x];
            musd[threadIdx.x] = P.mu[(size_t)q * P.n_mu + threadIdx.x];
        }
        __syncthreads();
        const int tx0 = (tile % ntx) * BX::X;
        const int ty0 = ((tile / ntx) % nty) * BX::Y;
        const int tz0 = (tile / (ntx * nty)) * BX::Z;
        const T* src = src_base + (size_t)q * g.n;
        T* dst = dst_base + (size_t)q * g.n;
        const T* bT = RBI ? nullptr : vec1<T>(P.r, P, q);
        // Polak-Ribiere needs (A p)^T y with the direction p of the step just taken
        const bool need_ap = !RBI && LAST && P.beta_form == RB_BETA_PR && !s.start;
        const T* pdir = need_ap ? vec<T>(P.p, P, q, s.ppar) : nullptr;
        auto bval = [&](long long i) -> T {
            if constexpr (RBI) return (T)load_value(P, musd, i);
            else return bT[i];
        };
        auto getsrc = [&](long long k) { return src[k]; };
        if (KIND == SM_RBGS) {
            // red half-sweep on the tile plus halo
            for (int e = threadIdx.x; e < NEXT; e += THREADS) {
                const int ex = e % EX, ey = (e / EX) % EY, ez = e / (EX * EY);
                const int ix = tx0 + ex - 1, iy = ty0 + ey - 1, iz = DIM == 3 ? tz0 + ez - 1 : 0;
                T val = T(0);
                if (ix >= 0 && ix < g.mx && iy >= 0 && iy < g.my && iz >= 0 && iz < g.mz &&
                    ((ix + iy + iz) & 1) == 0) {
                    const long long i = ix + (long long)g.mx * (iy + (long long)g.my * iz);
                    Coef<T> c;
                    node_coef(g, mus, ix, iy, iz, c);
                    val = (bval(i) + offdiag_sum(g, c, i, ix, iy, iz, getsrc)) / c.diag;
                }
                red_ext[e] = val;
            }
            __syncthreads();
        }
        T ry = T(0), roy = T(0);
        {
            const int t = threadIdx.x;
            const int lx = t % BX::X, ly = (t / BX::X) % BX::Y, lz = t / (BX::X * BX::Y);
            const int ix = tx0 + lx, iy = ty0 + ly, iz = tz0 + lz;
            if (ix < g.mx && iy < g.my && iz < g.mz) {
                const long long i = ix + (long long)g.mx * (iy + (long long)g.my * iz);
                T z;
                if (KIND == SM_RBGS) {
                    const int e = (lx + 1) + EX * ((ly + 1) + EY * (DIM == 3 ? lz + 1 : 0));
                    if (((ix + iy + iz) & 1) == 0) {
                        z = red_ext[e];
                    } else {
                        Coef<T> c;
                        node_coef(g, mus, ix, iy, iz, c);
                        T sum = T(0);
                        if (ix > 0) sum += c.kxm * red_ext[e - 1];
                        if (ix < g.mx - 1) sum += c.kxp * red_ext[e + 1];
                        if (iy > 0) sum += c.kym * red_ext[e - EX];
                        if (iy < g.my - 1) sum += c.kyp * red_ext[e + EX];
                        if (DIM == 3) {
                            if (iz > 0) sum += c.kzm * red_ext[e - EX * EY];
                            if (iz < g.mz - 1) sum += c.kzp * red_ext[e + EX * EY];
                        }
                        z = (bval(i) + sum) / c.diag;
                    }
                } else if (KIND == SM_JACOBI) {
                    Coef<T> c;
                    node_coef(g, mus, ix, iy, iz, c);
                    const T yi = src[i];
                    const T ay = c.diag * yi - offdiag_sum(g, c, i, ix, iy, iz, getsrc);
                    z = yi + (T)P.omega * (bval(i) - ay) / c.diag;
                } else {
                    z = src[i];
                }
                dst[i] = z;
                if constexpr (!RBI && LAST) {
                    ry += bT[i] * z;
                    if (need_ap) {
                        Coef<T> c;
                        node_coef(g, mus, ix, iy, iz, c);
                        const T ap = c.diag * pdir[i] -
                                     offdiag_sum(g, c, i, ix, iy, iz, [&](long long k) { return pdir[k]; });
                        roy += ap * z;
                    }
                }
            }
        }
        if constexpr (LAST) {
            double v[2];
            if constexpr (!RBI) {
                v[0] = block_sum_d(ry, red);
                v[1] = block_sum_d(roy, red);
            } else {
                v[0] = v[1] = 0.0;
            }
            if (arrive(P, q, tile, ntiles, v, RBI ? 0 : 2)) {
                double tot[2] = {0.0, 0.0};
                if constexpr (!RBI) gather_partials(P, q, ntiles, 2, tot, red);
                if (threadIdx.x == 0) {
                    if constexpr (RBI) {
                        list_push(P, L_OUT, q);
                    } else {
                        finalize_prec_state(P, q, tot[0], tot[1]);
                    }
                    P.tick[q] = 0;
                }
            }
        }
    }
}

template <typename T, int DIM, int KIND, bool RBI>
static void smooth_sweeps(const Params& P, const Launch& L, int nu) {
    T* ypro = reinterpret_cast<T*>(P.ypro);
    T* tmp = reinterpret_cast<T*>(P.tmp);
    T* out = RBI ? reinterpret_cast<T*>(P.x64) : reinterpret_cast<T*>(P.y);
    const int sweeps = KIND == SM_NONE ? 1 : (nu < 1 ? 1 : nu);
    const T* src = ypro;
    for (int s = 1; s <= sweeps; ++s) {
        const bool last = s == sweeps;
        T* dst = last ? out : ((s & 1) ? tmp : ypro);
        if (last)
            k_smooth<T, DIM, KIND, RBI, true><<<L.grid, THREADS, 0, L.s>>>(P, src, dst);
        else
            k_smooth<T, DIM, KIND, RBI, false><<<L.grid, THREADS, 0, L.s>>>(P, src, dst);
        src = dst;
    }
}

template <typename T, int DIM>
static void smooth_dispatch(const Params& P, const Launch& L, int nu, bool rbi) {
    const int kind = P.smoother == RB_SMOOTH_RBGS ? SM_RBGS : (P.smoother == RB_SMOOTH_JACOBI ? SM_JACOBI : SM_NONE);
    if (rbi) {
        if constexpr (sizeof(T) == 8) {
            if (kind == SM_RBGS) smooth_sweeps<T, DIM, SM_RBGS, true>(P, L, nu);
            else if (kind == SM_JACOBI) smooth_sweeps<T, DIM, SM_JACOBI, true>(P, L, nu);
            else smooth_sweeps<T, DIM, SM_NONE, true>(P, L, nu);
        }
    } else {
        if (kind == SM_RBGS) smooth_sweeps<T, DIM, SM_RBGS, false>(P, L, nu);
        else if (kind == SM_JACOBI) smooth_sweeps<T, DIM, SM_JACOBI, false>(P, L, nu);
        else smooth_sweeps<T, DIM, SM_NONE, false>(P, L, nu);
    }
}

template <typename T>
void launch_smoother(const Params& P, const Launch& L, int nu, bool rbi) {
    if (P.g.dim == 2) smooth_dispatch<T, 2>(P, L, nu, rbi);
    else smooth_dispatch<T, 3>(P, L, nu, rbi);
}
template void launch_smoother<float>(const Params&, const Launch&, int, bool);
template void launch_smoother<double>(const Params&, const Launch&, int, bool);

// ----------------------------------------------------------------------------
// RBI residual r = f - A x (Alg. 2 steps 2-3): the true residual every iteration.

__device__ void finalize_rbi(const Params& P, int q, double rr, double ff) {
    QState& s = P.st[q];
    if (s.outer == 0) s.fnorm = sqrt(ff);
    s.outer += 1;
    const double rn = sqrt(rr);
    const double fn = s.fnorm > 0.0 ? s.fnorm : 1.0;
    s.rel_res = rn / fn;
    s.rnorm = rn;
    s.xzero = 0;
    if (!(rn == rn)) { mark_done(P, s, RB_EBREAKDOWN); return; }
    if (s.rel_res < P.tol) { mark_done(P, s, RB_OK); return; }
    if (s.iters >= P.max_iter) { mark_done(P, s, RB_ENOCONV); return; }
    s.iters += 1;
    s.phase = PH_PREC;
    list_push(P, L_PREC, q);
}

__global__ void __launch_bounds__(THREADS) k_rbi_residual(Params P) {
    __shared__ double mus[MAX_MU];
    __shared__ double red[32];
    const int cnt = P.lcnt[L_OUT];
    const int ntiles = d_tiles_flat(P.g.n);
    const long long total = (long long)cnt * ntiles;
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        const int slot = (int)(w / ntiles), tile = (int)(w % ntiles);
        const int q = P.lidx[L_OUT * P.Bmax + slot];
        if (P.st[q].phase == PH_DONE) continue;
        load_mu(P, q, mus);
        const QState& s = P.st[q];
        const int xzero = s.xzero;
        double* rout = vec1<double>(P.r, P, q);
        const double* x = P.x64 + (size_t)q * P.g.n;
        double rr = 0.0, ff = 0.0;
#pragma unroll
        for (int j = 0; j < TILE / THREADS; ++j) {
            const long long i = (long long)tile * TILE + j * THREADS + threadIdx.x;
            if (i < P.g.n) {
                const double b = load_value(P, mus, i);
                double ax = 0.0;
                if (!xzero) {
                    int ix, iy, iz;
                    node_xyz(P.g, i, ix, iy, iz);
                    Coef<double> c;
                    node_coef(P.g, mus, ix, iy, iz, c);
                    ax = c.diag * x[i] - offdiag_sum(P.g, c, i, ix, iy, iz, [&](long long k) { return x[k]; });
                }
                const double rv = b - ax;
                rout[i] = rv;
                rr += rv * rv;
                ff += b * b;
            }
        }
        double v[2];
        v[0] = block_sum_d(rr, red);
        v[1] = block_sum_d(ff, red);
        if (arrive(P, q, tile, ntiles, v, 2)) {
            double tot[2];
            gather_partials(P, q, ntiles, 2, tot, red);
            if (threadIdx.x == 0) {
                finalize_rbi(P, q, tot[0], tot[1]);
                P.tick[q] = 0;
            }
        }
    }
}

// ----------------------------------------------------------------------------
// y = A(mu) x for a batch (rb_apply and the offline affine terms)

__global__ void __launch_bounds__(THREADS) k_apply(Geo g, int n_mu, const double* __restrict__ mu,
                                                   const double* __restrict__ x, double* __restrict__ y) {
    __shared__ double mus[MAX_MU];
    const int q = blockIdx.y;
    if (threadIdx.x < n_mu) mus[threadIdx.x] = mu[(size_t)q * n_mu + threadIdx.x];
    __syncthreads();
    const double* xq = x + (size_t)q * g.n;
    double* yq = y + (size_t)q * g.n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.n;
         i += (long long)gridDim.x * blockDim.x) {
        int ix, iy, iz;
        node_xyz(g, i, ix, iy, iz);
        Coef<double> c;
        node_coef(g, mus, ix, iy, iz, c);
        yq[i] = c.diag * xq[i] - offdiag_sum(g, c, i, ix, iy, iz, [&](long long k) { return xq[k]; });
    }
}

void launch_apply(const Geo& g, int B, int n_mu, const double* mu, const double* x, double* y, cudaStream_t s) {
    long long blocks = (g.n + THREADS - 1) / THREADS;
    if (blocks > 4096) blocks = 4096;
    dim3 grid((unsigned)blocks, (unsigned)B);
    k_apply<<<grid, THREADS, 0, s>>>(g, n_mu, mu, x, y);
}

// load terms f_r at the nodes
__global__ void k_fill_loads(Geo g, int R, const int* kind, const double* center, const double* sigma, double* fr) {
    const int r = blockIdx.y;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.n;
         i += (long long)gridDim.x * blockDim.x) {
        double v = kind[r] == RB_LOAD_CONST ? 1.0 : 0.0;   // array and boundary loads: copied by the host
        if (kind[r] == RB_LOAD_GAUSS) {
            int ix, iy, iz;
            node_xyz(g, i, ix, iy, iz);
            const double x = (ix + 1.0) / (g.mx + 1.0);
            const double y = (iy + 1.0) / (g.my + 1.0);
            double d2 = (x - center[3 * r]) * (x - center[3 * r]) + (y - center[3 * r + 1]) * (y - center[3 * r + 1]);
            if (g.dim == 3) {
                const double z = (iz + 1.0) / (g.mz + 1.0);
                d2 += (z - center[3 * r + 2]) * (z - center[3 * r + 2]);
            }
            v = exp(-d2 / (2.0 * sigma[r] * sigma[r]));
        }
        fr[(size_t)r * g.n + i] = v;
    }
}

// kappa(mu) at the nodes of each query slot, in FP64 and rounded to FP32 (the 3D tile kernels
// read the node values of their tile's neighbourhood from these instead of the fields)
__global__ void k_field_kappa(Geo g, int n_mu, const double* __restrict__ mu) {
    const int b = blockIdx.y;
    const double* m = mu + (size_t)b * n_mu;
    double* k64 = const_cast<double*>(g.kap64) + (size_t)b * g.n;
    float* k32 = const_cast<float*>(g.kap32) + (size_t)b * g.n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.n;
         i += (long long)gridDim.x * blockDim.x) {
        double k = 0.0;
        for (int q = 0; q < g.nf; ++q) k += m[q] * __ldg(g.kf64 + (size_t)q * g.n + i);
        k64[i] = k;
        k32[i] = (float)k;
    }
}

void launch_field_kappa(const Geo& g, int B, int n_mu, const double* mu, cudaStream_t s) {
    if (g.nf <= 0 || !g.kap64 || !g.kap32 || B <= 0) return;
    long long blocks = (g.n + THREADS - 1) / THREADS;
    if (blocks > 1024) blocks = 1024;
    k_field_kappa<<<dim3((unsigned)blocks, (unsigned)B), THREADS, 0, s>>>(g, n_mu, mu);
}

void launch_fill_loads(const Geo& g, int R, const int* kind, const double* center, const double* sigma, double* fr,
                       cudaStream_t s) {
    long long blocks = (g.n + THREADS - 1) / THREADS;
    if (blocks > 4096) blocks = 4096;
    k_fill_loads<<<dim3((unsigned)blocks, (unsigned)R), THREADS, 0, s>>>(g, R, kind, center, sigma, fr);
}

// ----------------------------------------------------------------------------
// launch wrappers

template <typename T>
void launch_outer_residual(const Params& P, const Launch& L) {
    k_outer_residual<T><<<L.grid, THREADS, 0, L.s>>>(P);
}
template void launch_outer_residual<float>(const Params&, const Launch&);
template void launch_outer_residual<double>(const Params&, const Launch&);

void launch_outer_update(const Params& P, const Launch& L) { k_outer_update<<<L.grid, THREADS, 0, L.s>>>(P); }

template <typename T>
void launch_cg_a(const Params& P, const Launch& L) { k_cg_a<T><<<L.grid, THREADS, 0, L.s>>>(P); }
template <typename T>
void launch_cg_b(const Params& P, const Launch& L) { k_cg_b<T><<<L.grid, THREADS, 0, L.s>>>(P); }
template void launch_cg_a<float>(const Params&, const Launch&);
template void launch_cg_a<double>(const Params&, const Launch&);
template void launch_cg_b<float>(const Params&, const Launch&);
template void launch_cg_b<double>(const Params&, const Launch&);

void launch_rbi_residual(const Params& P, const Launch& L) { k_rbi_residual<<<L.grid, THREADS, 0, L.s>>>(P); }

}  // namespace rbk
