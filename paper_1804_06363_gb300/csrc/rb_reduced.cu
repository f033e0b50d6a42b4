// Reduced-space kernels: projection W^T r (eq. 5), reduced solve A_N e_N = r_N
// (eq. 6) with the Cholesky factor of A_N(mu) (eq. 12b), prolongation W e_N
// (eq. 7), plus the offline-build helpers (Gram-Schmidt, greedy scores).
// CUDA-core versions, used for FP64 and as the reference engine of the mixed path.
#include <cuda_bf16.h>

#include <algorithm>

#include "rb_common.cuh"

namespace rbk {

constexpr int PG = 8;      // queries per CTA in the projection / prolongation
constexpr int PC = 32;     // points per shared-memory chunk of the projection

template <typename T>
__device__ __forceinline__ const T* cur_r(const Params& P, int q) {
    return reinterpret_cast<const T*>(P.r) + (size_t)q * (size_t)P.g.n;
}

template <typename T> __device__ __forceinline__ const T* basis_c(const Params& P);
template <> __device__ __forceinline__ const double* basis_c<double>(const Params& P) { return P.W64c; }
template <> __device__ __forceinline__ const float* basis_c<float>(const Params& P) { return P.W32c; }

// partial r_N: proj[s][q][k] = sum over split s of W[i][k] r_q[i]
template <typename T>
__global__ void __launch_bounds__(THREADS) k_project(Params P) {
    __shared__ T Wsm[PC][MAX_N + 1];
    __shared__ T Rsm[PG][PC];
    __shared__ int qs[PG];
    __shared__ const T* rp[PG];
    const T* Wc = basis_c<T>(P);
    const int nb = P.nb, nbp = P.nbp;
    const long long n = P.g.n;
    const int cnt = P.lcnt[L_PREC];
    const int groups = (cnt + PG - 1) / PG;
    const long long span = ((n + P.nsplit - 1) / P.nsplit + PC - 1) / PC * PC;
    const long long total = (long long)groups * P.nsplit;
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        const int grp = (int)(w / P.nsplit), sp = (int)(w % P.nsplit);
        __syncthreads();
        if (threadIdx.x < PG) {
            const int sl = grp * PG + threadIdx.x;
            const int q = sl < cnt ? P.lidx[L_PREC * P.Bmax + sl] : -1;
            qs[threadIdx.x] = q;
            rp[threadIdx.x] = q >= 0 ? cur_r<T>(P, q) : nullptr;
        }
        __syncthreads();
        const long long i0 = (long long)sp * span;
        const long long i1 = i0 + span < n ? i0 + span : n;
        T acc[4] = {T(0), T(0), T(0), T(0)};
        for (long long c0 = i0; c0 < i1; c0 += PC) {
            __syncthreads();
            for (int idx = threadIdx.x; idx < nbp * PC; idx += THREADS) {
                const int k = idx / PC, i = idx % PC;
                Wsm[i][k] = (k < nb && c0 + i < i1) ? Wc[(size_t)k * n + c0 + i] : T(0);
            }
            for (int idx = threadIdx.x; idx < PG * PC; idx += THREADS) {
                const int gq = idx / PC, i = idx % PC;
                Rsm[gq][i] = (rp[gq] != nullptr && c0 + i < i1) ? rp[gq][c0 + i] : T(0);
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int o = threadIdx.x + j * THREADS;
                if (o < PG * nbp) {
                    const int gq = o / nbp, k = o % nbp;
                    T a = acc[j];
#pragma unroll 8
                    for (int i = 0; i < PC; ++i) a += Wsm[i][k] * Rsm[gq][i];
                    acc[j] = a;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int o = threadIdx.x + j * THREADS;
            if (o < PG * nbp) {
                const int gq = o / nbp, k = o % nbp;
                if (qs[gq] >= 0) P.proj[((size_t)sp * P.Bmax + qs[gq]) * nbp + k] = (double)acc[j];
            }
        }
    }
}

// e_N = A_N(mu)^{-1} r_N (eq. 6).  r_N is the fixed-order sum of the projection
// partials; A_N^{-1} was formed from the Cholesky factor when the query started
// (k_cholesky), so each iteration is one dense matvec (one warp per query,
// coalesced rows of the symmetric inverse).
template <typename T>
__global__ void __launch_bounds__(THREADS) k_reduced_solve(Params P) {
    __shared__ double buf[THREADS / 32][MAX_N];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int cnt = P.lcnt[L_PREC];
    const int nb = P.nb, nbp = P.nbp;
    double* v = buf[wib];
    for (int sl = blockIdx.x * (THREADS / 32) + wib; sl < cnt; sl += gridDim.x * (THREADS / 32)) {
        const int q = P.lidx[L_PREC * P.Bmax + sl];
        for (int k = lane; k < nb; k += 32) {
            double s = 0.0;
            for (int sp = 0; sp < P.nsplit; ++sp) s += P.proj[((size_t)sp * P.Bmax + q) * nbp + k];
            v[k] = s;
        }
        __syncwarp();
        const double* Ai = P.L + (size_t)q * nbp * nbp;
        double acc[MAX_N / 32];
#pragma unroll
        for (int t = 0; t < MAX_N / 32; ++t) acc[t] = 0.0;
        int nu_ = nb;   // basis vectors used by this application
        if (P.adaptive) {
            // e = M_k^T (M_k v_k) with the inverse factor M stored as X (k_cholesky):
            // z_i = sum_{j <= i} X[j][i] v_j, then e_j = sum_{i >= j} X[i][j] z_i, i, j < k
            nu_ = P.st[q].n_used;
            for (int j = 0; j < nu_; ++j) {
                const double vj = v[j];
                const double* row = Ai + (size_t)j * nbp;
#pragma unroll
                for (int t = 0; t < MAX_N / 32; ++t) {
                    const int k = lane + 32 * t;
                    if (k >= j && k < nu_) acc[t] += row[k] * vj;
                }
            }
            __syncwarp();
#pragma unroll
            for (int t = 0; t < MAX_N / 32; ++t) {
                const int k = lane + 32 * t;
                if (k < nu_) v[k] = acc[t];
                acc[t] = 0.0;
            }
            __syncwarp();
            for (int i = 0; i < nu_; ++i) {
                const double zi = v[i];
                const double* row = Ai + (size_t)i * nbp;
#pragma unroll
                for (int t = 0; t < MAX_N / 32; ++t) {
                    const int k = lane + 32 * t;
                    if (k <= i) acc[t] += row[k] * zi;
                }
            }
        } else {
            for (int j = 0; j < nb; ++j) {
                const double vj = v[j];
                const double* row = Ai + (size_t)j * nbp;
#pragma unroll
                for (int t = 0; t < MAX_N / 32; ++t) {
                    const int k = lane + 32 * t;
                    if (k < nb) acc[t] += row[k] * vj;
                }
            }
        }
        T* e = reinterpret_cast<T*>(P.e) + (size_t)q * P.lde;
#pragma unroll
        for (int t = 0; t < MAX_N / 32; ++t) {
            const int k = lane + 32 * t;
            if (k < P.lde) e[k] = k < nu_ ? (T)acc[t] : T(0);
        }
        __syncwarp();
    }
}

// ypro = (RBI ? x : 0) + W e_N
template <typename T, bool ADDX>
__global__ void __launch_bounds__(THREADS) k_prolong(Params P) {
    __shared__ T es[PG][MAX_N];
    __shared__ int qs[PG];
    const T* Wc = basis_c<T>(P);
    const int nb = P.nb, nbp = P.nbp;
    const long long n = P.g.n;
    const int cnt = P.lcnt[L_PREC];
    const int groups = (cnt + PG - 1) / PG;
    const int nchunk = (int)((n + TILE - 1) / TILE);
    const long long total = (long long)groups * nchunk;
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        const int grp = (int)(w / nchunk), ch = (int)(w % nchunk);
        __syncthreads();
        if (threadIdx.x < PG) {
            const int sl = grp * PG + threadIdx.x;
            qs[threadIdx.x] = sl < cnt ? P.lidx[L_PREC * P.Bmax + sl] : -1;
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < PG * nb; idx += THREADS) {
            const int gq = idx / nb, k = idx % nb;
            es[gq][k] = qs[gq] >= 0 ? reinterpret_cast<const T*>(P.e)[(size_t)qs[gq] * P.lde + k] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < TILE / THREADS; ++j) {
            const long long i = (long long)ch * TILE + j * THREADS + threadIdx.x;
            if (i >= n) continue;
            T acc[PG];
#pragma unroll
            for (int gq = 0; gq < PG; ++gq) acc[gq] = T(0);
            for (int k = 0; k < nb; ++k) {
                const T wv = Wc[(size_t)k * n + i];
#pragma unroll
                for (int gq = 0; gq < PG; ++gq) acc[gq] += wv * es[gq][k];
            }
#pragma unroll
            for (int gq = 0; gq < PG; ++gq) {
                const int q = qs[gq];
                if (q < 0) continue;
                T v = acc[gq];
                if constexpr (ADDX) v += (T)P.x64[(size_t)q * n + i];
                if (sizeof(T) == 4 && P.ybf16)
                    reinterpret_cast<__nv_bfloat16*>(P.ypro)[(size_t)q * n + i] = __float2bfloat16_rn((float)v);
                else
                    reinterpret_cast<T*>(P.ypro)[(size_t)q * n + i] = v;
            }
        }
    }
}

template <typename T>
void launch_project(const Params& P, const Launch& L) {
    if (P.nb > 0) k_project<T><<<L.grid, THREADS, 0, L.s>>>(P);
}
template <typename T>
void launch_reduced_solve(const Params& P, const Launch& L) {
    if (P.nb > 0) k_reduced_solve<T><<<L.grid, THREADS, 0, L.s>>>(P);
}
template <typename T>
void launch_prolong(const Params& P, const Launch& L, bool rbi_mode) {
    if (rbi_mode) {
        if constexpr (sizeof(T) == 8) k_prolong<T, true><<<L.grid, THREADS, 0, L.s>>>(P);
    } else {
        k_prolong<T, false><<<L.grid, THREADS, 0, L.s>>>(P);
    }
}
template void launch_project<float>(const Params&, const Launch&);
template void launch_project<double>(const Params&, const Launch&);
template void launch_reduced_solve<float>(const Params&, const Launch&);
template void launch_reduced_solve<double>(const Params&, const Launch&);
template void launch_prolong<float>(const Params&, const Launch&, bool);
template void launch_prolong<double>(const Params&, const Launch&, bool);

// ----------------------------------------------------------------------------
// A_N(mu) = sum_q mu_q A_{N,q}, its Cholesky factor (breakdown on a non-positive
// pivot) and, from the factor, A_N^{-1} written to [q][nbp][nbp]; one CTA per query.

__global__ void __launch_bounds__(THREADS) k_cholesky(Params P, const double* __restrict__ ANq, int Q) {
    extern __shared__ double A[];
    __shared__ int bad;
    const int q = blockIdx.x;
    if (q >= P.B) return;
    const int nb = P.nb, nbp = P.nbp;
    const double* mu = P.mu + (size_t)q * P.n_mu;
    for (int idx = threadIdx.x; idx < nb * nb; idx += THREADS) {
        double s = 0.0;
        for (int t = 0; t < Q; ++t) s += mu[t] * ANq[(size_t)t * nb * nb + idx];
        A[idx] = s;
    }
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (threadIdx.x == 0) {
            const double dj = A[j * nb + j];
            if (!(dj > 0.0)) bad = 1;
            else A[j * nb + j] = sqrt(dj);
        }
        __syncthreads();
        if (bad) break;
        const double ljj = A[j * nb + j];
        for (int i = j + 1 + threadIdx.x; i < nb; i += THREADS) A[i * nb + j] /= ljj;
        __syncthreads();
        const int m = nb - j - 1;
        for (int idx = threadIdx.x; idx < m * m; idx += THREADS) {
            const int i = j + 1 + idx / m, k = j + 1 + idx % m;
            if (k <= i) A[i * nb + k] -= A[i * nb + j] * A[k * nb + j];
        }
        __syncthreads();
    }
    // A_N^{-1} = L^{-T} L^{-1}, column j by the two triangular solves L z = e_j,
    // L^T x = z (thread j owns column j of the output; the output doubles as z)
    double* Ai = const_cast<double*>(P.L) + (size_t)q * nbp * nbp;
    if (!bad && P.adaptive) {
        // adaptive N: the inverse factor M = L^{-1}, stored as X = M + M^T - diag(M).  The
        // leading k x k block of M is the inverse factor of the leading block of A_N (W_k is
        // nested in W_N), so one X serves every N <= nb: e = M_k^T (M_k r_k).
        for (int j = threadIdx.x; j < nb; j += THREADS) {
            for (int i = 0; i < nb; ++i) {
                double sacc = (i == j) ? 1.0 : 0.0;
                for (int k = j; k < i; ++k) sacc -= A[i * nb + k] * Ai[(size_t)k * nbp + j];
                if (i >= j) Ai[(size_t)i * nbp + j] = sacc / A[i * nb + i];
            }
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < nb * nb; idx += THREADS) {
            const int i = idx / nb, j = idx % nb;
            if (j > i) Ai[(size_t)i * nbp + j] = Ai[(size_t)j * nbp + i];
        }
    } else if (!bad) {
        for (int j = threadIdx.x; j < nb; j += THREADS) {
            for (int i = 0; i < nb; ++i) {
                double sacc = (i == j) ? 1.0 : 0.0;
                for (int k = j; k < i; ++k) sacc -= A[i * nb + k] * Ai[(size_t)k * nbp + j];
                Ai[(size_t)i * nbp + j] = i < j ? 0.0 : sacc / A[i * nb + i];
            }
            for (int i = nb - 1; i >= 0; --i) {
                double sacc = Ai[(size_t)i * nbp + j];
                for (int k = i + 1; k < nb; ++k) sacc -= A[k * nb + i] * Ai[(size_t)k * nbp + j];
                Ai[(size_t)i * nbp + j] = sacc / A[i * nb + i];
            }
        }
    }
    if (bad && threadIdx.x == 0) {
        QState& s = P.st[q];
        if (s.phase != PH_DONE) mark_done(P, s, RB_EBREAKDOWN);
    }
}

void launch_cholesky(const Params& P, cudaStream_t s, const double* ANq, int Q) {
    if (P.nb == 0) return;
    const size_t smem = (size_t)P.nb * P.nb * sizeof(double);
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(k_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_N * MAX_N * 8);
        configured = true;
    }
    k_cholesky<<<P.B, THREADS, smem, s>>>(P, ANq, Q);
}

// ----------------------------------------------------------------------------
// offline helpers (FP64)

// out[v][k] = sum_i W[k][i] V[v][i]; split partials then a fixed-order sum.
constexpr int OSPLIT = 128;

__global__ void __launch_bounds__(THREADS) k_project_cols_part(Geo g, int nb, const double* __restrict__ Wc,
                                                               const double* __restrict__ V, double* part) {
    __shared__ double red[32];
    const int sp = blockIdx.x, v = blockIdx.y;
    const long long span = (g.n + OSPLIT - 1) / OSPLIT;
    const long long i0 = (long long)sp * span, i1 = i0 + span < g.n ? i0 + span : g.n;
    const double* Vv = V + (size_t)v * g.n;
    for (int k = 0; k < nb; ++k) {
        double a = 0.0;
        for (long long i = i0 + threadIdx.x; i < i1; i += THREADS) a += Wc[(size_t)k * g.n + i] * Vv[i];
        a = block_sum(a, red);
        if (threadIdx.x == 0) part[((size_t)v * nb + k) * OSPLIT + sp] = a;
    }
}

__global__ void k_project_cols_sum(int nv, int nb, const double* part, double* out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nv * nb) return;
    double s = 0.0;
    for (int sp = 0; sp < OSPLIT; ++sp) s += part[(size_t)idx * OSPLIT + sp];
    out[idx] = s;
}

// scratch: nv * nb * 128 doubles
void launch_project_cols(const Geo& g, int nb, const double* W64c, int nv, const double* V, double* out,
                         double* scratch, cudaStream_t s) {
    if (nb == 0 || nv == 0) return;
    k_project_cols_part<<<dim3(OSPLIT, nv), THREADS, 0, s>>>(g, nb, W64c, V, scratch);
    k_project_cols_sum<<<(nv * nb + 127) / 128, 128, 0, s>>>(nv, nb, scratch, out);
}

// v -= sum_k c[k] W[:,k]
__global__ void k_sub_cols(Geo g, int nb, const double* __restrict__ Wc, const double* __restrict__ c, double* v) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.n;
         i += (long long)gridDim.x * blockDim.x) {
        double s = v[i];
        for (int k = 0; k < nb; ++k) s -= c[k] * Wc[(size_t)k * g.n + i];
        v[i] = s;
    }
}

void launch_sub_cols(const Geo& g, int nb, const double* W64c, const double* c, double* v, cudaStream_t s) {
    if (nb == 0) return;
    long long blocks = (g.n + THREADS - 1) / THREADS;
    if (blocks > 4096) blocks = 4096;
    k_sub_cols<<<(unsigned)blocks, THREADS, 0, s>>>(g, nb, W64c, c, v);
}

__global__ void k_norm_part(long long n, const double* __restrict__ v, double* part) {
    __shared__ double red[32];
    const long long span = (n + OSPLIT - 1) / OSPLIT;
    const long long i0 = (long long)blockIdx.x * span, i1 = i0 + span < n ? i0 + span : n;
    double a = 0.0;
    for (long long i = i0 + threadIdx.x; i < i1; i += THREADS) a += v[i] * v[i];
    a = block_sum(a, red);
    if (threadIdx.x == 0) part[blockIdx.x] = a;
}

double launch_norm(const Geo& g, const double* v, double* scratch, cudaStream_t s) {
    k_norm_part<<<OSPLIT, THREADS, 0, s>>>(g.n, v, scratch);
    double h[OSPLIT];
    cudaMemcpyAsync(h, scratch, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    double t = 0.0;
    for (int i = 0; i < OSPLIT; ++i) t += h[i];
    return sqrt(t);
}

// Greedy step 5-6 criterion for every training parameter (one CTA each):
// a = A_N(mu)^{-1} f_N(mu), c = Rsnap^{-1} a (or c = a), score = sum |c|.
__global__ void __launch_bounds__(THREADS) k_scores(int P_, int R, const int* __restrict__ load_param, int n_mu, int nb,
                                                    const double* __restrict__ ANq, const double* __restrict__ fNr,
                                                    const double* __restrict__ Rsnap, const double* __restrict__ mus,
                                                    int literal, double* score, int* bad_out) {
    extern __shared__ double A[];
    double* f = A + nb * nb;
    __shared__ int bad;
    __shared__ double red[32];
    const int t = blockIdx.x;
    const double* mu = mus + (size_t)t * n_mu;
    for (int idx = threadIdx.x; idx < nb * nb; idx += THREADS) {
        double s = 0.0;
        for (int q = 0; q < P_; ++q) s += mu[q] * ANq[(size_t)q * nb * nb + idx];
        A[idx] = s;
    }
    for (int k = threadIdx.x; k < nb; k += THREADS) {
        double s = 0.0;
        for (int r = 0; r < R; ++r) s += (load_param[r] < 0 ? 1.0 : mu[load_param[r]]) * fNr[(size_t)r * nb + k];
        f[k] = s;
    }
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (threadIdx.x == 0) {
            const double dj = A[j * nb + j];
            if (!(dj > 0.0)) bad = 1;
            else A[j * nb + j] = sqrt(dj);
        }
        __syncthreads();
        if (bad) break;
        const double ljj = A[j * nb + j];
        for (int i = j + 1 + threadIdx.x; i < nb; i += THREADS) A[i * nb + j] /= ljj;
        __syncthreads();
        const int m = nb - j - 1;
        for (int idx = threadIdx.x; idx < m * m; idx += THREADS) {
            const int i = j + 1 + idx / m, k = j + 1 + idx % m;
            if (k <= i) A[i * nb + k] -= A[i * nb + j] * A[k * nb + j];
        }
        __syncthreads();
    }
    if (bad) {
        if (threadIdx.x == 0) { score[t] = -1.0; bad_out[t] = 1; }
        return;
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < nb; ++i) {           // L z = f
            double s = f[i];
            for (int k = 0; k < i; ++k) s -= A[i * nb + k] * f[k];
            f[i] = s / A[i * nb + i];
        }
        for (int i = nb - 1; i >= 0; --i) {      // L^T a = z
            double s = f[i];
            for (int k = i + 1; k < nb; ++k) s -= A[k * nb + i] * f[k];
            f[i] = s / A[i * nb + i];
        }
        if (!literal) {
            for (int i = nb - 1; i >= 0; --i) {  // Rsnap c = a
                double s = f[i];
                for (int k = i + 1; k < nb; ++k) s -= Rsnap[i * nb + k] * f[k];
                f[i] = s / Rsnap[i * nb + i];
            }
        }
    }
    __syncthreads();
    double a = 0.0;
    for (int k = threadIdx.x; k < nb; k += THREADS) a += fabs(f[k]);
    a = block_sum(a, red);
    if (threadIdx.x == 0) { score[t] = a; bad_out[t] = 0; }
}

void launch_scores(const Geo& g, int P_, int R, const int* load_param, int n_mu, int nb, int nbp, const double* ANq,
                   const double* fNr, const double* Rsnap, int ntrain, const double* mu, int literal, double* score,
                   int* bad, cudaStream_t s) {
    (void)g;
    (void)nbp;
    const size_t smem = ((size_t)nb * nb + nb) * sizeof(double);
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(k_scores, cudaFuncAttributeMaxDynamicSharedMemorySize, (MAX_N * MAX_N + MAX_N) * 8);
        configured = true;
    }
    k_scores<<<ntrain, THREADS, smem, s>>>(P_, R, load_param, n_mu, nb, ANq, fNr, Rsnap, mu, literal, score, bad);
}

}  // namespace rbk

// ----------------------------------------------------------------------------
// Starting vectors and reduced coefficients of given vectors (rb_warm_start,
// rb_coefficients).

namespace rbk {

// a_N(mu) of eq. 2: A_N(mu) a = f_N(mu) with A_N(mu) = sum_q mu_q A_{N,q} and
// f_N(mu) = sum_r Phi_r(mu) f_{N,r} (eq. 12b), by Cholesky; one CTA per query.
// A non-positive pivot zeroes the query's coefficients and sets *bad.
__global__ void __launch_bounds__(128) k_galerkin(int nb, int Q, const double* __restrict__ ANq, int R, LoadMap lm,
                                                   const double* __restrict__ fNr, int n_mu,
                                                   const double* __restrict__ mu, double* coef, int* bad) {
    extern __shared__ double A[];      // [nb][nb], then f [nb]
    __shared__ int brk;
    double* f = A + (size_t)nb * nb;
    const int q = blockIdx.x;
    const double* m = mu + (size_t)q * n_mu;
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
        double s = 0.0;
        for (int t = 0; t < Q; ++t) s += m[t] * ANq[(size_t)t * nb * nb + idx];
        A[idx] = s;
    }
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        double s = 0.0;
        for (int r = 0; r < R; ++r) s += (lm.param[r] < 0 ? 1.0 : m[lm.param[r]]) * fNr[(size_t)r * nb + k];
        f[k] = s;
    }
    if (threadIdx.x == 0) brk = 0;
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (threadIdx.x == 0) {
            const double d = A[j * nb + j];
            if (!(d > 0.0)) brk = 1;
            else A[j * nb + j] = sqrt(d);
        }
        __syncthreads();
        if (brk) break;
        const double ljj = A[j * nb + j];
        for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) A[i * nb + j] /= ljj;
        __syncthreads();
        const int rem = nb - j - 1;
        for (int idx = threadIdx.x; idx < rem * rem; idx += blockDim.x) {
            const int i = j + 1 + idx / rem, k = j + 1 + idx % rem;
            if (k <= i) A[i * nb + k] -= A[i * nb + j] * A[k * nb + j];
        }
        __syncthreads();
    }
    double* c = coef + (size_t)q * nb;
    if (brk) {
        for (int k = threadIdx.x; k < nb; k += blockDim.x) c[k] = 0.0;
        if (threadIdx.x == 0) atomicExch(bad, 1);
        return;
    }
    if (threadIdx.x == 0) {
        // L z = f, then L^T a = z (in place in f)
        for (int i = 0; i < nb; ++i) {
            double s = f[i];
            for (int k = 0; k < i; ++k) s -= A[i * nb + k] * f[k];
            f[i] = s / A[i * nb + i];
        }
        for (int i = nb - 1; i >= 0; --i) {
            double s = f[i];
            for (int k = i + 1; k < nb; ++k) s -= A[k * nb + i] * f[k];
            f[i] = s / A[i * nb + i];
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nb; k += blockDim.x) c[k] = f[k];
}

void launch_galerkin(int nb, int Q, const double* ANq, int R, const LoadMap& lm, const double* fNr, int n_mu, int B,
                     const double* mu, double* coef, int* bad, cudaStream_t s) {
    if (nb == 0 || B == 0) return;
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(k_galerkin, cudaFuncAttributeMaxDynamicSharedMemorySize, (MAX_N * MAX_N + MAX_N) * 8);
        configured = true;
    }
    k_galerkin<<<B, 128, (size_t)(nb * nb + nb) * sizeof(double), s>>>(nb, Q, ANq, R, lm, fNr, n_mu, mu, coef, bad);
}

// x_b = W c_b for B queries (products and sums in the precision of the given copy of W,
// written as FP64): one pass over W per group of LQ queries, points coalesced.
constexpr int LQ = 16;

template <typename TW>
__global__ void __launch_bounds__(THREADS) k_lift(long long n, int nb, const TW* __restrict__ Wc, int B,
                                                  const double* __restrict__ coef, double* __restrict__ x) {
    __shared__ TW cs[LQ][MAX_N];
    const int groups = (B + LQ - 1) / LQ;
    const long long chunks = (n + TILE - 1) / TILE;
    for (long long w = blockIdx.x; w < (long long)groups * chunks; w += gridDim.x) {
        const int grp = (int)(w / chunks);
        const long long ch = w % chunks;
        __syncthreads();
        for (int idx = threadIdx.x; idx < LQ * nb; idx += THREADS) {
            const int g = idx / nb, k = idx % nb, b = grp * LQ + g;
            cs[g][k] = b < B ? (TW)coef[(size_t)b * nb + k] : TW(0);
        }
        __syncthreads();
#pragma unroll 1
        for (int j = 0; j < TILE / THREADS; ++j) {
            const long long i = ch * TILE + (long long)j * THREADS + threadIdx.x;
            if (i >= n) continue;
            TW acc[LQ];
#pragma unroll
            for (int g = 0; g < LQ; ++g) acc[g] = TW(0);
            for (int k = 0; k < nb; ++k) {
                const TW wv = Wc[(size_t)k * n + i];
#pragma unroll
                for (int g = 0; g < LQ; ++g) acc[g] = fma(cs[g][k], wv, acc[g]);
            }
#pragma unroll
            for (int g = 0; g < LQ; ++g) {
                const int b = grp * LQ + g;
                if (b < B) x[(size_t)b * n + i] = (double)acc[g];
            }
        }
    }
}

void launch_lift(long long n, int nb, const float* W32c, int B, const double* coef, double* x, int grid,
                 cudaStream_t s) {
    if (B == 0) return;
    if (nb == 0) {
        cudaMemsetAsync(x, 0, (size_t)B * n * sizeof(double), s);
        return;
    }
    k_lift<float><<<grid, THREADS, 0, s>>>(n, nb, W32c, B, coef, x);
}

// the same with the FP64 basis (products and sums in FP64): the RB approximation as a start
void launch_lift64(long long n, int nb, const double* W64c, int B, const double* coef, double* x, int grid,
                   cudaStream_t s) {
    if (B == 0) return;
    if (nb == 0) {
        cudaMemsetAsync(x, 0, (size_t)B * n * sizeof(double), s);
        return;
    }
    k_lift<double><<<grid, THREADS, 0, s>>>(n, nb, W64c, B, coef, x);
}

// part[sp][b][k] = sum over split sp of W[i][k] x_b[i]: FP32 products summed in
// FP32 over chunks of CPC points, chunk sums added in FP64.
constexpr int CQ = 8;
constexpr int CPC = 32;

__global__ void __launch_bounds__(THREADS) k_coef_part(long long n, int nb, const float* __restrict__ Wc, int B,
                                                       const double* __restrict__ X, int nsplit, double* part) {
    __shared__ float Ws[CPC][MAX_N + 1];
    __shared__ float Xs[CQ][CPC];
    const int groups = (B + CQ - 1) / CQ;
    const long long span = ((n + nsplit - 1) / nsplit + CPC - 1) / CPC * CPC;
    for (long long w = blockIdx.x; w < (long long)groups * nsplit; w += gridDim.x) {
        const int grp = (int)(w / nsplit), sp = (int)(w % nsplit);
        const long long i0 = (long long)sp * span;
        const long long i1 = i0 + span < n ? i0 + span : n;
        double acc[CQ * MAX_N / THREADS];
#pragma unroll
        for (int j = 0; j < CQ * MAX_N / THREADS; ++j) acc[j] = 0.0;
        for (long long c0 = i0; c0 < i1; c0 += CPC) {
            __syncthreads();
            for (int idx = threadIdx.x; idx < nb * CPC; idx += THREADS) {
                const int k = idx / CPC, i = idx % CPC;
                Ws[i][k] = c0 + i < i1 ? Wc[(size_t)k * n + c0 + i] : 0.0f;
            }
            for (int idx = threadIdx.x; idx < CQ * CPC; idx += THREADS) {
                const int g = idx / CPC, i = idx % CPC, b = grp * CQ + g;
                Xs[g][i] = (b < B && c0 + i < i1) ? (float)X[(size_t)b * n + c0 + i] : 0.0f;
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < CQ * MAX_N / THREADS; ++j) {
                const int o = threadIdx.x + j * THREADS;
                if (o < CQ * nb) {
                    const int g = o / nb, k = o % nb;
                    float a = 0.0f;
#pragma unroll 8
                    for (int i = 0; i < CPC; ++i) a = fmaf(Ws[i][k], Xs[g][i], a);
                    acc[j] += (double)a;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < CQ * MAX_N / THREADS; ++j) {
            const int o = threadIdx.x + j * THREADS;
            if (o < CQ * nb) {
                const int g = o / nb, k = o % nb, b = grp * CQ + g;
                if (b < B) part[((size_t)sp * B + b) * nb + k] = acc[j];
            }
        }
    }
}

__global__ void k_coef_sum(int nsplit, int B, int nb, const double* __restrict__ part, double* coef) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * nb) return;
    double s = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) s += part[(size_t)sp * B * nb + idx];
    coef[idx] = s;
}

// coef [B][nb] = W^T X_b; scratch must hold coef_splits(B, num_sms) * B * nb doubles
int coef_splits(int B, int num_sms) {
    const int groups = (B + CQ - 1) / CQ;
    return std::max(1, std::min(64, (4 * num_sms + groups - 1) / groups));
}

void launch_coefficients(long long n, int nb, const float* W32c, int B, const double* X, double* coef,
                         double* scratch, int num_sms, cudaStream_t s) {
    if (B == 0 || nb == 0) return;
    const int nsplit = coef_splits(B, num_sms);
    const long long work = (long long)((B + CQ - 1) / CQ) * nsplit;
    const int grid = (int)std::min<long long>(work, 8LL * num_sms);
    k_coef_part<<<grid, THREADS, 0, s>>>(n, nb, W32c, B, X, nsplit, scratch);
    k_coef_sum<<<(B * nb + 255) / 256, 256, 0, s>>>(nsplit, B, nb, scratch, coef);
}

}  // namespace rbk
