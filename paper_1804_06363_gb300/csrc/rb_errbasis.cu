// Error basis of the learned warm start.
//
// A start in span(W) is sent by the first RB correction of Alg. 3 to about the same
// iterate, so the start that can gain leaves span(W): x_0 = x_hat(mu) + V z(mu), with
// x_hat = W a_N(mu) the RB approximation of eq. 3 (Galerkin coefficients of eq. 2) and V
// an orthonormal basis of the errors e_s = x_s - x_hat(mu_s) of training solutions.
// V comes from the method of snapshots: the Gram matrix G = E^T E (S x S, FP64 on the
// device, fixed-order partial sums), its eigenpairs (cyclic Jacobi on the host, S <= 512),
// V = E Phi_m diag(lambda_m)^{-1/2}; the network's targets are Z = V^T E =
// diag(lambda_m)^{1/2} Phi_m^T.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "rb_common.cuh"

namespace rbk {

namespace {

constexpr int EB_Q = 8;      // queries per CTA of the error and lift kernels
constexpr int EB_T = 32;     // Gram tile (32 x 32 entries per CTA, 4 per thread)
constexpr int EB_CH = 64;    // points per staged chunk of the Gram kernel
constexpr int EB_SPLIT = 96; // point ranges of the Gram partial sums

// E[s][i] = X[s][i] - sum_k W64c[k][i] a[s][k], FP64
__global__ void __launch_bounds__(THREADS) k_eb_errors(long long n, int nb, const double* __restrict__ W64c, int S,
                                                       const double* __restrict__ a, const double* __restrict__ X,
                                                       double* __restrict__ E) {
    __shared__ double as[EB_Q][MAX_N];
    const int groups = (S + EB_Q - 1) / EB_Q;
    const long long chunks = (n + TILE - 1) / TILE;
    for (long long w = blockIdx.x; w < (long long)groups * chunks; w += gridDim.x) {
        const int grp = (int)(w / chunks);
        const long long ch = w % chunks;
        __syncthreads();
        for (int idx = threadIdx.x; idx < EB_Q * nb; idx += THREADS) {
            const int g = idx / nb, k = idx % nb, s = grp * EB_Q + g;
            as[g][k] = s < S ? a[(size_t)s * nb + k] : 0.0;
        }
        __syncthreads();
        for (int j = 0; j < TILE / THREADS; ++j) {
            const long long i = ch * TILE + (long long)j * THREADS + threadIdx.x;
            if (i >= n) continue;
            double acc[EB_Q];
#pragma unroll
            for (int g = 0; g < EB_Q; ++g) acc[g] = 0.0;
            for (int k = 0; k < nb; ++k) {
                const double wv = W64c[(size_t)k * n + i];
#pragma unroll
                for (int g = 0; g < EB_Q; ++g) acc[g] += as[g][k] * wv;
            }
#pragma unroll
            for (int g = 0; g < EB_Q; ++g) {
                const int s = grp * EB_Q + g;
                if (s < S) E[(size_t)s * n + i] = X[(size_t)s * n + i] - acc[g];
            }
        }
    }
}

// part[sp][s][t] = sum over the points of split sp of E[s][i] E[t][i] for the tiles with
// ts <= tt (32 x 32 entries per CTA, 4 per thread)
__global__ void __launch_bounds__(THREADS) k_eb_gram_part(long long n, int S, const double* __restrict__ E,
                                                          double* __restrict__ part) {
    __shared__ double es[EB_T][EB_CH + 1];
    __shared__ double et[EB_T][EB_CH + 1];
    const int nt = (S + EB_T - 1) / EB_T;
    const int npairs = nt * (nt + 1) / 2;
    const long long span = (n + EB_SPLIT - 1) / EB_SPLIT;
    for (long long w = blockIdx.x; w < (long long)npairs * EB_SPLIT; w += gridDim.x) {
        const int pr = (int)(w / EB_SPLIT), sp = (int)(w % EB_SPLIT);
        int ts = 0, rem = pr;
        while (rem >= nt - ts) { rem -= nt - ts; ++ts; }
        const int tt = ts + rem;
        const long long i0 = (long long)sp * span, i1 = min(n, i0 + span);
        // thread -> entries (r, c), (r + 8, c), (r + 16, c), (r + 24, c) of the tile
        const int c = threadIdx.x % EB_T, r = threadIdx.x / EB_T;
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (long long c0 = i0; c0 < i1; c0 += EB_CH) {
            __syncthreads();
            for (int idx = threadIdx.x; idx < EB_T * EB_CH; idx += THREADS) {
                const int row = idx / EB_CH, col = idx % EB_CH;
                const long long i = c0 + col;
                const int s = ts * EB_T + row, t = tt * EB_T + row;
                es[row][col] = (s < S && i < i1) ? E[(size_t)s * n + i] : 0.0;
                et[row][col] = (t < S && i < i1) ? E[(size_t)t * n + i] : 0.0;
            }
            __syncthreads();
            for (int col = 0; col < EB_CH; ++col) {
                const double b = et[c][col];
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[u] += es[r + 8 * u][col] * b;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int s = ts * EB_T + r + 8 * u, t = tt * EB_T + c;
            if (s < S && t < S) part[((size_t)sp * S + s) * S + t] = acc[u];
        }
    }
}

// G[s][t] = sum_sp part[sp][s][t] in split order, for s in the tile row <= t's tile; mirrored
__global__ void k_eb_gram_sum(int S, const double* __restrict__ part, double* __restrict__ G) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)S * S) return;
    const int s = (int)(idx / S), t = (int)(idx % S);
    if (s / EB_T > t / EB_T) return;   // filled from its mirror
    double acc = 0.0;
    for (int sp = 0; sp < EB_SPLIT; ++sp) acc += part[((size_t)sp * S + s) * S + t];
    G[(size_t)s * S + t] = acc;
    if (s / EB_T < t / EB_T) G[(size_t)t * S + s] = acc;
}

// V[k][i] = sum_s E[s][i] C[s][k] (C = Phi_m diag(lambda)^{-1/2}), FP64 and an FP32 copy
__global__ void __launch_bounds__(THREADS) k_eb_modes(long long n, int S, int m, const double* __restrict__ E,
                                                      const double* __restrict__ C, double* __restrict__ V64,
                                                      float* __restrict__ V32) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        for (int k0 = 0; k0 < m; k0 += 8) {
            double acc[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] = 0.0;
            for (int s = 0; s < S; ++s) {
                const double e = E[(size_t)s * n + i];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (k0 + u < m) acc[u] += e * __ldg(C + (size_t)s * m + k0 + u);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (k0 + u < m) {
                    V64[(size_t)(k0 + u) * n + i] = acc[u];
                    V32[(size_t)(k0 + u) * n + i] = (float)acc[u];
                }
        }
    }
}

// x_b += sum_k V32[k][i] z_b[k]  (the error part of the warm start)
__global__ void __launch_bounds__(THREADS) k_eb_lift_add(long long n, int m, const float* __restrict__ V32, int B,
                                                         const double* __restrict__ z, double* __restrict__ x) {
    __shared__ float zs[EB_Q][64];
    const int groups = (B + EB_Q - 1) / EB_Q;
    const long long chunks = (n + TILE - 1) / TILE;
    for (long long w = blockIdx.x; w < (long long)groups * chunks; w += gridDim.x) {
        const int grp = (int)(w / chunks);
        const long long ch = w % chunks;
        __syncthreads();
        for (int idx = threadIdx.x; idx < EB_Q * m; idx += THREADS) {
            const int g = idx / m, k = idx % m, b = grp * EB_Q + g;
            zs[g][k] = b < B ? (float)z[(size_t)b * m + k] : 0.0f;
        }
        __syncthreads();
        for (int j = 0; j < TILE / THREADS; ++j) {
            const long long i = ch * TILE + (long long)j * THREADS + threadIdx.x;
            if (i >= n) continue;
            float acc[EB_Q];
#pragma unroll
            for (int g = 0; g < EB_Q; ++g) acc[g] = 0.0f;
            for (int k = 0; k < m; ++k) {
                const float v = V32[(size_t)k * n + i];
#pragma unroll
                for (int g = 0; g < EB_Q; ++g) acc[g] = fmaf(zs[g][k], v, acc[g]);
            }
#pragma unroll
            for (int g = 0; g < EB_Q; ++g) {
                const int b = grp * EB_Q + g;
                if (b < B) x[(size_t)b * n + i] += (double)acc[g];
            }
        }
    }
}

}  // namespace

// Eigenpairs of the symmetric S x S matrix A (row-major, destroyed) by cyclic Jacobi
// rotations: lam[S], Phi [S][S] (column k = eigenvector k), sorted by decreasing lambda.
void jacobi_eigen(int S, std::vector<double>& A, std::vector<double>& lam, std::vector<double>& Phi) {
    std::vector<double> V((size_t)S * S, 0.0);
    for (int i = 0; i < S; ++i) V[(size_t)i * S + i] = 1.0;
    auto a = [&](int i, int j) -> double& { return A[(size_t)i * S + j]; };
    double fro = 0.0;
    for (size_t i = 0; i < A.size(); ++i) fro += A[i] * A[i];
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < S; ++i)
            for (int j = i + 1; j < S; ++j) off += a(i, j) * a(i, j);
        if (off <= 1e-30 * fro) break;
        for (int p = 0; p < S - 1; ++p)
            for (int q = p + 1; q < S; ++q) {
                const double apq = a(p, q);
                if (std::fabs(apq) <= 1e-300) continue;
                const double theta = (a(q, q) - a(p, p)) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < S; ++k) {   // columns p, q
                    const double akp = a(k, p), akq = a(k, q);
                    a(k, p) = c * akp - s * akq;
                    a(k, q) = s * akp + c * akq;
                }
                for (int k = 0; k < S; ++k) {   // rows p, q
                    const double apk = a(p, k), aqk = a(q, k);
                    a(p, k) = c * apk - s * aqk;
                    a(q, k) = s * apk + c * aqk;
                }
                for (int k = 0; k < S; ++k) {
                    const double vkp = V[(size_t)k * S + p], vkq = V[(size_t)k * S + q];
                    V[(size_t)k * S + p] = c * vkp - s * vkq;
                    V[(size_t)k * S + q] = s * vkp + c * vkq;
                }
            }
    }
    std::vector<int> order(S);
    for (int i = 0; i < S; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return a(x, x) > a(y, y); });
    lam.resize(S);
    Phi.assign((size_t)S * S, 0.0);
    for (int k = 0; k < S; ++k) {
        lam[k] = a(order[k], order[k]);
        for (int i = 0; i < S; ++i) Phi[(size_t)i * S + k] = V[(size_t)i * S + order[k]];
    }
}

void launch_eb_errors(long long n, int nb, const double* W64c, int S, const double* a, const double* X, double* E,
                      int grid, cudaStream_t s) {
    k_eb_errors<<<grid, THREADS, 0, s>>>(n, nb, W64c, S, a, X, E);
}
size_t eb_gram_part_elems(int S) { return (size_t)EB_SPLIT * S * S; }
void launch_eb_gram(long long n, int S, const double* E, double* part, double* G, int grid, cudaStream_t s) {
    k_eb_gram_part<<<grid, THREADS, 0, s>>>(n, S, E, part);
    const long long tot = (long long)S * S;
    k_eb_gram_sum<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(S, part, G);
}
void launch_eb_modes(long long n, int S, int m, const double* E, const double* C, double* V64, float* V32, int grid,
                     cudaStream_t s) {
    k_eb_modes<<<grid, THREADS, 0, s>>>(n, S, m, E, C, V64, V32);
}
void launch_eb_lift_add(long long n, int m, const float* V32, int B, const double* z, double* x, int grid,
                        cudaStream_t s) {
    if (B > 0 && m > 0) k_eb_lift_add<<<grid, THREADS, 0, s>>>(n, m, V32, B, z, x);
}

}  // namespace rbk
