// Learned warm start: a multilayer perceptron c(mu) that predicts the reduced
// coefficients of the solution, so that the RB solvers (Alg. 2, Alg. 3) can
// start from x_0 = W c(mu) instead of x_0 = 0.  The paper has no learned
// component; its iterations accept any start.
//
// Network: features of the parameter vector (log of the P diffusion
// coefficients, the load parameters as they are), standardised by the training
// set's per-column mean and standard deviation, two hidden layers of width H
// with GELU, a linear output layer giving standardised coefficients.
//
// Precision: weights are used as BF16 values (the FP32 master copies rounded to
// nearest, ties to even), biases and activations are FP32, every product is
// accumulated in FP32.  Training: mean squared error over the standardised
// targets, full batch, back-propagation, Adam (Kingma & Ba 2015) on the FP32
// masters; the gradient treats the BF16 rounding as the identity.
//
// Kernels:
//   k_mlp_moments  per-column mean and standard deviation of features / targets
//   k_mlp_tile     TS samples per CTA, everything in shared memory: the forward
//                  pass through all layers; in training also the loss, the
//                  back-propagation and the tile's partial weight gradients
//   k_mlp_adam     fixed-order sum of the partials over tiles, then Adam
// Flat parameter vector: W1 [H][I], b1 [H], W2 [H][H], b2 [H], W3 [O][H], b3 [O].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "rb_common.cuh"

namespace rbk {
void set_global_error(const std::string& m);
}

namespace {

constexpr int TS = 32;            // samples per CTA tile
constexpr int SG = 8;             // samples per thread in the dense products
constexpr int MT = 256;           // threads per CTA
constexpr int MAX_IN = 32;
constexpr int MAX_H = 128;
constexpr int MAX_OUT = 128;
constexpr int LOSS_CAP = 1 << 16; // steps per rb_mlp_fit call
constexpr int GRAPH_STEPS = 16;   // training steps per captured graph

// Leading dimension of a transposed BF16 weight tile Wt[k][j]: at least n, and
// n/2 odd in 4-byte words, so that threads that differ in k hit distinct banks.
__host__ __device__ inline int ldpad(int n) {
    int ld = (n + 1) & ~1;
    if (((ld / 2) & 1) == 0) ld += 2;
    return ld;
}

__host__ __device__ inline size_t al16(size_t b) { return (b + 15) & ~size_t(15); }

struct Layout {
    int ld1, ld2, ld3;
    size_t wt1, wt2, wt3, bias, x, z1, a1, z2, a2, y, red, total;
};

__host__ __device__ inline Layout layout(int I, int H, int O) {
    Layout L;
    L.ld1 = ldpad(H);
    L.ld2 = ldpad(H);
    L.ld3 = ldpad(O);
    size_t o = 0;
    L.wt1 = o; o = al16(o + (size_t)I * L.ld1 * 2);
    L.wt2 = o; o = al16(o + (size_t)H * L.ld2 * 2);
    L.wt3 = o; o = al16(o + (size_t)H * L.ld3 * 2);
    L.bias = o; o = al16(o + (size_t)(2 * H + O) * 4);
    L.x = o; o = al16(o + (size_t)TS * I * 4);
    L.z1 = o; o = al16(o + (size_t)TS * H * 4);
    L.a1 = o; o = al16(o + (size_t)TS * H * 4);
    L.z2 = o; o = al16(o + (size_t)TS * H * 4);
    L.a2 = o; o = al16(o + (size_t)TS * H * 4);
    L.y = o; o = al16(o + (size_t)TS * O * 4);
    L.red = o; o = al16(o + 32 * 8);
    L.total = o;
    return L;
}

struct Net {
    int I, P, H, O;
    long long np;
    long long ow1, ob1, ow2, ob2, ow3, ob3;   // offsets in the flat parameter vector
    const float* w;                           // FP32 masters
    const __nv_bfloat16* wb;                  // BF16 copies (same offsets)
    const double* scale;                      // in_mean [I], in_scale [I], out_mean [O], out_scale [O]
};

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

// d/dz z Phi(z) = Phi(z) + z phi(z)
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// out[s][j] = bias[j] + sum_k in[s][k] W[j][k] for the TS samples; Wt[k * ldw + j] = W[j][k].
// With a != nullptr the pre-activation goes to z and GELU of it to a.
__device__ void dense_fwd(const float* in, int ldi, int nin, const __nv_bfloat16* Wt, int ldw, const float* bias,
                          int nout, float* z, float* a, int ldz) {
    for (int c = threadIdx.x; c < nout * (TS / SG); c += MT) {
        const int j = c % nout, g = c / nout;
        const float* ip = in + (size_t)g * SG * ldi;
        float acc[SG];
#pragma unroll
        for (int u = 0; u < SG; ++u) acc[u] = bias[j];
        for (int k = 0; k < nin; ++k) {
            const float w = __bfloat162float(Wt[k * ldw + j]);
#pragma unroll
            for (int u = 0; u < SG; ++u) acc[u] = fmaf(ip[u * ldi + k], w, acc[u]);
        }
#pragma unroll
        for (int u = 0; u < SG; ++u) {
            const int o = (g * SG + u) * ldz + j;
            z[o] = acc[u];
            if (a) a[o] = gelu(acc[u]);
        }
    }
}

// dz[s][k] = (sum_j d[s][j] W[j][k]) * GELU'(z[s][k])   (back-propagation through
// a layer with nout outputs into a GELU layer of width nin)
__device__ void dense_bwd(const float* d, int ldd, int nout, const __nv_bfloat16* Wt, int ldw, int nin,
                          const float* z, float* dz, int ldz) {
    for (int c = threadIdx.x; c < nin * (TS / SG); c += MT) {
        const int k = c % nin, g = c / nin;
        const float* dp = d + (size_t)g * SG * ldd;
        float acc[SG];
#pragma unroll
        for (int u = 0; u < SG; ++u) acc[u] = 0.0f;
        for (int j = 0; j < nout; ++j) {
            const float w = __bfloat162float(Wt[k * ldw + j]);
#pragma unroll
            for (int u = 0; u < SG; ++u) acc[u] = fmaf(dp[u * ldd + j], w, acc[u]);
        }
#pragma unroll
        for (int u = 0; u < SG; ++u) {
            const int o = (g * SG + u) * ldz + k;
            dz[o] = acc[u] * gelu_grad(z[o]);
        }
    }
}

// gW[j][k] = sum_s d[s][j] in[s][k], gb[j] = sum_s d[s][j] over the tile (global memory)
__device__ void dense_wgrad(const float* d, int ldd, int nout, const float* in, int ldi, int nin, float* gW,
                            float* gb) {
    for (int c = threadIdx.x; c < nout * nin; c += MT) {
        const int j = c / nin, k = c % nin;
        float acc = 0.0f;
#pragma unroll 8
        for (int s = 0; s < TS; ++s) acc = fmaf(d[s * ldd + j], in[s * ldi + k], acc);
        gW[c] = acc;
    }
    for (int j = threadIdx.x; j < nout; j += MT) {
        float acc = 0.0f;
        for (int s = 0; s < TS; ++s) acc += d[s * ldd + j];
        gb[j] = acc;
    }
}

__device__ double block_sum_d(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;   // valid in thread 0
}

// Per-column mean and population standard deviation (floored at 1e-12); column
// c < I is feature c of mu, column I + j is target j.  One CTA per column.
__global__ void __launch_bounds__(MT) k_mlp_moments(int S, int I, int P, int O, const double* __restrict__ mu,
                                                     int ld_mu, const double* __restrict__ tgt, double* scale) {
    __shared__ double red[32];
    __shared__ double mean_s;
    const int c = blockIdx.x;
    auto val = [&](int s) -> double {
        if (c < I) {
            const double m = mu[(size_t)s * ld_mu + c];
            return c < P ? log(m) : m;
        }
        return tgt[(size_t)s * O + (c - I)];
    };
    double a = 0.0;
    for (int s = threadIdx.x; s < S; s += MT) a += val(s);
    a = block_sum_d(a, red);
    if (threadIdx.x == 0) mean_s = a / S;
    __syncthreads();
    const double mean = mean_s;
    double q = 0.0;
    for (int s = threadIdx.x; s < S; s += MT) {
        const double d = val(s) - mean;
        q += d * d;
    }
    q = block_sum_d(q, red);
    if (threadIdx.x == 0) {
        const double sd = fmax(sqrt(q / S), 1e-12);
        if (c < I) {
            scale[c] = mean;
            scale[I + c] = sd;
        } else {
            scale[2 * I + (c - I)] = mean;
            scale[2 * I + O + (c - I)] = sd;
        }
    }
}

// One tile of TS samples.  Inference (TRAIN = false): out[s][j] = out_mean[j] +
// out_scale[j] * network(x_s)[j].  Training: loss partial sum of (y - t)^2 over
// the tile into loss_part[tile], weight-gradient partials into part[tile][np].
template <bool TRAIN>
__global__ void __launch_bounds__(MT) k_mlp_tile(Net M, int S, const double* __restrict__ mu, int ld_mu,
                                                  const double* __restrict__ tgt, double* __restrict__ out,
                                                  float* __restrict__ part, double* __restrict__ loss_part,
                                                  int* __restrict__ step, int bump) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int I = M.I, H = M.H, O = M.O;
    const Layout L = layout(I, H, O);
    __nv_bfloat16* Wt1 = reinterpret_cast<__nv_bfloat16*>(smem + L.wt1);
    __nv_bfloat16* Wt2 = reinterpret_cast<__nv_bfloat16*>(smem + L.wt2);
    __nv_bfloat16* Wt3 = reinterpret_cast<__nv_bfloat16*>(smem + L.wt3);
    float* b1 = reinterpret_cast<float*>(smem + L.bias);
    float* b2 = b1 + H;
    float* b3 = b2 + H;
    float* X = reinterpret_cast<float*>(smem + L.x);
    float* Z1 = reinterpret_cast<float*>(smem + L.z1);
    float* A1 = reinterpret_cast<float*>(smem + L.a1);
    float* Z2 = reinterpret_cast<float*>(smem + L.z2);
    float* A2 = reinterpret_cast<float*>(smem + L.a2);
    float* Y = reinterpret_cast<float*>(smem + L.y);
    double* red = reinterpret_cast<double*>(smem + L.red);

    const int s0 = blockIdx.x * TS;
    const int ns = min(TS, S - s0);
    if (TRAIN && bump && blockIdx.x == 0 && threadIdx.x == 0) *step += 1;

    // weights, transposed into shared memory: Wt[k][j] = W[j][k]
    for (int idx = threadIdx.x; idx < H * I; idx += MT) Wt1[(idx % I) * L.ld1 + idx / I] = M.wb[M.ow1 + idx];
    for (int idx = threadIdx.x; idx < H * H; idx += MT) Wt2[(idx % H) * L.ld2 + idx / H] = M.wb[M.ow2 + idx];
    for (int idx = threadIdx.x; idx < O * H; idx += MT) Wt3[(idx % H) * L.ld3 + idx / H] = M.wb[M.ow3 + idx];
    for (int j = threadIdx.x; j < H; j += MT) {
        b1[j] = M.w[M.ob1 + j];
        b2[j] = M.w[M.ob2 + j];
    }
    for (int j = threadIdx.x; j < O; j += MT) b3[j] = M.w[M.ob3 + j];
    // standardised features; rows past the end of the set are zero
    for (int idx = threadIdx.x; idx < TS * I; idx += MT) {
        const int s = idx / I, i = idx % I;
        float v = 0.0f;
        if (s < ns) {
            const double m = mu[(size_t)(s0 + s) * ld_mu + i];
            const double f = i < M.P ? log(m) : m;
            v = (float)((f - M.scale[i]) / M.scale[I + i]);
        }
        X[idx] = v;
    }
    __syncthreads();
    dense_fwd(X, I, I, Wt1, L.ld1, b1, H, Z1, A1, H);
    __syncthreads();
    dense_fwd(A1, H, H, Wt2, L.ld2, b2, H, Z2, A2, H);
    __syncthreads();
    dense_fwd(A2, H, H, Wt3, L.ld3, b3, O, Y, nullptr, O);
    __syncthreads();
    const double* om = M.scale + 2 * I;
    const double* os = om + O;
    if constexpr (!TRAIN) {
        for (int idx = threadIdx.x; idx < ns * O; idx += MT) {
            const int s = idx / O, j = idx % O;
            out[(size_t)(s0 + s) * O + j] = om[j] + os[j] * (double)Y[idx];
        }
        return;
    } else {
        // loss and output gradient dL/dy = 2 (y - t) / (S O); zero for padding rows
        const float gs = (float)(2.0 / ((double)S * (double)O));
        double lsum = 0.0;
        for (int idx = threadIdx.x; idx < TS * O; idx += MT) {
            const int s = idx / O, j = idx % O;
            float d = 0.0f;
            if (s < ns) {
                const float t = (float)((tgt[(size_t)(s0 + s) * O + j] - om[j]) / os[j]);
                const float e = Y[idx] - t;
                lsum += (double)e * (double)e;
                d = gs * e;
            }
            Y[idx] = d;
        }
        lsum = block_sum_d(lsum, red);
        if (threadIdx.x == 0) loss_part[blockIdx.x] = lsum;
        __syncthreads();
        float* G = part + (size_t)blockIdx.x * M.np;
        dense_wgrad(Y, O, O, A2, H, H, G + M.ow3, G + M.ob3);       // layer 3
        __syncthreads();
        dense_bwd(Y, O, O, Wt3, L.ld3, H, Z2, A2, H);                 // A2 <- dL/dz2
        __syncthreads();
        dense_wgrad(A2, H, H, A1, H, H, G + M.ow2, G + M.ob2);      // layer 2
        __syncthreads();
        dense_bwd(A2, H, H, Wt2, L.ld2, H, Z1, A1, H);                // A1 <- dL/dz1
        __syncthreads();
        dense_wgrad(A1, H, H, X, I, I, G + M.ow1, G + M.ob1);       // layer 1
    }
}

// g = sum over tiles of the partials (fixed order, FP64).  update = 1: Adam on
// the FP32 master and its BF16 copy, loss of this step into lossh; update = 0:
// the gradient into grad and the loss into *loss.
__global__ void __launch_bounds__(MT) k_mlp_adam(long long np, int tiles, const float* __restrict__ part,
                                                  const double* __restrict__ loss_part, double inv_so,
                                                  float* w, __nv_bfloat16* wb, float* m, float* v,
                                                  const int* __restrict__ step, int t0, double* lossh, int update,
                                                  double* grad, double* loss, float lr, float b1, float b2,
                                                  float eps) {
    const long long p = (long long)blockIdx.x * MT + threadIdx.x;
    const int t = *step;
    if (p < np) {
        double g = 0.0;
        for (int k = 0; k < tiles; ++k) g += part[(size_t)k * np + p];
        if (update) {
            const float gf = (float)g;
            const float mm = b1 * m[p] + (1.0f - b1) * gf;
            const float vv = b2 * v[p] + (1.0f - b2) * gf * gf;
            m[p] = mm;
            v[p] = vv;
            const float c1 = (float)(1.0 - pow((double)b1, (double)t));
            const float c2 = (float)(1.0 - pow((double)b2, (double)t));
            const float nw = w[p] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
            w[p] = nw;
            wb[p] = __float2bfloat16_rn(nw);
        } else {
            grad[p] = g;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double L = 0.0;
        for (int k = 0; k < tiles; ++k) L += loss_part[k];
        L *= inv_so;
        if (update) {
            const int i = t - 1 - t0;
            if (i >= 0 && i < LOSS_CAP) lossh[i] = L;
        } else {
            *loss = L;
        }
    }
}

__global__ void k_mlp_round(long long np, const float* w, __nv_bfloat16* wb) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x)
        wb[p] = __float2bfloat16_rn(w[p]);
}

bool is_dev(const void* p) { return rbk::pointer_kind(p) == rbk::PTR_DEVICE; }

}  // namespace

struct rb_mlp {
    int I = 0, P = 0, H = 0, O = 0, Smax = 0, tiles_max = 0;
    long long np = 0;
    float* d_w = nullptr;
    __nv_bfloat16* d_wb = nullptr;
    float *d_m = nullptr, *d_v = nullptr;
    double* d_scale = nullptr;
    float* d_part = nullptr;
    double* d_loss_part = nullptr;
    double* d_lossh = nullptr;
    double* d_grad = nullptr;
    double* d_loss = nullptr;
    int* d_step = nullptr;
    double* d_mu = nullptr;
    double* d_tgt = nullptr;
    double* d_out = nullptr;
    int t = 0;               // Adam steps taken
    bool scaled = false;     // standardisation computed
    cudaStream_t own = nullptr;
    std::vector<void*> allocs;
    size_t smem = 0;
};

namespace {

Net net_view(const rb_mlp* n) {
    Net M;
    M.I = n->I; M.P = n->P; M.H = n->H; M.O = n->O; M.np = n->np;
    M.ow1 = 0;
    M.ob1 = M.ow1 + (long long)n->H * n->I;
    M.ow2 = M.ob1 + n->H;
    M.ob2 = M.ow2 + (long long)n->H * n->H;
    M.ow3 = M.ob2 + n->H;
    M.ob3 = M.ow3 + (long long)n->O * n->H;
    M.w = n->d_w; M.wb = n->d_wb; M.scale = n->d_scale;
    return M;
}

rb_status fail(rb_status s, const std::string& m) {
    rbk::set_global_error(m);
    return s;
}

#define MCK(call)                                                                                \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return fail(RB_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
rb_status malloc_into(rb_mlp* n, T** p, size_t count) {
    *p = nullptr;
    if (cudaMalloc((void**)p, std::max<size_t>(1, count) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(RB_ENOMEM, "device allocation of the network failed");
    }
    n->allocs.push_back((void*)*p);
    return RB_OK;
}

void destroy(rb_mlp* n) {
    if (!n) return;
    if (n->own) cudaStreamSynchronize(n->own);
    for (void* p : n->allocs) cudaFree(p);
    if (n->own) cudaStreamDestroy(n->own);
    delete n;
}

rb_status check_mu(const rb_mlp* n, int B, const double* mu) {
    for (long long i = 0; i < (long long)B * n->I; ++i) {
        const double v = mu[i];
        if (!std::isfinite(v) || ((i % n->I) < n->P && !(v > 0.0)))
            return fail(RB_EINVAL, "parameter vectors must be finite, with positive diffusion coefficients");
    }
    return RB_OK;
}

// Stage S training pairs on the device; the first call also fixes the standardisation.
rb_status stage_pairs(rb_mlp* n, int S, const double* mu, const double* Y, cudaStream_t s) {
    if (S < 1 || S > n->Smax || !mu || !Y) return fail(RB_EINVAL, "need 1 <= S <= max_samples and non-NULL mu, Y");
    if (rbk::pointer_kind(mu) != rbk::PTR_HOST) return fail(RB_EINVAL, "mu must be host memory");
    if (check_mu(n, S, mu) != RB_OK) return RB_EINVAL;
    MCK(cudaMemcpyAsync(n->d_mu, mu, (size_t)S * n->I * sizeof(double), cudaMemcpyHostToDevice, s));
    MCK(cudaMemcpyAsync(n->d_tgt, Y, (size_t)S * n->O * sizeof(double), cudaMemcpyDefault, s));
    if (!n->scaled) {
        k_mlp_moments<<<n->I + n->O, MT, 0, s>>>(S, n->I, n->P, n->O, n->d_mu, n->I, n->d_tgt, n->d_scale);
        MCK(cudaGetLastError());
        n->scaled = true;
    }
    return RB_OK;
}

void enqueue_train_step(rb_mlp* n, const Net& M, int S, int t0, cudaStream_t s, float lr) {
    const int tiles = (S + TS - 1) / TS;
    k_mlp_tile<true><<<tiles, MT, n->smem, s>>>(M, S, n->d_mu, n->I, n->d_tgt, nullptr, n->d_part, n->d_loss_part,
                                               n->d_step, 1);
    const unsigned blocks = (unsigned)((n->np + MT - 1) / MT);
    k_mlp_adam<<<blocks, MT, 0, s>>>(n->np, tiles, n->d_part, n->d_loss_part, 1.0 / ((double)S * n->O), n->d_w,
                                    n->d_wb, n->d_m, n->d_v, n->d_step, t0, n->d_lossh, 1, nullptr, nullptr, lr,
                                    0.9f, 0.999f, 1e-8f);
}

}  // namespace

namespace rbk {

int mlp_n_in(const rb_mlp* n) { return n ? n->I : -1; }
int mlp_n_out(const rb_mlp* n) { return n ? n->O : -1; }
bool mlp_ready(const rb_mlp* n) { return n && n->scaled; }

// out [B][O] = c(mu_b) for device mu [B][ld_mu] (the first I entries are used)
rb_status mlp_predict_device(rb_mlp* n, int B, const double* d_mu, int ld_mu, double* d_out, cudaStream_t s) {
    if (B <= 0) return RB_OK;
    const Net M = net_view(n);
    k_mlp_tile<false><<<(B + TS - 1) / TS, MT, n->smem, s>>>(M, B, d_mu, ld_mu, nullptr, d_out, nullptr, nullptr,
                                                            nullptr, 0);
    MCK(cudaGetLastError());
    return RB_OK;
}

}  // namespace rbk

extern "C" {

rb_status rb_mlp_create(rb_mlp** out, int n_in, int n_log, int hidden, int n_out, const double* params,
                        int max_samples) {
    if (!out) return fail(RB_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_in < 1 || n_in > MAX_IN || n_log < 0 || n_log > n_in || hidden < 1 || hidden > MAX_H || n_out < 1 ||
        n_out > MAX_OUT || !params || max_samples < 1)
        return fail(RB_EINVAL, "network sizes out of range (n_in <= 32, hidden <= 128, n_out <= 128) or NULL params");
    const long long np = (long long)hidden * n_in + hidden + (long long)hidden * hidden + hidden +
                         (long long)n_out * hidden + n_out;
    for (long long p = 0; p < np; ++p)
        if (!std::isfinite(params[p])) return fail(RB_EINVAL, "initial parameters must be finite");
    rb_mlp* n = new rb_mlp();
    n->I = n_in; n->P = n_log; n->H = hidden; n->O = n_out; n->Smax = max_samples;
    n->np = np;
    n->tiles_max = (max_samples + TS - 1) / TS;
    n->smem = layout(n_in, hidden, n_out).total;
    rb_status st = RB_OK;
    auto run = [&]() -> rb_status {
        if (cudaStreamCreateWithFlags(&n->own, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            n->own = nullptr;
            return fail(RB_ECUDA, "stream creation failed");
        }
        if (malloc_into(n, &n->d_w, n->np) || malloc_into(n, &n->d_wb, n->np) || malloc_into(n, &n->d_m, n->np) ||
            malloc_into(n, &n->d_v, n->np) || malloc_into(n, &n->d_scale, 2 * n_in + 2 * n_out) ||
            malloc_into(n, &n->d_part, (size_t)n->tiles_max * n->np) ||
            malloc_into(n, &n->d_loss_part, n->tiles_max) || malloc_into(n, &n->d_lossh, LOSS_CAP) ||
            malloc_into(n, &n->d_grad, n->np) || malloc_into(n, &n->d_loss, 1) || malloc_into(n, &n->d_step, 1) ||
            malloc_into(n, &n->d_mu, (size_t)max_samples * n_in) ||
            malloc_into(n, &n->d_tgt, (size_t)max_samples * n_out) ||
            malloc_into(n, &n->d_out, (size_t)max_samples * n_out))
            return RB_ENOMEM;
        std::vector<float> w32(n->np);
        for (long long p = 0; p < n->np; ++p) w32[p] = (float)params[p];
        MCK(cudaMemcpy(n->d_w, w32.data(), n->np * sizeof(float), cudaMemcpyHostToDevice));
        MCK(cudaMemset(n->d_m, 0, n->np * sizeof(float)));
        MCK(cudaMemset(n->d_v, 0, n->np * sizeof(float)));
        MCK(cudaMemset(n->d_step, 0, sizeof(int)));
        k_mlp_round<<<256, 256, 0, n->own>>>(n->np, n->d_w, n->d_wb);
        MCK(cudaGetLastError());
        // the largest layout any network can have, so that networks of different sizes coexist
        const int smax = (int)layout(MAX_IN, MAX_H, MAX_OUT).total;
        MCK(cudaFuncSetAttribute(k_mlp_tile<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
        MCK(cudaFuncSetAttribute(k_mlp_tile<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
        MCK(cudaStreamSynchronize(n->own));
        return RB_OK;
    };
    st = run();
    if (st != RB_OK) {
        destroy(n);
        return st;
    }
    *out = n;
    return RB_OK;
}

rb_status rb_mlp_fit(rb_mlp* n, int S, const double* mu, const double* Y, int steps, double lr, double* loss,
                     void* stream) {
    if (!n) return fail(RB_EINVAL, "network is NULL");
    if (steps < 0 || steps > LOSS_CAP || !(lr > 0.0)) return fail(RB_EINVAL, "need 0 <= steps <= 65536 and lr > 0");
    cudaStream_t s = stream ? (cudaStream_t)stream : n->own;
    rb_status st = stage_pairs(n, S, mu, Y, s);
    if (st != RB_OK) return st;
    const Net M = net_view(n);
    const int t0 = n->t;
    int done = 0;
    if (steps >= GRAPH_STEPS) {
        // the step body is replayed as a CUDA graph (the Adam count lives on the device)
        cudaGraph_t g;
        cudaGraphExec_t exec = nullptr;
        MCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k < GRAPH_STEPS; ++k) enqueue_train_step(n, M, S, t0, s, (float)lr);
        MCK(cudaStreamEndCapture(s, &g));
        const cudaError_t ie = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) return fail(RB_ECUDA, std::string("graph instantiation: ") + cudaGetErrorString(ie));
        for (; done + GRAPH_STEPS <= steps; done += GRAPH_STEPS) {
            const cudaError_t e = cudaGraphLaunch(exec, s);
            if (e != cudaSuccess) {
                cudaGraphExecDestroy(exec);
                return fail(RB_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
            }
        }
        cudaGraphExecDestroy(exec);
    }
    for (; done < steps; ++done) enqueue_train_step(n, M, S, t0, s, (float)lr);
    MCK(cudaGetLastError());
    n->t += steps;
    if (loss && steps > 0) MCK(cudaMemcpyAsync(loss, n->d_lossh, (size_t)steps * sizeof(double), cudaMemcpyDefault, s));
    MCK(cudaStreamSynchronize(s));
    return RB_OK;
}

rb_status rb_mlp_gradient(rb_mlp* n, int S, const double* mu, const double* Y, double* loss, double* grad,
                          void* stream) {
    if (!n) return fail(RB_EINVAL, "network is NULL");
    cudaStream_t s = stream ? (cudaStream_t)stream : n->own;
    rb_status st = stage_pairs(n, S, mu, Y, s);
    if (st != RB_OK) return st;
    const Net M = net_view(n);
    const int tiles = (S + TS - 1) / TS;
    k_mlp_tile<true><<<tiles, MT, n->smem, s>>>(M, S, n->d_mu, n->I, n->d_tgt, nullptr, n->d_part, n->d_loss_part,
                                               n->d_step, 0);
    k_mlp_adam<<<(unsigned)((n->np + MT - 1) / MT), MT, 0, s>>>(n->np, tiles, n->d_part, n->d_loss_part,
                                                               1.0 / ((double)S * n->O), n->d_w, n->d_wb, n->d_m,
                                                               n->d_v, n->d_step, n->t, n->d_lossh, 0, n->d_grad,
                                                               n->d_loss, 0.f, 0.9f, 0.999f, 1e-8f);
    MCK(cudaGetLastError());
    if (loss) MCK(cudaMemcpyAsync(loss, n->d_loss, sizeof(double), cudaMemcpyDefault, s));
    if (grad) MCK(cudaMemcpyAsync(grad, n->d_grad, n->np * sizeof(double), cudaMemcpyDefault, s));
    MCK(cudaStreamSynchronize(s));
    return RB_OK;
}

rb_status rb_mlp_predict(rb_mlp* n, int B, const double* mu, double* Y, void* stream) {
    if (!n) return fail(RB_EINVAL, "network is NULL");
    if (B < 0 || (B > 0 && (!mu || !Y))) return fail(RB_EINVAL, "B < 0 or NULL mu / Y");
    if (!n->scaled) return fail(RB_EINVAL, "the network has no standardisation yet: fit it first");
    if (rbk::pointer_kind(mu) != rbk::PTR_HOST) return fail(RB_EINVAL, "mu must be host memory");
    if (check_mu(n, B, mu) != RB_OK) return RB_EINVAL;
    if (rbk::pointer_kind(Y) == rbk::PTR_OTHER_DEVICE) return fail(RB_EINVAL, "Y lives on another device");
    cudaStream_t s = stream ? (cudaStream_t)stream : n->own;
    const bool dev_y = is_dev(Y);
    for (int b0 = 0; b0 < B; b0 += n->Smax) {
        const int nb = std::min(n->Smax, B - b0);
        MCK(cudaMemcpyAsync(n->d_mu, mu + (size_t)b0 * n->I, (size_t)nb * n->I * sizeof(double),
                            cudaMemcpyHostToDevice, s));
        double* dst = dev_y ? Y + (size_t)b0 * n->O : n->d_out;
        rb_status st = rbk::mlp_predict_device(n, nb, n->d_mu, n->I, dst, s);
        if (st != RB_OK) return st;
        if (!dev_y)
            MCK(cudaMemcpyAsync(Y + (size_t)b0 * n->O, n->d_out, (size_t)nb * n->O * sizeof(double),
                                cudaMemcpyDeviceToHost, s));
        MCK(cudaStreamSynchronize(s));
    }
    return RB_OK;
}

rb_status rb_mlp_get(const rb_mlp* n, double* params, double* scaling, int* adam_steps) {
    if (!n) return fail(RB_EINVAL, "network is NULL");
    if (cudaStreamSynchronize(n->own) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return fail(RB_ECUDA, "device synchronisation failed");
    }
    if (params) {
        std::vector<float> w(n->np);
        MCK(cudaMemcpy(w.data(), n->d_w, n->np * sizeof(float), cudaMemcpyDeviceToHost));
        for (long long p = 0; p < n->np; ++p) params[p] = w[p];
    }
    if (scaling) {
        if (!n->scaled) {
            for (int i = 0; i < 2 * n->I + 2 * n->O; ++i) scaling[i] = 0.0;
        } else {
            MCK(cudaMemcpy(scaling, n->d_scale, (2 * n->I + 2 * n->O) * sizeof(double), cudaMemcpyDeviceToHost));
        }
    }
    if (adam_steps) *adam_steps = n->t;
    return RB_OK;
}

int rb_mlp_num_params(const rb_mlp* n) { return n ? (int)n->np : -1; }

void rb_mlp_free(rb_mlp* n) { destroy(n); }

}  // extern "C"
