// rb_probe.cu - measured FMA rate of the device.
//
// The FP64 outer residual of the mixed solver (f - A x in FP64, Alg. 3 with
// residual refinement) does about 21 FP64 operations per point on 12 bytes per
// point: on GB300, whose FP64 rate is a small fraction of its FP32 rate, that
// kernel is bound by the FP64 pipe, not by HBM.  Its roofline needs the rate
// this device actually reaches, which this probe measures: every thread runs
// eight independent chains of dependent FMAs x <- a x + b (no loads or stores
// in the loop), the grid fills every SM several times over, and the rate is
// 2 flops per FMA over the CUDA-event time of the launch.
#include <cuda_runtime.h>

#include "../../include/rb.h"

namespace {

constexpr int CHAINS = 8;
constexpr int UNROLL = 16;
constexpr int THREADS = 256;
constexpr int MAX_ITERS = 1 << 16;   // bounds a launch to seconds even at 1 TFLOP/s FP64

template <typename T>
__global__ void __launch_bounds__(THREADS, 8) k_fma_rate(T* out, int iters, T a, T b) {
    T x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
#pragma unroll
            for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
        }
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    out[(size_t)blockIdx.x * THREADS + threadIdx.x] = s;   // keeps every chain live
}

template <typename T>
rb_status run(int blocks, double* flops_per_s, cudaStream_t stream) {
    T* out = nullptr;
    if (cudaMalloc(&out, (size_t)blocks * THREADS * sizeof(T)) != cudaSuccess) return RB_ENOMEM;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    rb_status st = RB_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = RB_ECUDA;
    // |a| < 1: the chains converge to b / (1 - a), no overflow or subnormals
    const T a = (T)0.999999, b = (T)1e-7;
    int iters = 64, timed_iters = 0;
    float ms = 0.f;
    for (int attempt = 0; st == RB_OK && attempt < 12; ++attempt) {
        k_fma_rate<T><<<blocks, THREADS, 0, stream>>>(out, iters, a, b);   // warm-up of this size
        cudaEventRecord(e0, stream);
        k_fma_rate<T><<<blocks, THREADS, 0, stream>>>(out, iters, a, b);
        cudaEventRecord(e1, stream);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            st = RB_ECUDA;
            break;
        }
        cudaEventElapsedTime(&ms, e0, e1);
        timed_iters = iters;
        if (ms >= 20.f || iters >= MAX_ITERS) break;
        iters *= ms > 0.5f ? (int)(25.f / ms) + 1 : 8;   // aim at 20-50 ms
        if (iters > MAX_ITERS) iters = MAX_ITERS;
    }
    if (st == RB_OK && ms <= 0.f) st = RB_ECUDA;
    if (st == RB_OK) {
        const double fmas = (double)blocks * THREADS * (double)timed_iters * UNROLL * CHAINS;
        *flops_per_s = 2.0 * fmas / (ms * 1e-3);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return st;
}

}  // namespace

extern "C" rb_status rb_fma_rate(int fp64, double* flops_per_s, void* stream) {
    if (!flops_per_s) return RB_EINVAL;
    *flops_per_s = 0.0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return RB_ECUDA;
    const int blocks = sms * 8;   // 8 CTAs of 256 threads per SM: 64 warps of 8 independent chains
    cudaStream_t s = (cudaStream_t)stream;
    return fp64 ? run<double>(blocks, flops_per_s, s) : run<float>(blocks, flops_per_s, s);
}
