// Building blocks of the staged row-march kernels on 2D grids (the smoother and
// the CG body): rows move from global to shared memory by bulk asynchronous
// copies (cp.async.bulk) that complete on mbarriers, issued by one producer
// lane; every wait on a copy is bounded in time.
//
// Common plan of a staged kernel.  A work item is one band of rows of one query
// (TB_ROWS rows, fewer when the work list is short: band_rows).  The CTA has
// mx/4 consumer threads (thread t owns the points x0 = 4t .. 4t+3 of every row)
// and one producer warp, and walks its items (grid-stride order) as one
// continuous march: the item's steps k each consume one stage (the rows that
// step needs), stages are numbered across items, and stage u lands in ring
// slot u mod RING.  Every thread passes one CTA barrier per step.  A stage is
// read in its own step and at most LAG-1 following ones, so after the barrier
// of global step g the producer refills the slot of stage g-LAG with the next
// stage of its cursor, which runs ahead into the next item: the copies of a
// new band are in flight before the previous band ends.  Staged rows are
// padded with 16 bytes of zeros on both sides (x = -1 and x = mx read the
// Dirichlet zero); rows outside the grid are copied from a zero row.
#pragma once

#include "rb_common.cuh"

namespace rbk {
namespace stg {

#ifndef RB_STAGE_RING
#define RB_STAGE_RING 8
#endif
#ifndef RB_STAGE_ROWS
#define RB_STAGE_ROWS 128
#endif
constexpr int RING = RB_STAGE_RING;      // stages in flight
constexpr int TB_ROWS = RB_STAGE_ROWS;   // rows per band (even)
static_assert(TB_ROWS % 2 == 0, "bands start on even rows");
static_assert(RING >= 3, "a slot is refilled two steps after its stage");
constexpr unsigned long long WAIT_NS = 2000000000ull;   // bounded mbarrier wait
constexpr unsigned long long DRAIN_NS = 500000000ull;   // bounded drain after an expired wait
constexpr int MAX_MX = 1024;

// source of the rows outside the grid (zero-initialised, never written; one per translation unit)
static __device__ __align__(128) double g_zero_row[MAX_MX];

__device__ __forceinline__ uint32_t s2u(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ uint64_t gtime() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mb_init(uint64_t* b, uint32_t count = 1) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s2u(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s2u(b)) : "memory");
}
__device__ __forceinline__ void mb_arrive_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s2u(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mb_test(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(s2u(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait (limit_ns of globaltimer); false (and the error flag raised) on expiry
static __device__ __noinline__ bool mb_wait_slow(uint64_t* b, uint32_t parity, int* err, unsigned long long limit_ns) {
    const uint64_t t0 = gtime();
    while (!mb_test(b, parity)) {
        if (gtime() - t0 > limit_ns) {
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ bool mb_wait(uint64_t* b, uint32_t parity, int* err, unsigned long long limit_ns = WAIT_NS) {
    return mb_test(b, parity) || mb_wait_slow(b, parity, err, limit_ns);
}
__device__ __forceinline__ void bulk_row(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(s2u(dst)),
        "l"(src), "r"(bytes), "r"(s2u(bar))
        : "memory");
}
// After an expired wait: let the copies of the last RING stages land (bounded in time:
// the drain limit, or the wait limit when that is shorter).
__device__ __forceinline__ void drain(uint64_t* bar, unsigned seq, unsigned long long limit_ns = DRAIN_NS) {
    const uint64_t t0 = gtime();
    const unsigned long long lim = limit_ns < DRAIN_NS ? limit_ns : DRAIN_NS;
    for (unsigned u = seq > (unsigned)RING ? seq - RING : 0u; u < seq; ++u)
        while (!mb_test(bar + u % RING, (u / RING) & 1u) && gtime() - t0 < lim) {
        }
}

// The same for a ring of `ring` stages (kernels whose ring is not RING).
__device__ __forceinline__ void drain_ring(uint64_t* bar, unsigned seq, unsigned ring,
                                           unsigned long long limit_ns = DRAIN_NS) {
    const uint64_t t0 = gtime();
    const unsigned long long lim = limit_ns < DRAIN_NS ? limit_ns : DRAIN_NS;
    for (unsigned u = seq > ring ? seq - ring : 0u; u < seq; ++u)
        while (!mb_test(bar + u % ring, (u / ring) & 1u) && gtime() - t0 < lim) {
        }
}

template <typename T> struct V4t { T v[4]; };
__device__ __forceinline__ V4t<float> lds4(const float* p) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    return V4t<float>{{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ V4t<double> lds4(const double* p) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    return V4t<double>{{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void stg4(float* p, const V4t<float>& a) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(a.v[0], a.v[1], a.v[2], a.v[3]));
}
__device__ __forceinline__ void stg4(double* p, const V4t<double>& a) {
    __stcs(reinterpret_cast<double2*>(p), make_double2(a.v[0], a.v[1]));
    __stcs(reinterpret_cast<double2*>(p) + 1, make_double2(a.v[2], a.v[3]));
}
template <typename T> __device__ __forceinline__ V4t<T> zero4() { return V4t<T>{{T(0), T(0), T(0), T(0)}}; }

// Face coefficients kappa_f / h^2 of the thread's 4 points in one row (eq. 1 on the
// grid: face value = mean of the two cells' mu), the diagonal and its inverse.
template <typename T>
struct TCoef {
    T kx[5];   // x faces: kx[j] between points j-1 and j (kx[0], kx[4] reach the neighbour threads)
    T kym[4], kyp[4], diag[4], idiag[4];
};

template <typename T>
__device__ __forceinline__ void tcoef(const Geo& g, const T* mus, int x0, int k, TCoef<T>& c) {
    const int nbx = g.nbx, mx = g.mx;
    const bool left = x0 > 0, right = x0 + 4 < mx;
    const int byc = nbx * __ldg(g.by + k);
    const bool up = k > 0, dn = k < g.my - 1;
    const int bym = up ? nbx * __ldg(g.by + k - 1) : byc;
    const int byp = dn ? nbx * __ldg(g.by + k + 1) : byc;
    int bxs[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) bxs[j] = __ldg(g.bx + min(max(x0 - 1 + j, 0), mx - 1));
    T m[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) m[j] = mus[bxs[j] + byc];
    const T hx = (T)g.ihx2, hy = (T)g.ihy2, half = T(0.5);
    c.kx[0] = hx * (left ? half * (m[0] + m[1]) : m[1]);
#pragma unroll
    for (int j = 1; j < 4; ++j) c.kx[j] = hx * half * (m[j] + m[j + 1]);
    c.kx[4] = hx * (right ? half * (m[4] + m[5]) : m[4]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const T mc = m[j + 1];
        c.kym[j] = hy * (up ? half * (mc + mus[bxs[j + 1] + bym]) : mc);
        c.kyp[j] = hy * (dn ? half * (mc + mus[bxs[j + 1] + byp]) : mc);
        c.diag[j] = c.kx[j] + c.kx[j + 1] + c.kym[j] + c.kyp[j];
        c.idiag[j] = T(1) / c.diag[j];
    }
}

// The block rows that a row's coefficients depend on (the row and its two
// neighbours): rows with equal keys share their coefficients.
__device__ __forceinline__ int tkey(const Geo& g, int k) {
    const int c = __ldg(g.by + k);
    const int m = k > 0 ? __ldg(g.by + k - 1) : 0xFF;
    const int p = k < g.my - 1 ? __ldg(g.by + k + 1) : 0xFF;
    return c | (m << 8) | (p << 16);
}

// (A v) at the thread's 4 points of a row from rows k-1, k, k+1 and the two x neighbours
template <typename T>
__device__ __forceinline__ T apply_pt(const TCoef<T>& c, int j, const T* vm, const T* vc, const T* vp, T left,
                                      T right) {
    const T xl = j == 0 ? left : vc[j - 1];
    const T xr = j == 3 ? right : vc[j + 1];
    return c.diag[j] * vc[j] - (c.kx[j] * xl + c.kx[j + 1] * xr + c.kym[j] * vm[j] + c.kyp[j] * vp[j]);
}

// Shared-memory layout: RING stages of `arrays` padded rows, then `extra`
// elements (kernel-specific), then RING mbarriers.
template <typename T>
struct Layout {
    int pad, stride, arrays, nthr;
    size_t stage_elems, ring_elems, extra, bytes;
    __host__ __device__ Layout(int mx, int narrays, size_t extra_elems) {
        pad = 16 / (int)sizeof(T);
        stride = mx + 2 * pad;
        arrays = narrays;
        nthr = mx / 4;
        stage_elems = (size_t)arrays * stride;
        ring_elems = (size_t)RING * stage_elems;
        extra = (extra_elems + 1) & ~(size_t)1;
        bytes = (ring_elems + extra) * sizeof(T) + RING * sizeof(uint64_t);
    }
    __device__ uint64_t* bars(unsigned char* smem) const {
        return reinterpret_cast<uint64_t*>(smem + (ring_elems + extra) * sizeof(T));
    }
};

// zero the pads of every staged row and `extra` elements after the ring; init the barriers
// (ends with a CTA barrier)
template <typename T>
__device__ __forceinline__ void setup(const Layout<T>& lay, T* ring, uint64_t* bar, int mx) {
    for (int i = threadIdx.x; i < RING * lay.arrays; i += blockDim.x) {
        T* row = ring + (size_t)i * lay.stride;
        for (int j = 0; j < lay.pad; ++j) {
            row[j] = T(0);
            row[lay.pad + mx + j] = T(0);
        }
    }
    T* extra = ring + lay.ring_elems;
    for (int i = threadIdx.x; i < (int)lay.extra; i += blockDim.x) extra[i] = T(0);
    if (threadIdx.x == 0) {
        for (int i = 0; i < RING; ++i) mb_init(bar + i);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();   // barriers initialised and pads zeroed before the first copy is issued
}

// Rows per band: TB_ROWS, halved (down to 16) while the work items (queries x
// bands) would leave part of the grid idle, and never more bands than a query
// has partial-sum slots.  Uniform across the grid; always even.
__device__ __forceinline__ int band_rows(int my, int cnt, int max_tiles) {
    int rows = TB_ROWS;
    while (rows > 16 && (long long)cnt * ((my + rows - 1) / rows) < (long long)gridDim.x) rows >>= 1;
    while ((my + rows - 1) / rows > max_tiles) rows <<= 1;
    return rows;
}

// ---- warp-specialised kernels: the consumer threads are the first nthr threads
// (a multiple of 32) and synchronise among themselves on named barrier 1; the
// producer warp never takes part after set-up.

__device__ __forceinline__ void cbar(int nthr) { asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory"); }

// consumer sum of two per-thread partials (FP64 across warps); result in thread 0
template <typename T>
__device__ __forceinline__ void csum2(T a, T b, double* red, double out[2], int nthr) {
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    cbar(nthr);   // red[] free
    if (lane == 0) {
        red[wi] = (double)a;
        red[16 + wi] = (double)b;
    }
    cbar(nthr);
    out[0] = out[1] = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < nthr / 32; ++i) {
            out[0] += red[i];
            out[1] += red[16 + i];
        }
}

// Thread 0 publishes the consumer partials of (q, tile); true in every consumer
// thread of the CTA that arrives last for q (then all partials of q are visible).
__device__ __forceinline__ bool carrive(const Params& P, int q, int tile, int ntiles, const double* vals, int nv,
                                        int nthr, int* s_flag) {
    if (threadIdx.x == 0) {
        double* dst = P.part + ((size_t)q * P.max_tiles + tile) * 4;
        for (int j = 0; j < nv; ++j) dst[j] = vals[j];
        __threadfence();
        const unsigned prev = atomicAdd(P.tick + q, 1u);
        *s_flag = (prev == (unsigned)ntiles - 1u);
    }
    cbar(nthr);
    const bool last = *s_flag != 0;
    if (last) __threadfence();
    return last;
}

// fixed-order consumer sum of the nv partials of q over its tiles; result in thread 0
__device__ __forceinline__ void cgather(const Params& P, int q, int ntiles, int nv, double* out, double* red,
                                        int nthr) {
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    for (int j = 0; j < nv; ++j) {
        double s = 0.0;
        for (int t = threadIdx.x; t < ntiles; t += nthr) s += __ldcg(P.part + ((size_t)q * P.max_tiles + t) * 4 + j);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        cbar(nthr);
        if (lane == 0) red[wi] = s;
        cbar(nthr);
        if (threadIdx.x == 0) {
            double tot = 0.0;
            for (int i = 0; i < nthr / 32; ++i) tot += red[i];
            out[j] = tot;
        }
    }
}

// CTA sum of per-thread partials (FP64 across warps); result in thread 0
template <typename T>
__device__ __forceinline__ void cta_sum2(T a, T b, double* red, double out[2]) {
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        red[wi] = (double)a;
        red[16 + wi] = (double)b;
    }
    __syncthreads();
    out[0] = out[1] = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            out[0] += red[i];
            out[1] += red[16 + i];
        }
}

// resident grid of a staged kernel: SM count x CTAs per SM at (threads, smem)
template <typename K>
inline int resident(K kernel, int threads, size_t smem) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0, sms = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    return sms * (per_sm > 0 ? per_sm : 1);
}

struct Par0 { static constexpr int value = 0; };
struct Par1 { static constexpr int value = 1; };

}  // namespace stg
}  // namespace rbk
