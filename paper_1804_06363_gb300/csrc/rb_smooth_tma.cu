// One red-black Gauss-Seidel sweep (eq. 8) on 2D grids, with the rows staged in
// shared memory by bulk asynchronous copies (cp.async.bulk, completion on
// mbarriers).
//
// A work item is one band of TB_ROWS rows of one query.  A CTA has mx/4
// consumer threads (thread t owns the points x0 = 4t .. 4t+3 of every row) and
// one producer warp.  The item marches over steps k = y0-3 .. y1; stage k brings
// source row k+1, residual row k and, on the last sweep under Polak-Ribiere,
// direction row k into ring slot (stage number mod RING).  At step k a consumer
//   - shifts its register window of old black source values and adds row k+1
//     (only the values that the red updates of rows k .. k+2 read),
//   - updates the red points of row k (red: x + y even) from old black values,
//   - after the CTA barrier, updates the black points of row k-1 from the new
//     red values of rows k-2 .. k (registers) and writes row k-1.
// Neighbours owned by the adjacent threads come from the staged source row
// (zero-padded at both ends, so x = -1 and x = mx read the Dirichlet zero) or
// from a small shared array of new red values.  The march is unrolled by two so
// that the colour pattern of a row is a compile-time constant.
//
// The producer refills the slot of stage k-2 (every read of it ended before the
// barrier of step k) with stage k-2+RING after that barrier.  Rows outside the
// grid are copied from a zero row in global memory.  Every mbarrier wait is
// bounded in time: on expiry the device error flag is raised, the thread stops
// waiting and marches on whatever the slots hold (the CTA barriers stay
// matched), then the copies in flight are drained (bounded) and the CTA returns.
#include "rb_common.cuh"

namespace rbk {

#ifndef RB_TMA_RING
#define RB_TMA_RING 8
#endif
#ifndef RB_TMA_ROWS
#define RB_TMA_ROWS 128
#endif
constexpr int RING = RB_TMA_RING;     // stages in flight
constexpr int TB_ROWS = RB_TMA_ROWS;  // rows per band (even)
static_assert(TB_ROWS % 2 == 0, "bands start on even rows");
static_assert(RING >= 3, "a slot is refilled two steps after its stage");
constexpr unsigned long long TMA_WAIT_NS = 2000000000ull;
constexpr int TMA_MAX_MX = 1024;

// source of the rows outside the grid (zero-initialised, never written)
__device__ __align__(128) double g_tma_zero_row[TMA_MAX_MX];

namespace {

__device__ __forceinline__ uint32_t s2u(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ uint64_t gtime() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mb_init(uint64_t* b) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s2u(b)) : "memory");
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
// bounded wait; false (and the error flag raised) on expiry
__device__ __noinline__ bool mb_wait_slow(uint64_t* b, uint32_t parity, int* err) {
    const uint64_t t0 = gtime();
    while (!mb_test(b, parity)) {
        if (gtime() - t0 > TMA_WAIT_NS) {
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ bool mb_wait(uint64_t* b, uint32_t parity, int* err) {
    return mb_test(b, parity) || mb_wait_slow(b, parity, err);
}
__device__ __forceinline__ void bulk_row(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(s2u(dst)),
        "l"(src), "r"(bytes), "r"(s2u(bar))
        : "memory");
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

// face coefficients of the thread's 4 points in one row (same arithmetic as the other 2D kernels)
template <typename T, bool LAST>
struct TCoef {
    T kx[5], kym[4], kyp[4], idiag[4];
    T diag[LAST ? 4 : 1];
};

template <typename T, bool LAST>
__device__ __forceinline__ void tcoef(const Geo& g, const T* mus, int x0, int k, TCoef<T, LAST>& c) {
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
        const T d = c.kx[j] + c.kx[j + 1] + c.kym[j] + c.kyp[j];
        c.idiag[j] = T(1) / d;
        if constexpr (LAST) c.diag[j] = d;
    }
}

// the block rows that a row's coefficients depend on (the row and its two neighbours)
__device__ __forceinline__ int tkey(const Geo& g, int k) {
    const int c = __ldg(g.by + k);
    const int m = k > 0 ? __ldg(g.by + k - 1) : 0xFF;
    const int p = k < g.my - 1 ? __ldg(g.by + k + 1) : 0xFF;
    return c | (m << 8) | (p << 16);
}

struct Par0 { static constexpr int value = 0; };
struct Par1 { static constexpr int value = 1; };

}  // namespace

// Shared-memory layout: RING stages of (source, residual[, direction]) rows,
// each row padded by 16 bytes of zeros on both sides; 4 rows of new red edge
// values (thread t at index t+1, zeros at both ends); RING mbarriers.
template <typename T>
struct TmaLayout {
    int pad, stride, arrays, nthr, zstride;
    size_t stage_elems, ring_elems, zedge_elems, bytes;
    __host__ __device__ TmaLayout(int mx, bool last) {
        pad = 16 / (int)sizeof(T);
        stride = mx + 2 * pad;
        arrays = last ? 3 : 2;
        nthr = mx / 4;
        zstride = (nthr + 2 + 3) & ~3;
        stage_elems = (size_t)arrays * stride;
        ring_elems = (size_t)RING * stage_elems;
        zedge_elems = (size_t)4 * zstride;
        bytes = (ring_elems + zedge_elems) * sizeof(T) + RING * sizeof(uint64_t);
    }
};

template <typename T, bool LAST>
__global__ void __launch_bounds__(TMA_MAX_MX / 4 + 32) k2_smooth_tma(Params P, const T* __restrict__ src_base,
                                                                    T* dst_base) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ T mus[MAX_MU];
    __shared__ double red[32];
    const Geo& g = P.g;
    const int mx = g.mx, my = g.my;
    const TmaLayout<T> lay(mx, LAST);
    T* ring = reinterpret_cast<T*>(smem_raw);
    T* zedge = ring + lay.ring_elems;
    uint64_t* bar = reinterpret_cast<uint64_t*>(zedge + lay.zedge_elems);
    const int nthr = lay.nthr;
    const bool producer = (int)threadIdx.x >= nthr;
    const bool issuer = producer && (threadIdx.x & 31) == 0;
    const int t = producer ? 0 : (int)threadIdx.x;
    const int x0 = 4 * t;
    const uint32_t row_bytes = (uint32_t)(mx * sizeof(T));
    const T* zero_row = reinterpret_cast<const T*>(g_tma_zero_row);

    // zero the pads of every staged row and the edge rows, set up the barriers
    for (int i = threadIdx.x; i < RING * lay.arrays; i += blockDim.x) {
        T* row = ring + (size_t)i * lay.stride;
        for (int j = 0; j < lay.pad; ++j) {
            row[j] = T(0);
            row[lay.pad + mx + j] = T(0);
        }
    }
    for (int i = threadIdx.x; i < (int)lay.zedge_elems; i += blockDim.x) zedge[i] = T(0);
    if (threadIdx.x == 0) {
        for (int i = 0; i < RING; ++i) mb_init(bar + i);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }

    const int nband = (my + TB_ROWS - 1) / TB_ROWS;
    const int cnt = P.lcnt[L_PREC];
    const long long total = (long long)cnt * nband;
    unsigned seq = 0;   // stages requested so far by this CTA (all threads agree)
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        const int slot = (int)(w / nband), band = (int)(w % nband);
        const int q = P.lidx[L_PREC * P.Bmax + slot];
        const QState& s = P.st[q];
        const bool need_ap = LAST && P.beta_form == RB_BETA_PR && !s.start;
        const int y0 = band * TB_ROWS, y1 = min(my, y0 + TB_ROWS);
        const int kfirst = y0 - 3;   // first stage and step (odd)
        const size_t base = (size_t)q * g.n;
        const T* src = src_base + base;
        const T* rg = reinterpret_cast<const T*>(P.r) + base;
        const T* pg = reinterpret_cast<const T*>(P.p) + ((size_t)q * 2 + s.ppar) * g.n;
        T* dst = dst_base + base;
        const uint32_t stage_bytes = row_bytes * (need_ap ? 3u : 2u);
        __syncthreads();   // the previous item no longer reads the ring, the edges or mus
        for (int j = threadIdx.x; j < P.n_mu; j += blockDim.x) mus[j] = (T)P.mu[(size_t)q * P.n_mu + j];

        // stage kk of this item into its slot (producer lane 0)
        auto issue = [&](int kk) {
            const unsigned u = seq + (unsigned)(kk - kfirst);
            T* sg = ring + (size_t)(u % RING) * lay.stage_elems + lay.pad;
            uint64_t* b = bar + u % RING;
            mb_arrive_tx(b, stage_bytes);
            const int ms = kk + 1, mr = kk;
            bulk_row(sg, (ms >= 0 && ms < my) ? src + (size_t)ms * mx : zero_row, row_bytes, b);
            bulk_row(sg + lay.stride, (mr >= 0 && mr < my) ? rg + (size_t)mr * mx : zero_row, row_bytes, b);
            if (need_ap)
                bulk_row(sg + 2 * lay.stride, (mr >= 0 && mr < my) ? pg + (size_t)mr * mx : zero_row, row_bytes, b);
        };
        if (issuer)
            for (int kk = kfirst; kk <= y1 && kk < kfirst + RING; ++kk) issue(kk);
        __syncthreads();   // mus visible

        TCoef<T, LAST> cf[2];     // coefficients of the last even / odd row updated
        int key[2] = {-1, -1};
        T sbm[2] = {T(0), T(0)}, sbc[2] = {T(0), T(0)}, sbp[2] = {T(0), T(0)};   // old black source values
        T rr[2][4];               // residual rows of even / odd parity
        T zm[2] = {T(0), T(0)}, zc[2] = {T(0), T(0)}, zp[2] = {T(0), T(0)};      // new red rows k-2, k-1, k
        T pm[4], pc[4], pn[4];    // direction rows k-2, k-1, k
#pragma unroll
        for (int j = 0; j < 4; ++j) rr[0][j] = rr[1][j] = pm[j] = pc[j] = pn[j] = T(0);
        T ry = T(0), apy = T(0);
        bool ok = true;
        unsigned cslot = seq % RING, cpar = (seq / RING) & 1u;

        // one step of the march; PAR = k & 1
        auto step = [&](auto par_tag, int k) {
            constexpr int PAR = decltype(par_tag)::value;
            constexpr int R0 = PAR, R1 = PAR + 2;   // red columns of row k = black columns of row k-1
            if (!producer) {
                const T* stg = ring + (size_t)cslot * lay.stage_elems + lay.pad;
                const unsigned pslot = cslot == 0 ? RING - 1 : cslot - 1;
                const T* prev = ring + (size_t)pslot * lay.stage_elems + lay.pad;   // stage k-1
                if (ok && !mb_wait(bar + cslot, cpar, P.err)) ok = false;
                // source row k+1 at the red columns of row k (its black points)
                const V4t<T> sn = lds4(stg + x0);
                sbm[0] = sbc[0];
                sbm[1] = sbc[1];
                sbc[0] = sbp[0];
                sbc[1] = sbp[1];
                sbp[0] = sn.v[R0];
                sbp[1] = sn.v[R1];
                if (k >= y0 - 1) {
                    const V4t<T> rk = lds4(stg + lay.stride + x0);
#pragma unroll
                    for (int j = 0; j < 4; ++j) rr[PAR][j] = rk.v[j];
                    if (need_ap) {
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            pm[j] = pc[j];
                            pc[j] = pn[j];
                        }
                        const V4t<T> pv = lds4(stg + 2 * lay.stride + x0);
#pragma unroll
                        for (int j = 0; j < 4; ++j) pn[j] = pv.v[j];
                    }
                    // red half-sweep of row k
                    zm[0] = zc[0];
                    zm[1] = zc[1];
                    zc[0] = zp[0];
                    zc[1] = zp[1];
                    if (k >= 0 && k < my) {
                        const int kk = tkey(g, k);
                        if (kk != key[PAR]) {
                            tcoef<T, LAST>(g, mus, x0, k, cf[PAR]);
                            key[PAR] = kk;
                        }
                        const TCoef<T, LAST>& c = cf[PAR];
                        // source row k (previous stage): the horizontal neighbour across the thread edge
                        const T halo = PAR == 0 ? prev[x0 - 1] : prev[x0 + 4];
                        // PAR 0: red 0 (halo, sbc0), red 2 (sbc0, sbc1); PAR 1: red 1 (sbc0, sbc1), red 3 (sbc1, halo)
                        const T l0 = PAR == 0 ? halo : sbc[0], r0 = PAR == 0 ? sbc[0] : sbc[1];
                        const T l1 = PAR == 0 ? sbc[0] : sbc[1], r1 = PAR == 0 ? sbc[1] : halo;
                        const T n0 = rk.v[R0] + c.kx[R0] * l0 + c.kx[R0 + 1] * r0 + c.kym[R0] * sbm[0] +
                                     c.kyp[R0] * sbp[0];
                        const T n1 = rk.v[R1] + c.kx[R1] * l1 + c.kx[R1 + 1] * r1 + c.kym[R1] * sbm[1] +
                                     c.kyp[R1] * sbp[1];
                        zp[0] = n0 * c.idiag[R0];
                        zp[1] = n1 * c.idiag[R1];
                    } else {
                        zp[0] = T(0);
                        zp[1] = T(0);
                    }
                    // the value a neighbour thread needs for the black update of row k:
                    // PAR 0: red point 0 (read by thread t-1); PAR 1: red point 3 (read by thread t+1)
                    zedge[(k & 3) * lay.zstride + t + 1] = PAR == 0 ? zp[0] : zp[1];
                    __syncthreads();
                    // black half-sweep of row b = k-1 (black columns of b = red columns of k)
                    const int b = k - 1;
                    if (b >= y0 && b < y1) {
                        const TCoef<T, LAST>& c = cf[1 - PAR];
                        const T* rb = rr[1 - PAR];
                        const T* ze = zedge + (b & 3) * lay.zstride;
                        // PAR 0 (b odd): black 0 (t-1's red 3, zc0), black 2 (zc0, zc1)
                        // PAR 1 (b even): black 1 (zc0, zc1), black 3 (zc1, t+1's red 0)
                        const T zh = PAR == 0 ? ze[t] : ze[t + 2];
                        const T l0 = PAR == 0 ? zh : zc[0], r0 = PAR == 0 ? zc[0] : zc[1];
                        const T l1 = PAR == 0 ? zc[0] : zc[1], r1 = PAR == 0 ? zc[1] : zh;
                        const T n0 = rb[R0] + c.kx[R0] * l0 + c.kx[R0 + 1] * r0 + c.kym[R0] * zm[0] +
                                     c.kyp[R0] * zp[0];
                        const T n1 = rb[R1] + c.kx[R1] * l1 + c.kx[R1 + 1] * r1 + c.kym[R1] * zm[1] +
                                     c.kyp[R1] * zp[1];
                        V4t<T> out;
                        out.v[R0] = n0 * c.idiag[R0];
                        out.v[R1] = n1 * c.idiag[R1];
                        out.v[1 - PAR] = zc[0];
                        out.v[3 - PAR] = zc[1];
                        stg4(dst + (size_t)b * mx + x0, out);
                        if constexpr (LAST) {
#pragma unroll
                            for (int j = 0; j < 4; ++j) ry += rb[j] * out.v[j];
                            if (need_ap) {
                                // direction row b (previous stage): neighbours across the thread edges
                                const T* pb = prev + 2 * lay.stride;
                                const T pl = pb[x0 - 1], pr = pb[x0 + 4];
#pragma unroll
                                for (int j = 0; j < 4; ++j) {
                                    const T xl = j == 0 ? pl : pc[j - 1];
                                    const T xr = j == 3 ? pr : pc[j + 1];
                                    const T ap = c.diag[j] * pc[j] - (c.kx[j] * xl + c.kx[j + 1] * xr +
                                                                      c.kym[j] * pm[j] + c.kyp[j] * pn[j]);
                                    apy += ap * out.v[j];
                                }
                            }
                        }
                    }
                } else {
                    __syncthreads();
                }
            } else {
                __syncthreads();
                // refill: stage k-2 is no longer read
                if (issuer && k - 2 >= kfirst && k - 2 + RING <= y1) issue(k - 2 + RING);
            }
            if (++cslot == RING) {
                cslot = 0;
                cpar ^= 1u;
            }
        };
        for (int k = kfirst; k <= y1; k += 2) {
            step(Par1{}, k);
            if (k + 1 <= y1) step(Par0{}, k + 1);
        }
        seq += (unsigned)(y1 - kfirst + 1);
        // an expired wait anywhere in the CTA: let the requested copies land (bounded), then stop
        if (__syncthreads_or(!ok)) {
            if (issuer) {
                const uint64_t t0 = gtime();
                for (unsigned u = seq > RING ? seq - RING : 0u; u < seq; ++u)
                    while (!mb_test(bar + u % RING, (u / RING) & 1u) && gtime() - t0 < 500000000ull) {
                    }
            }
            __syncthreads();
            return;
        }
        if (LAST) {
            T a = ry, bs = apy;
            for (int o = 16; o > 0; o >>= 1) {
                a += __shfl_down_sync(0xffffffffu, a, o);
                bs += __shfl_down_sync(0xffffffffu, bs, o);
            }
            const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
            __syncthreads();
            if (lane == 0) {
                red[wi] = (double)a;
                red[16 + wi] = (double)bs;
            }
            __syncthreads();
            double v[2] = {0.0, 0.0};
            if (threadIdx.x == 0)
                for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
                    v[0] += red[i];
                    v[1] += red[16 + i];
                }
            if (arrive(P, q, band, nband, v, 2)) {
                double tot[2];
                gather_partials(P, q, nband, 2, tot, red);
                if (threadIdx.x == 0) {
                    finalize_prec_state(P, q, tot[0], tot[1]);
                    P.tick[q] = 0;
                }
            }
        }
    }
}

template <typename T>
static size_t tma_smem(const Geo& g, bool last) {
    return TmaLayout<T>(g.mx, last).bytes;
}

// 2D, rows of 128 .. 1024 points (a multiple of 128), stages within 200 KB of shared memory
bool use_tma_smoother(const Geo& g) {
    return g.dim == 2 && g.mx % 128 == 0 && g.mx <= TMA_MAX_MX && tma_smem<double>(g, true) <= 200u * 1024u;
}

template <typename T, bool LAST>
static void launch_tma_one(const Params& P, const Launch& L, const T* src, T* dst) {
    const size_t smem = tma_smem<T>(P.g, LAST);
    const int threads = P.g.mx / 4 + 32;
    static size_t conf_smem = 0;
    static int conf_threads = 0;
    static int grid = 0;
    if (conf_smem != smem || conf_threads != threads) {
        cudaFuncSetAttribute(k2_smooth_tma<T, LAST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int dev = 0, sms = 1, per_sm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k2_smooth_tma<T, LAST>, threads, smem);
        grid = sms * (per_sm > 0 ? per_sm : 1);
        conf_smem = smem;
        conf_threads = threads;
    }
    k2_smooth_tma<T, LAST><<<grid, threads, smem, L.s>>>(P, src, dst);
}

template <typename T>
void launch2d_smooth_tma(const Params& P, const Launch& L, int nu) {
    T* ypro = reinterpret_cast<T*>(P.ypro);
    T* tmp = reinterpret_cast<T*>(P.tmp);
    T* out = reinterpret_cast<T*>(P.y);
    const int sweeps = nu < 1 ? 1 : nu;
    const T* src = ypro;
    for (int s = 1; s <= sweeps; ++s) {
        const bool last = s == sweeps;
        T* dst = last ? out : ((s & 1) ? tmp : ypro);
        if (last) launch_tma_one<T, true>(P, L, src, dst);
        else launch_tma_one<T, false>(P, L, src, dst);
        src = dst;
    }
}
template void launch2d_smooth_tma<float>(const Params&, const Launch&, int);
template void launch2d_smooth_tma<double>(const Params&, const Launch&, int);

}  // namespace rbk
