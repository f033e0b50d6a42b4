// One red-black Gauss-Seidel sweep (eq. 8) on 2D grids, with the rows staged in
// shared memory by bulk asynchronous copies (plan and helpers in rb_stage.cuh).
//
// Item = band y0 .. y1-1 of one query; steps k = y0-3 .. y1.  Stage k brings
// source row k+1 and, from k = y0-1 on, residual row k and (last sweep under
// Polak-Ribiere) direction row k.  At step k a consumer
//   - shifts its register window of old black source values and adds row k+1
//     (only the values that the red updates of rows k .. k+2 read),
//   - updates the red points of row k (red: x + y even) from old black values,
//   - after the CTA barrier, updates the black points of row k-1 from the new
//     red values of rows k-2 .. k (registers) and the residual row k-1 (stage
//     k-1), and writes row k-1.
// Neighbours owned by the adjacent threads come from the staged source row or
// from a small shared array of new red values.  The march is unrolled by two
// so that the colour pattern of a row is a compile-time constant.
//
// The last sweep also accumulates r^T y and, under Polak-Ribiere, (A p)^T y
// with the direction rows k-2 .. k read from their stages (a stage is then read
// for three steps: LAG 3) and the diagonal rebuilt from the face coefficients,
// which keeps it near the register budget of the other sweeps.
//
// Storage S of the smoother's iterates (the prolongation output and the
// intermediate sweeps): FP32, or BF16 in the mixed solver when the caller asks
// for it (half the bytes of those rows; the arithmetic stays FP32 and the last
// sweep writes an FP32 y).  Residual and direction rows are always T.
//
// Every mbarrier wait is bounded in time: on expiry the device error flag is
// raised, the thread stops waiting and marches on whatever the slots hold (the
// CTA barriers stay matched), then the copies in flight are drained (bounded)
// and the CTA returns.
#include <cuda_bf16.h>

#include "rb_stage.cuh"

namespace rbk {

using namespace stg;

namespace {

// Shared memory, in bytes: RING stages of (source row in S, residual row in T
// [, direction row in T]), every row with 16 zero bytes on both sides; then 4
// rows of new red edge values (T; thread t at index t+1, zeros at both ends);
// then the mbarriers full[RING] (a stage landed) and empty[RING] (every consumer
// warp is done with the stage in that slot).
template <typename T, typename S>
struct SmoothLayout {
    int nthr, zstride, arrays_t;
    size_t s_stride, t_stride, stage, zedge_off, bar_off, bytes;
    __host__ __device__ constexpr SmoothLayout(int mx, bool last)
        : nthr(mx / 4),
          zstride((mx / 4 + 2 + 3) & ~3),
          arrays_t(last ? 2 : 1),
          s_stride((size_t)mx * sizeof(S) + 32),
          t_stride((size_t)mx * sizeof(T) + 32),
          stage(s_stride + (size_t)arrays_t * t_stride),
          zedge_off((size_t)RING * stage),
          bar_off(zedge_off + (size_t)4 * zstride * sizeof(T)),
          bytes(bar_off + (size_t)2 * RING * sizeof(uint64_t)) {}   // full[RING], empty[RING]
};

// loads of 4 consecutive staged values as T, and their stores
__device__ __forceinline__ V4t<float> lds4s(const float* p) { return lds4(p); }
__device__ __forceinline__ V4t<double> lds4s(const double* p) { return lds4(p); }
__device__ __forceinline__ V4t<float> lds4s(const __nv_bfloat16* p) {
    const uint2 u = *reinterpret_cast<const uint2*>(p);   // bf16 = upper half of the FP32 pattern
    return V4t<float>{{__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u), __uint_as_float(u.y << 16),
                       __uint_as_float(u.y & 0xffff0000u)}};
}
__device__ __forceinline__ float lds1s(const float* p) { return *p; }
__device__ __forceinline__ double lds1s(const double* p) { return *p; }
__device__ __forceinline__ float lds1s(const __nv_bfloat16* p) {
    return __uint_as_float((uint32_t)(*reinterpret_cast<const unsigned short*>(p)) << 16);
}
__device__ __forceinline__ void stg4s(float* p, const V4t<float>& a) { stg4(p, a); }
__device__ __forceinline__ void stg4s(double* p, const V4t<double>& a) { stg4(p, a); }
__device__ __forceinline__ void stg4s(__nv_bfloat16* p, const V4t<float>& a) {
    const __nv_bfloat162 lo = __floats2bfloat162_rn(a.v[0], a.v[1]), hi = __floats2bfloat162_rn(a.v[2], a.v[3]);
    uint2 u;
    u.x = *reinterpret_cast<const uint32_t*>(&lo);
    u.y = *reinterpret_cast<const uint32_t*>(&hi);
    __stcs(reinterpret_cast<uint2*>(p), u);
}

}  // namespace

// The producer (one lane): every stage of the CTA's items in order; a slot is
// reused once all consumer warps have released the stage it held.  Kept out of
// line so that its registers do not add to the consumers'.
template <typename T, bool LAST, typename S>
__device__ __noinline__ void smooth_producer(const Params& P, const S* __restrict__ src_base, unsigned char* smem_raw,
                                             const SmoothLayout<T, S>& lay, uint64_t* full, uint64_t* empty, int rows,
                                             int nband, long long total) {
    const Geo& g = P.g;
    const int mx = g.mx, my = g.my;
    const uint32_t row_bytes = (uint32_t)(mx * sizeof(T)), srow_bytes = (uint32_t)(mx * sizeof(S));
    const void* zero_row = g_zero_row;
    unsigned u = 0;
    bool ok = true;
    for (long long w = blockIdx.x; w < total && ok; w += gridDim.x) {
        const int slot = (int)(w / nband), band = (int)(w % nband);
        const int q = P.lidx[L_PREC * P.Bmax + slot];
        const QState& s = P.st[q];
        const size_t base = (size_t)q * g.n;
        const S* src = src_base + base;
        const T* rg = reinterpret_cast<const T*>(P.r) + base;
        const T* pg = reinterpret_cast<const T*>(P.p) + ((size_t)q * 2 + s.ppar) * g.n;
        const bool need_ap = LAST && P.beta_form == RB_BETA_PR && !s.start;
        const int y0 = band * rows, y1 = min(my, y0 + rows);
        for (int kk = y0 - 3; kk <= y1; ++kk, ++u) {
            const unsigned i = u % RING;
            if (u >= (unsigned)RING && !mb_wait(empty + i, ((u / RING) + 1) & 1u, P.err, P.wait_ns)) {
                ok = false;
                break;
            }
            unsigned char* st = smem_raw + (size_t)i * lay.stage + 16;
            const int ms = kk + 1;
            const bool rp = kk >= y0 - 1;   // residual (and direction) rows from y0-1 on
            const bool in = kk >= 0 && kk < my;
            const bool ap = rp && need_ap;
            mb_arrive_tx(full + i, srow_bytes + row_bytes * ((rp ? 1u : 0u) + (ap ? 1u : 0u)));
            bulk_row(st, (ms >= 0 && ms < my) ? (const void*)(src + (size_t)ms * mx) : zero_row, srow_bytes, full + i);
            if (rp) bulk_row(st + lay.s_stride, in ? (const void*)(rg + (size_t)kk * mx) : zero_row, row_bytes, full + i);
            if (ap)
                bulk_row(st + lay.s_stride + lay.t_stride, in ? (const void*)(pg + (size_t)kk * mx) : zero_row,
                         row_bytes, full + i);
        }
    }
    drain(full, u, P.wait_ns);   // copies still in flight (only after an expired wait do any remain)
}

// S: storage of the source rows (and of dst unless LAST); dst of the last sweep is T.
// MX: the row length as a compile-time constant (all shared-memory offsets become
// immediates), or 0 for the runtime P.g.mx.
template <typename T, bool LAST, typename S, int MX>
__global__ void __maxnreg__(sizeof(T) == 4 ? 96 : 168) k2_smooth_tma(Params P, const S* __restrict__ src_base,
                                                                    std::conditional_t<LAST, T, S>* dst_base) {
    using D = std::conditional_t<LAST, T, S>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ T mus[MAX_MU];
    __shared__ double red[32];
    __shared__ int s_flag;
    constexpr int LAG = LAST ? 3 : 2;
    const Geo& g = P.g;
    const int mx = MX > 0 ? MX : g.mx, my = g.my;
    const SmoothLayout<T, S> lay(mx, LAST);
    unsigned char* ring = smem_raw;
    T* zedge = reinterpret_cast<T*>(smem_raw + lay.zedge_off);   // zeroed once; then by byte offset
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + lay.bar_off);
    uint64_t* empty = full + RING;
    const int nthr = lay.nthr;
    const bool producer = (int)threadIdx.x >= nthr;
    const int t = producer ? 0 : (int)threadIdx.x;
    const int x0 = 4 * t;

    // zero the pads of every staged row and the edge rows, set up the barriers
    for (int i = threadIdx.x; i < RING * (1 + lay.arrays_t); i += blockDim.x) {
        const int slot = i / (1 + lay.arrays_t), a = i % (1 + lay.arrays_t);
        unsigned char* row = ring + (size_t)slot * lay.stage + (a == 0 ? 0 : lay.s_stride + (a - 1) * lay.t_stride);
        const size_t len = a == 0 ? lay.s_stride : lay.t_stride;
        for (int j = 0; j < 16; ++j) {
            row[j] = 0;
            row[len - 16 + j] = 0;
        }
    }
    for (int i = threadIdx.x; i < 4 * lay.zstride; i += blockDim.x) zedge[i] = T(0);
    if (threadIdx.x == 0) {
        for (int i = 0; i < RING; ++i) {
            mb_init(full + i, 1);
            mb_init(empty + i, (uint32_t)(nthr / 32));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();   // the last CTA-wide barrier: from here on producer and consumers run apart

    const int cnt = P.lcnt[L_PREC];
    const int rows = band_rows(my, cnt, P.max_tiles);
    const int nband = (my + rows - 1) / rows;
    const long long total = (long long)cnt * nband;

    // ---- producer: lane 0 of the last warp issues every stage of this CTA's items in
    // order; a slot is reused once all consumer warps released the stage it held.
    if (producer) {
        if ((threadIdx.x & 31) == 0)
            smooth_producer<T, LAST, S>(P, src_base, smem_raw, lay, full, empty, rows, nband, total);
        return;
    }

    // ---- consumers
    unsigned seq = 0;   // global step (= stage) number of this CTA
    bool ok = true;
    const int lane = threadIdx.x & 31;
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        const int slot = (int)(w / nband), band = (int)(w % nband);
        const int q = P.lidx[L_PREC * P.Bmax + slot];
        const QState& s = P.st[q];
        const bool need_ap = LAST && P.beta_form == RB_BETA_PR && !s.start;
        const int y0 = band * rows, y1 = min(my, y0 + rows);
        const int kfirst = y0 - 3;   // odd
        D* dst = dst_base + (size_t)q * g.n;
        cbar(nthr);   // the previous item no longer reads mus or the edge rows
        for (int j = threadIdx.x; j < P.n_mu; j += nthr) mus[j] = (T)P.mu[(size_t)q * P.n_mu + j];
        cbar(nthr);
        TCoef<T> cf[2];   // coefficients of the last even / odd row updated
        int key[2] = {-1, -1};
        int kpf = __ldg(g.rkey + max(y0 - 1, 0));   // key of the next red row, loaded a step ahead
        T sbm[2] = {T(0), T(0)}, sbc[2] = {T(0), T(0)}, sbp[2] = {T(0), T(0)};   // old black source values
        T zm[2] = {T(0), T(0)}, zc[2] = {T(0), T(0)}, zp[2] = {T(0), T(0)};      // new red rows k-2, k-1, k
        T ry = T(0), apy = T(0);
        unsigned cslot = seq % RING, cpar = (seq / RING) & 1u;
        // byte offsets in shared memory of the stages k, k-1, k-2 and of this thread's columns
        const uint32_t stage_b = (uint32_t)lay.stage;
        uint32_t o_cur = cslot * stage_b, o_prev = ((cslot + RING - 1) % RING) * stage_b,
                 o_prev2 = ((cslot + RING - 2) % RING) * stage_b;
        const uint32_t sx0 = 16 + (uint32_t)(x0 * sizeof(S));
        const uint32_t rx0 = (uint32_t)lay.s_stride + 16 + (uint32_t)(x0 * sizeof(T));
        const uint32_t px0 = rx0 + (uint32_t)lay.t_stride;
        const uint32_t zsb = (uint32_t)(lay.zstride * sizeof(T));
        auto ld_s4 = [&](uint32_t off) { return lds4s(reinterpret_cast<const S*>(smem_raw + off)); };
        auto ld_s1 = [&](uint32_t off) { return lds1s(reinterpret_cast<const S*>(smem_raw + off)); };
        auto ld_t4 = [&](uint32_t off) { return lds4(reinterpret_cast<const T*>(smem_raw + off)); };
        auto ld_t1 = [&](uint32_t off) { return *reinterpret_cast<const T*>(smem_raw + off); };

        // one step of the march; PAR = k & 1
        auto step = [&](auto par_tag, int k) {
            constexpr int PAR = decltype(par_tag)::value;
            constexpr int R0 = PAR, R1 = PAR + 2;   // red columns of row k = black columns of row k-1
            {
                if (ok && !mb_wait(full + cslot, cpar, P.err, P.wait_ns)) ok = false;
                // source row k+1 at the red columns of row k (its black points)
                const V4t<T> sn = ld_s4(o_cur + sx0);
                sbm[0] = sbc[0];
                sbm[1] = sbc[1];
                sbc[0] = sbp[0];
                sbc[1] = sbp[1];
                sbp[0] = sn.v[R0];
                sbp[1] = sn.v[R1];
                if (k >= y0 - 1) {
                    // red half-sweep of row k
                    zm[0] = zc[0];
                    zm[1] = zc[1];
                    zc[0] = zp[0];
                    zc[1] = zp[1];
                    if (k >= 0 && k < my) {
                        const int kk = kpf;
                        kpf = __ldg(g.rkey + min(k + 1, my - 1));
                        if (kk != key[PAR]) {
                            tcoef<T>(g, mus, x0, k, cf[PAR]);
                            key[PAR] = kk;
                        }
                        const TCoef<T>& c = cf[PAR];
                        const V4t<T> rk = ld_t4(o_cur + rx0);
                        // source row k (previous stage): the horizontal neighbour across the thread edge
                        const T halo = PAR == 0 ? ld_s1(o_prev + sx0 - (uint32_t)sizeof(S))
                                                : ld_s1(o_prev + sx0 + 4 * (uint32_t)sizeof(S));
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
                    *reinterpret_cast<T*>(smem_raw + lay.zedge_off + (uint32_t)(k & 3) * zsb +
                                          (uint32_t)((t + 1) * sizeof(T))) = PAR == 0 ? zp[0] : zp[1];
                    cbar(nthr);
                    // black half-sweep of row b = k-1 (black columns of b = red columns of k)
                    const int b = k - 1;
                    if (b >= y0 && b < y1) {
                        const TCoef<T>& c = cf[1 - PAR];
                        const V4t<T> rb = ld_t4(o_prev + rx0);   // residual row b
                        // PAR 0 (b odd): black 0 (t-1's red 3, zc0), black 2 (zc0, zc1)
                        // PAR 1 (b even): black 1 (zc0, zc1), black 3 (zc1, t+1's red 0)
                        const T zh = ld_t1((uint32_t)lay.zedge_off + (uint32_t)(b & 3) * zsb +
                                           (uint32_t)((PAR == 0 ? t : t + 2) * sizeof(T)));
                        const T l0 = PAR == 0 ? zh : zc[0], r0 = PAR == 0 ? zc[0] : zc[1];
                        const T l1 = PAR == 0 ? zc[0] : zc[1], r1 = PAR == 0 ? zc[1] : zh;
                        const T n0 = rb.v[R0] + c.kx[R0] * l0 + c.kx[R0 + 1] * r0 + c.kym[R0] * zm[0] +
                                     c.kyp[R0] * zp[0];
                        const T n1 = rb.v[R1] + c.kx[R1] * l1 + c.kx[R1 + 1] * r1 + c.kym[R1] * zm[1] +
                                     c.kyp[R1] * zp[1];
                        V4t<T> out;
                        out.v[R0] = n0 * c.idiag[R0];
                        out.v[R1] = n1 * c.idiag[R1];
                        out.v[1 - PAR] = zc[0];
                        out.v[3 - PAR] = zc[1];
                        stg4s(dst + (unsigned)(b * mx + x0), out);
                        if constexpr (LAST) {
#pragma unroll
                            for (int j = 0; j < 4; ++j) ry += rb.v[j] * out.v[j];
                            if (need_ap) {
                                // direction rows b-1, b, b+1 from stages k-2, k-1, k
                                const V4t<T> pm = ld_t4(o_prev2 + px0);
                                const V4t<T> pc = ld_t4(o_prev + px0);
                                const V4t<T> pn = ld_t4(o_cur + px0);
                                const T pl = ld_t1(o_prev + px0 - (uint32_t)sizeof(T)),
                                        pr = ld_t1(o_prev + px0 + 4 * (uint32_t)sizeof(T));
#pragma unroll
                                for (int j = 0; j < 4; ++j) {
                                    const T xl = j == 0 ? pl : pc.v[j - 1];
                                    const T xr = j == 3 ? pr : pc.v[j + 1];
                                    const T dg = c.kx[j] + c.kx[j + 1] + c.kym[j] + c.kyp[j];
                                    const T ap = dg * pc.v[j] - (c.kx[j] * xl + c.kx[j + 1] * xr + c.kym[j] * pm.v[j] +
                                                                 c.kyp[j] * pn.v[j]);
                                    apy += ap * out.v[j];
                                }
                            }
                        }
                    }
                } else {
                    cbar(nthr);
                }
            }
            // stage seq-LAG+1 has had its last read in this step: release its slot
            if (seq >= (unsigned)(LAG - 1)) {
                __syncwarp();
                if (lane == 0) mb_arrive(empty + (seq - (LAG - 1)) % RING);
            }
            ++seq;
            o_prev2 = o_prev;
            o_prev = o_cur;
            o_cur += stage_b;
            if (++cslot == RING) {
                cslot = 0;
                cpar ^= 1u;
                o_cur = 0;
            }
        };
        for (int k = kfirst; k <= y1; k += 2) {
            step(Par1{}, k);
            if (k + 1 <= y1) step(Par0{}, k + 1);
        }
        if (LAST) {
            double v[2];
            csum2(ry, apy, red, v, nthr);
            if (carrive(P, q, band, nband, v, 2, nthr, &s_flag)) {
                double tot[2];
                cgather(P, q, nband, 2, tot, red, nthr);
                if (threadIdx.x == 0) {
                    finalize_prec_state(P, q, tot[0], tot[1]);
                    P.tick[q] = 0;
                }
            }
        }
    }
}

template <typename T, typename S>
static size_t tma_smem(const Geo& g, bool last) {
    return SmoothLayout<T, S>(g.mx, last).bytes;
}

// 2D, rows of 128 .. 1024 points (a multiple of 128), fewer than 2^31 points (32-bit offsets),
// stages within 200 KB of shared memory
bool use_tma_smoother(const Geo& g) {
    return g.dim == 2 && g.mx % 128 == 0 && g.mx <= MAX_MX && g.n < (1LL << 31) &&
           tma_smem<double, double>(g, true) <= 200u * 1024u;
}

template <typename T, bool LAST, typename S, int MX>
static void launch_tma_mx(const Params& P, const Launch& L, const S* src, std::conditional_t<LAST, T, S>* dst) {
    const size_t smem = tma_smem<T, S>(P.g, LAST);
    const int threads = P.g.mx / 4 + 32;
    static size_t conf_smem = 0;
    static int conf_threads = 0, grid = 0;
    if (conf_smem != smem || conf_threads != threads) {
        grid = resident(k2_smooth_tma<T, LAST, S, MX>, threads, smem);
        conf_smem = smem;
        conf_threads = threads;
    }
    k2_smooth_tma<T, LAST, S, MX><<<grid, threads, smem, L.s>>>(P, src, dst);
}

template <typename T, bool LAST, typename S>
static void launch_tma_one(const Params& P, const Launch& L, const S* src, std::conditional_t<LAST, T, S>* dst) {
    if (sizeof(T) == 4 && P.g.mx == 512) launch_tma_mx<T, LAST, S, 512>(P, L, src, dst);
    else launch_tma_mx<T, LAST, S, 0>(P, L, src, dst);
}

// nu sweeps: ypro -> tmp -> ypro ... -> y; the iterates before y are stored as S
template <typename T, typename S>
static void smooth_sweeps(const Params& P, const Launch& L, int nu) {
    S* ypro = reinterpret_cast<S*>(P.ypro);
    S* tmp = reinterpret_cast<S*>(P.tmp);
    T* out = reinterpret_cast<T*>(P.y);
    const int sweeps = nu < 1 ? 1 : nu;
    const S* src = ypro;
    for (int s = 1; s <= sweeps; ++s) {
        if (s == sweeps) {
            launch_tma_one<T, true, S>(P, L, src, out);
        } else {
            S* dst = (s & 1) ? tmp : ypro;
            launch_tma_one<T, false, S>(P, L, src, dst);
            src = dst;
        }
    }
}

template <typename T>
void launch2d_smooth_tma(const Params& P, const Launch& L, int nu) {
    if constexpr (sizeof(T) == 4) {
        if (P.ybf16) {
            smooth_sweeps<float, __nv_bfloat16>(P, L, nu);
            return;
        }
    }
    smooth_sweeps<T, T>(P, L, nu);
}
template void launch2d_smooth_tma<float>(const Params&, const Launch&, int);
template void launch2d_smooth_tma<double>(const Params&, const Launch&, int);

}  // namespace rbk
