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
#include "rb_stage.cuh"

namespace rbk {

using namespace stg;

namespace {

// Shared memory: the stage ring (source, residual[, direction] rows), then 4
// rows of new red edge values (thread t at index t+1, zeros at both ends).
template <typename T>
struct SmoothLayout : Layout<T> {
    int zstride;
    __host__ __device__ SmoothLayout(int mx, bool last)
        : Layout<T>(mx, last ? 3 : 2, (size_t)4 * ((mx / 4 + 2 + 3) & ~3)), zstride((mx / 4 + 2 + 3) & ~3) {}
};

}  // namespace

template <typename T, bool LAST>
__global__ void __launch_bounds__(MAX_MX / 4 + 32) k2_smooth_tma(Params P, const T* __restrict__ src_base,
                                                                    T* dst_base) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ T mus[MAX_MU];
    __shared__ double red[32];
    const Geo& g = P.g;
    const int mx = g.mx, my = g.my;
    const SmoothLayout<T> lay(mx, LAST);
    T* ring = reinterpret_cast<T*>(smem_raw);
    T* zedge = ring + lay.ring_elems;
    uint64_t* bar = lay.bars(smem_raw);
    const int nthr = lay.nthr;
    const bool producer = (int)threadIdx.x >= nthr;
    const bool issuer = producer && (threadIdx.x & 31) == 0;
    const int t = producer ? 0 : (int)threadIdx.x;
    const int x0 = 4 * t;
    const uint32_t row_bytes = (uint32_t)(mx * sizeof(T));
    const T* zero_row = reinterpret_cast<const T*>(g_zero_row);

    setup(lay, ring, bar, mx);   // zero pads and edge rows, barriers

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

        TCoef<T> cf[2];     // coefficients of the last even / odd row updated
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
                            tcoef<T>(g, mus, x0, k, cf[PAR]);
                            key[PAR] = kk;
                        }
                        const TCoef<T>& c = cf[PAR];
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
                        const TCoef<T>& c = cf[1 - PAR];
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
            if (issuer) drain(bar, seq);
            __syncthreads();
            return;
        }
        if (LAST) {
            double v[2];
            cta_sum2(ry, apy, red, v);
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
    return SmoothLayout<T>(g.mx, last).bytes;
}

// 2D, rows of 128 .. 1024 points (a multiple of 128), stages within 200 KB of shared memory
bool use_tma_smoother(const Geo& g) {
    return g.dim == 2 && g.mx % 128 == 0 && g.mx <= MAX_MX && tma_smem<double>(g, true) <= 200u * 1024u;
}

template <typename T, bool LAST>
static void launch_tma_one(const Params& P, const Launch& L, const T* src, T* dst) {
    const size_t smem = tma_smem<T>(P.g, LAST);
    const int threads = P.g.mx / 4 + 32;
    static size_t conf_smem = 0;
    static int conf_threads = 0, grid = 0;
    if (conf_smem != smem || conf_threads != threads) {
        grid = resident(k2_smooth_tma<T, LAST>, threads, smem);
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
