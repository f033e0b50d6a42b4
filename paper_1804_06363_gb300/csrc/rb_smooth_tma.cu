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
// Every mbarrier wait is bounded in time: on expiry the device error flag is
// raised, the thread stops waiting and marches on whatever the slots hold (the
// CTA barriers stay matched), then the copies in flight are drained (bounded)
// and the CTA returns.
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
    constexpr int LAG = LAST ? 3 : 2;
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

    const int cnt = P.lcnt[L_PREC];
    const int rows = band_rows(my, cnt, P.max_tiles);
    const int nband = (my + rows - 1) / rows;
    const long long total = (long long)cnt * nband;

    // ---- producer cursor: the next stage in this CTA's order.  Only lane 0 of the
    // producer warp touches it; it lives in shared memory so that it costs the
    // consumers no registers.
    struct Cursor {
        const T* src;
        const T* rg;
        const T* pg;
        long long w;
        int y0, y1, k;
        unsigned issued;
        bool need_ap;
    };
    __shared__ Cursor cur;
    auto cursor_item = [&](long long w) {
        cur.w = w;
        if (w >= total) return;
        const int slot = (int)(w / nband), band = (int)(w % nband);
        const int q = P.lidx[L_PREC * P.Bmax + slot];
        const QState& s = P.st[q];
        const size_t base = (size_t)q * g.n;
        cur.src = src_base + base;
        cur.rg = reinterpret_cast<const T*>(P.r) + base;
        cur.pg = reinterpret_cast<const T*>(P.p) + ((size_t)q * 2 + s.ppar) * g.n;
        cur.y0 = band * rows;
        cur.y1 = min(my, cur.y0 + rows);
        cur.k = cur.y0 - 3;
        cur.need_ap = LAST && P.beta_form == RB_BETA_PR && !s.start;
    };
    auto issue_next = [&]() {
        if (cur.w >= total) return;
        const unsigned u = cur.issued++;
        T* sg = ring + (size_t)(u % RING) * lay.stage_elems + lay.pad;
        uint64_t* b = bar + u % RING;
        const int kk = cur.k, ms = kk + 1;
        const bool rp = kk >= cur.y0 - 1;   // residual (and direction) rows from y0-1 on
        const bool in = kk >= 0 && kk < my;
        const bool ap = rp && cur.need_ap;
        mb_arrive_tx(b, row_bytes * (1u + (rp ? 1u : 0u) + (ap ? 1u : 0u)));
        bulk_row(sg, (ms >= 0 && ms < my) ? cur.src + (size_t)ms * mx : zero_row, row_bytes, b);
        if (rp) bulk_row(sg + lay.stride, in ? cur.rg + (size_t)kk * mx : zero_row, row_bytes, b);
        if (ap) bulk_row(sg + 2 * lay.stride, in ? cur.pg + (size_t)kk * mx : zero_row, row_bytes, b);
        if (++cur.k > cur.y1) cursor_item(cur.w + gridDim.x);
    };
    if (issuer) {
        cur.issued = 0;
        cursor_item(blockIdx.x);
        for (int i = 0; i < RING; ++i) issue_next();
    }

    unsigned seq = 0;   // global step (= stage) number of this CTA (all threads agree)
    bool ok = true;
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        const int slot = (int)(w / nband), band = (int)(w % nband);
        const int q = P.lidx[L_PREC * P.Bmax + slot];
        const QState& s = P.st[q];
        const bool need_ap = LAST && P.beta_form == RB_BETA_PR && !s.start;
        const int y0 = band * rows, y1 = min(my, y0 + rows);
        const int kfirst = y0 - 3;   // odd
        T* dst = dst_base + (size_t)q * g.n;
        __syncthreads();   // the previous item no longer reads mus or the edge rows
        for (int j = threadIdx.x; j < P.n_mu; j += blockDim.x) mus[j] = (T)P.mu[(size_t)q * P.n_mu + j];
        __syncthreads();

        TCoef<T> cf[2];   // coefficients of the last even / odd row updated
        int key[2] = {-1, -1};
        int kpf = __ldg(g.rkey + max(y0 - 1, 0));   // key of the next red row, loaded a step ahead
        T sbm[2] = {T(0), T(0)}, sbc[2] = {T(0), T(0)}, sbp[2] = {T(0), T(0)};   // old black source values
        T zm[2] = {T(0), T(0)}, zc[2] = {T(0), T(0)}, zp[2] = {T(0), T(0)};      // new red rows k-2, k-1, k
        T ry = T(0), apy = T(0);
        unsigned cslot = seq % RING, cpar = (seq / RING) & 1u;

        // one step of the march; PAR = k & 1
        auto step = [&](auto par_tag, int k) {
            constexpr int PAR = decltype(par_tag)::value;
            constexpr int R0 = PAR, R1 = PAR + 2;   // red columns of row k = black columns of row k-1
            if (!producer) {
                const T* stg = ring + (size_t)cslot * lay.stage_elems + lay.pad;
                const T* prev = ring + (size_t)(cslot == 0 ? RING - 1 : cslot - 1) * lay.stage_elems + lay.pad;
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
                        const V4t<T> rk = lds4(stg + lay.stride + x0);
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
                        const V4t<T> rb = lds4(prev + lay.stride + x0);   // residual row b
                        const T* ze = zedge + (b & 3) * lay.zstride;
                        // PAR 0 (b odd): black 0 (t-1's red 3, zc0), black 2 (zc0, zc1)
                        // PAR 1 (b even): black 1 (zc0, zc1), black 3 (zc1, t+1's red 0)
                        const T zh = PAR == 0 ? ze[t] : ze[t + 2];
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
                        stg4(dst + (size_t)b * mx + x0, out);
                        if constexpr (LAST) {
#pragma unroll
                            for (int j = 0; j < 4; ++j) ry += rb.v[j] * out.v[j];
                            if (need_ap) {
                                // direction rows b-1, b, b+1 from stages k-2, k-1, k
                                const T* prev2 =
                                    ring + (size_t)(cslot >= 2 ? cslot - 2 : cslot + RING - 2) * lay.stage_elems +
                                    lay.pad;
                                const V4t<T> pm = lds4(prev2 + 2 * lay.stride + x0);
                                const V4t<T> pc = lds4(prev + 2 * lay.stride + x0);
                                const V4t<T> pn = lds4(stg + 2 * lay.stride + x0);
                                const T pl = prev[2 * lay.stride + x0 - 1], pr = prev[2 * lay.stride + x0 + 4];
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
                    __syncthreads();
                }
            } else {
                __syncthreads();
                if (issuer && seq >= (unsigned)LAG) issue_next();   // stage seq-LAG is no longer read
            }
            ++seq;
            if (++cslot == RING) {
                cslot = 0;
                cpar ^= 1u;
            }
        };
        for (int k = kfirst; k <= y1; k += 2) {
            step(Par1{}, k);
            if (k + 1 <= y1) step(Par0{}, k + 1);
        }
        // an expired wait anywhere in the CTA: let the requested copies land (bounded), then stop
        if (__syncthreads_or(!ok)) {
            if (issuer) drain(bar, cur.issued);
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
