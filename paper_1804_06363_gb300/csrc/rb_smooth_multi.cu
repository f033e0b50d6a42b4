// Several red-black Gauss-Seidel sweeps (eq. 8) in ONE pass over memory on 2D
// grids (FP32, the mixed solver's inner precision), with the rows staged in
// shared memory by bulk asynchronous copies (plan and helpers in rb_stage.cuh).
//
// The 2 NF half-sweeps H_0 (red), H_1 (black), H_2 (red), ... of NF sweeps form
// a pipeline marching down a band of rows, one row per step and ONE consumer
// barrier per step: at step k, H_i updates row k - i.  H_i needs the values of
// H_{i-1} at rows k-i-1, k-i, k-i+1: the thread's own points come from a
// three-row register window (H_{i-1} produced row k-i+1 earlier in the same
// step), the two values across the thread's edges from a small shared array
// that H_{i-1} filled in the previous step (so one barrier per step orders all
// exchanges).  H_0 reads the old source values like the one-sweep kernel.  In
// step k every half-sweep updates the same two columns of its row (those with
// x = k mod 2), so the coefficient subset is common to all of them.
//
// Band [y0, y1) (trapezoid in y): H_i is computed on rows y0 - e_i .. y1 + e_i - 1
// with e_i = 2 NF - 1 - i, so the last half-sweep produces exactly the band; the
// extra rows are recomputed by the neighbouring band instead of being exchanged.
// Rows outside the grid hold zero in every half-sweep (Dirichlet).  Stage k
// brings source row k+1, residual row k and (last pass under Polak-Ribiere)
// direction row k.  A residual row is read by every half-sweep as the pipeline
// passes it (2 NF steps), a direction row by the output of rows k-1 .. k+1.
// Reads and writes per point and pass: source, residual (direction) and output
// once each, whatever NF is.
//
// Coefficients: the face coefficients of a row depend on its block row and its
// two neighbours' (the row key).  While the 2 NF rows in flight share a key
// (away from block boundaries) one register set serves every half-sweep; in the
// few steps that straddle a boundary each half-sweep forms its own.
//
// The producer is one lane of a warp of its own, reusing a slot once every
// consumer warp has released it; every wait is bounded (rb_stage.cuh).
#include "rb_stage.cuh"

namespace rbk {

using namespace stg;

namespace {

constexpr int MS_MAX_NF = 3;
struct Par2 { static constexpr int value = 2; };   // step tag: uniform key, every row inside
// Steps of one band: its rows plus 2 NH.  A band has at most TB_ROWS rows, since the
// partial-sum slots (at least one per TILE points) outnumber the bands of 128-point rows.
constexpr int MS_MAX_STEPS = TB_ROWS + 2 * 2 * MS_MAX_NF;
static_assert(TILE <= 128 * TB_ROWS, "bands of the multi-sweep smoother would outgrow TB_ROWS");

template <int NF, bool LAST>
struct MsShape {
    static constexpr int NH = 2 * NF;                       // half-sweeps
    static constexpr int LAG = LAST ? NH + 1 : NH;          // steps a stage is read in
    static constexpr int RING = LAG + 3;                    // stages in the ring
};

// Shared memory: RING stages of (source row, residual row [, direction row]), each row
// with 16 zero bytes on both sides; then NH x 4 rows of edge values (thread t at index
// t + 1, zeros at both ends); then the mbarriers full[RING] and empty[RING].
template <int NF, bool LAST>
struct MsLayout {
    int nthr, zstride;
    size_t row_stride, stage, edge_off, bar_off, bytes;
    __host__ __device__ MsLayout(int mx)
        : nthr(mx / 4),
          zstride((mx / 4 + 2 + 3) & ~3),
          row_stride((size_t)mx * sizeof(float) + 32),
          stage(row_stride * (LAST ? 3 : 2)),
          edge_off((size_t)MsShape<NF, LAST>::RING * stage),
          bar_off(edge_off + (size_t)MsShape<NF, LAST>::NH * 4 * zstride * sizeof(float)),
          bytes(bar_off + (size_t)2 * MsShape<NF, LAST>::RING * sizeof(uint64_t)) {}
};

// Coefficients of the two points of a row a step updates (columns J, J + 2): the x faces
// on both sides, the y faces, the reciprocal diagonal.
struct MsCoef {
    float kl0, kr0, kl1, kr1, kym0, kyp0, kym1, kyp1, id0, id1;
};

template <int J>
__device__ __forceinline__ MsCoef ms_pick(const TCoef<float>& c) {
    return MsCoef{c.kx[J], c.kx[J + 1], c.kx[J + 2], c.kx[J + 3], c.kym[J], c.kyp[J],
                  c.kym[J + 2], c.kyp[J + 2], c.idiag[J], c.idiag[J + 2]};
}

}  // namespace

template <int NF, bool LAST>
__device__ __noinline__ void multi_producer(const Params& P, const float* __restrict__ src_base,
                                            unsigned char* smem_raw, const MsLayout<NF, LAST>& lay, uint64_t* full,
                                            uint64_t* empty, int rows, int nband, long long total) {
    using S = MsShape<NF, LAST>;
    const Geo& g = P.g;
    const int mx = g.mx, my = g.my;
    const uint32_t row_bytes = (uint32_t)(mx * sizeof(float));
    const void* zero_row = g_zero_row;
    unsigned u = 0;
    bool ok = true;
    for (long long w = blockIdx.x; w < total && ok; w += gridDim.x) {
        const int slot = (int)(w / nband), band = (int)(w % nband);
        const int q = P.lidx[L_PREC * P.Bmax + slot];
        const QState& s = P.st[q];
        const size_t base = (size_t)q * g.n;
        const float* src = src_base + base;
        const float* rg = reinterpret_cast<const float*>(P.r) + base;
        const float* pg = reinterpret_cast<const float*>(P.p) + ((size_t)q * 2 + s.ppar) * g.n;
        const bool need_ap = LAST && P.beta_form == RB_BETA_PR && !s.start;
        const int y0 = band * rows, y1 = min(my, y0 + rows);
        for (int kk = y0 - S::NH - 1; kk <= y1 + S::NH - 2; ++kk, ++u) {
            const unsigned i = u % S::RING;
            if (u >= (unsigned)S::RING && !mb_wait(empty + i, ((u / S::RING) + 1) & 1u, P.err, P.wait_ns)) {
                ok = false;
                break;
            }
            unsigned char* st = smem_raw + (size_t)i * lay.stage + 16;
            const int ms = kk + 1;
            const bool rp = kk >= y0 - S::NH + 1;                      // residual rows of H_0 on
            const bool ap = need_ap && kk >= y0 - 1 && kk <= y1;         // direction rows of the output
            const bool in = kk >= 0 && kk < my;
            mb_arrive_tx(full + i, row_bytes * (1u + (rp ? 1u : 0u) + (ap ? 1u : 0u)));
            bulk_row(st, (ms >= 0 && ms < my) ? (const void*)(src + (size_t)ms * mx) : zero_row, row_bytes, full + i);
            if (rp) bulk_row(st + lay.row_stride, in ? (const void*)(rg + (size_t)kk * mx) : zero_row, row_bytes, full + i);
            if (ap)
                bulk_row(st + 2 * lay.row_stride, in ? (const void*)(pg + (size_t)kk * mx) : zero_row, row_bytes,
                         full + i);
        }
    }
    drain_ring(full, u, (unsigned)S::RING, P.wait_ns);
}

// The 512-point instantiations know their thread count (160) and the CTAs per SM their shared
// memory allows (4 for a pass before the last, 3 for the last, which stages p as well): the
// register cap follows (96 and 128 registers a thread).  Build-time tunables.
#ifndef RB_MS_BLOCKS_MID
#define RB_MS_BLOCKS_MID 4
#endif
#ifndef RB_MS_BLOCKS_LAST
#define RB_MS_BLOCKS_LAST 3
#endif
template <int MX>
constexpr int ms_threads() { return MX > 0 ? MX / 4 + 32 : MAX_MX / 4 + 32; }
template <int MX, bool LAST>
constexpr int ms_min_blocks() { return MX > 0 ? (LAST ? RB_MS_BLOCKS_LAST : RB_MS_BLOCKS_MID) : 1; }

template <int NF, bool LAST, int MX>
__global__ void __launch_bounds__(ms_threads<MX>(), ms_min_blocks<MX, LAST>()) k2_smooth_multi(
    Params P, const float* __restrict__ src_base, float* dst_base) {
    using S = MsShape<NF, LAST>;
    constexpr int NH = S::NH, RING_N = S::RING, LAG = S::LAG;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ float mus[MAX_MU];
    __shared__ double red[32];
    __shared__ int s_flag;
    __shared__ int ukey[MS_MAX_STEPS];   // per step of the item: the common key of the rows in flight, or -1
    const Geo& g = P.g;
    const int mx = MX > 0 ? MX : g.mx, my = g.my;
    const MsLayout<NF, LAST> lay(mx);
    float* edge = reinterpret_cast<float*>(smem_raw + lay.edge_off);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + lay.bar_off);
    uint64_t* empty = full + RING_N;
    const int nthr = lay.nthr;
    const bool producer = (int)threadIdx.x >= nthr;
    const int t = producer ? 0 : (int)threadIdx.x;
    const int x0 = 4 * t;

    // zero the pads of every staged row and the edge rows, set up the barriers
    for (int i = threadIdx.x; i < RING_N * (LAST ? 3 : 2); i += blockDim.x) {
        unsigned char* row = smem_raw + (size_t)i * lay.row_stride;
        for (int j = 0; j < 16; ++j) {
            row[j] = 0;
            row[lay.row_stride - 16 + j] = 0;
        }
    }
    for (int i = threadIdx.x; i < NH * 4 * lay.zstride; i += blockDim.x) edge[i] = 0.0f;
    if (threadIdx.x == 0) {
        for (int i = 0; i < RING_N; ++i) {
            mb_init(full + i, 1);
            mb_init(empty + i, (uint32_t)(nthr / 32));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    const int cnt = P.lcnt[L_PREC];
    const int rows = band_rows(my, cnt, P.max_tiles);
    const int nband = (my + rows - 1) / rows;
    const long long total = (long long)cnt * nband;

    if (producer) {
        if ((threadIdx.x & 31) == 0)
            multi_producer<NF, LAST>(P, src_base, smem_raw, lay, full, empty, rows, nband, total);
        return;
    }

    unsigned seq = 0;
    bool ok = true;
    const int lane = threadIdx.x & 31;
    const uint32_t stage_b = (uint32_t)lay.stage;
    const uint32_t sx0 = 16 + (uint32_t)(x0 * sizeof(float));
    const uint32_t rx0 = (uint32_t)lay.row_stride + sx0;
    const uint32_t px0 = 2 * (uint32_t)lay.row_stride + sx0;
    const uint32_t zsb = (uint32_t)(lay.zstride * sizeof(float));
    auto ld4 = [&](uint32_t off) { return lds4(reinterpret_cast<const float*>(smem_raw + off)); };
    auto ld1 = [&](uint32_t off) { return *reinterpret_cast<const float*>(smem_raw + off); };
    auto eoff = [&](int h, int r) {   // byte offset of the edge row of half-sweep h, row r
        return (uint32_t)lay.edge_off + (uint32_t)(h * 4 + (r & 3)) * zsb;
    };

    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        const int slot = (int)(w / nband), band = (int)(w % nband);
        const int q = P.lidx[L_PREC * P.Bmax + slot];
        const QState& s = P.st[q];
        const bool need_ap = LAST && P.beta_form == RB_BETA_PR && !s.start;
        const int y0 = band * rows, y1 = min(my, y0 + rows);
        const int kfirst = y0 - NH - 1, klast = y1 + NH - 2;   // kfirst odd (y0 even)
        float* dst = dst_base + (size_t)q * g.n;
        cbar(nthr);   // the previous item no longer reads mus or the edge rows
        for (int j = threadIdx.x; j < P.n_mu; j += nthr) mus[j] = (float)P.mu[(size_t)q * P.n_mu + j];
        for (int i = threadIdx.x; i < NH * 4 * lay.zstride; i += nthr) edge[i] = 0.0f;
        for (int i = threadIdx.x; i <= klast - kfirst && i < MS_MAX_STEPS; i += nthr) {
            const int k = kfirst + i;
            const int kt = min(max(k, 0), my - 1), kb = min(max(k - NH + 1, 0), my - 1);
            const int a = __ldg(g.rkey + kt), b = __ldg(g.rkey + kb);
            ukey[i] = a == b ? a : -1;
        }
        cbar(nthr);
        TCoef<float> cf;   // coefficients of the rows in flight while they share a key
        int ckey = -1;
        float sbm[2] = {0.f, 0.f}, sbc[2] = {0.f, 0.f}, sbp[2] = {0.f, 0.f};   // old source values (H_0)
        // windows of the half-sweep outputs: H_i's rows (m, c, p) = k-i-2, k-i-1, k-i after step k
        float hm[NH][2], hc[NH][2], hp[NH][2];
#pragma unroll
        for (int h = 0; h < NH; ++h) hm[h][0] = hm[h][1] = hc[h][0] = hc[h][1] = hp[h][0] = hp[h][1] = 0.f;
        float ry = 0.f, apy = 0.f;
        unsigned cslot = seq % RING_N, cpar = (seq / RING_N) & 1u;

        // one step of the march; PAR = k & 1: every half-sweep updates columns PAR, PAR + 2
        // UNI: the rows k .. k-NH+1 share one key (uniform across the CTA), so every half-sweep
        // uses cf; otherwise each forms its own coefficients
        // slot of the stage d steps back (d <= RING_N, both known at compile time after unrolling)
        auto ring_back = [&](unsigned slot, int d) -> unsigned {
            return slot >= (unsigned)d ? slot - (unsigned)d : slot + (unsigned)(RING_N - d);
        };
        auto step = [&](auto par_tag, auto uni_tag, int k, int kkey) {
            constexpr int PAR = decltype(par_tag)::value;
            constexpr bool UNI = decltype(uni_tag)::value != 0;
            constexpr bool FULL = decltype(uni_tag)::value == 2;   // every half-sweep's row is inside
            constexpr int J0 = PAR, J1 = PAR + 2;          // updated columns
            constexpr int K0 = 1 - PAR, K1 = 3 - PAR;      // the other colour's columns
            if (ok && !mb_wait(full + cslot, cpar, P.err, P.wait_ns)) ok = false;
            const uint32_t o_cur = cslot * stage_b;
            const uint32_t o_prev = ring_back(cslot, 1) * stage_b;
            if constexpr (UNI) {
                if (kkey != ckey) {
                    tcoef<float>(g, mus, x0, min(max(k, 0), my - 1), cf);
                    ckey = kkey;
                }
            }
            // ---- H_0: red half-sweep of row k from the old source values
            {
                const V4t<float> sn = ld4(o_cur + sx0);   // source row k+1
                sbm[0] = sbc[0];
                sbm[1] = sbc[1];
                sbc[0] = sbp[0];
                sbc[1] = sbp[1];
                sbp[0] = sn.v[J0];
                sbp[1] = sn.v[J1];
                hm[0][0] = hc[0][0];
                hm[0][1] = hc[0][1];
                hc[0][0] = hp[0][0];
                hc[0][1] = hp[0][1];
                float n0 = 0.f, n1 = 0.f;
                if (FULL || (k >= y0 - NH + 1 && k >= 0 && k < my)) {
                    MsCoef c;
                    if constexpr (UNI) {
                        c = ms_pick<J0>(cf);
                    } else {
                        TCoef<float> own;
                        tcoef<float>(g, mus, x0, k, own);
                        c = ms_pick<J0>(own);
                    }
                    const V4t<float> rk = ld4(o_cur + rx0);
                    // source row k (previous stage) across the thread edge
                    const float halo = PAR == 0 ? ld1(o_prev + sx0 - 4) : ld1(o_prev + sx0 + 16);
                    const float l0 = PAR == 0 ? halo : sbc[0], r0 = PAR == 0 ? sbc[0] : sbc[1];
                    const float l1 = PAR == 0 ? sbc[0] : sbc[1], r1 = PAR == 0 ? sbc[1] : halo;
                    n0 = (rk.v[J0] + c.kl0 * l0 + c.kr0 * r0 + c.kym0 * sbm[0] + c.kyp0 * sbp[0]) * c.id0;
                    n1 = (rk.v[J1] + c.kl1 * l1 + c.kr1 * r1 + c.kym1 * sbm[1] + c.kyp1 * sbp[1]) * c.id1;
                }
                hp[0][0] = n0;
                hp[0][1] = n1;
                // the value a neighbour thread needs: PAR 0 -> point 0 (thread t-1); PAR 1 -> point 3 (t+1)
                *reinterpret_cast<float*>(smem_raw + eoff(0, k) + (uint32_t)((t + 1) * 4)) = PAR == 0 ? n0 : n1;
            }
            // ---- H_i, i >= 1: row k - i from H_{i-1}'s rows k-i-1 .. k-i+1
#pragma unroll
            for (int h = 1; h < NH; ++h) {
                const int r = k - h;
                // H_{i-1} produced row k-i+1 in this step: its window is (hm, hc, hp) = rows
                // k-i-1, k-i, k-i+1.  H_i's own window shifts to make room for row k-i.
                hm[h][0] = hc[h][0];
                hm[h][1] = hc[h][1];
                hc[h][0] = hp[h][0];
                hc[h][1] = hp[h][1];
                float n0 = 0.f, n1 = 0.f;
                if (FULL || (r >= y0 - (NH - 1 - h) && r >= 0 && r < my)) {
                    MsCoef c;
                    if constexpr (UNI) {
                        c = ms_pick<J0>(cf);
                    } else {
                        TCoef<float> own;
                        tcoef<float>(g, mus, x0, r, own);
                        c = ms_pick<J0>(own);
                    }
                    const uint32_t o_r = ring_back(cslot, h) * stage_b;   // stage of row r
                    const V4t<float> rb = ld4(o_r + rx0);
                    // H_{i-1}'s value across the thread edge of row r (written in the previous step)
                    const float zh = ld1(eoff(h - 1, r) + (uint32_t)((PAR == 0 ? t : t + 2) * 4));
                    const float c0 = hc[h - 1][0], c1 = hc[h - 1][1];
                    const float l0 = PAR == 0 ? zh : c0, r0 = PAR == 0 ? c0 : c1;
                    const float l1 = PAR == 0 ? c0 : c1, r1 = PAR == 0 ? c1 : zh;
                    n0 = (rb.v[J0] + c.kl0 * l0 + c.kr0 * r0 + c.kym0 * hm[h - 1][0] + c.kyp0 * hp[h - 1][0]) * c.id0;
                    n1 = (rb.v[J1] + c.kl1 * l1 + c.kr1 * r1 + c.kym1 * hm[h - 1][1] + c.kyp1 * hp[h - 1][1]) * c.id1;
                }
                hp[h][0] = n0;
                hp[h][1] = n1;
                if (h < NH - 1)
                    *reinterpret_cast<float*>(smem_raw + eoff(h, r) + (uint32_t)((t + 1) * 4)) = PAR == 0 ? n0 : n1;
            }
            // ---- output row k - (NH - 1): the last black values and the last red values
            {
                const int r = k - (NH - 1);
                if (r >= y0 && r < y1) {
                    V4t<float> out;
                    out.v[J0] = hp[NH - 1][0];
                    out.v[J1] = hp[NH - 1][1];
                    out.v[K0] = hc[NH - 2][0];
                    out.v[K1] = hc[NH - 2][1];
                    stg4(dst + (unsigned)(r * mx + x0), out);
                    if constexpr (LAST) {
                        const uint32_t o_r = ring_back(cslot, NH - 1) * stage_b;
                        const V4t<float> rb = ld4(o_r + rx0);
#pragma unroll
                        for (int j = 0; j < 4; ++j) ry += rb.v[j] * out.v[j];
                        if (need_ap) {
                            // direction rows r-1, r, r+1 from their stages
                            const uint32_t o_m = ring_back(cslot, NH) * stage_b;
                            const uint32_t o_p = ring_back(cslot, NH - 2) * stage_b;
                            const V4t<float> pm = ld4(o_m + px0), pc = ld4(o_r + px0), pn = ld4(o_p + px0);
                            const float pl = ld1(o_r + px0 - 4), pr = ld1(o_r + px0 + 16);
                            TCoef<float> own;
                            if constexpr (!UNI) tcoef<float>(g, mus, x0, r, own);
                            const TCoef<float>& c = UNI ? cf : own;
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const float xl = j == 0 ? pl : pc.v[j - 1];
                                const float xr = j == 3 ? pr : pc.v[j + 1];
                                const float dg = c.kx[j] + c.kx[j + 1] + c.kym[j] + c.kyp[j];
                                const float ap =
                                    dg * pc.v[j] - (c.kx[j] * xl + c.kx[j + 1] * xr + c.kym[j] * pm.v[j] + c.kyp[j] * pn.v[j]);
                                apy += ap * out.v[j];
                            }
                        }
                    }
                }
            }
            cbar(nthr);
            // stage seq-LAG+1 has had its last read in this step: release its slot
            if (seq >= (unsigned)(LAG - 1)) {
                __syncwarp();
                if (lane == 0) mb_arrive(empty + (seq - (LAG - 1)) % RING_N);
            }
            ++seq;
            if (++cslot == RING_N) {
                cslot = 0;
                cpar ^= 1u;
            }
        };
        for (int k = kfirst; k <= klast; k += 2) {
            // u >= 0: rows k .. k-NH+1 (clamped to the grid) share a key, uniform over the CTA; when
            // they are also all inside the band's trapezoid and the grid (most steps) the step
            // skips its row tests
            const int u0 = ukey[k - kfirst];
            if (u0 >= 0 && k >= y0 + NH - 1 && k < my) step(Par1{}, Par2{}, k, u0);
            else if (u0 >= 0) step(Par1{}, Par1{}, k, u0);
            else step(Par1{}, Par0{}, k, u0);
            if (k + 1 <= klast) {
                const int u1 = ukey[k + 1 - kfirst];
                if (u1 >= 0 && k + 1 >= y0 + NH - 1 && k + 1 < my) step(Par0{}, Par2{}, k + 1, u1);
                else if (u1 >= 0) step(Par0{}, Par1{}, k + 1, u1);
                else step(Par0{}, Par0{}, k + 1, u1);
            }
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
    (void)ok;
}

namespace {

template <int NF, bool LAST, int MX>
void launch_multi_mx(const Params& P, const Launch& L, const float* src, float* dst) {
    const size_t smem = MsLayout<NF, LAST>(P.g.mx).bytes;
    const int threads = P.g.mx / 4 + 32;
    static size_t conf_smem = 0;
    static int grid = 0;
    if (conf_smem != smem) {
        grid = resident(k2_smooth_multi<NF, LAST, MX>, threads, smem);
        conf_smem = smem;
    }
    k2_smooth_multi<NF, LAST, MX><<<grid, threads, smem, L.s>>>(P, src, dst);
}

template <int NF, bool LAST>
void launch_multi(const Params& P, const Launch& L, const float* src, float* dst) {
    if (P.g.mx == 512) launch_multi_mx<NF, LAST, 512>(P, L, src, dst);
    else launch_multi_mx<NF, LAST, 0>(P, L, src, dst);
}

template <bool LAST>
void launch_multi_nf(int nf, const Params& P, const Launch& L, const float* src, float* dst) {
    if (nf == 1) launch_multi<1, LAST>(P, L, src, dst);
    else if (nf == 2) launch_multi<2, LAST>(P, L, src, dst);
    else launch_multi<3, LAST>(P, L, src, dst);
}

}  // namespace

// FP32, 2D, rows of 128 .. 1024 points (a multiple of 128), stages within 200 KB
bool use_multi_smoother(const Geo& g) {
    return g.dim == 2 && g.mx % 128 == 0 && g.mx <= MAX_MX && g.n < (1LL << 31) &&
           MsLayout<MS_MAX_NF, true>(g.mx).bytes <= 200u * 1024u;
}

// nu sweeps in passes of at most max_nf (<= 3; e.g. 6 = 3 + 3, 5 = 3 + 2): ypro -> tmp -> ... -> y
void launch2d_smooth_multi(const Params& P, const Launch& L, int nu, int max_nf) {
    max_nf = max_nf < 1 ? 1 : (max_nf > MS_MAX_NF ? MS_MAX_NF : max_nf);
    float* ypro = reinterpret_cast<float*>(P.ypro);
    float* tmp = reinterpret_cast<float*>(P.tmp);
    float* out = reinterpret_cast<float*>(P.y);
    int left = nu < 1 ? 1 : nu;
    const float* src = ypro;
    bool to_tmp = true;
    while (left > 0) {
        const int passes = (left + max_nf - 1) / max_nf;
        const int nf = (left + passes - 1) / passes;   // spread the sweeps evenly over the passes
        left -= nf;
        if (left == 0) {
            launch_multi_nf<true>(nf, P, L, src, out);
        } else {
            float* dst = to_tmp ? tmp : ypro;
            launch_multi_nf<false>(nf, P, L, src, dst);
            src = dst;
            to_tmp = !to_tmp;
        }
    }
}

}  // namespace rbk
