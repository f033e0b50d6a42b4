// All nu sweeps of the red-black Gauss-Seidel smoother S(A, r, y) (eq. 8) in one
// pass over memory, FP32, 2D grids.
//
// The 2 nu half-sweeps (red, black, red, black, ...) form a pipeline marching
// down a band of rows: half-sweep t works one row behind half-sweep t-1, since
// it needs the rows above and below its own in t-1's output.  Each stage keeps
// its last three rows in registers.  A warp owns a strip of 64 columns, 2 per
// lane; a point's x-neighbours come from the adjacent lanes by shuffle, so no
// shared memory or CTA barrier is touched inside the march.  The outermost
// columns of a strip have no neighbour lane: every half-sweep therefore loses one
// valid column on each side and the warp writes only the central
// 64 - 4 nu columns ("trapezoid"); neighbouring strips overlap by 4 nu columns.
// Source, residual and direction are read once and the result written once,
// whatever nu is: 16 B per point instead of 16 + 12 (nu - 1).
// The update of one point uses the same arithmetic as the one-sweep kernels.
// Trade-off measured on 512x512: per output point this kernel issues about 2.4x
// the instructions of nu one-sweep passes (each lane updates one of its two
// points per half-sweep, plus the strip and band overlap), so it is an option
// (rb_opts.kernels = 1) that the autotuner weighs, not the default.
#include "rb_common.cuh"

namespace rbk {

constexpr int FS_BAND = 64;    // output rows per band
constexpr int FS_WARPS = 4;    // strips per CTA (same query and band)
constexpr int FS_KEYS = FS_BAND + 2 * 12 + 2;

__device__ __forceinline__ int fs_row_key(const Geo& g, int j) {
    const int c = __ldg(g.by + j);
    const int m = j > 0 ? __ldg(g.by + j - 1) : 0xFF;
    const int p = j < g.my - 1 ? __ldg(g.by + j + 1) : 0xFF;
    return c | (m << 8) | (p << 16);
}

// coefficients of the point at column c0 + u of a row with the given key
struct FsCoef {
    float kxm, kxp, kym, kyp, diag, idiag;
};

__device__ __forceinline__ FsCoef fs_coef(const Geo& g, const float* mus, int key, int bxl, int bxc, int bxr, bool hasl,
                                          bool hasr) {
    const int nbx = g.nbx;
    const int byc = key & 0xFF, bym = (key >> 8) & 0xFF, byp = (key >> 16) & 0xFF;
    const float hx = (float)g.ihx2, hy = (float)g.ihy2, half = 0.5f;
    const float m = mus[bxc + nbx * byc];
    FsCoef c;
    c.kxm = hx * (hasl ? half * (mus[bxl + nbx * byc] + m) : m);
    c.kxp = hx * (hasr ? half * (m + mus[bxr + nbx * byc]) : m);
    c.kym = hy * (bym != 0xFF ? half * (m + mus[bxc + nbx * bym]) : m);
    c.kyp = hy * (byp != 0xFF ? half * (m + mus[bxc + nbx * byp]) : m);
    c.diag = c.kxm + c.kxp + c.kym + c.kyp;
    c.idiag = 1.0f / c.diag;
    return c;
}

template <int NU>
__global__ void __launch_bounds__(FS_WARPS * 32) k2_smooth_fused(Params P, const float* __restrict__ src_base,
                                                                 float* dst_base) {
    constexpr int NS = 2 * NU;          // half-sweeps
    constexpr int S = 64 - 2 * NS;      // output columns of a strip
    __shared__ float mus[MAX_MU];
    __shared__ int skey[FS_KEYS];
    __shared__ double red[2][FS_WARPS];
    const Geo& g = P.g;
    const int mx = g.mx, my = g.my;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nstrip = (mx + S - 1) / S;
    const int ngroup = (nstrip + FS_WARPS - 1) / FS_WARPS;
    const int nband = (my + FS_BAND - 1) / FS_BAND;
    const int per_q = nband * ngroup;
    const int cnt = P.lcnt[L_PREC];
    const long long total = (long long)cnt * per_q;
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        const int slot = (int)(w / per_q), rem = (int)(w % per_q);
        const int band = rem / ngroup, grp = rem % ngroup;
        const int q = P.lidx[L_PREC * P.Bmax + slot];
        const QState& s = P.st[q];
        const int y0 = band * FS_BAND, y1 = min(my, y0 + FS_BAND);
        const int kb = y0 - NS, ke = y1 - 1 + NS;   // input rows of the band
        __syncthreads();
        if (threadIdx.x < P.n_mu) mus[threadIdx.x] = (float)P.mu[(size_t)q * P.n_mu + threadIdx.x];
        for (int i = threadIdx.x; i <= ke - kb; i += blockDim.x) {
            const int j = kb + i;
            skey[i] = (j >= 0 && j < my) ? fs_row_key(g, j) : -1;
        }
        __syncthreads();
        const int strip = grp * FS_WARPS + warp;
        const bool need_ap = P.beta_form == RB_BETA_PR && !s.start;
        float ry = 0.0f, apy = 0.0f;
        if (strip < nstrip) {   // warp-uniform
            const int xs = strip * S;
            const int c0 = xs - NS + 2 * lane;                 // even; points c0, c0 + 1
            const bool in = c0 >= 0 && c0 < mx;                // mx even: c0 + 1 is inside too
            const bool outc = in && c0 >= xs && c0 < xs + S;   // this lane writes its points
            const bool hasl = c0 > 0, hasr = c0 + 2 < mx;
            const int cl = min(max(c0 - 1, 0), mx - 1), cc0 = min(max(c0, 0), mx - 1);
            const int cc1 = min(max(c0 + 1, 0), mx - 1), cr = min(max(c0 + 2, 0), mx - 1);
            const int bxl = __ldg(g.bx + cl), bx0 = __ldg(g.bx + cc0), bx1 = __ldg(g.bx + cc1),
                      bxr = __ldg(g.bx + cr);
            const size_t base = (size_t)q * g.n;
            const float* src = src_base + base;
            float* dst = dst_base + base;
            const float* r = reinterpret_cast<const float*>(P.r) + base;
            const float* pd = reinterpret_cast<const float*>(P.p) + ((size_t)q * 2 + s.ppar) * g.n;
            auto ld2 = [&](const float* v, int row) -> float2 {
                if (!in || row < 0 || row >= my) return make_float2(0.0f, 0.0f);
                return __ldg(reinterpret_cast<const float2*>(v + (size_t)row * mx + c0));
            };
            // win[t]: the last three rows half-sweep t produced (win[0]: input rows);
            // at step k half-sweep t produces row k - t
            float2 win[NS + 1][3];
#pragma unroll
            for (int t = 0; t <= NS; ++t) win[t][0] = win[t][1] = win[t][2] = make_float2(0.0f, 0.0f);
            float2 rw[NS];   // rw[i] = r row k - 1 - i
#pragma unroll
            for (int t = 0; t < NS; ++t) rw[t] = make_float2(0.0f, 0.0f);
            float2 pw0 = make_float2(0.0f, 0.0f), pw1 = pw0, pw2 = pw0;
            int ckey = -2;
            FsCoef cf0 = {0, 0, 0, 0, 1, 1}, cf1 = cf0;
            for (int k = kb; k <= ke; ++k) {
                win[0][0] = win[0][1];
                win[0][1] = win[0][2];
                win[0][2] = ld2(src, k);
#pragma unroll
                for (int t = NS - 1; t > 0; --t) rw[t] = rw[t - 1];
                rw[0] = ld2(r, k - 1);
                if (need_ap) {
                    pw0 = pw1;
                    pw1 = pw2;
                    pw2 = ld2(pd, k - NS + 1);
                }
#pragma unroll
                for (int t = 1; t <= NS; ++t) {
                    const int j = k - t;
                    win[t][0] = win[t][1];
                    win[t][1] = win[t][2];
                    const float2 cur = win[t - 1][1];
                    const float nl = __shfl_up_sync(0xffffffffu, cur.y, 1);     // column c0 - 1
                    const float nr = __shfl_down_sync(0xffffffffu, cur.x, 1);   // column c0 + 2
                    float2 out = make_float2(0.0f, 0.0f);
                    if (j >= kb && j >= 0 && j < my) {   // j is warp-uniform
                        const int key = skey[j - kb];
                        if (key != ckey) {
                            cf0 = fs_coef(g, mus, key, bxl, bx0, bx1, hasl, true);
                            cf1 = fs_coef(g, mus, key, bx0, bx1, bxr, true, hasr);
                            ckey = key;
                        }
                        // red stages (t odd) update the point with (c + j) even, black ones the other
                        const int par = j & 1;                          // colour of column c0 (c0 even)
                        const int u = (t & 1) ? par : 1 - par;
                        const float rr = u ? rw[t - 1].y : rw[t - 1].x;
                        if (in) {
                            out = cur;
                            if (u == 0) {
                                const float xl = hasl ? nl : 0.0f;
                                const float num = rr + cf0.kxm * xl + cf0.kxp * cur.y + cf0.kym * win[t - 1][0].x +
                                                  cf0.kyp * win[t - 1][2].x;
                                out.x = num * cf0.idiag;
                            } else {
                                const float xr = hasr ? nr : 0.0f;
                                const float num = rr + cf1.kxm * cur.x + cf1.kxp * xr + cf1.kym * win[t - 1][0].y +
                                                  cf1.kyp * win[t - 1][2].y;
                                out.y = num * cf1.idiag;
                            }
                        }
                    }
                    win[t][2] = out;
                }
                // output row jo = k - NS (coefficients of that row are in the cache)
                const int jo = k - NS;
                const float apl = __shfl_up_sync(0xffffffffu, pw1.y, 1);
                const float apr = __shfl_down_sync(0xffffffffu, pw1.x, 1);
                if (jo >= y0 && jo < y1) {
                    const float2 y = win[NS][2];
                    if (outc) {
                        __stcs(reinterpret_cast<float2*>(dst + (size_t)jo * mx + c0), y);
                        ry += rw[NS - 1].x * y.x + rw[NS - 1].y * y.y;
                        if (need_ap) {
                            const float pl = hasl ? apl : 0.0f, pr = hasr ? apr : 0.0f;
                            const float a0 = cf0.diag * pw1.x -
                                             (cf0.kxm * pl + cf0.kxp * pw1.y + cf0.kym * pw0.x + cf0.kyp * pw2.x);
                            const float a1 = cf1.diag * pw1.y -
                                             (cf1.kxm * pw1.x + cf1.kxp * pr + cf1.kym * pw0.y + cf1.kyp * pw2.y);
                            apy += a0 * y.x + a1 * y.y;
                        }
                    }
                }
            }
        }
        // CTA reduction of the two dot products, then the per-query finalizer
        float a = ry, b = apy;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            b += __shfl_down_sync(0xffffffffu, b, o);
        }
        __syncthreads();
        if (lane == 0) {
            red[0][warp] = (double)a;
            red[1][warp] = (double)b;
        }
        __syncthreads();
        double v[2] = {0.0, 0.0};
        if (threadIdx.x == 0)
            for (int i = 0; i < FS_WARPS; ++i) {
                v[0] += red[0][i];
                v[1] += red[1][i];
            }
        if (arrive(P, q, rem, per_q, v, 2)) {
            double tot[2];
            gather_partials(P, q, per_q, 2, tot, &red[0][0]);
            if (threadIdx.x == 0) {
                finalize_prec_state(P, q, tot[0], tot[1]);
                P.tick[q] = 0;
            }
        }
    }
}

bool use_fused_smoother(const Geo& g, int nu) {
    return g.dim == 2 && g.mx % 2 == 0 && nu >= 1 && nu <= 6 && g.nbx <= 255 && g.nby <= 255;
}

template <int NU>
static void launch_nu(const Params& P, const Launch& L) {
    static int grid = 0;
    if (!grid) {
        int dev = 0, sms = 1, per_sm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k2_smooth_fused<NU>, FS_WARPS * 32, 0);
        grid = sms * (per_sm > 0 ? per_sm : 1);
    }
    k2_smooth_fused<NU><<<grid, FS_WARPS * 32, 0, L.s>>>(P, reinterpret_cast<const float*>(P.ypro),
                                                         reinterpret_cast<float*>(P.y));
}

void launch2d_smooth_fused(const Params& P, const Launch& L, int nu) {
    switch (nu) {
        case 1: launch_nu<1>(P, L); break;
        case 2: launch_nu<2>(P, L); break;
        case 3: launch_nu<3>(P, L); break;
        case 4: launch_nu<4>(P, L); break;
        case 5: launch_nu<5>(P, L); break;
        default: launch_nu<6>(P, L); break;
    }
}

int fused_tiles(const Geo& g, int nu) {
    const int S = 64 - 4 * nu;
    const int nstrip = (g.mx + S - 1) / S;
    return ((g.my + FS_BAND - 1) / FS_BAND) * ((nstrip + FS_WARPS - 1) / FS_WARPS);
}

}  // namespace rbk
