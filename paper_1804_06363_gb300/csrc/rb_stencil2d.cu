// Row-marching 2D kernels for the CG body and the preconditioner's smoother.
//
// A CTA owns one band of rows of one query; thread t owns the 4 consecutive
// points x0 = 4t..4t+3 of every row (16-byte vector loads for FP32, two for
// FP64) and marches down the band keeping the rows above and below in
// registers, so each vector is read from memory once per pass.  The x
// neighbours of a thread's first and last point come from the adjacent lanes
// (shuffles) and, at warp edges, through a small double-buffered shared array:
// one __syncthreads per row.  Coefficients are rebuilt per row from the block
// map (x-blocks of the thread's columns are fixed for the whole band).
// Used when dim == 2 and mx is a multiple of 128 (mx <= 1024); other grids take
// the generic kernels.
#include "rb_common.cuh"

namespace rbk {

#ifndef RB_BAND_ROWS
#define RB_BAND_ROWS 32
#endif
#ifndef RB_MIN_BLOCKS
#define RB_MIN_BLOCKS 1
#endif
constexpr int RB_ROWS = RB_BAND_ROWS;   // rows per band

template <typename T> struct V4 { T v[4]; };

__device__ __forceinline__ V4<float> ld4(const float* p) {
    const float4 a = __ldcs(reinterpret_cast<const float4*>(p));
    return V4<float>{{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ V4<double> ld4(const double* p) {
    const double2 a = __ldcs(reinterpret_cast<const double2*>(p));
    const double2 b = __ldcs(reinterpret_cast<const double2*>(p) + 1);
    return V4<double>{{a.x, a.y, b.x, b.y}};
}
// loads of vectors that neighbouring rows / bands read again (keep in L2)
__device__ __forceinline__ V4<float> ld4k(const float* p) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    return V4<float>{{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ V4<double> ld4k(const double* p) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    return V4<double>{{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st4(float* p, const V4<float>& a) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(a.v[0], a.v[1], a.v[2], a.v[3]));
}
__device__ __forceinline__ void st4(double* p, const V4<double>& a) {
    __stcs(reinterpret_cast<double2*>(p), make_double2(a.v[0], a.v[1]));
    __stcs(reinterpret_cast<double2*>(p) + 1, make_double2(a.v[2], a.v[3]));
}
template <typename T> __device__ __forceinline__ V4<T> zero4() { return V4<T>{{T(0), T(0), T(0), T(0)}}; }

// Coefficients of the thread's 4 points in one row: face terms kappa/h^2 and diagonal.
template <typename T>
struct RowCoef {
    T kx[5];     // x faces: kx[j] between points j-1 and j (kx[0], kx[4] reach the neighbour threads)
    T kym[4], kyp[4], diag[4], idiag[4];
};

// The coefficients of row k depend only on the y-blocks of rows k-1, k, k+1 (and on
// whether those rows exist): rows with equal keys share their coefficients.
__device__ __forceinline__ int row_key(const Geo& g, int k) {
    const int c = __ldg(g.by + k);
    const int m = k > 0 ? __ldg(g.by + k - 1) : 0xFF;
    const int p = k < g.my - 1 ? __ldg(g.by + k + 1) : 0xFF;
    return c | (m << 8) | (p << 16);
}

template <typename T>
struct ColMap {
    int b[6];      // x-block of columns x0-1 .. x0+4 (clamped at the grid edge)
    bool left, right;   // neighbour column exists on the left of point 0 / right of point 3
};

template <typename T>
__device__ __forceinline__ void row_coef(const Geo& g, const T* mus, const ColMap<T>& cm, int k, RowCoef<T>& c) {
    const int nbx = g.nbx;
    const int byc = nbx * __ldg(g.by + k);
    const bool up = k > 0, dn = k < g.my - 1;
    const int bym = up ? nbx * __ldg(g.by + k - 1) : byc;
    const int byp = dn ? nbx * __ldg(g.by + k + 1) : byc;
    T m[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) m[j] = mus[cm.b[j] + byc];
    const T hx = (T)g.ihx2, hy = (T)g.ihy2, half = T(0.5);
    c.kx[0] = hx * (cm.left ? half * (m[0] + m[1]) : m[1]);
#pragma unroll
    for (int j = 1; j < 4; ++j) c.kx[j] = hx * half * (m[j] + m[j + 1]);
    c.kx[4] = hx * (cm.right ? half * (m[4] + m[5]) : m[4]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const T mc = m[j + 1];
        c.kym[j] = hy * (up ? half * (mc + mus[cm.b[j + 1] + bym]) : mc);
        c.kyp[j] = hy * (dn ? half * (mc + mus[cm.b[j + 1] + byp]) : mc);
        c.diag[j] = c.kx[j] + c.kx[j + 1] + c.kym[j] + c.kyp[j];
        c.idiag[j] = T(1) / c.diag[j];
    }
}

// row_coef with a one-entry cache keyed by row_key (uniform across the CTA)
template <typename T>
__device__ __forceinline__ void row_coef_cached(const Geo& g, const T* mus, const ColMap<T>& cm, int k, int& ckey,
                                                RowCoef<T>& c) {
    const int key = row_key(g, k);
    if (key != ckey) {
        row_coef(g, mus, cm, k, c);
        ckey = key;
    }
}

template <typename T>
__device__ __forceinline__ void col_map(const Geo& g, int x0, ColMap<T>& cm) {
    cm.left = x0 > 0;
    cm.right = x0 + 4 < g.mx;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        int xx = x0 - 1 + j;
        xx = xx < 0 ? 0 : (xx >= g.mx ? g.mx - 1 : xx);
        cm.b[j] = __ldg(g.bx + xx);
    }
}

// Exchange the first / last value of each thread's 4 points with the
// neighbouring threads: returns (value left of point 0, value right of point 3).
// sx / sw: shared arrays [2][warps], buf selects the half (double buffering).
template <typename T>
__device__ __forceinline__ void xhalo(const V4<T>& a, T* sx, T* sw, int buf, int nwarps, T& left, T& right) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    left = __shfl_up_sync(0xffffffffu, a.v[3], 1);
    right = __shfl_down_sync(0xffffffffu, a.v[0], 1);
    if (lane == 31) sw[buf * 32 + w] = a.v[3];
    if (lane == 0) sx[buf * 32 + w] = a.v[0];
    __syncthreads();
    if (lane == 0) left = w > 0 ? sw[buf * 32 + w - 1] : T(0);
    if (lane == 31) right = w + 1 < nwarps ? sx[buf * 32 + w + 1] : T(0);
}

template <typename T>
__device__ __forceinline__ double block_sum2d(T v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = (double)v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;
}

// A v at the thread's 4 points of row k, given rows k-1, k, k+1 and the x-halo
template <typename T>
__device__ __forceinline__ V4<T> apply_row(const RowCoef<T>& c, const V4<T>& vm, const V4<T>& vc, const V4<T>& vp,
                                           T left, T right) {
    V4<T> out;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const T xl = j == 0 ? left : vc.v[j - 1];
        const T xr = j == 3 ? right : vc.v[j + 1];
        out.v[j] = c.diag[j] * vc.v[j] - (c.kx[j] * xl + c.kx[j + 1] * xr + c.kym[j] * vm.v[j] + c.kyp[j] * vp.v[j]);
    }
    return out;
}

// ---------------------------------------------------------------------------
// CG part A: p_new = y + beta p_old; accumulate p_new^T A p_new

template <typename T>
__global__ void __launch_bounds__(256, RB_MIN_BLOCKS) k2_cg_a(Params P) {
    __shared__ T mus[MAX_MU];
    __shared__ T sx[64], sw[64];
    __shared__ double red[32];
    const Geo& g = P.g;
    const int mx = g.mx, my = g.my;
    const int nwarps = blockDim.x >> 5;
    const int x0 = 4 * threadIdx.x;
    const int nband = (my + RB_ROWS - 1) / RB_ROWS;
    const int cnt = P.lcnt[L_ITER];
    const long long total = (long long)cnt * nband;
    ColMap<T> cm;
    col_map(g, x0, cm);
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        const int slot = (int)(w / nband), band = (int)(w % nband);
        const int q = P.lidx[L_ITER * P.Bmax + slot];
        const QState& s = P.st[q];
        if (s.phase != PH_ITER) continue;
        __syncthreads();
        if (threadIdx.x < P.n_mu) mus[threadIdx.x] = (T)P.mu[(size_t)q * P.n_mu + threadIdx.x];
        __syncthreads();
        const T beta = (T)s.beta;
        const bool use_old = beta != T(0);
        const size_t base = (size_t)q * g.n;
        const T* y = reinterpret_cast<const T*>(P.y) + base + x0;
        const T* po = reinterpret_cast<const T*>(P.p) + ((size_t)q * 2 + s.ppar) * g.n + x0;
        T* pn = reinterpret_cast<T*>(P.p) + ((size_t)q * 2 + (s.ppar ^ 1)) * g.n + x0;
        auto prow = [&](int k) -> V4<T> {
            if (k < 0 || k >= my) return zero4<T>();
            V4<T> a = ld4k(y + (size_t)k * mx);
            if (use_old) {
                const V4<T> b = ld4k(po + (size_t)k * mx);
#pragma unroll
                for (int j = 0; j < 4; ++j) a.v[j] += beta * b.v[j];
            }
            return a;
        };
        const int y0 = band * RB_ROWS, y1 = min(my, y0 + RB_ROWS);
        V4<T> vm = prow(y0 - 1), vc = prow(y0);
        T acc = T(0);
        int buf = 0;
        RowCoef<T> c;
        int ckey = -1;
        for (int k = y0; k < y1; ++k) {
            const V4<T> vp = prow(k + 1);
            T left, right;
            xhalo(vc, sx, sw, buf, nwarps, left, right);
            buf ^= 1;
            if (!cm.left) left = T(0);
            if (!cm.right) right = T(0);
            row_coef_cached(g, mus, cm, k, ckey, c);
            const V4<T> av = apply_row(c, vm, vc, vp, left, right);
            st4(pn + (size_t)k * mx, vc);
#pragma unroll
            for (int j = 0; j < 4; ++j) acc += vc.v[j] * av.v[j];
            vm = vc;
            vc = vp;
        }
        double v = block_sum2d(acc, red);
        if (arrive(P, q, band, nband, &v, 1)) {
            double tot;
            gather_partials(P, q, nband, 1, &tot, red);
            if (threadIdx.x == 0) {
                finalize_cg_a_state(P, q, tot);
                P.tick[q] = 0;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// CG part B: d += alpha p; r_new = r_old - alpha A p; accumulate ||r_new||^2

template <typename T>
__global__ void __launch_bounds__(256, RB_MIN_BLOCKS) k2_cg_b(Params P) {
    __shared__ T mus[MAX_MU];
    __shared__ T sx[64], sw[64];
    __shared__ double red[32];
    const Geo& g = P.g;
    const int mx = g.mx, my = g.my;
    const int nwarps = blockDim.x >> 5;
    const int x0 = 4 * threadIdx.x;
    const int nband = (my + RB_ROWS - 1) / RB_ROWS;
    const int cnt = P.lcnt[L_ITER];
    const long long total = (long long)cnt * nband;
    ColMap<T> cm;
    col_map(g, x0, cm);
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        const int slot = (int)(w / nband), band = (int)(w % nband);
        const int q = P.lidx[L_ITER * P.Bmax + slot];
        const QState& s = P.st[q];
        if (s.phase != PH_ITER) continue;
        __syncthreads();
        if (threadIdx.x < P.n_mu) mus[threadIdx.x] = (T)P.mu[(size_t)q * P.n_mu + threadIdx.x];
        __syncthreads();
        const T alpha = (T)s.alpha;
        const size_t base = (size_t)q * g.n;
        const T* p = reinterpret_cast<const T*>(P.p) + ((size_t)q * 2 + s.ppar) * g.n + x0;
        T* rr = reinterpret_cast<T*>(P.r) + base + x0;
        T* d = (P.mixed ? reinterpret_cast<T*>(P.d) : reinterpret_cast<T*>(P.x64)) + base + x0;
        auto prow = [&](int k) -> V4<T> { return (k < 0 || k >= my) ? zero4<T>() : ld4k(p + (size_t)k * mx); };
        const int y0 = band * RB_ROWS, y1 = min(my, y0 + RB_ROWS);
        V4<T> vm = prow(y0 - 1), vc = prow(y0);
        T acc = T(0);
        int buf = 0;
        RowCoef<T> c;
        int ckey = -1;
        for (int k = y0; k < y1; ++k) {
            const V4<T> vp = prow(k + 1);
            const V4<T> dk = ld4(d + (size_t)k * mx);
            const V4<T> rk = ld4(rr + (size_t)k * mx);
            T left, right;
            xhalo(vc, sx, sw, buf, nwarps, left, right);
            buf ^= 1;
            if (!cm.left) left = T(0);
            if (!cm.right) right = T(0);
            row_coef_cached(g, mus, cm, k, ckey, c);
            const V4<T> av = apply_row(c, vm, vc, vp, left, right);
            V4<T> dn, rnew;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                dn.v[j] = dk.v[j] + alpha * vc.v[j];
                rnew.v[j] = rk.v[j] - alpha * av.v[j];
                acc += rnew.v[j] * rnew.v[j];
            }
            st4(d + (size_t)k * mx, dn);
            st4(rr + (size_t)k * mx, rnew);
            vm = vc;
            vc = vp;
        }
        double v = block_sum2d(acc, red);
        if (arrive(P, q, band, nband, &v, 1)) {
            double tot;
            gather_partials(P, q, nband, 1, &tot, red);
            if (threadIdx.x == 0) {
                finalize_cg_b_state(P, q, tot);
                P.tick[q] = 0;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// One red-black Gauss-Seidel sweep on A z = r starting from src, with the
// black half-sweep one row behind the red one:
//   step k: red points of row k (needs src rows k-1..k+1, r row k), then black
//   points of row k-1 (needs the new red values of rows k-2..k).
// The band's first and last rows need red values one row outside the band:
// those are recomputed (never read from another CTA's output).

template <typename T, bool LAST>
__global__ void __launch_bounds__(256, RB_MIN_BLOCKS) k2_smooth(Params P, const T* __restrict__ src_base, T* dst_base) {
    __shared__ T mus[MAX_MU];
    __shared__ T sx[3][64], sw[3][64];
    __shared__ double red[32];
    const Geo& g = P.g;
    const int mx = g.mx, my = g.my;
    const int nwarps = blockDim.x >> 5;
    const int x0 = 4 * threadIdx.x;
    const int nband = (my + RB_ROWS - 1) / RB_ROWS;
    const int cnt = P.lcnt[L_PREC];
    const long long total = (long long)cnt * nband;
    ColMap<T> cm;
    col_map(g, x0, cm);
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    // colour of point j of row k: (x0 + j + k) & 1, x0 even: (j + k) & 1
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        const int slot = (int)(w / nband), band = (int)(w % nband);
        const int q = P.lidx[L_PREC * P.Bmax + slot];
        const QState& s = P.st[q];
        __syncthreads();
        if (threadIdx.x < P.n_mu) mus[threadIdx.x] = (T)P.mu[(size_t)q * P.n_mu + threadIdx.x];
        __syncthreads();
        const size_t base = (size_t)q * g.n;
        const T* src = src_base + base + x0;
        T* dst = dst_base + base + x0;
        const T* r = reinterpret_cast<const T*>(P.r) + base + x0;
        // Polak-Ribiere needs (A p)^T y with the direction p of the step just taken
        const bool need_ap = LAST && P.beta_form == RB_BETA_PR && !s.start;
        const T* pd = reinterpret_cast<const T*>(P.p) + ((size_t)q * 2 + s.ppar) * g.n + x0;
        auto srow = [&](int k) -> V4<T> { return (k < 0 || k >= my) ? zero4<T>() : ld4k(src + (size_t)k * mx); };
        auto rrow = [&](int k) -> V4<T> { return (k < 0 || k >= my) ? zero4<T>() : ld4k(r + (size_t)k * mx); };
        auto prow = [&](int k) -> V4<T> {
            return (!need_ap || k < 0 || k >= my) ? zero4<T>() : ld4k(pd + (size_t)k * mx);
        };
        const int y0 = band * RB_ROWS, y1 = min(my, y0 + RB_ROWS);
        // src rows k-1, k, k+1 around the red row k; new red rows k-2, k-1, k; r row k-1;
        // p rows k-2, k-1, k around the black row k-1
        V4<T> sm = srow(y0 - 2), sc = srow(y0 - 1);
        V4<T> zm = zero4<T>(), zc = zero4<T>();
        V4<T> rc = zero4<T>();
        V4<T> pm = zero4<T>(), pc = zero4<T>();
        RowCoef<T> cprev, ccache;
        int ckey = -1;
        T ry = T(0), apy = T(0);
        int buf = 0;
        for (int k = y0 - 1; k <= y1; ++k) {
            const V4<T> sp = srow(k + 1);
            const V4<T> rk = rrow(k);
            const V4<T> pk = prow(k);
            // one exchange for the src row k (red update), the new red row k-1 (black
            // update) and the direction row k-1 (A p at the black row)
            T v0[3] = {sc.v[0], zc.v[0], pc.v[0]};
            T v3[3] = {sc.v[3], zc.v[3], pc.v[3]};
            T lft[3], rgt[3];
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                lft[t] = __shfl_up_sync(0xffffffffu, v3[t], 1);
                rgt[t] = __shfl_down_sync(0xffffffffu, v0[t], 1);
                if (lane == 31) sw[t][buf * 32 + wi] = v3[t];
                if (lane == 0) sx[t][buf * 32 + wi] = v0[t];
            }
            __syncthreads();
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                if (lane == 0) lft[t] = wi > 0 ? sw[t][buf * 32 + wi - 1] : T(0);
                if (lane == 31) rgt[t] = wi + 1 < nwarps ? sx[t][buf * 32 + wi + 1] : T(0);
                if (!cm.left) lft[t] = T(0);
                if (!cm.right) rgt[t] = T(0);
            }
            buf ^= 1;
            // red half-sweep on row k (inside the grid)
            V4<T> zk = zero4<T>();
            if (k >= 0 && k < my) {
                row_coef_cached(g, mus, cm, k, ckey, ccache);
                const RowCoef<T>& ck = ccache;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (((j + k) & 1) == 0) {
                        const T xl = j == 0 ? lft[0] : sc.v[j - 1];
                        const T xr = j == 3 ? rgt[0] : sc.v[j + 1];
                        const T num = rk.v[j] + ck.kx[j] * xl + ck.kx[j + 1] * xr + ck.kym[j] * sm.v[j] +
                                      ck.kyp[j] * sp.v[j];
                        zk.v[j] = num * ck.idiag[j];
                    }
                }
            }
            // black half-sweep on row k-1 (inside the band), output of row k-1
            const int kb = k - 1;
            if (kb >= y0 && kb < y1) {
                V4<T> out;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (((j + kb) & 1) == 0) {
                        out.v[j] = zc.v[j];
                    } else {
                        const T xl = j == 0 ? lft[1] : zc.v[j - 1];
                        const T xr = j == 3 ? rgt[1] : zc.v[j + 1];
                        const T num = rc.v[j] + cprev.kx[j] * xl + cprev.kx[j + 1] * xr + cprev.kym[j] * zm.v[j] +
                                      cprev.kyp[j] * zk.v[j];
                        out.v[j] = num * cprev.idiag[j];
                    }
                }
                st4(dst + (size_t)kb * mx, out);
                if (LAST) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) ry += rc.v[j] * out.v[j];
                    if (need_ap) {
                        const V4<T> ap = apply_row(cprev, pm, pc, pk, lft[2], rgt[2]);
#pragma unroll
                        for (int j = 0; j < 4; ++j) apy += ap.v[j] * out.v[j];
                    }
                }
            }
            sm = sc;
            sc = sp;
            zm = zc;
            zc = zk;
            rc = rk;
            pm = pc;
            pc = pk;
            cprev = ccache;
        }
        if (LAST) {
            double v[2];
            v[0] = block_sum2d(ry, red);
            v[1] = block_sum2d(apy, red);
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

bool use_rowmarch(const Geo& g) { return g.dim == 2 && g.mx % 128 == 0 && g.mx <= 1024; }

// persistent grid: every CTA resident at once (occupancy of the kernel times the SM count)
template <typename K>
static int resident_grid(K kernel, int threads) {
    int dev = 0, sms = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    return sms * (per_sm > 0 ? per_sm : 1);
}

template <typename T>
void launch2d_cg_a(const Params& P, const Launch& L) {
    static int grid = 0;
    if (!grid) grid = resident_grid(k2_cg_a<T>, P.g.mx / 4);
    k2_cg_a<T><<<grid, P.g.mx / 4, 0, L.s>>>(P);
}
template <typename T>
void launch2d_cg_b(const Params& P, const Launch& L) {
    static int grid = 0;
    if (!grid) grid = resident_grid(k2_cg_b<T>, P.g.mx / 4);
    k2_cg_b<T><<<grid, P.g.mx / 4, 0, L.s>>>(P);
}

template <typename T>
void launch2d_smooth(const Params& P, const Launch& L, int nu) {
    T* ypro = reinterpret_cast<T*>(P.ypro);
    T* tmp = reinterpret_cast<T*>(P.tmp);
    T* out = reinterpret_cast<T*>(P.y);
    const int sweeps = nu < 1 ? 1 : nu;
    const T* src = ypro;
    for (int s = 1; s <= sweeps; ++s) {
        const bool last = s == sweeps;
        T* dst = last ? out : ((s & 1) ? tmp : ypro);
        static int grid_l = 0, grid_n = 0;
        if (!grid_l) grid_l = resident_grid(k2_smooth<T, true>, P.g.mx / 4);
        if (!grid_n) grid_n = resident_grid(k2_smooth<T, false>, P.g.mx / 4);
        if (last) k2_smooth<T, true><<<grid_l, P.g.mx / 4, 0, L.s>>>(P, src, dst);
        else k2_smooth<T, false><<<grid_n, P.g.mx / 4, 0, L.s>>>(P, src, dst);
        src = dst;
    }
}

template void launch2d_cg_a<float>(const Params&, const Launch&);
template void launch2d_cg_a<double>(const Params&, const Launch&);
template void launch2d_cg_b<float>(const Params&, const Launch&);
template void launch2d_cg_b<double>(const Params&, const Launch&);
template void launch2d_smooth<float>(const Params&, const Launch&, int);
template void launch2d_smooth<double>(const Params&, const Launch&, int);

int bands2d(const Geo& g) { return (g.my + RB_ROWS - 1) / RB_ROWS; }

}  // namespace rbk
