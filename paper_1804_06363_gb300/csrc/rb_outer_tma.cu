// Outer (true) residual r = f(mu) - A(mu) x in FP64 on 2D grids with the rows
// of x staged in shared memory by bulk asynchronous copies (plan and helpers in
// rb_stage.cuh); r is stored as TR (FP32 for the mixed solver, FP64 otherwise)
// and ||r||^2, ||f||^2 go to the outer finalizer (Alg. 3 step 8 on the true
// residual).
//
// Step k (k = y0-2 .. y1-1) consumes stage k = x row k+1 (LAG 2) and, for rows of the
// band, forms f(mu) = sum_r phi_r(mu) f_r at the thread's 4 points (eq. 3; the
// load vectors stay in L2 across queries) and A x from the register window of
// x rows k-1 .. k+1 with the face coefficients cached per row key.  FP64 runs
// at a small fraction of the FP32 rate on this part, so the work per point is
// kept to the load sum, the 5-point stencil and the two squares.  A query that
// starts from x = 0 stages nothing: r = f.
#include "rb_stage.cuh"

namespace rbk {

using namespace stg;

template <typename TR>
__global__ void __launch_bounds__(MAX_MX / 4 + 32) k2s_outer_residual(Params P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double mus[MAX_MU];
    __shared__ double red[32];
    const Geo& g = P.g;
    const int mx = g.mx, my = g.my;
    const Layout<double> lay(mx, 1, 0);
    double* ring = reinterpret_cast<double*>(smem_raw);
    uint64_t* bar = lay.bars(smem_raw);
    const bool producer = (int)threadIdx.x >= lay.nthr;
    const bool issuer = producer && (threadIdx.x & 31) == 0;
    const int x0 = producer ? 0 : 4 * (int)threadIdx.x;
    const uint32_t row_bytes = (uint32_t)(mx * sizeof(double));
    const double* zero_row = g_zero_row;
    setup(lay, ring, bar, mx);

    const int cnt = P.lcnt[L_OUT];
    const int rows = band_rows(my, cnt, P.max_tiles);
    const int nband = (my + rows - 1) / rows;
    const long long total = (long long)cnt * nband;
    constexpr int LAG = 2;

    // producer cursor (shared memory; lane 0 of the producer warp only).  Items of
    // queries that start from x = 0 have no stages.
    struct Cursor {
        const double* xg;
        long long w;
        int y1, k;
        unsigned issued;
    };
    __shared__ Cursor cur;
    auto cursor_item = [&](long long w) {
        for (; w < total; w += gridDim.x) {
            const int slot = (int)(w / nband), band = (int)(w % nband);
            const int q = P.lidx[L_OUT * P.Bmax + slot];
            const QState& s = P.st[q];
            if (s.phase == PH_DONE || s.xzero) continue;
            cur.xg = P.x64 + (size_t)q * g.n;
            const int y0 = band * rows;
            cur.y1 = min(my, y0 + rows);
            cur.k = y0 - 2;
            break;
        }
        cur.w = w;
    };
    auto issue_next = [&]() {
        if (cur.w >= total) return;
        const unsigned u = cur.issued++;
        double* sg = ring + (size_t)(u % RING) * lay.stage_elems + lay.pad;
        uint64_t* b = bar + u % RING;
        const int m = cur.k + 1;
        mb_arrive_tx(b, row_bytes);
        bulk_row(sg, (m >= 0 && m < my) ? cur.xg + (size_t)m * mx : zero_row, row_bytes, b);
        if (++cur.k > cur.y1 - 1) cursor_item(cur.w + gridDim.x);
    };
    if (issuer) {
        cur.issued = 0;
        cursor_item(blockIdx.x);
        for (int i = 0; i < RING; ++i) issue_next();
    }

    unsigned seq = 0;
    bool ok = true;
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        const int slot = (int)(w / nband), band = (int)(w % nband);
        const int q = P.lidx[L_OUT * P.Bmax + slot];
        const QState& s = P.st[q];
        if (s.phase == PH_DONE) continue;   // uniform across the CTA
        const bool xzero = s.xzero != 0;
        const int y0 = band * rows, y1 = min(my, y0 + rows);
        const int kfirst = y0 - 2, klast = y1 - 1;
        TR* rout = reinterpret_cast<TR*>(P.r) + (size_t)q * g.n;
        __syncthreads();
        for (int j = threadIdx.x; j < P.n_mu; j += blockDim.x) mus[j] = P.mu[(size_t)q * P.n_mu + j];
        __syncthreads();
        double phi[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) phi[r] = (r < P.R) ? (P.load_param[r] < 0 ? 1.0 : mus[P.load_param[r]]) : 0.0;
        // f(mu) at the thread's 4 points of row k (same summation order as the generic kernel)
        auto load_row = [&](int k, double* f) {
            const size_t off = (size_t)k * mx + x0;
#pragma unroll
            for (int j = 0; j < 4; ++j) f[j] = 0.0;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                if (r >= P.R) break;
                const double2* src = reinterpret_cast<const double2*>(P.fr + (size_t)r * g.n + off);
                const double2 a = __ldg(src), b = __ldg(src + 1);
                f[0] += phi[r] * a.x;
                f[1] += phi[r] * a.y;
                f[2] += phi[r] * b.x;
                f[3] += phi[r] * b.y;
            }
        };
        double rr = 0.0, ff = 0.0;
        if (xzero) {
            if (!producer)
                for (int k = y0; k < y1; ++k) {
                    double f[4];
                    load_row(k, f);
                    V4t<TR> o;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        o.v[j] = (TR)f[j];
                        rr += f[j] * f[j];
                        ff += f[j] * f[j];
                    }
                    stg4(rout + (size_t)k * mx + x0, o);
                }
        } else {
            double vm[4], vc[4], vp[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) vm[j] = vc[j] = vp[j] = 0.0;
            TCoef<double> c;
            int key = -1;
            int kpf = __ldg(g.rkey + y0);
            unsigned cslot = seq % RING, cpar = (seq / RING) & 1u;
            for (int k = kfirst; k <= klast; ++k) {
                if (!producer) {
                    const double* sg = ring + (size_t)cslot * lay.stage_elems + lay.pad;
                    const double* sprev =
                        ring + (size_t)(cslot == 0 ? RING - 1 : cslot - 1) * lay.stage_elems + lay.pad;
                    if (ok && !mb_wait(bar + cslot, cpar, P.err, P.wait_ns)) ok = false;
                    const V4t<double> a = lds4(sg + x0);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        vm[j] = vc[j];
                        vc[j] = vp[j];
                        vp[j] = a.v[j];
                    }
                    if (k >= y0) {
                        const double left = sprev[x0 - 1], right = sprev[x0 + 4];   // x row k
                        const int kk = kpf;
                        kpf = __ldg(g.rkey + min(k + 1, my - 1));
                        if (kk != key) {
                            tcoef<double>(g, mus, x0, k, c);
                            key = kk;
                        }
                        double f[4];
                        load_row(k, f);
                        V4t<TR> o;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const double rv = f[j] - apply_pt(c, j, vm, vc, vp, left, right);
                            o.v[j] = (TR)rv;
                            rr += rv * rv;
                            ff += f[j] * f[j];
                        }
                        stg4(rout + (size_t)k * mx + x0, o);
                    }
                }
                __syncthreads();
                if (issuer && seq >= (unsigned)LAG) issue_next();
                ++seq;
                if (++cslot == RING) {
                    cslot = 0;
                    cpar ^= 1u;
                }
            }
        }
        if (__syncthreads_or(!ok)) {
            if (issuer) drain(bar, cur.issued, P.wait_ns);
            __syncthreads();
            return;
        }
        double v[2];
        cta_sum2(rr, ff, red, v);
        if (arrive(P, q, band, nband, v, 2)) {
            double tot[2];
            gather_partials(P, q, nband, 2, tot, red);
            if (threadIdx.x == 0) {
                finalize_outer_state(P, q, tot[0], tot[1]);
                P.tick[q] = 0;
            }
        }
    }
}

bool use_staged_outer(const Geo& g) {
    return g.dim == 2 && g.mx % 128 == 0 && g.mx <= MAX_MX && Layout<double>(g.mx, 1, 0).bytes <= 200u * 1024u;
}

template <typename TR>
void launch2d_outer_residual_staged(const Params& P, const Launch& L) {
    const size_t smem = Layout<double>(P.g.mx, 1, 0).bytes;
    const int threads = P.g.mx / 4 + 32;
    static size_t conf_smem = 0;
    static int grid = 0;
    if (conf_smem != smem) {
        grid = resident(k2s_outer_residual<TR>, threads, smem);
        conf_smem = smem;
    }
    k2s_outer_residual<TR><<<grid, threads, smem, L.s>>>(P);
}
template void launch2d_outer_residual_staged<float>(const Params&, const Launch&);
template void launch2d_outer_residual_staged<double>(const Params&, const Launch&);

}  // namespace rbk
