// The CG body (Alg. 3 steps 5-8 and 11) on 2D grids with the rows staged in
// shared memory by bulk asynchronous copies (plan and helpers in rb_stage.cuh).
//
// Part A: p_new = y + beta p_old and p_new^T A p_new.  Step k (k = y0-2 .. y1-1)
// consumes stage k = (y row k+1, p_old row k+1): the thread forms p_new of row
// k+1 at its 4 points, writes it (rows of the band), and applies A at row k
// from its register window of p_new rows k-1 .. k+1.  The two x neighbours of
// row k are rebuilt from the staged y and p_old rows of the previous stage (the
// same expression as in the neighbour thread), so threads exchange nothing.
//
// Part B: d += alpha p, r_new = r_old - alpha A p and ||r_new||^2.  Stage k =
// (p row k+1; r and d rows k inside the band); step k applies A at row k from
// the register window of p rows k-1 .. k+1 and the x neighbours read from the
// staged p row k.
//
// Both read a stage in its own step and the next one (LAG 2).
#include "rb_stage.cuh"

namespace rbk {

using namespace stg;

template <typename T>
__global__ void __launch_bounds__(MAX_MX / 4 + 32) k2s_cg_a(Params P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ T mus[MAX_MU];
    __shared__ double red[32];
    constexpr int LAG = 2;
    const Geo& g = P.g;
    const int mx = g.mx, my = g.my;
    const Layout<T> lay(mx, 2, 0);
    T* ring = reinterpret_cast<T*>(smem_raw);
    uint64_t* bar = lay.bars(smem_raw);
    const bool producer = (int)threadIdx.x >= lay.nthr;
    const bool issuer = producer && (threadIdx.x & 31) == 0;
    const int x0 = producer ? 0 : 4 * (int)threadIdx.x;
    const uint32_t row_bytes = (uint32_t)(mx * sizeof(T));
    const T* zero_row = reinterpret_cast<const T*>(g_zero_row);
    setup(lay, ring, bar, mx);

    const int cnt = P.lcnt[L_ITER];
    const int rows = band_rows(my, cnt, P.max_tiles);
    const int nband = (my + rows - 1) / rows;
    const long long total = (long long)cnt * nband;

    // producer cursor (shared memory; lane 0 of the producer warp only)
    struct Cursor {
        const T* yg;
        const T* po;
        long long w;
        int y1, k;
        unsigned issued;
        bool use_old;
    };
    __shared__ Cursor cur;
    auto cursor_item = [&](long long w) {
        for (; w < total; w += gridDim.x) {   // skip the items of queries not in the CG body
            const int slot = (int)(w / nband), band = (int)(w % nband);
            const int q = P.lidx[L_ITER * P.Bmax + slot];
            const QState& s = P.st[q];
            if (s.phase != PH_ITER) continue;
            cur.yg = reinterpret_cast<const T*>(P.y) + (size_t)q * g.n;
            cur.po = reinterpret_cast<const T*>(P.p) + ((size_t)q * 2 + s.ppar) * g.n;
            const int y0 = band * rows;
            cur.y1 = min(my, y0 + rows);
            cur.k = y0 - 2;
            cur.use_old = (T)s.beta != T(0);
            break;
        }
        cur.w = w;
    };
    auto issue_next = [&]() {
        if (cur.w >= total) return;
        const unsigned u = cur.issued++;
        T* sg = ring + (size_t)(u % RING) * lay.stage_elems + lay.pad;
        uint64_t* b = bar + u % RING;
        const int m = cur.k + 1;
        const bool in = m >= 0 && m < my;
        mb_arrive_tx(b, row_bytes * (cur.use_old ? 2u : 1u));
        bulk_row(sg, in ? cur.yg + (size_t)m * mx : zero_row, row_bytes, b);
        if (cur.use_old) bulk_row(sg + lay.stride, in ? cur.po + (size_t)m * mx : zero_row, row_bytes, b);
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
        const int q = P.lidx[L_ITER * P.Bmax + slot];
        const QState& s = P.st[q];
        if (s.phase != PH_ITER) continue;   // uniform across the CTA
        const T beta = (T)s.beta;
        const bool use_old = beta != T(0);
        const int y0 = band * rows, y1 = min(my, y0 + rows);
        const int kfirst = y0 - 2, klast = y1 - 1;
        T* pnew = reinterpret_cast<T*>(P.p) + ((size_t)q * 2 + (s.ppar ^ 1)) * g.n;
        __syncthreads();
        for (int j = threadIdx.x; j < P.n_mu; j += blockDim.x) mus[j] = (T)P.mu[(size_t)q * P.n_mu + j];
        __syncthreads();

        T vm[4], vc[4], vp[4];   // p_new rows k-1, k, k+1
#pragma unroll
        for (int j = 0; j < 4; ++j) vm[j] = vc[j] = vp[j] = T(0);
        TCoef<T> c;
        int key = -1;
        int kpf = __ldg(g.rkey + y0);
        T acc = T(0);
        unsigned cslot = seq % RING, cpar = (seq / RING) & 1u;
        for (int k = kfirst; k <= klast; ++k) {
            if (!producer) {
                const T* sg = ring + (size_t)cslot * lay.stage_elems + lay.pad;
                const T* sprev = ring + (size_t)(cslot == 0 ? RING - 1 : cslot - 1) * lay.stage_elems + lay.pad;
                if (ok && !mb_wait(bar + cslot, cpar, P.err, P.wait_ns)) ok = false;
                V4t<T> a = lds4(sg + x0);
                if (use_old) {
                    const V4t<T> b = lds4(sg + lay.stride + x0);
#pragma unroll
                    for (int j = 0; j < 4; ++j) a.v[j] += beta * b.v[j];
                }
                if (k + 1 >= y0 && k + 1 < y1) stg4(pnew + (size_t)(k + 1) * mx + x0, a);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    vm[j] = vc[j];
                    vc[j] = vp[j];
                    vp[j] = a.v[j];
                }
                if (k >= y0) {
                    const int kk = kpf;
                    kpf = __ldg(g.rkey + min(k + 1, my - 1));
                    if (kk != key) {
                        tcoef<T>(g, mus, x0, k, c);
                        key = kk;
                    }
                    // x neighbours of row k, formed like the neighbour threads form them
                    T left = sprev[x0 - 1], right = sprev[x0 + 4];
                    if (use_old) {
                        left += beta * sprev[lay.stride + x0 - 1];
                        right += beta * sprev[lay.stride + x0 + 4];
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc += vc[j] * apply_pt(c, j, vm, vc, vp, left, right);
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
        if (__syncthreads_or(!ok)) {
            if (issuer) drain(bar, cur.issued, P.wait_ns);
            __syncthreads();
            return;
        }
        double v[2];
        cta_sum2(acc, T(0), red, v);
        if (arrive(P, q, band, nband, v, 1)) {
            double tot;
            gather_partials(P, q, nband, 1, &tot, red);
            if (threadIdx.x == 0) {
                finalize_cg_a_state(P, q, tot);
                P.tick[q] = 0;
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(MAX_MX / 4 + 32) k2s_cg_b(Params P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ T mus[MAX_MU];
    __shared__ double red[32];
    constexpr int LAG = 2;
    const Geo& g = P.g;
    const int mx = g.mx, my = g.my;
    const Layout<T> lay(mx, 3, 0);
    T* ring = reinterpret_cast<T*>(smem_raw);
    uint64_t* bar = lay.bars(smem_raw);
    const bool producer = (int)threadIdx.x >= lay.nthr;
    const bool issuer = producer && (threadIdx.x & 31) == 0;
    const int x0 = producer ? 0 : 4 * (int)threadIdx.x;
    const uint32_t row_bytes = (uint32_t)(mx * sizeof(T));
    const T* zero_row = reinterpret_cast<const T*>(g_zero_row);
    setup(lay, ring, bar, mx);

    const int cnt = P.lcnt[L_ITER];
    const int rows = band_rows(my, cnt, P.max_tiles);
    const int nband = (my + rows - 1) / rows;
    const long long total = (long long)cnt * nband;

    struct Cursor {
        const T* pg;
        const T* rg;
        const T* dg;
        long long w;
        int y0, y1, k;
        unsigned issued;
    };
    __shared__ Cursor cur;
    auto cursor_item = [&](long long w) {
        for (; w < total; w += gridDim.x) {
            const int slot = (int)(w / nband), band = (int)(w % nband);
            const int q = P.lidx[L_ITER * P.Bmax + slot];
            const QState& s = P.st[q];
            if (s.phase != PH_ITER) continue;
            const size_t base = (size_t)q * g.n;
            cur.pg = reinterpret_cast<const T*>(P.p) + ((size_t)q * 2 + s.ppar) * g.n;
            cur.rg = reinterpret_cast<const T*>(P.r) + base;
            cur.dg = (P.mixed ? reinterpret_cast<const T*>(P.d) : reinterpret_cast<const T*>(P.x64)) + base;
            cur.y0 = band * rows;
            cur.y1 = min(my, cur.y0 + rows);
            cur.k = cur.y0 - 2;
            break;
        }
        cur.w = w;
    };
    auto issue_next = [&]() {
        if (cur.w >= total) return;
        const unsigned u = cur.issued++;
        T* sg = ring + (size_t)(u % RING) * lay.stage_elems + lay.pad;
        uint64_t* b = bar + u % RING;
        const int kk = cur.k, m = kk + 1;
        const bool rows_rd = kk >= cur.y0;   // r and d rows of the band (kk < y1 always)
        if (P.dbg_skip >= 0 && blockIdx.x == 0 && (long long)u == P.dbg_skip) {
            // test hook: this stage is never issued, so the consumers' bounded wait on it runs out
            if (++cur.k > cur.y1 - 1) cursor_item(cur.w + gridDim.x);
            return;
        }
        mb_arrive_tx(b, row_bytes * (rows_rd ? 3u : 1u));
        bulk_row(sg, (m >= 0 && m < my) ? cur.pg + (size_t)m * mx : zero_row, row_bytes, b);
        if (rows_rd) {
            bulk_row(sg + lay.stride, cur.dg + (size_t)kk * mx, row_bytes, b);
            bulk_row(sg + 2 * lay.stride, cur.rg + (size_t)kk * mx, row_bytes, b);
        }
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
        const int q = P.lidx[L_ITER * P.Bmax + slot];
        const QState& s = P.st[q];
        if (s.phase != PH_ITER) continue;   // uniform across the CTA
        const T alpha = (T)s.alpha;
        const int y0 = band * rows, y1 = min(my, y0 + rows);
        const int kfirst = y0 - 2, klast = y1 - 1;
        const size_t base = (size_t)q * g.n;
        T* rg = reinterpret_cast<T*>(P.r) + base;
        T* dg = (P.mixed ? reinterpret_cast<T*>(P.d) : reinterpret_cast<T*>(P.x64)) + base;
        __syncthreads();
        for (int j = threadIdx.x; j < P.n_mu; j += blockDim.x) mus[j] = (T)P.mu[(size_t)q * P.n_mu + j];
        __syncthreads();

        T vm[4], vc[4], vp[4];   // p rows k-1, k, k+1
#pragma unroll
        for (int j = 0; j < 4; ++j) vm[j] = vc[j] = vp[j] = T(0);
        TCoef<T> c;
        int key = -1;
        int kpf = __ldg(g.rkey + y0);
        T acc = T(0);
        unsigned cslot = seq % RING, cpar = (seq / RING) & 1u;
        for (int k = kfirst; k <= klast; ++k) {
            if (!producer) {
                const T* sg = ring + (size_t)cslot * lay.stage_elems + lay.pad;
                const T* sprev = ring + (size_t)(cslot == 0 ? RING - 1 : cslot - 1) * lay.stage_elems + lay.pad;
                if (ok && !mb_wait(bar + cslot, cpar, P.err, P.wait_ns)) ok = false;
                const V4t<T> a = lds4(sg + x0);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    vm[j] = vc[j];
                    vc[j] = vp[j];
                    vp[j] = a.v[j];
                }
                if (k >= y0) {
                    const int kk = kpf;
                    kpf = __ldg(g.rkey + min(k + 1, my - 1));
                    if (kk != key) {
                        tcoef<T>(g, mus, x0, k, c);
                        key = kk;
                    }
                    const T left = sprev[x0 - 1], right = sprev[x0 + 4];   // p row k
                    const V4t<T> dk = lds4(sg + lay.stride + x0);
                    const V4t<T> rk = lds4(sg + 2 * lay.stride + x0);
                    V4t<T> dn, rn;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const T av = apply_pt(c, j, vm, vc, vp, left, right);
                        dn.v[j] = dk.v[j] + alpha * vc[j];
                        rn.v[j] = rk.v[j] - alpha * av;
                        acc += rn.v[j] * rn.v[j];
                    }
                    stg4(dg + (size_t)k * mx + x0, dn);
                    stg4(rg + (size_t)k * mx + x0, rn);
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
        if (__syncthreads_or(!ok)) {
            if (issuer) drain(bar, cur.issued, P.wait_ns);
            __syncthreads();
            return;
        }
        double v[2];
        cta_sum2(acc, T(0), red, v);
        if (arrive(P, q, band, nband, v, 1)) {
            double tot;
            gather_partials(P, q, nband, 1, &tot, red);
            if (threadIdx.x == 0) {
                finalize_cg_b_state(P, q, tot);
                P.tick[q] = 0;
            }
        }
    }
}

// same grids as the staged smoother
bool use_staged_cg(const Geo& g) {
    return g.dim == 2 && g.mx % 128 == 0 && g.mx <= MAX_MX && Layout<double>(g.mx, 3, 0).bytes <= 200u * 1024u;
}

template <typename T>
void launch2d_cg_a_staged(const Params& P, const Launch& L) {
    const size_t smem = Layout<T>(P.g.mx, 2, 0).bytes;
    const int threads = P.g.mx / 4 + 32;
    static size_t conf_smem = 0;
    static int grid = 0;
    if (conf_smem != smem) {
        grid = resident(k2s_cg_a<T>, threads, smem);
        conf_smem = smem;
    }
    k2s_cg_a<T><<<grid, threads, smem, L.s>>>(P);
}

template <typename T>
void launch2d_cg_b_staged(const Params& P, const Launch& L) {
    const size_t smem = Layout<T>(P.g.mx, 3, 0).bytes;
    const int threads = P.g.mx / 4 + 32;
    static size_t conf_smem = 0;
    static int grid = 0;
    if (conf_smem != smem) {
        grid = resident(k2s_cg_b<T>, threads, smem);
        conf_smem = smem;
    }
    k2s_cg_b<T><<<grid, threads, smem, L.s>>>(P);
}
template void launch2d_cg_a_staged<float>(const Params&, const Launch&);
template void launch2d_cg_a_staged<double>(const Params&, const Launch&);
template void launch2d_cg_b_staged<float>(const Params&, const Launch&);
template void launch2d_cg_b_staged<double>(const Params&, const Launch&);

}  // namespace rbk
