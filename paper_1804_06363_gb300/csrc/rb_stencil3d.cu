// Red-black Gauss-Seidel smoother S(A, b, y) of eq. 8 on 3D grids, marching in z.
//
// One work item is (query, 32 x 8 tile in x-y, chunk of ZC planes in z).  The
// CTA walks its chunk plane by plane and keeps a ring of three planes of NEW red
// values, each on the tile plus a one-node ring around it (34 x 10), in shared
// memory:
//   red(z+1) on the extended plane  <- old black values of src at z, z+1, z+2
//   black(z) on the tile            <- new red values of planes z-1, z, z+1
// so a point's new value never depends on another CTA of the same launch (the
// ring is recomputed by each CTA that needs it).  Work per point: about 1.5
// red evaluations (ring and chunk ends) against about 2.5 for a 16 x 4 x 4 box
// with a full halo.  Colour, update order and the floating-point expression of
// every update are those of the generic smoother (red = (i_x + i_y + i_z) even
// first, neighbours in the order x-, x+, y-, y+, z-, z+), so both give the same
// values.
// PCG mode only (b = r, output y; the last sweep adds r^T y and (A p)^T y and
// runs the preconditioner finalizer).  RBI keeps the generic kernel.
#include "rb_common.cuh"

namespace rbk {

namespace {

constexpr int TX = 32, TY = 8;             // tile, one point per thread and plane
constexpr int EX = TX + 2, EY = TY + 2;    // tile plus the one-node ring
constexpr int ZC = 16;                     // planes per work item

template <typename T>
__device__ __forceinline__ double bsum(T v, double* red) {
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

__host__ __device__ inline int tiles3(const Geo& g) {
    return ((g.mx + TX - 1) / TX) * ((g.my + TY - 1) / TY) * ((g.mz + ZC - 1) / ZC);
}

template <typename T, bool LAST>
__global__ void __launch_bounds__(THREADS) k3_smooth(Params P, const T* __restrict__ src_base, T* dst_base) {
    __shared__ T mus[MAX_MU];
    __shared__ T ring[3][EY][EX];
    __shared__ double red[32];
    const Geo& g = P.g;
    const int ntx = (g.mx + TX - 1) / TX, nty = (g.my + TY - 1) / TY;
    const int ntiles = tiles3(g);
    const long long plane = (long long)g.mx * g.my;
    const int cnt = P.lcnt[L_PREC];
    const long long total = (long long)cnt * ntiles;
    const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        const int slot = (int)(w / ntiles), tile = (int)(w % ntiles);
        const int q = P.lidx[L_PREC * P.Bmax + slot];
        const QState& s = P.st[q];
        __syncthreads();
        if (threadIdx.x < P.n_mu) mus[threadIdx.x] = (T)P.mu[(size_t)q * P.n_mu + threadIdx.x];
        __syncthreads();
        const int tx0 = (tile % ntx) * TX;
        const int ty0 = ((tile / ntx) % nty) * TY;
        const int z0 = (tile / (ntx * nty)) * ZC;
        const int z1 = min(z0 + ZC, g.mz);
        const T* src = src_base + (size_t)q * g.n;
        T* dst = dst_base + (size_t)q * g.n;
        const T* b = reinterpret_cast<const T*>(P.r) + (size_t)q * g.n;
        const bool need_ap = LAST && P.beta_form == RB_BETA_PR && !s.start;
        const T* pdir = need_ap ? reinterpret_cast<const T*>(P.p) + ((size_t)q * 2 + s.ppar) * (size_t)g.n : nullptr;

        // new red values of plane zz on the extended tile (zero at black points and outside)
        auto red_plane = [&](int zz) {
            T(*rp)[EX] = ring[(zz + 3) % 3];
            for (int e = threadIdx.x; e < EX * EY; e += THREADS) {
                const int ex = e % EX, ey = e / EX;
                const int ix = tx0 + ex - 1, iy = ty0 + ey - 1;
                T val = T(0);
                if (zz >= 0 && zz < g.mz && ix >= 0 && ix < g.mx && iy >= 0 && iy < g.my && ((ix + iy + zz) & 1) == 0) {
                    const long long i = ix + (long long)g.mx * iy + plane * zz;
                    Coef<T> c;
                    node_coef(g, mus, ix, iy, zz, c);
                    val = (b[i] + offdiag_sum(g, c, i, ix, iy, zz, [&](long long k) { return src[k]; })) / c.diag;
                }
                rp[ey][ex] = val;
            }
        };

        red_plane(z0 - 1);
        red_plane(z0);
        T ry = T(0), roy = T(0);
        for (int z = z0; z < z1; ++z) {
            red_plane(z + 1);
            __syncthreads();
            const int ix = tx0 + lx, iy = ty0 + ly;
            if (ix < g.mx && iy < g.my) {
                const long long i = ix + (long long)g.mx * iy + plane * z;
                const T(*rc)[EX] = ring[z % 3];
                T v;
                if (((ix + iy + z) & 1) == 0) {
                    v = rc[ly + 1][lx + 1];
                } else {
                    const T(*rm)[EX] = ring[(z + 2) % 3];
                    const T(*rpz)[EX] = ring[(z + 1) % 3];
                    Coef<T> c;
                    node_coef(g, mus, ix, iy, z, c);
                    T sum = T(0);
                    if (ix > 0) sum += c.kxm * rc[ly + 1][lx];
                    if (ix < g.mx - 1) sum += c.kxp * rc[ly + 1][lx + 2];
                    if (iy > 0) sum += c.kym * rc[ly][lx + 1];
                    if (iy < g.my - 1) sum += c.kyp * rc[ly + 2][lx + 1];
                    if (z > 0) sum += c.kzm * rm[ly + 1][lx + 1];
                    if (z < g.mz - 1) sum += c.kzp * rpz[ly + 1][lx + 1];
                    v = (b[i] + sum) / c.diag;
                }
                dst[i] = v;
                if constexpr (LAST) {
                    ry += b[i] * v;
                    if (need_ap) {
                        Coef<T> c;
                        node_coef(g, mus, ix, iy, z, c);
                        const T ap = c.diag * pdir[i] -
                                     offdiag_sum(g, c, i, ix, iy, z, [&](long long k) { return pdir[k]; });
                        roy += ap * v;
                    }
                }
            }
            __syncthreads();
        }
        if constexpr (LAST) {
            double v[2];
            v[0] = bsum(ry, red);
            v[1] = bsum(roy, red);
            if (arrive(P, q, tile, ntiles, v, 2)) {
                double tot[2];
                gather_partials(P, q, ntiles, 2, tot, red);
                if (threadIdx.x == 0) {
                    finalize_prec_state(P, q, tot[0], tot[1]);
                    P.tick[q] = 0;
                }
            }
        }
    }
}

}  // namespace

bool use_zmarch_smoother(const Geo& g) { return g.dim == 3 && tiles3(g) <= tiles_flat(g.n); }

// nu sweeps ypro -> tmp -> ypro ... -> y, as the generic smoother
template <typename T>
void launch3d_smooth(const Params& P, const Launch& L, int nu) {
    T* ypro = reinterpret_cast<T*>(P.ypro);
    T* tmp = reinterpret_cast<T*>(P.tmp);
    T* out = reinterpret_cast<T*>(P.y);
    const int sweeps = nu < 1 ? 1 : nu;
    const T* src = ypro;
    for (int s = 1; s <= sweeps; ++s) {
        const bool last = s == sweeps;
        T* dst = last ? out : ((s & 1) ? tmp : ypro);
        if (last) k3_smooth<T, true><<<L.grid, THREADS, 0, L.s>>>(P, src, dst);
        else k3_smooth<T, false><<<L.grid, THREADS, 0, L.s>>>(P, src, dst);
        src = dst;
    }
}
template void launch3d_smooth<float>(const Params&, const Launch&, int);
template void launch3d_smooth<double>(const Params&, const Launch&, int);

}  // namespace rbk
