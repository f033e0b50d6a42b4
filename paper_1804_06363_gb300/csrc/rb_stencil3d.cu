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

// ----------------------------------------------------------------------------
// Staged variants: the planes a step needs are prefetched into rings of shared
// memory by asynchronous copies (cp.async, one element per copy, zero-filled
// outside the grid), issued a few planes ahead of the march, so the loads of
// plane z+3 are in flight while plane z is computed.  Regions of a plane:
//   E1 = tile + 1-node ring (34 x 10), origin (x0 - 1, y0 - 1)
//   E2 = tile + 2-node ring (36 x 12), origin (x0 - 2, y0 - 2)
//   I  = tile (32 x 8), origin (x0, y0)
// The floating-point expressions and their order are those of the generic
// kernels; zero-filled neighbours outside the grid are never read (the same
// bounds tests decide which faces enter a sum).

constexpr int E2X = TX + 4, E2Y = TY + 4;

__device__ __forceinline__ uint32_t sh_addr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// one element global -> shared, asynchronously; zero-filled when !valid (no global read)
template <typename T>
__device__ __forceinline__ void cp_elem(T* sdst, const T* gsrc, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(sh_addr(sdst)), "l"(gsrc),
                 "n"((int)sizeof(T)), "r"(valid ? (int)sizeof(T) : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Per-thread plan for staging one RX x RY region: the in-plane offsets of the
// thread's elements and which of them lie in the grid (computed once per work
// item; a plane then costs one address and one copy per element).
template <int RX, int RY>
struct StagePlan {
    static constexpr int MAXE = (RX * RY + THREADS - 1) / THREADS;
    int off[MAXE];
    unsigned ok;
    __device__ __forceinline__ void init(const Geo& g, int x0, int y0) {
        ok = 0u;
#pragma unroll
        for (int j = 0; j < MAXE; ++j) {
            const int e = threadIdx.x + j * THREADS;
            off[j] = 0;
            const int ix = x0 + e % RX, iy = y0 + e / RX;
            if (e < RX * RY && ix >= 0 && ix < g.mx && iy >= 0 && iy < g.my) {
                off[j] = ix + g.mx * iy;
                ok |= 1u << j;
            }
        }
    }
    // plane zz of v into s (zero outside the grid)
    template <typename T>
    __device__ __forceinline__ void stage(T* s, const T* __restrict__ v, const Geo& g, int zz) const {
        const bool zin = zz >= 0 && zz < g.mz;
        const T* vp = v + (long long)g.mx * g.my * (zin ? zz : 0);
#pragma unroll
        for (int j = 0; j < MAXE; ++j) {
            const int e = threadIdx.x + j * THREADS;
            if (e < RX * RY) {
                const bool valid = zin && ((ok >> j) & 1u);
                cp_elem(s + e, valid ? vp + off[j] : v, valid);
            }
        }
    }
};

__host__ __device__ inline int wrap(int k, int n) { return ((k % n) + n) % n; }

// Key of the z-dependence of a node's face coefficients: the blocks of planes
// k-1, k, k+1 (0xFF where the face lies on the boundary).  Equal keys at the
// same (x, y) give equal coefficients, so a thread rebuilds its Coef only when
// the key changes (at block boundaries in z).
constexpr int ZK = ZC + 4;   // planes z0-2 .. z0+ZC+1
__device__ __forceinline__ void fill_zkeys(int* zk, const Geo& g, int z0) {
    for (int t = threadIdx.x; t < ZK; t += THREADS) {
        const int k = z0 - 2 + t;
        int key = -1;
        if (k >= 0 && k < g.mz)
            key = ((k > 0 ? __ldg(g.bz + k - 1) : 0xFF) << 16) | (__ldg(g.bz + k) << 8) |
                  (k < g.mz - 1 ? __ldg(g.bz + k + 1) : 0xFF);
        zk[t] = key;
    }
}

template <typename T>
__device__ __forceinline__ void cached_coef(const Geo& g, const T* mus, int ix, int iy, int k, int key, Coef<T>& c,
                                            int& ckey) {
    if (ckey != key) {
        node_coef(g, mus, ix, iy, k, c);
        ckey = key;
    }
}

// ---- smoother, staged: ring of NSS planes of {src on E2, b on E1, p on E1 (PR only)}
constexpr int NSS = 5;
constexpr int RED_PTS = EY * (EX / 2);   // red points of an E1 plane (EX even)

template <typename T>
struct SmoothSmem {
    T src[NSS][E2Y][E2X];
    T b[NSS][EY][EX];
    T pd[NSS][EY][EX];
    T red[3][EY][EX];
};

template <typename T, bool LAST>
__global__ void __launch_bounds__(THREADS, 3) k3s_smooth(Params P, const T* __restrict__ src_base, T* dst_base) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmoothSmem<T>& S = *reinterpret_cast<SmoothSmem<T>*>(smem_raw);
    __shared__ T mus[MAX_MU];
    __shared__ int zk[ZK];
    __shared__ double red[32];
    const Geo& g = P.g;
    const int ntx = (g.mx + TX - 1) / TX, nty = (g.my + TY - 1) / TY;
    const int ntiles = tiles3(g);
    const long long plane = (long long)g.mx * g.my;
    const int cnt = P.lcnt[L_PREC];
    const long long total = (long long)cnt * ntiles;
    const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
    // this thread's red point of an E1 plane: row rey, x = 2 rj + parity
    const int rey = threadIdx.x / (EX / 2), rj = threadIdx.x % (EX / 2);
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        const int slot = (int)(w / ntiles), tile = (int)(w % ntiles);
        const int q = P.lidx[L_PREC * P.Bmax + slot];
        const QState& s = P.st[q];
        const int tx0 = (tile % ntx) * TX;
        const int ty0 = ((tile / ntx) % nty) * TY;
        const int z0 = (tile / (ntx * nty)) * ZC;
        const int z1 = min(z0 + ZC, g.mz);
        __syncthreads();
        if (threadIdx.x < P.n_mu) mus[threadIdx.x] = (T)P.mu[(size_t)q * P.n_mu + threadIdx.x];
        fill_zkeys(zk, g, z0);
        const T* src = src_base + (size_t)q * g.n;
        T* dst = dst_base + (size_t)q * g.n;
        const T* b = reinterpret_cast<const T*>(P.r) + (size_t)q * g.n;
        const bool need_ap = LAST && P.beta_form == RB_BETA_PR && !s.start;
        const T* pdir = need_ap ? reinterpret_cast<const T*>(P.p) + ((size_t)q * 2 + s.ppar) * (size_t)g.n : b;
        StagePlan<E2X, E2Y> p2;
        StagePlan<EX, EY> p1;
        p2.init(g, tx0 - 2, ty0 - 2);
        p1.init(g, tx0 - 1, ty0 - 1);
        auto stage = [&](int k) {
            const int sl = wrap(k, NSS);
            if (k <= z1 + 1) {
                p2.stage(&S.src[sl][0][0], src, g, k);
                p1.stage(&S.b[sl][0][0], b, g, k);
                if (need_ap) p1.stage(&S.pd[sl][0][0], pdir, g, k);
            }
            cp_commit();
        };
        // coefficient caches: the red point of even / odd planes, the tile point
        Coef<T> cr0, cr1, ci;
        int kr0 = -1, kr1 = -1, ki = -1;
        // new red values of plane k on E1; black entries and points outside the grid are
        // never read, so only the RED_PTS red points are computed (one per thread)
        auto red_plane = [&](int k) {
            if (k < 0 || k >= g.mz || threadIdx.x >= RED_PTS) return;
            const int iy = ty0 - 1 + rey;
            const int ex = 2 * rj + ((1 + tx0 + iy + k) & 1);
            const int ix = tx0 - 1 + ex;
            if (ix < 0 || ix >= g.mx || iy < 0 || iy >= g.my) return;
            const int key = zk[k - z0 + 2];
            Coef<T> c;
            if (k & 1) {
                cached_coef(g, mus, ix, iy, k, key, cr1, kr1);
                c = cr1;
            } else {
                cached_coef(g, mus, ix, iy, k, key, cr0, kr0);
                c = cr0;
            }
            const T(*sc)[E2X] = S.src[wrap(k, NSS)];
            const T(*sm)[E2X] = S.src[wrap(k - 1, NSS)];
            const T(*sp)[E2X] = S.src[wrap(k + 1, NSS)];
            T sum = T(0);
            if (ix > 0) sum += c.kxm * sc[rey + 1][ex];
            if (ix < g.mx - 1) sum += c.kxp * sc[rey + 1][ex + 2];
            if (iy > 0) sum += c.kym * sc[rey][ex + 1];
            if (iy < g.my - 1) sum += c.kyp * sc[rey + 2][ex + 1];
            if (k > 0) sum += c.kzm * sm[rey + 1][ex + 1];
            if (k < g.mz - 1) sum += c.kzp * sp[rey + 1][ex + 1];
            S.red[wrap(k, 3)][rey][ex] = (S.b[wrap(k, NSS)][rey][ex] + sum) / c.diag;
        };
        for (int k = z0 - 2; k <= z0 + 2; ++k) stage(k);
        cp_wait<2>();               // planes z0-2 .. z0 (and mus, zk)
        __syncthreads();
        red_plane(z0 - 1);
        cp_wait<1>();               // plane z0+1
        __syncthreads();
        red_plane(z0);
        T ry = T(0), roy = T(0);
        const int ix = tx0 + lx, iy = ty0 + ly;
        const bool inside = ix < g.mx && iy < g.my;
        for (int z = z0; z < z1; ++z) {
            stage(z + 3);           // into the slot of plane z-2, last read before the previous barrier
            cp_wait<1>();           // plane z+2
            __syncthreads();
            red_plane(z + 1);
            __syncthreads();
            if (inside) {
                const long long i = ix + (long long)g.mx * iy + plane * z;
                const T(*rc)[EX] = S.red[wrap(z, 3)];
                const T bi = S.b[wrap(z, NSS)][ly + 1][lx + 1];
                const bool is_red = ((ix + iy + z) & 1) == 0;
                if (!is_red || need_ap) cached_coef(g, mus, ix, iy, z, zk[z - z0 + 2], ci, ki);
                T v;
                if (is_red) {
                    v = rc[ly + 1][lx + 1];
                } else {
                    const T(*rm)[EX] = S.red[wrap(z - 1, 3)];
                    const T(*rpz)[EX] = S.red[wrap(z + 1, 3)];
                    T sum = T(0);
                    if (ix > 0) sum += ci.kxm * rc[ly + 1][lx];
                    if (ix < g.mx - 1) sum += ci.kxp * rc[ly + 1][lx + 2];
                    if (iy > 0) sum += ci.kym * rc[ly][lx + 1];
                    if (iy < g.my - 1) sum += ci.kyp * rc[ly + 2][lx + 1];
                    if (z > 0) sum += ci.kzm * rm[ly + 1][lx + 1];
                    if (z < g.mz - 1) sum += ci.kzp * rpz[ly + 1][lx + 1];
                    v = (bi + sum) / ci.diag;
                }
                dst[i] = v;
                if constexpr (LAST) {
                    ry += bi * v;
                    if (need_ap) {
                        const T(*pc)[EX] = S.pd[wrap(z, NSS)];
                        const T(*pm)[EX] = S.pd[wrap(z - 1, NSS)];
                        const T(*pp)[EX] = S.pd[wrap(z + 1, NSS)];
                        T sum = T(0);
                        if (ix > 0) sum += ci.kxm * pc[ly + 1][lx];
                        if (ix < g.mx - 1) sum += ci.kxp * pc[ly + 1][lx + 2];
                        if (iy > 0) sum += ci.kym * pc[ly][lx + 1];
                        if (iy < g.my - 1) sum += ci.kyp * pc[ly + 2][lx + 1];
                        if (z > 0) sum += ci.kzm * pm[ly + 1][lx + 1];
                        if (z < g.mz - 1) sum += ci.kzp * pp[ly + 1][lx + 1];
                        const T ap = ci.diag * pc[ly + 1][lx + 1] - sum;
                        roy += ap * v;
                    }
                }
            }
            __syncthreads();
        }
        cp_wait<0>();               // nothing of this item may land in the next one's slots
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

// ---- CG body, staged: ring of NSC planes on E1 (p or y, p_old) and on I (r, d)
constexpr int NSC = 4;

template <typename T>
struct CgSmem {
    T a[NSC][EY][EX];      // cg_a: y; cg_b: p
    T c[NSC][EY][EX];      // cg_a: p_old
    T r[NSC][TY][TX];      // cg_b: r
    T d[NSC][TY][TX];      // cg_b: d
};

// part A: p_new = y + beta p_old on the tile, p_new^T A p_new (Alg. 3 steps 11, 5);
// part B: d += alpha p, r -= alpha A p, ||r||^2 (steps 6-8)
template <typename T, bool PART_A>
__global__ void __launch_bounds__(THREADS) k3s_cg(Params P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CgSmem<T>& S = *reinterpret_cast<CgSmem<T>*>(smem_raw);
    __shared__ T mus[MAX_MU];
    __shared__ int zk[ZK];
    __shared__ double red[32];
    const Geo& g = P.g;
    const int ntx = (g.mx + TX - 1) / TX, nty = (g.my + TY - 1) / TY;
    const int ntiles = tiles3(g);
    const long long plane = (long long)g.mx * g.my;
    const int cnt = P.lcnt[L_ITER];
    const long long total = (long long)cnt * ntiles;
    const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        const int slot = (int)(w / ntiles), tile = (int)(w % ntiles);
        const int q = P.lidx[L_ITER * P.Bmax + slot];
        const QState& s = P.st[q];
        if (s.phase != PH_ITER) continue;          // uniform across the CTA
        const int tx0 = (tile % ntx) * TX;
        const int ty0 = ((tile / ntx) % nty) * TY;
        const int z0 = (tile / (ntx * nty)) * ZC;
        const int z1 = min(z0 + ZC, g.mz);
        __syncthreads();
        if (threadIdx.x < P.n_mu) mus[threadIdx.x] = (T)P.mu[(size_t)q * P.n_mu + threadIdx.x];
        fill_zkeys(zk, g, z0);
        const T beta = (T)s.beta;
        const T alpha = (T)s.alpha;
        const bool use_old = PART_A && beta != T(0);
        const size_t qn = (size_t)q * g.n;
        const T* va = PART_A ? reinterpret_cast<const T*>(P.y) + qn
                             : reinterpret_cast<const T*>(P.p) + ((size_t)q * 2 + s.ppar) * (size_t)g.n;
        const T* vc = reinterpret_cast<const T*>(P.p) + ((size_t)q * 2 + s.ppar) * (size_t)g.n;   // p_old (A)
        T* pnew = reinterpret_cast<T*>(P.p) + ((size_t)q * 2 + (s.ppar ^ 1)) * (size_t)g.n;
        T* rr = reinterpret_cast<T*>(P.r) + qn;
        T* dd = P.mixed ? reinterpret_cast<T*>(P.d) + qn : reinterpret_cast<T*>(P.x64 + qn);
        StagePlan<EX, EY> p1;
        StagePlan<TX, TY> p0;
        p1.init(g, tx0 - 1, ty0 - 1);
        if (!PART_A) p0.init(g, tx0, ty0);
        auto stage = [&](int k) {
            const int sl = wrap(k, NSC);
            if (k <= z1) {
                p1.stage(&S.a[sl][0][0], va, g, k);
                if (use_old) p1.stage(&S.c[sl][0][0], vc, g, k);
                if (!PART_A && k >= z0 && k < z1) {
                    p0.stage(&S.r[sl][0][0], rr, g, k);
                    p0.stage(&S.d[sl][0][0], dd, g, k);
                }
            }
            cp_commit();
        };
        // the operand of the stencil at E1 position (ex, ey) of plane k
        auto opv = [&](int k, int ex, int ey) -> T {
            const int sl = wrap(k, NSC);
            if (PART_A) return use_old ? S.a[sl][ey][ex] + beta * S.c[sl][ey][ex] : S.a[sl][ey][ex];
            return S.a[sl][ey][ex];
        };
        for (int k = z0 - 1; k <= z0 + 1; ++k) stage(k);
        Coef<T> c;
        int ckey = -1;
        T acc = T(0);
        const int ix = tx0 + lx, iy = ty0 + ly;
        const bool inside = ix < g.mx && iy < g.my;
        for (int z = z0; z < z1; ++z) {
            stage(z + 2);           // into the slot of plane z-2, last read before the previous barrier
            cp_wait<1>();           // planes up to z+1 (and mus, zk)
            __syncthreads();
            if (inside) {
                const long long i = ix + (long long)g.mx * iy + plane * z;
                cached_coef(g, mus, ix, iy, z, zk[z - z0 + 2], c, ckey);
                const T pi = opv(z, lx + 1, ly + 1);
                T sum = T(0);
                if (ix > 0) sum += c.kxm * opv(z, lx, ly + 1);
                if (ix < g.mx - 1) sum += c.kxp * opv(z, lx + 2, ly + 1);
                if (iy > 0) sum += c.kym * opv(z, lx + 1, ly);
                if (iy < g.my - 1) sum += c.kyp * opv(z, lx + 1, ly + 2);
                if (z > 0) sum += c.kzm * opv(z - 1, lx + 1, ly + 1);
                if (z < g.mz - 1) sum += c.kzp * opv(z + 1, lx + 1, ly + 1);
                const T api = c.diag * pi - sum;
                if constexpr (PART_A) {
                    pnew[i] = pi;
                    acc += pi * api;
                } else {
                    const int sl = wrap(z, NSC);
                    dd[i] = S.d[sl][ly][lx] + alpha * pi;
                    const T rv = S.r[sl][ly][lx] - alpha * api;
                    rr[i] = rv;
                    acc += rv * rv;
                }
            }
            __syncthreads();
        }
        cp_wait<0>();
        double v = bsum(acc, red);
        if (arrive(P, q, tile, ntiles, &v, 1)) {
            double tot;
            gather_partials(P, q, ntiles, 1, &tot, red);
            if (threadIdx.x == 0) {
                if constexpr (PART_A) finalize_cg_a_state(P, q, tot);
                else finalize_cg_b_state(P, q, tot);
                P.tick[q] = 0;
            }
        }
    }
}

template <typename K>
void allow_smem(K kernel, size_t bytes) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

bool use_zmarch_smoother(const Geo& g) { return g.dim == 3 && tiles3(g) <= tiles_flat(g.n); }

template <typename T>
void launch3d_smooth_staged(const Params& P, const Launch& L, int nu) {
    if (use_ztile(P.g, sizeof(T) == 8) && launch3d_smooth_tile<T>(P, L, nu)) return;
    if (P.g.nf > 0) {   // the kernels below take block coefficients only
        launch_smoother<T>(P, L, nu, false);
        return;
    }
    static bool configured = false;
    const size_t sm = sizeof(SmoothSmem<T>);
    if (!configured) {
        allow_smem(k3s_smooth<T, true>, sm);
        allow_smem(k3s_smooth<T, false>, sm);
        configured = true;
    }
    T* ypro = reinterpret_cast<T*>(P.ypro);
    T* tmp = reinterpret_cast<T*>(P.tmp);
    T* out = reinterpret_cast<T*>(P.y);
    const int sweeps = nu < 1 ? 1 : nu;
    const T* src = ypro;
    for (int s = 1; s <= sweeps; ++s) {
        const bool last = s == sweeps;
        T* dst = last ? out : ((s & 1) ? tmp : ypro);
        if (last) k3s_smooth<T, true><<<L.grid, THREADS, sm, L.s>>>(P, src, dst);
        else k3s_smooth<T, false><<<L.grid, THREADS, sm, L.s>>>(P, src, dst);
        src = dst;
    }
}
template void launch3d_smooth_staged<float>(const Params&, const Launch&, int);
template void launch3d_smooth_staged<double>(const Params&, const Launch&, int);

template <typename T>
void launch3d_cg_a(const Params& P, const Launch& L) {
    if (use_ztile(P.g, sizeof(T) == 8) && launch3d_cg_tile<T>(P, L, true)) return;
    if (P.g.nf > 0) {
        launch_cg_a<T>(P, L);
        return;
    }
    static bool configured = false;
    if (!configured) {
        allow_smem(k3s_cg<T, true>, sizeof(CgSmem<T>));
        configured = true;
    }
    k3s_cg<T, true><<<L.grid, THREADS, sizeof(CgSmem<T>), L.s>>>(P);
}
template <typename T>
void launch3d_cg_b(const Params& P, const Launch& L) {
    if (use_ztile(P.g, sizeof(T) == 8) && launch3d_cg_tile<T>(P, L, false)) return;
    if (P.g.nf > 0) {
        launch_cg_b<T>(P, L);
        return;
    }
    static bool configured = false;
    if (!configured) {
        allow_smem(k3s_cg<T, false>, sizeof(CgSmem<T>));
        configured = true;
    }
    k3s_cg<T, false><<<L.grid, THREADS, sizeof(CgSmem<T>), L.s>>>(P);
}
template void launch3d_cg_a<float>(const Params&, const Launch&);
template void launch3d_cg_a<double>(const Params&, const Launch&);
template void launch3d_cg_b<float>(const Params&, const Launch&);
template void launch3d_cg_b<double>(const Params&, const Launch&);

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
