// The CG body (Alg. 3 steps 5-8 and 11) and the red-black Gauss-Seidel smoother
// S(A, r, y) (eq. 8) on 3D grids, marching in z over tiles of whole x-rows.
//
// Plan.  A work item is one query x one tile of TY rows in y (all mx points of
// each row) x one chunk of planes in z.  Thread (tx, tr) owns the points
// x0 = 4 tx .. 4 tx + 3 of row y = y0 + tr (smoother: y0 - 1 + tr) in every
// plane, and the CTA marches down z one plane per step with ONE CTA barrier
// per step.  The rows of a plane that a step needs reach shared memory as ONE
// tensor copy per array (cp.async.bulk.tensor, a box of whole rows of a 4D map
// [query][z][y][x], completion on an mbarrier), issued by a producer lane that
// runs RING-2 planes ahead, its cursor continuing into the next work item; rows
// and planes outside the grid arrive as zeros (the map's out-of-bounds fill),
// the Dirichlet neighbours x = -1 and x = mx are zero by selection.  (One copy
// per row instead runs into the copy engine's request rate on rows this short.)
// Each thread keeps its own
// points of planes z-1, z, z+1 in registers (a window over z); the y
// neighbours (rows y +- 1) and the two x neighbours across the thread's edges
// come from the staged planes.  A stage is read in its own step and the next
// one (LAG 2).
//
// CG part A: stage z = (y, p_old) of plane z+1 on rows y0-1 .. y0+TY.  Step z
//   forms p_new = y + beta p_old of plane z+1 at the thread's points (window,
//   written out) and applies A at plane z; the y and x neighbours of plane z are
//   rebuilt from stage z-1 with the same expression.  Accumulates p^T A p.
// CG part B: stage z = p of plane z+1 on rows y0-1 .. y0+TY, and r, d of plane z
//   on the tile rows.  Step z applies A to p at plane z: d += alpha p,
//   r -= alpha A p, ||r||^2.
// Smoother: thread rows cover y0-1 .. y0+TY (the tile and one halo row on each
//   side).  Stage z = source of plane z+2 on rows y0-2 .. y0+TY+1, b = r of
//   plane z+1 on rows y0-1 .. y0+TY [, direction p of plane z+1 for the last
//   sweep under Polak-Ribiere].  Step z computes the new RED values of plane
//   z+1 (red: x + y + z even) from old black source values (own points of planes
//   z, z+2 from the register window, rows y +- 1 of plane z+1 and the x edges
//   from stage z-1), keeps them in a window and writes them to a shared row
//   buffer of plane z+1; then the BLACK values of plane z (tile rows only) from
//   the new red values: own points of planes z-1, z+1 (window), rows y +- 1 and
//   x edges of plane z (row buffer written in the previous step).  The halo
//   rows compute red values only: each CTA recomputes the red values its black
//   points need, so no value depends on another CTA of the same launch.  The
//   columns a thread updates alternate with the parity of y + z; the thread
//   mapping puts rows of one parity in each warp, so the branch on it is
//   uniform.  The last sweep also accumulates r^T y and (A p)^T y.
// Colour order, neighbour sets and face coefficients are those of the generic
// kernels; a point is updated as (b + sum of kappa_f v_j) / diag with the
// reciprocal of the diagonal formed once per coefficient set.
//
// Every mbarrier wait is bounded in time (rb_stage.cuh): on expiry the device
// error flag is raised, the CTA keeps its barriers matched, drains its copies
// (bounded) and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "rb_stage.cuh"

namespace rbk {

using namespace stg;

namespace {

// FP32 consumer threads per CTA at most and copies in flight per CTA (build-time tunables)
#ifndef RB_Z_THREADS32
#define RB_Z_THREADS32 448
#endif
#ifndef RB_Z_FLIGHT_KB
#define RB_Z_FLIGHT_KB 96
#endif
constexpr int ZRING_MIN = 4;    // stages (planes) in the ring: at least 4, ...
constexpr int ZRING_MAX = 10;
constexpr size_t ZFLIGHT = (size_t)RB_Z_FLIGHT_KB * 1024;   // ... and about this many bytes in flight per CTA
constexpr int ZMAX_MX = 256;    // row length limit of these kernels
// consumer threads at most (FP32 / FP64), plus one producer warp: 15 (8) warps keep 4 (2)
// warps per SM sub-partition, 128 (255) registers per thread
template <typename T> constexpr int zmax_consumers() { return sizeof(T) == 4 ? RB_Z_THREADS32 : 224; }
// two FP32 CTAs per SM when they fit in the register file (each then keeps half the shared memory)
template <typename T> constexpr int zmin_blocks() { return sizeof(T) == 4 && RB_Z_THREADS32 <= 224 ? 2 : 1; }
template <typename T> constexpr size_t zsmem_cap() {
    return zmin_blocks<T>() == 2 ? 110u * 1024u : 200u * 1024u;
}

// Shape of a launch, fixed on the host per geometry and kernel kind.
struct ZPlan {
    int txp;         // thread columns per row: mx/4 rounded up to 16 or a multiple of 32
    int rows;        // thread rows: TY (CG) or TY + 2 (smoother)
    int ty;          // tile rows in y (even)
    int nthr;        // consumer threads = txp * rows (a multiple of 32)
    int ntile_y;     // tiles per plane column
    int pad;         // 16 bytes in elements (red row buffer of the smoother)
    int rsr;         // red row buffer stride in elements (mx + 2 pad)
    int a_rows, b_rows, c_rows;   // rows of the boxes of the three staged arrays (0: unused)
    int ring;                     // stages in the ring (a stage is read in two steps, the rest are in flight)
    uint32_t off_a, off_b, off_c; // element offsets of the arrays in a stage (128-byte aligned)
    size_t stage_elems, ring_elems, rbuf_elems, bytes;
};

constexpr int ZLEAD = 128;   // bytes before the ring (reads at x0-1 of a first row stay inside)

template <typename T>
size_t zalign(size_t elems) {   // round up to a multiple of 128 bytes
    const size_t q = 128 / sizeof(T);
    return (elems + q - 1) / q * q;
}

// outer = true: the FP64 outer residual (only x with its halo rows is staged)
template <typename T>
ZPlan zplan(const Geo& g, bool smoother, bool last, bool outer = false) {
    ZPlan z{};
    const int tx = g.mx / 4;
    z.txp = tx <= 16 ? 16 : ((tx + 31) / 32) * 32;
    const int max_thr = zmax_consumers<T>();
    int rows = max_thr / z.txp;
    if (z.txp == 16) rows &= ~3;          // row pairs of one parity per warp
    z.ty = smoother ? rows - 2 : rows;
    if (z.ty & 1) z.ty -= 1;               // tiles start on even rows
    if (z.ty > g.my + (g.my & 1)) z.ty = g.my + (g.my & 1);
    if (z.ty < 2) z.ty = 2;
    // 16 columns: warps pair two rows of one parity, so the thread rows come in fours
    if (z.txp == 16 && ((smoother ? z.ty + 2 : z.ty) & 3)) z.ty += 2;
    z.rows = smoother ? z.ty + 2 : z.ty;
    z.nthr = z.txp * z.rows;
    if (z.nthr % 32) z.nthr += 32 - z.nthr % 32;
    z.ntile_y = (g.my + z.ty - 1) / z.ty;
    z.pad = 16 / (int)sizeof(T);
    z.rsr = g.mx + 2 * z.pad;
    if (smoother) {            // a: source, b: b = r, c: direction p (last sweep)
        z.a_rows = z.ty + 4;
        z.b_rows = z.ty + 2;
        z.c_rows = last ? z.ty + 2 : 0;
    } else if (last) {         // part A: a: y, b: p_old
        z.a_rows = z.ty + 2;
        z.b_rows = z.ty + 2;
        z.c_rows = 0;
    } else if (outer) {        // outer residual: a: x
        z.a_rows = z.ty + 2;
        z.b_rows = 0;
        z.c_rows = 0;
    } else {                   // part B: a: p, b: r, c: d
        z.a_rows = z.ty + 2;
        z.b_rows = z.ty;
        z.c_rows = z.ty;
    }
    z.off_a = 0;
    z.off_b = (uint32_t)zalign<T>((size_t)z.a_rows * g.mx);
    z.off_c = z.off_b + (uint32_t)zalign<T>((size_t)z.b_rows * g.mx);
    z.stage_elems = z.off_c + zalign<T>((size_t)z.c_rows * g.mx);
    // the copies in flight per CTA (ring - 2 stages) hide the latency of HBM: a CTA keeps about
    // ZFLIGHT bytes in flight within 200 KB of shared memory
    z.rbuf_elems = smoother ? (size_t)2 * z.rows * z.rsr : 0;
    const size_t sb = z.stage_elems * sizeof(T);
    int ring = 2 + (int)((ZFLIGHT + sb - 1) / sb);
    ring = ring < ZRING_MIN ? ZRING_MIN : (ring > ZRING_MAX ? ZRING_MAX : ring);
    while (ring > ZRING_MIN && ZLEAD + (ring * z.stage_elems + z.rbuf_elems) * sizeof(T) + ring * sizeof(uint64_t) >
                                   zsmem_cap<T>())
        --ring;
    z.ring = ring;
    z.ring_elems = (size_t)ring * z.stage_elems;
    z.bytes = ZLEAD + (z.ring_elems + z.rbuf_elems) * sizeof(T) + ring * sizeof(uint64_t);
    return z;
}

// The tensor maps of a launch: 4D [queries][z][y][x] over a batch buffer, boxes of whole rows.
struct ZMaps {
    CUtensorMap a, b, c;
};

// thread -> (column tx, thread row tr); every warp holds rows of one parity
__device__ __forceinline__ void zmap(const ZPlan& z, int t, int& tx, int& tr) {
    if (z.txp == 16) {
        const int w = t >> 5, l = t & 31;
        tx = l & 15;
        tr = 4 * (w >> 1) + (w & 1) + 2 * (l >> 4);
    } else {
        tx = t % z.txp;
        tr = t / z.txp;
    }
}

// Chunk of planes per work item: whole columns unless the items would leave part of
// the grid idle; even (the march is unrolled by two) and within the partial-sum slots.
__device__ __forceinline__ int zchunk(const Geo& g, const ZPlan& z, int cnt, int max_tiles) {
    int zc = g.mz + (g.mz & 1);
    while (zc > 8 && (long long)cnt * z.ntile_y * ((g.mz + zc - 1) / zc) < 2LL * gridDim.x) zc = ((zc / 2) + 1) & ~1;
    while ((long long)z.ntile_y * ((g.mz + zc - 1) / zc) > max_tiles) zc *= 2;
    return zc;
}

// Face coefficients kappa_f / h^2 of the thread's 4 points in row y of plane k and the
// reciprocal diagonal (the definition of node_coef, four points at a time).
template <typename T>
struct ZCoef {
    T kx[5];   // kx[j]: face between points j-1 and j
    T kym[4], kyp[4], kzm[4], kzp[4], idiag[4];
};

template <typename T>
__device__ __forceinline__ void zcoef(const Geo& g, const T* mus, int x0, int y, int k, ZCoef<T>& c) {
    const int nbx = g.nbx, nbxy = g.nbx * g.nby, mx = g.mx;
    const int byc = __ldg(g.by + y), bzc = __ldg(g.bz + k);
    const bool up = y > 0, dn = y < g.my - 1, zb = k > 0, zf = k < g.mz - 1;
    const int bym = up ? __ldg(g.by + y - 1) : byc, byp = dn ? __ldg(g.by + y + 1) : byc;
    const int bzm = zb ? __ldg(g.bz + k - 1) : bzc, bzp = zf ? __ldg(g.bz + k + 1) : bzc;
    const int pc = nbx * byc + nbxy * bzc;
    int bxs[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) bxs[j] = __ldg(g.bx + min(max(x0 - 1 + j, 0), mx - 1));
    T m[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) m[j] = mus[bxs[j] + pc];
    const T hx = (T)g.ihx2, hy = (T)g.ihy2, hz = (T)g.ihz2, half = T(0.5);
    c.kx[0] = hx * (x0 > 0 ? half * (m[1] + m[0]) : m[1]);
#pragma unroll
    for (int j = 1; j < 4; ++j) c.kx[j] = hx * half * (m[j] + m[j + 1]);
    c.kx[4] = hx * (x0 + 4 < mx ? half * (m[4] + m[5]) : m[4]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const T mc = m[j + 1];
        const int bx = bxs[j + 1];
        c.kym[j] = hy * (up ? half * (mc + mus[bx + nbx * bym + nbxy * bzc]) : mc);
        c.kyp[j] = hy * (dn ? half * (mc + mus[bx + nbx * byp + nbxy * bzc]) : mc);
        c.kzm[j] = hz * (zb ? half * (mc + mus[bx + nbx * byc + nbxy * bzm]) : mc);
        c.kzp[j] = hz * (zf ? half * (mc + mus[bx + nbx * byc + nbxy * bzp]) : mc);
        T dg = c.kx[j] + c.kx[j + 1] + c.kym[j] + c.kyp[j];
        dg += c.kzm[j] + c.kzp[j];
        c.idiag[j] = T(1) / dg;
    }
}

template <typename T>
__device__ __forceinline__ V4t<T> ldg4(const T* p);
template <>
__device__ __forceinline__ V4t<float> ldg4<float>(const float* p) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p));
    return V4t<float>{{a.x, a.y, a.z, a.w}};
}
template <>
__device__ __forceinline__ V4t<double> ldg4<double>(const double* p) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p)), b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    return V4t<double>{{a.x, a.y, b.x, b.y}};
}

template <typename T>
__device__ __forceinline__ const T* query_kappa(const Geo& g, int q);
template <>
__device__ __forceinline__ const float* query_kappa<float>(const Geo& g, int q) { return g.kap32 + (size_t)q * g.n; }
template <>
__device__ __forceinline__ const double* query_kappa<double>(const Geo& g, int q) { return g.kap64 + (size_t)q * g.n; }

// zcoef for coefficient fields: the same face rule on the node values kappa(mu) of the query
// (kq), read around the thread's 4 points of row y, plane k (mostly L1 hits: neighbouring threads,
// rows and planes read the same values)
template <typename T>
__device__ __forceinline__ void zcoef_field(const Geo& g, const T* __restrict__ kq, int x0, int y, int k,
                                            ZCoef<T>& c) {
    const int mx = g.mx;
    const size_t plane = (size_t)mx * g.my;
    const size_t rb = (size_t)k * plane + (size_t)y * mx + x0;
    const bool left = x0 > 0, right = x0 + 4 < mx, up = y > 0, dn = y < g.my - 1, zb = k > 0, zf = k < g.mz - 1;
    const V4t<T> m = ldg4(kq + rb);
    const V4t<T> mu_ = up ? ldg4(kq + rb - mx) : m, md = dn ? ldg4(kq + rb + mx) : m;
    const V4t<T> mb = zb ? ldg4(kq + rb - plane) : m, mf = zf ? ldg4(kq + rb + plane) : m;
    const T ml = left ? __ldg(kq + rb - 1) : m.v[0], mr = right ? __ldg(kq + rb + 4) : m.v[3];
    const T hx = (T)g.ihx2, hy = (T)g.ihy2, hz = (T)g.ihz2, half = T(0.5);
    c.kx[0] = hx * (left ? half * (m.v[0] + ml) : m.v[0]);
#pragma unroll
    for (int j = 1; j < 4; ++j) c.kx[j] = hx * half * (m.v[j - 1] + m.v[j]);
    c.kx[4] = hx * (right ? half * (m.v[3] + mr) : m.v[3]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const T mc = m.v[j];
        c.kym[j] = hy * (up ? half * (mc + mu_.v[j]) : mc);
        c.kyp[j] = hy * (dn ? half * (mc + md.v[j]) : mc);
        c.kzm[j] = hz * (zb ? half * (mc + mb.v[j]) : mc);
        c.kzp[j] = hz * (zf ? half * (mc + mf.v[j]) : mc);
        T dg = c.kx[j] + c.kx[j + 1] + c.kym[j] + c.kyp[j];
        dg += c.kzm[j] + c.kzp[j];
        c.idiag[j] = T(1) / dg;
    }
}

// key of the z-dependence of a row's coefficients: the blocks of planes k-1, k, k+1
__device__ __forceinline__ int zkey(const Geo& g, int k) {
    if (k < 0 || k >= g.mz) return -1;
    const int c = __ldg(g.bz + k);
    const int m = k > 0 ? __ldg(g.bz + k - 1) : 0xFF;
    const int p = k < g.mz - 1 ? __ldg(g.bz + k + 1) : 0xFF;
    return c | (m << 8) | (p << 16);
}

// (A v) at point j of the thread from its plane window and the staged neighbours
template <typename T>
__device__ __forceinline__ T zapply(const ZCoef<T>& c, int j, const V4t<T>& vm, const V4t<T>& vc, const V4t<T>& vp,
                                    const V4t<T>& yu, const V4t<T>& yd, T left, T right) {
    const T xl = j == 0 ? left : vc.v[j - 1];
    const T xr = j == 3 ? right : vc.v[j + 1];
    const T dg = (c.kx[j] + c.kx[j + 1] + c.kym[j] + c.kyp[j]) + (c.kzm[j] + c.kzp[j]);
    return dg * vc.v[j] -
           (c.kx[j] * xl + c.kx[j + 1] * xr + c.kym[j] * yu.v[j] + c.kyp[j] * yd.v[j] + c.kzm[j] * vm.v[j] +
            c.kzp[j] * vp.v[j]);
}

// one box of whole rows: rows y .. y+box-1 of plane zz of query (map coordinate) qq
__device__ __forceinline__ void tma4d(void* dst, const CUtensorMap* m, uint64_t* bar, int y, int zz, int qq) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, "
        "%6}], [%2];" ::"r"(s2u(dst)),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(s2u(bar)), "r"(0), "r"(y), "r"(zz), "r"(qq)
        : "memory");
}

// After an expired wait: let the copies of the last `ring` stages land (bounded in time).
__device__ __forceinline__ void zdrain(uint64_t* bar, unsigned issued, unsigned ring, unsigned long long limit_ns) {
    const uint64_t t0 = gtime();
    const unsigned long long lim = limit_ns < DRAIN_NS ? limit_ns : DRAIN_NS;
    for (unsigned u = issued > ring ? issued - ring : 0u; u < issued; ++u)
        while (!mb_test(bar + u % ring, (u / ring) & 1u) && gtime() - t0 < lim) {
        }
}

// zero the red row buffers (their pads stay zero: the Dirichlet neighbours), init the barriers
template <typename T>
__device__ __forceinline__ void zsetup(const ZPlan& z, T* ring, uint64_t* bar) {
    for (size_t i = threadIdx.x; i < z.rbuf_elems; i += blockDim.x) ring[z.ring_elems + i] = T(0);
    if (threadIdx.x == 0) {
        for (int i = 0; i < z.ring; ++i) mb_init(bar + i, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
}

// staged value at column x of a row starting at p (zero outside the grid in x)
template <typename T>
__device__ __forceinline__ T xat(const T* row, int x, int mx) {
    return (x >= 0 && x < mx) ? row[x] : T(0);
}

// ---------------------------------------------------------------------------
// CG body.  PART_A: p_new = y + beta p_old, p^T A p.  Part B: d += alpha p,
// r -= alpha A p, ||r||^2.

template <typename T, bool PART_A, bool FIELD>
__global__ void __launch_bounds__(zmax_consumers<T>() + 32, zmin_blocks<T>()) k3z_cg(Params P, ZPlan z, const __grid_constant__ ZMaps maps) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ T mus[MAX_MU];
    __shared__ double red[32];
    const Geo& g = P.g;
    const int mx = g.mx;
    T* ring = reinterpret_cast<T*>(smem_raw + ZLEAD);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + ZLEAD + (z.ring_elems + z.rbuf_elems) * sizeof(T));
    const bool producer = (int)threadIdx.x >= z.nthr;
    const bool issuer = producer && (int)threadIdx.x == z.nthr;
    int tx = 0, tr = 0;
    if (!producer) zmap(z, threadIdx.x, tx, tr);
    const int x0 = 4 * tx;
    const bool col_ok = !producer && x0 < mx;
    zsetup<T>(z, ring, bar);

    const int cnt = P.lcnt[L_ITER];
    const int zc = zchunk(g, z, cnt, P.max_tiles);
    const int nchunk = (g.mz + zc - 1) / zc;
    const int per_q = z.ntile_y * nchunk;
    const long long total = (long long)cnt * per_q;
    const size_t plane = (size_t)mx * g.my;
    const uint32_t tbytes_a = (uint32_t)(z.a_rows * mx * sizeof(T));
    const uint32_t tbytes_b = (uint32_t)(z.b_rows * mx * sizeof(T));
    const uint32_t tbytes_c = (uint32_t)(z.c_rows * mx * sizeof(T));

    // ---- producer (one lane): cursor over (item, step); one stage = up to three tensor copies
    long long pw = blockIdx.x;
    int pz = 0, pz1 = 0, pz0 = 0, py0 = 0, pqa = 0, pqb = 0;
    bool puse_old = false;
    unsigned issued = 0, pslot = 0;   // stages issued, slot of the next one
    auto cursor_item = [&](long long w) {
        for (; w < total; w += gridDim.x) {
            const int slot = (int)(w / per_q), rem = (int)(w % per_q);
            const int q = P.lidx[L_ITER * P.Bmax + slot];
            const QState& s = P.st[q];
            if (s.phase != PH_ITER) continue;
            const int chunk = rem / z.ntile_y, yt = rem % z.ntile_y;
            py0 = yt * z.ty;
            pz0 = chunk * zc;
            pz1 = min(g.mz, pz0 + zc);
            pz = pz0 - 2;
            if (PART_A) {
                pqa = q;                   // y
                pqb = 2 * q + s.ppar;      // p_old
                puse_old = (T)s.beta != T(0);
            } else {
                pqa = 2 * q + s.ppar;      // p
                pqb = q;                   // r, d
            }
            break;
        }
        pw = w;
    };
    auto issue_next = [&]() {
        if (pw >= total) return;
        const unsigned u = issued++;
        (void)u;
        T* st = ring + (size_t)pslot * z.stage_elems;
        uint64_t* b = bar + pslot;
        if (++pslot == (unsigned)z.ring) pslot = 0;
        const int pl = pz + 1;   // plane of the stencil operand (out of the grid: zeros)
        if (PART_A) {
            mb_arrive_tx(b, tbytes_a + (puse_old ? tbytes_b : 0u));
            tma4d(st + z.off_a, &maps.a, b, py0 - 1, pl, pqa);
            if (puse_old) tma4d(st + z.off_b, &maps.b, b, py0 - 1, pl, pqb);
        } else {
            const bool rd = pz >= pz0;
            mb_arrive_tx(b, tbytes_a + (rd ? tbytes_b + tbytes_c : 0u));
            tma4d(st + z.off_a, &maps.a, b, py0 - 1, pl, pqa);
            if (rd) {
                tma4d(st + z.off_b, &maps.b, b, py0, pz, pqb);
                tma4d(st + z.off_c, &maps.c, b, py0, pz, pqb);
            }
        }
        if (++pz > pz1 - 1) cursor_item(pw + gridDim.x);
    };
    if (issuer) {
        cursor_item(blockIdx.x);
        for (int i = 0; i < z.ring; ++i) issue_next();
    }

    unsigned seq = 0, cs = 0, cph = 0;   // steps so far, slot and phase parity of the current stage
    bool ok = true;
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        const int slot = (int)(w / per_q), rem = (int)(w % per_q);
        const int q = P.lidx[L_ITER * P.Bmax + slot];
        const QState& s = P.st[q];
        if (s.phase != PH_ITER) continue;   // uniform across the CTA
        const int chunk = rem / z.ntile_y, yt = rem % z.ntile_y;
        const int y0 = yt * z.ty, z0 = chunk * zc, z1 = min(g.mz, z0 + zc);
        const int y = y0 + tr;
        const bool row_ok = col_ok && y < g.my;
        const T beta = (T)s.beta, alpha = (T)s.alpha;
        const bool use_old = PART_A && beta != T(0);
        const size_t qn = (size_t)q * g.n;
        T* pnew = reinterpret_cast<T*>(P.p) + ((size_t)q * 2 + (s.ppar ^ 1)) * (size_t)g.n;
        T* rg = reinterpret_cast<T*>(P.r) + qn;
        T* dg = (P.mixed ? reinterpret_cast<T*>(P.d) : reinterpret_cast<T*>(P.x64)) + qn;
        __syncthreads();
        for (int j = threadIdx.x; j < P.n_mu; j += blockDim.x) mus[j] = (T)P.mu[(size_t)q * P.n_mu + j];
        __syncthreads();
        V4t<T> vm = zero4<T>(), vc = zero4<T>(), vp = zero4<T>();
        ZCoef<T> c;
        int ckey = -2;
        T acc = T(0);
        const uint32_t own = (uint32_t)((tr + 1) * mx + x0);   // row y of the a (and b) box (rows from y0-1)
        for (int k = z0 - 2; k <= z1 - 1; ++k) {
            if (!producer) {
                const T* sg = ring + (size_t)cs * z.stage_elems;
                const T* sp = ring + (size_t)(cs == 0 ? z.ring - 1 : cs - 1) * z.stage_elems;   // stage k-1
                if (ok && !mb_wait(bar + cs, cph, P.err, P.wait_ns)) ok = false;
                if (col_ok) {
                    V4t<T> a = lds4(sg + z.off_a + own);
                    if (use_old) {
                        const V4t<T> b = lds4(sg + z.off_b + own);
#pragma unroll
                        for (int j = 0; j < 4; ++j) a.v[j] += beta * b.v[j];
                    }
                    if (PART_A && row_ok && k + 1 >= z0 && k + 1 < z1)
                        stg4(pnew + (size_t)(k + 1) * plane + (size_t)y * mx + x0, a);
                    vm = vc;
                    vc = vp;
                    vp = a;
                    if (k >= z0 && row_ok) {
                        if constexpr (FIELD) {
                            zcoef_field<T>(g, query_kappa<T>(g, q), x0, y, k, c);
                        } else {
                            const int kk = zkey(g, k);
                            if (kk != ckey) {
                                zcoef<T>(g, mus, x0, y, k, c);
                                ckey = kk;
                            }
                        }
                        // plane k neighbours from stage k-1: rows y-1, y+1 and the x edges of row y
                        const T* ra = sp + z.off_a + own;
                        V4t<T> yu = lds4(ra - mx), yd = lds4(ra + mx);
                        T left = x0 > 0 ? ra[-1] : T(0), right = x0 + 4 < mx ? ra[4] : T(0);
                        if (use_old) {
                            const T* rb = sp + z.off_b + own;
                            const V4t<T> bu = lds4(rb - mx), bd = lds4(rb + mx);
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                yu.v[j] += beta * bu.v[j];
                                yd.v[j] += beta * bd.v[j];
                            }
                            if (x0 > 0) left += beta * rb[-1];
                            if (x0 + 4 < mx) right += beta * rb[4];
                        }
                        if constexpr (PART_A) {
#pragma unroll
                            for (int j = 0; j < 4; ++j) acc += vc.v[j] * zapply(c, j, vm, vc, vp, yu, yd, left, right);
                        } else {
                            const uint32_t orow = (uint32_t)(tr * mx + x0);   // r, d boxes start at row y0
                            const V4t<T> rk = lds4(sg + z.off_b + orow);
                            const V4t<T> dk = lds4(sg + z.off_c + orow);
                            V4t<T> dn, rn;
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const T av = zapply(c, j, vm, vc, vp, yu, yd, left, right);
                                dn.v[j] = dk.v[j] + alpha * vc.v[j];
                                rn.v[j] = rk.v[j] - alpha * av;
                                acc += rn.v[j] * rn.v[j];
                            }
                            const size_t gi = (size_t)k * plane + (size_t)y * mx + x0;
                            stg4(dg + gi, dn);
                            stg4(rg + gi, rn);
                        }
                    }
                }
            }
            __syncthreads();
            // stage seq-1 had its last read in this step: refill its slot
            if (issuer && seq >= 1) issue_next();
            ++seq;
            if (++cs == (unsigned)z.ring) {
                cs = 0;
                cph ^= 1u;
            }
        }
        if (__syncthreads_or(!ok)) {
            if (issuer) zdrain(bar, issued, (unsigned)z.ring, P.wait_ns);
            __syncthreads();
            return;
        }
        double v[2];
        cta_sum2(acc, T(0), red, v);
        if (arrive(P, q, rem, per_q, v, 1)) {
            double tot;
            gather_partials(P, q, per_q, 1, &tot, red);
            if (threadIdx.x == 0) {
                if constexpr (PART_A) finalize_cg_a_state(P, q, tot);
                else finalize_cg_b_state(P, q, tot);
                P.tick[q] = 0;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Outer residual r = f(mu) - A(mu) x in FP64 (stored as TR), ||r||^2 and ||f||^2: the
// march of part B with x in place of p and the load terms read at the thread's points.

template <typename TR, bool FIELD>
__global__ void __launch_bounds__(zmax_consumers<double>() + 32) k3z_outer(Params P, ZPlan z,
                                                                            const __grid_constant__ ZMaps maps) {
    using T = double;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ T mus[MAX_MU];
    __shared__ double red[32];
    const Geo& g = P.g;
    const int mx = g.mx;
    T* ring = reinterpret_cast<T*>(smem_raw + ZLEAD);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + ZLEAD + (z.ring_elems + z.rbuf_elems) * sizeof(T));
    const bool producer = (int)threadIdx.x >= z.nthr;
    const bool issuer = producer && (int)threadIdx.x == z.nthr;
    int tx = 0, tr = 0;
    if (!producer) zmap(z, threadIdx.x, tx, tr);
    const int x0 = 4 * tx;
    const bool col_ok = !producer && x0 < mx;
    zsetup<T>(z, ring, bar);

    const int cnt = P.lcnt[L_OUT];
    const int zc = zchunk(g, z, cnt, P.max_tiles);
    const int nchunk = (g.mz + zc - 1) / zc;
    const int per_q = z.ntile_y * nchunk;
    const long long total = (long long)cnt * per_q;
    const size_t plane = (size_t)mx * g.my;
    const uint32_t tbytes_a = (uint32_t)(z.a_rows * mx * sizeof(T));

    // ---- producer (one lane): one tensor copy of x per stage
    long long pw = blockIdx.x;
    int pz = 0, pz1 = 0, py0 = 0, pq = 0;
    unsigned issued = 0, pslot = 0;
    auto cursor_item = [&](long long w) {
        for (; w < total; w += gridDim.x) {
            const int slot = (int)(w / per_q), rem = (int)(w % per_q);
            const int q = P.lidx[L_OUT * P.Bmax + slot];
            if (P.st[q].phase == PH_DONE) continue;
            const int chunk = rem / z.ntile_y, yt = rem % z.ntile_y;
            py0 = yt * z.ty;
            const int pz0 = chunk * zc;
            pz1 = min(g.mz, pz0 + zc);
            pz = pz0 - 2;
            pq = q;
            break;
        }
        pw = w;
    };
    auto issue_next = [&]() {
        if (pw >= total) return;
        ++issued;
        T* st = ring + (size_t)pslot * z.stage_elems;
        uint64_t* b = bar + pslot;
        if (++pslot == (unsigned)z.ring) pslot = 0;
        mb_arrive_tx(b, tbytes_a);
        tma4d(st + z.off_a, &maps.a, b, py0 - 1, pz + 1, pq);
        if (++pz > pz1 - 1) cursor_item(pw + gridDim.x);
    };
    if (issuer) {
        cursor_item(blockIdx.x);
        for (int i = 0; i < z.ring; ++i) issue_next();
    }

    unsigned seq = 0, cs = 0, cph = 0;
    bool ok = true;
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        const int slot = (int)(w / per_q), rem = (int)(w % per_q);
        const int q = P.lidx[L_OUT * P.Bmax + slot];
        if (P.st[q].phase == PH_DONE) continue;   // uniform across the CTA
        const int chunk = rem / z.ntile_y, yt = rem % z.ntile_y;
        const int y0 = yt * z.ty, z0 = chunk * zc, z1 = min(g.mz, z0 + zc);
        const int y = y0 + tr;
        const bool row_ok = col_ok && y < g.my;
        TR* rg = reinterpret_cast<TR*>(P.r) + (size_t)q * g.n;
        __syncthreads();
        for (int j = threadIdx.x; j < P.n_mu; j += blockDim.x) mus[j] = P.mu[(size_t)q * P.n_mu + j];
        __syncthreads();
        double phi[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) phi[r] = (r < P.R) ? (P.load_param[r] < 0 ? 1.0 : mus[P.load_param[r]]) : 0.0;
        V4t<T> vm = zero4<T>(), vc = zero4<T>(), vp = zero4<T>();
        ZCoef<T> c;
        int ckey = -2;
        double rr = 0.0, ff = 0.0;
        const uint32_t own = (uint32_t)((tr + 1) * mx + x0);
        for (int k = z0 - 2; k <= z1 - 1; ++k) {
            if (!producer) {
                const T* sg = ring + (size_t)cs * z.stage_elems;
                const T* sp = ring + (size_t)(cs == 0 ? z.ring - 1 : cs - 1) * z.stage_elems;   // stage k-1
                if (ok && !mb_wait(bar + cs, cph, P.err, P.wait_ns)) ok = false;
                if (col_ok) {
                    const V4t<T> a = lds4(sg + z.off_a + own);
                    vm = vc;
                    vc = vp;
                    vp = a;
                    if (k >= z0 && row_ok) {
                        if constexpr (FIELD) {
                            zcoef_field<T>(g, query_kappa<T>(g, q), x0, y, k, c);
                        } else {
                            const int kk = zkey(g, k);
                            if (kk != ckey) {
                                zcoef<T>(g, mus, x0, y, k, c);
                                ckey = kk;
                            }
                        }
                        const T* ra = sp + z.off_a + own;
                        const V4t<T> yu = lds4(ra - mx), yd = lds4(ra + mx);
                        const T left = x0 > 0 ? ra[-1] : T(0), right = x0 + 4 < mx ? ra[4] : T(0);
                        const size_t gi = (size_t)k * plane + (size_t)y * mx + x0;
                        // f(mu) at the 4 points (same summation order as the generic kernel)
                        double f[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
                        for (int r = 0; r < 8; ++r) {
                            if (r >= P.R) break;
                            const V4t<double> fr = ldg4(P.fr + (size_t)r * g.n + gi);
#pragma unroll
                            for (int j = 0; j < 4; ++j) f[j] += phi[r] * fr.v[j];
                        }
                        V4t<TR> o;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const double rv = f[j] - zapply(c, j, vm, vc, vp, yu, yd, left, right);
                            o.v[j] = (TR)rv;
                            rr += rv * rv;
                            ff += f[j] * f[j];
                        }
                        stg4(rg + gi, o);
                    }
                }
            }
            __syncthreads();
            if (issuer && seq >= 1) issue_next();
            ++seq;
            if (++cs == (unsigned)z.ring) {
                cs = 0;
                cph ^= 1u;
            }
        }
        if (__syncthreads_or(!ok)) {
            if (issuer) zdrain(bar, issued, (unsigned)z.ring, P.wait_ns);
            __syncthreads();
            return;
        }
        double v[2];
        cta_sum2(rr, ff, red, v);
        if (arrive(P, q, rem, per_q, v, 2)) {
            double tot[2];
            gather_partials(P, q, per_q, 2, tot, red);
            if (threadIdx.x == 0) {
                finalize_outer_state(P, q, tot[0], tot[1]);
                P.tick[q] = 0;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Smoother: one red-black sweep from src to dst (LAST: dst = y, r^T y and
// (A p)^T y accumulated and the preconditioner finalised).

template <typename T, bool LAST, bool FIELD>
__global__ void __launch_bounds__(zmax_consumers<T>() + 32, zmin_blocks<T>()) k3z_smooth(Params P, ZPlan z, T* dst_base,
                                                                       const __grid_constant__ ZMaps maps) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ T mus[MAX_MU];
    __shared__ double red[32];
    const Geo& g = P.g;
    const int mx = g.mx;
    T* ring = reinterpret_cast<T*>(smem_raw + ZLEAD);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + ZLEAD + (z.ring_elems + z.rbuf_elems) * sizeof(T));
    T* rbuf = ring + z.ring_elems;   // [2][rows][rsr]: new red values of planes of each parity
    const bool producer = (int)threadIdx.x >= z.nthr;
    const bool issuer = producer && (int)threadIdx.x == z.nthr;
    int tx = 0, tr = 0;
    if (!producer) zmap(z, threadIdx.x, tx, tr);
    const int x0 = 4 * tx;
    const bool col_ok = !producer && x0 < mx && tr < z.rows;
    zsetup<T>(z, ring, bar);

    const int cnt = P.lcnt[L_PREC];
    const int zc = zchunk(g, z, cnt, P.max_tiles);
    const int nchunk = (g.mz + zc - 1) / zc;
    const int per_q = z.ntile_y * nchunk;
    const long long total = (long long)cnt * per_q;
    const size_t plane = (size_t)mx * g.my;
    const uint32_t tbytes_a = (uint32_t)(z.a_rows * mx * sizeof(T));
    const uint32_t tbytes_b = (uint32_t)(z.b_rows * mx * sizeof(T));
    const uint32_t tbytes_c = (uint32_t)(z.c_rows * mx * sizeof(T));

    // ---- producer cursor (one lane)
    long long pw = blockIdx.x;
    int pz = 0, pz1 = 0, pz0 = 0, py0 = 0, pq = 0, pqp = 0;
    bool pap = false;
    unsigned issued = 0, pslot = 0;   // stages issued, slot of the next one
    auto cursor_item = [&](long long w) {
        for (; w < total; w += gridDim.x) {
            const int slot = (int)(w / per_q), rem = (int)(w % per_q);
            const int q = P.lidx[L_PREC * P.Bmax + slot];
            const QState& s = P.st[q];
            const int chunk = rem / z.ntile_y, yt = rem % z.ntile_y;
            py0 = yt * z.ty;
            pz0 = chunk * zc;
            pz1 = min(g.mz, pz0 + zc);
            pz = pz0 - 4;
            pq = q;
            pqp = 2 * q + s.ppar;
            pap = LAST && P.beta_form == RB_BETA_PR && !s.start;
            break;
        }
        pw = w;
    };
    auto issue_next = [&]() {
        if (pw >= total) return;
        const unsigned u = issued++;
        (void)u;
        T* st = ring + (size_t)pslot * z.stage_elems;
        uint64_t* b = bar + pslot;
        if (++pslot == (unsigned)z.ring) pslot = 0;
        const bool rb = pz >= pz0 - 2;   // b (and p) of plane pz+1 are read from here on
        const bool rp = rb && pap;
        mb_arrive_tx(b, tbytes_a + (rb ? tbytes_b : 0u) + (rp ? tbytes_c : 0u));
        tma4d(st + z.off_a, &maps.a, b, py0 - 2, pz + 2, pq);
        if (rb) tma4d(st + z.off_b, &maps.b, b, py0 - 1, pz + 1, pq);
        if (rp) tma4d(st + z.off_c, &maps.c, b, py0 - 1, pz + 1, pqp);
        if (++pz > pz1 - 1) cursor_item(pw + gridDim.x);
    };
    if (issuer) {
        cursor_item(blockIdx.x);
        for (int i = 0; i < z.ring; ++i) issue_next();
    }

    unsigned seq = 0, cs = 0, cph = 0;   // steps so far, slot and phase parity of the current stage
    bool ok = true;
    for (long long w = blockIdx.x; w < total; w += gridDim.x) {
        const int slot = (int)(w / per_q), rem = (int)(w % per_q);
        const int q = P.lidx[L_PREC * P.Bmax + slot];
        const QState& s = P.st[q];
        const int chunk = rem / z.ntile_y, yt = rem % z.ntile_y;
        const int y0 = yt * z.ty, z0 = chunk * zc, z1 = min(g.mz, z0 + zc);
        const int y = y0 - 1 + tr;
        const bool in_y = col_ok && y >= 0 && y < g.my;
        const bool tile_row = in_y && tr >= 1 && tr <= z.ty;   // black update and output
        const bool need_ap = LAST && P.beta_form == RB_BETA_PR && !s.start;
        T* dst = dst_base + (size_t)q * g.n;
        __syncthreads();
        for (int j = threadIdx.x; j < P.n_mu; j += blockDim.x) mus[j] = (T)P.mu[(size_t)q * P.n_mu + j];
        __syncthreads();
        // old black source values of planes k, k+1, k+2 at the columns that are red in plane k+1
        T sbm[2] = {T(0), T(0)}, sbc[2] = {T(0), T(0)}, sbp[2] = {T(0), T(0)};
        // new red values of planes k-1, k, k+1 at the columns that are black in plane k
        T zm[2] = {T(0), T(0)}, zcv[2] = {T(0), T(0)}, zp[2] = {T(0), T(0)};
        V4t<T> pm = zero4<T>(), pcv = zero4<T>(), pn = zero4<T>();   // direction, planes k-1, k, k+1
        ZCoef<T> cf[2];
        int key[2] = {-2, -2};
        T ry = T(0), apy = T(0);
        const int rowpar = (y + 1024) & 1;
        const uint32_t own_s = (uint32_t)((tr + 1) * mx + x0);   // source row y (box rows from y0-2)
        const uint32_t own_b = (uint32_t)(tr * mx + x0);         // b / p row y (box rows from y0-1)
        const uint32_t own_r = (uint32_t)(z.pad + tr * z.rsr + x0);   // red row buffer, row y
        const bool has_l = x0 > 0, has_r = x0 + 4 < mx;

        // one step; PZ = k & 1, RP = rowpar: columns J = (y + k + 1) & 1 + {0, 2} are red in
        // plane k+1 and black in plane k
        auto step = [&](auto pz_tag, auto rp_tag, int k) {
            constexpr int PZ = decltype(pz_tag)::value, RP = decltype(rp_tag)::value;
            constexpr int J0 = (RP + PZ + 1) & 1, J1 = J0 + 2;   // updated columns of this step
            constexpr int K0 = 1 - J0, K1 = K0 + 2;              // the other two
            const T* sg = ring + (size_t)cs * z.stage_elems;
            const T* sp = ring + (size_t)(cs == 0 ? z.ring - 1 : cs - 1) * z.stage_elems;   // stage k-1
            if (ok && !mb_wait(bar + cs, cph, P.err, P.wait_ns)) ok = false;
            if (col_ok) {
                // source plane k+2 at the columns J (black there)
                const V4t<T> s2 = lds4(sg + z.off_a + own_s);
                sbm[0] = sbc[0];
                sbm[1] = sbc[1];
                sbc[0] = sbp[0];
                sbc[1] = sbp[1];
                sbp[0] = s2.v[J0];
                sbp[1] = s2.v[J1];
                zm[0] = zcv[0];
                zm[1] = zcv[1];
                zcv[0] = zp[0];
                zcv[1] = zp[1];
                if (LAST && need_ap) {
                    pm = pcv;
                    pcv = pn;
                    pn = lds4(sg + z.off_c + own_b);
                }
            }
            const int kr = k + 1;   // plane of the red update
            if (col_ok && k >= z0 - 2) {
                // ---- red half-sweep of plane k+1 at columns J
                T n0 = T(0), n1 = T(0);
                if (in_y && kr >= 0 && kr < g.mz) {
                    if constexpr (FIELD) {
                        zcoef_field<T>(g, query_kappa<T>(g, q), x0, y, kr, cf[1 - PZ]);
                    } else {
                        const int kk = zkey(g, kr);
                        if (kk != key[1 - PZ]) {   // (k + 1) & 1 == 1 - PZ
                            zcoef<T>(g, mus, x0, y, kr, cf[1 - PZ]);
                            key[1 - PZ] = kk;
                        }
                    }
                    const ZCoef<T>& c = cf[1 - PZ];
                    // source plane k+1 (stage k-1): rows y-1, y+1 and the own row with its x edges
                    const T* rs1 = sp + z.off_a + own_s;
                    const V4t<T> su = lds4(rs1 - mx), sd = lds4(rs1 + mx);
                    const V4t<T> sc = lds4(rs1);
                    const V4t<T> bk = lds4(sg + z.off_b + own_b);   // b of plane k+1
                    const T halo_l = has_l ? rs1[-1] : T(0), halo_r = has_r ? rs1[4] : T(0);
                    // x neighbours of the red points J0, J1 are the black columns K of plane k+1
                    const T l0 = J0 == 0 ? halo_l : sc.v[J0 - 1];
                    const T r0 = sc.v[J0 + 1];
                    const T l1 = sc.v[J1 - 1];
                    const T r1 = J1 == 3 ? halo_r : sc.v[J1 + 1];
                    n0 = bk.v[J0] + c.kx[J0] * l0 + c.kx[J0 + 1] * r0 + c.kym[J0] * su.v[J0] + c.kyp[J0] * sd.v[J0] +
                         c.kzm[J0] * sbm[0] + c.kzp[J0] * sbp[0];
                    n1 = bk.v[J1] + c.kx[J1] * l1 + c.kx[J1 + 1] * r1 + c.kym[J1] * su.v[J1] + c.kyp[J1] * sd.v[J1] +
                         c.kzm[J1] * sbm[1] + c.kzp[J1] * sbp[1];
                    n0 *= c.idiag[J0];
                    n1 *= c.idiag[J1];
                }
                zp[0] = n0;
                zp[1] = n1;
                T* rbw = rbuf + (size_t)(1 - PZ) * z.rows * z.rsr + own_r;
                rbw[J0] = n0;
                rbw[J1] = n1;
                // ---- black half-sweep of plane k at columns J (tile rows)
                if (tile_row && k >= z0) {
                    const ZCoef<T>& c = cf[PZ];
                    const T* rc = rbuf + (size_t)PZ * z.rows * z.rsr + own_r;   // red values of plane k
                    const V4t<T> ru = lds4(rc - z.rsr), rd = lds4(rc + z.rsr);
                    const T rl = rc[-1], rr = rc[4];   // the pads hold zeros
                    const V4t<T> bk = lds4(sp + z.off_b + own_b);   // b of plane k (stage k-1)
                    // x neighbours of J0, J1: columns K of plane k (red there) -> zcv; edges -> buffer
                    const T l0 = J0 == 0 ? rl : (K0 == J0 - 1 ? zcv[0] : zcv[1]);
                    const T r0 = K0 == J0 + 1 ? zcv[0] : zcv[1];
                    const T l1 = K0 == J1 - 1 ? zcv[0] : zcv[1];
                    const T r1 = J1 == 3 ? rr : zcv[1];
                    T b0 = bk.v[J0] + c.kx[J0] * l0 + c.kx[J0 + 1] * r0 + c.kym[J0] * ru.v[J0] + c.kyp[J0] * rd.v[J0] +
                           c.kzm[J0] * zm[0] + c.kzp[J0] * zp[0];
                    T b1 = bk.v[J1] + c.kx[J1] * l1 + c.kx[J1 + 1] * r1 + c.kym[J1] * ru.v[J1] + c.kyp[J1] * rd.v[J1] +
                           c.kzm[J1] * zm[1] + c.kzp[J1] * zp[1];
                    b0 *= c.idiag[J0];
                    b1 *= c.idiag[J1];
                    V4t<T> out;
                    out.v[J0] = b0;
                    out.v[J1] = b1;
                    out.v[K0] = zcv[0];
                    out.v[K1] = zcv[1];
                    stg4(dst + (size_t)k * plane + (size_t)y * mx + x0, out);
                    if constexpr (LAST) {
#pragma unroll
                        for (int j = 0; j < 4; ++j) ry += bk.v[j] * out.v[j];
                        if (need_ap) {
                            // direction plane k: rows y-1, y+1 and the x edges from stage k-1
                            const T* rp1 = sp + z.off_c + own_b;
                            const V4t<T> pu = lds4(rp1 - mx), pd = lds4(rp1 + mx);
                            const T pl = has_l ? rp1[-1] : T(0), pr = has_r ? rp1[4] : T(0);
#pragma unroll
                            for (int j = 0; j < 4; ++j) apy += zapply(c, j, pm, pcv, pn, pu, pd, pl, pr) * out.v[j];
                        }
                    }
                }
            }
            __syncthreads();
            if (issuer && seq >= 1) issue_next();
            ++seq;
            if (++cs == (unsigned)z.ring) {
                cs = 0;
                cph ^= 1u;
            }
        };
        // steps k = z0-4 .. z1-1 (z0 even): the first two only load the source planes z0-2, z0-1
        for (int k = z0 - 4; k <= z1 - 1; k += 2) {
            if (rowpar) step(Par0{}, Par1{}, k);
            else step(Par0{}, Par0{}, k);
            if (k + 1 <= z1 - 1) {
                if (rowpar) step(Par1{}, Par1{}, k + 1);
                else step(Par1{}, Par0{}, k + 1);
            }
        }
        if (__syncthreads_or(!ok)) {
            if (issuer) zdrain(bar, issued, (unsigned)z.ring, P.wait_ns);
            __syncthreads();
            return;
        }
        if constexpr (LAST) {
            double v[2];
            cta_sum2(ry, apy, red, v);
            if (arrive(P, q, rem, per_q, v, 2)) {
                double tot[2];
                gather_partials(P, q, per_q, 2, tot, red);
                if (threadIdx.x == 0) {
                    finalize_prec_state(P, q, tot[0], tot[1]);
                    P.tick[q] = 0;
                }
            }
        }
    }
}

template <typename K>
int zgrid(K kernel, int threads, size_t smem) {
    return resident(kernel, threads, smem);
}

PFN_cuTensorMapEncodeTiled_v12000 zencode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
        looked_up = true;
    }
    return fn;
}

// 4D map [nq][mz][my][mx] over a batch buffer, boxes of `rows` whole rows of one plane;
// out-of-bounds elements arrive as zeros.  An unused array gets a valid map over the same base.
template <typename T>
bool zencode(CUtensorMap* m, const void* base, const Geo& g, long long nq, int rows) {
    auto fn = zencode_fn();
    if (!fn || !base) return false;
    const cuuint64_t es = sizeof(T);
    cuuint64_t dims[4] = {(cuuint64_t)g.mx, (cuuint64_t)g.my, (cuuint64_t)g.mz, (cuuint64_t)nq};
    cuuint64_t strides[3] = {(cuuint64_t)g.mx * es, (cuuint64_t)g.mx * g.my * es, (cuuint64_t)g.n * es};
    cuuint32_t box[4] = {(cuuint32_t)g.mx, (cuuint32_t)(rows > 0 ? rows : 1), 1, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(m, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
              const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool outer_fits(const Geo& g) {
    const ZPlan z = zplan<double>(g, false, false, true);
    return z.bytes <= zsmem_cap<double>() && z.nthr <= zmax_consumers<double>() &&
           (long long)z.ntile_y <= tiles_flat(g.n) && z.a_rows <= 256;
}

template <typename T>
bool ztile_fits(const Geo& g) {
    for (int kind = 0; kind < 4; ++kind) {
        const ZPlan z = zplan<T>(g, kind < 2, (kind & 1) != 0);
        if (z.bytes > zsmem_cap<T>() || z.nthr > zmax_consumers<T>() || (long long)z.ntile_y > tiles_flat(g.n) ||
            z.a_rows > 256)
            return false;
    }
    return true;
}

}  // namespace

// 3D grids whose rows hold a multiple of 4 points (8 .. 256) and whose stages and thread
// rows fit, for the precision of the launch (and the tensor-map encoder is available)
bool use_ztile(const Geo& g, bool fp64) {
    if (g.dim != 3 || g.mx % 4 != 0 || g.mx > ZMAX_MX || g.mx < 8 || g.my < 2) return false;
    if (g.n >= (1LL << 31) || !zencode_fn()) return false;
    return fp64 ? ztile_fits<double>(g) : ztile_fits<float>(g);
}

bool use_ztile_outer(const Geo& g) {
    if (g.dim != 3 || g.mx % 4 != 0 || g.mx > ZMAX_MX || g.mx < 8 || g.my < 2) return false;
    if (g.n >= (1LL << 31) || !zencode_fn() || (g.nf > 0 && !g.kap64)) return false;
    return outer_fits(g);
}


// FIELD: coefficient fields (kappa(mu) read per row and plane) instead of block coefficients
template <typename T, bool FIELD>
void cg_tile_launch(const Params& P, const Launch& L, const ZPlan& z, const ZMaps& maps, bool part_a) {
    const int threads = z.nthr + 32;
    static size_t conf[2] = {0, 0};
    static int grid[2] = {0, 0};
    const int i = part_a ? 0 : 1;
    if (conf[i] != z.bytes) {
        grid[i] = part_a ? zgrid(k3z_cg<T, true, FIELD>, threads, z.bytes)
                         : zgrid(k3z_cg<T, false, FIELD>, threads, z.bytes);
        conf[i] = z.bytes;
    }
    if (part_a) k3z_cg<T, true, FIELD><<<grid[i], threads, z.bytes, L.s>>>(P, z, maps);
    else k3z_cg<T, false, FIELD><<<grid[i], threads, z.bytes, L.s>>>(P, z, maps);
}

template <typename T, bool FIELD>
void smooth_tile_launch(const Params& P, const Launch& L, const ZPlan& zl, const ZPlan& zi, const ZMaps& m_ypro,
                        const ZMaps& m_tmp, int nu) {
    T* ypro = reinterpret_cast<T*>(P.ypro);
    T* tmp = reinterpret_cast<T*>(P.tmp);
    T* out = reinterpret_cast<T*>(P.y);
    static size_t conf[2] = {0, 0};
    static int grid[2] = {0, 0};
    if (conf[0] != zl.bytes) {
        grid[0] = zgrid(k3z_smooth<T, true, FIELD>, zl.nthr + 32, zl.bytes);
        conf[0] = zl.bytes;
    }
    if (conf[1] != zi.bytes) {
        grid[1] = zgrid(k3z_smooth<T, false, FIELD>, zi.nthr + 32, zi.bytes);
        conf[1] = zi.bytes;
    }
    const int sweeps = nu < 1 ? 1 : nu;
    const T* src = ypro;
    for (int s = 1; s <= sweeps; ++s) {
        const bool last = s == sweeps;
        T* dst = last ? out : ((s & 1) ? tmp : ypro);
        const ZMaps& m = src == ypro ? m_ypro : m_tmp;
        if (last) k3z_smooth<T, true, FIELD><<<grid[0], zl.nthr + 32, zl.bytes, L.s>>>(P, zl, dst, m);
        else k3z_smooth<T, false, FIELD><<<grid[1], zi.nthr + 32, zi.bytes, L.s>>>(P, zi, dst, m);
        src = dst;
    }
}

template <typename TR, bool FIELD>
void outer_tile_launch(const Params& P, const Launch& L, const ZPlan& z, const ZMaps& maps) {
    const int threads = z.nthr + 32;
    static size_t conf = 0;
    static int grid = 0;
    if (conf != z.bytes) {
        grid = zgrid(k3z_outer<TR, FIELD>, threads, z.bytes);
        conf = z.bytes;
    }
    k3z_outer<TR, FIELD><<<grid, threads, z.bytes, L.s>>>(P, z, maps);
}

template <typename T>
bool launch3d_cg_tile(const Params& P, const Launch& L, bool part_a) {
    const ZPlan z = zplan<T>(P.g, false, part_a);
    ZMaps maps;
    const Geo& g = P.g;
    bool ok;
    if (part_a) {
        ok = zencode<T>(&maps.a, P.y, g, P.Bmax, z.a_rows) && zencode<T>(&maps.b, P.p, g, 2LL * P.Bmax, z.b_rows);
        maps.c = maps.b;
    } else {
        const void* d = P.mixed ? P.d : (const void*)P.x64;
        ok = zencode<T>(&maps.a, P.p, g, 2LL * P.Bmax, z.a_rows) && zencode<T>(&maps.b, P.r, g, P.Bmax, z.b_rows) &&
             zencode<T>(&maps.c, d, g, P.mixed ? P.Bmax : P.B, z.c_rows);
    }
    if (!ok) return false;
    if (g.nf > 0) cg_tile_launch<T, true>(P, L, z, maps, part_a);
    else cg_tile_launch<T, false>(P, L, z, maps, part_a);
    return true;
}
template bool launch3d_cg_tile<float>(const Params&, const Launch&, bool);
template bool launch3d_cg_tile<double>(const Params&, const Launch&, bool);

// nu sweeps ypro -> tmp -> ypro ... -> y, as the generic smoother
template <typename T>
bool launch3d_smooth_tile(const Params& P, const Launch& L, int nu) {
    const Geo& g = P.g;
    const ZPlan zl = zplan<T>(g, true, true), zi = zplan<T>(g, true, false);
    T* ypro = reinterpret_cast<T*>(P.ypro);
    T* tmp = reinterpret_cast<T*>(P.tmp);
    ZMaps m_ypro, m_tmp;
    if (!zencode<T>(&m_ypro.a, ypro, g, P.Bmax, zl.a_rows) || !zencode<T>(&m_ypro.b, P.r, g, P.Bmax, zl.b_rows) ||
        !zencode<T>(&m_ypro.c, P.p, g, 2LL * P.Bmax, zl.c_rows) || !zencode<T>(&m_tmp.a, tmp, g, P.Bmax, zl.a_rows))
        return false;
    m_tmp.b = m_ypro.b;
    m_tmp.c = m_ypro.c;
    if (g.nf > 0) smooth_tile_launch<T, true>(P, L, zl, zi, m_ypro, m_tmp, nu);
    else smooth_tile_launch<T, false>(P, L, zl, zi, m_ypro, m_tmp, nu);
    return true;
}
template bool launch3d_smooth_tile<float>(const Params&, const Launch&, int);
template bool launch3d_smooth_tile<double>(const Params&, const Launch&, int);


// FP64 outer residual on the tiles; r stored as TR (FP32 for the mixed solver)
template <typename TR>
bool launch3d_outer_tile(const Params& P, const Launch& L) {
    const ZPlan z = zplan<double>(P.g, false, false, true);
    ZMaps maps;
    if (!zencode<double>(&maps.a, P.x64, P.g, P.B, z.a_rows)) return false;
    maps.b = maps.a;
    maps.c = maps.a;
    if (P.g.nf > 0) outer_tile_launch<TR, true>(P, L, z, maps);
    else outer_tile_launch<TR, false>(P, L, z, maps);
    return true;
}
template bool launch3d_outer_tile<float>(const Params&, const Launch&);
template bool launch3d_outer_tile<double>(const Params&, const Launch&);

}  // namespace rbk
