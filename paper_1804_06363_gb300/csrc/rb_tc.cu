// Tensor-core engine of the mixed-precision preconditioner (see rb_tc.cuh).
//
// Both products are dense GEMMs once queries are batched:
//   projection    P[s] (128 queries x n) = R (128 x K-slice of points) * W32c^T
//                 split-K over the points (partials reduced in FP64 by the
//                 reduced-solve kernel, fixed order), one CTA per (query tile,
//                 split);
//   prolongation  Y^T (128 points x 128 queries) = W32r tile (128 x n) * E^T,
//                 one CTA per (query tile, range of point tiles), accumulators
//                 double-buffered in TMEM so the epilogue of one tile overlaps
//                 the MMAs of the next; the point is the TMEM lane, so stores of
//                 one query by a warp are contiguous.
// Operands are staged by TMA (128-byte swizzle) and consumed by
// tcgen05.mma.kind::tf32 issued by one thread; accumulators live in TMEM and
// are read back with tcgen05.ld by four epilogue warps.  Warp 0 is the TMA
// producer, warp 1 the MMA issuer, warps 2-5 the epilogue.  Every wait on an
// mbarrier is bounded in time: on expiry the kernel raises a device error flag,
// the other roles stop, in-flight copies are drained (bounded) and TMEM freed.
#include "rb_tc.cuh"

#include <cuda_bf16.h>

#include <cudaTypedefs.h>

#include <cstring>

namespace rbk {

namespace {

constexpr int TC_THREADS = 192;
constexpr uint64_t WAIT_NS = 2000000000ull;   // 2 s
constexpr uint64_t DRAIN_NS = 500000000ull;   // 0.5 s

__device__ __forceinline__ uint32_t s2u(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ uint64_t gtime() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s2u(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s2u(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s2u(b)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(s2u(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase with the given parity; false if another thread already gave
// up (err set) or the wait expired (then err is set here).
__device__ bool mbar_wait(uint64_t* b, uint32_t parity, int* err) {
    if (mbar_test(b, parity)) return true;
    const uint64_t t0 = gtime();
    while (true) {
        if (mbar_test(b, parity)) return true;
        if (*(volatile int*)err) return false;
        if (gtime() - t0 > WAIT_NS) {
            atomicExch(err, 1);
            return false;
        }
    }
}
// Bounded wait used only while draining after an error.
__device__ void mbar_drain(uint64_t* b, uint32_t parity) {
    const uint64_t t0 = gtime();
    while (!mbar_test(b, parity) && gtime() - t0 < DRAIN_NS) {
    }
}

__device__ __forceinline__ void tma2d(void* dst, const CUtensorMap* m, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
        "[%2];" ::"r"(s2u(dst)),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(s2u(bar)), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s2u(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void umma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s2u(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes grouped in 8-row (1024-byte) atoms.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4)      // start address
           | ((uint64_t)1 << 16)                    // leading-dimension offset (unused for swizzled K-major)
           | ((uint64_t)(1024 >> 4) << 32)          // stride between 8-row atoms
           | ((uint64_t)1 << 46)                    // descriptor version
           | ((uint64_t)2 << 61);                   // 128-byte swizzle
}
// Instruction descriptor, kind::tf32: D f32, A and B tf32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ unsigned char* align1024(unsigned char* p) {
    return reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// true in all threads if a query of rows [q0, q0+128) is waiting for the preconditioner
__device__ __forceinline__ bool tile_active(const Params& P, int q0) {
    int mine = 0;
    if (threadIdx.x < 128) {
        const int q = q0 + threadIdx.x;
        mine = (q < P.B && P.st[q].phase == PH_PREC) ? 1 : 0;
    }
    return __syncthreads_or(mine) != 0;
}

// ---------------------------------------------------------------------------
// projection: proj[split][q][k] = sum over the split's points of r_q[i] W[i][k]

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_project(const __grid_constant__ CUtensorMap tm_r, const __grid_constant__ CUtensorMap tm_wc, Params P,
                 int nsplit, int stages, long long kblocks, int* err) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = align1024(smem_raw);
    const int nbp = P.nbp;
    const uint32_t a_bytes = 128 * 128;
    const uint32_t b_bytes = (uint32_t)nbp * 128;
    unsigned char* sA = sm;
    unsigned char* sB = sm + (size_t)stages * a_bytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + (size_t)stages * b_bytes);
    uint64_t* empty = full + stages;
    uint64_t* done = empty + stages;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    const uint32_t tcols = nbp <= 32 ? 32 : (nbp <= 64 ? 64 : 128);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mtile = blockIdx.x / nsplit, sp = blockIdx.x % nsplit;
    const int q0 = mtile * 128;
    if (!tile_active(P, q0)) return;
    const long long per = (kblocks + nsplit - 1) / nsplit;
    const long long kb0 = (long long)sp * per;
    const long long kb1 = kb0 + per < kblocks ? kb0 + per : kblocks;
    const int nk = kb1 > kb0 ? (int)(kb1 - kb0) : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tslot, tcols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            int last_use[8];
            for (int s = 0; s < 8; ++s) last_use[s] = -1;
            for (int i = 0; i < nk; ++i) {
                const int s = i % stages;
                const int use = i / stages;
                if (use > 0 && !mbar_wait(empty + s, (use - 1) & 1, err)) break;
                mbar_expect_tx(full + s, a_bytes + b_bytes);
                const int x = (int)((kb0 + i) * 32);
                tma2d(sA + (size_t)s * a_bytes, &tm_r, full + s, x, q0);
                tma2d(sB + (size_t)s * b_bytes, &tm_wc, full + s, x, 0);
                last_use[s] = use;
            }
            if (*(volatile int*)err) {
                for (int s = 0; s < stages && s < 8; ++s)
                    if (last_use[s] >= 0) mbar_drain(full + s, last_use[s] & 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(128, nbp);
            for (int i = 0; i < nk; ++i) {
                const int s = i % stages;
                const int use = i / stages;
                if (!mbar_wait(full + s, use & 1, err)) break;
                tc_fence_after();
                const uint64_t ad = sdesc_sw128(s2u(sA + (size_t)s * a_bytes));
                const uint64_t bd = sdesc_sw128(s2u(sB + (size_t)s * b_bytes));
#pragma unroll
                for (int j = 0; j < 4; ++j)   // K = 8 TF32 values (32 bytes) per MMA
                    umma_tf32(tmem, ad + 2 * j, bd + 2 * j, idesc, (i > 0 || j > 0) ? 1u : 0u);
                umma_commit(empty + s);
            }
            umma_commit(done);   // arrives once every MMA issued above has completed
        }
        __syncwarp();
    } else {
        const int quad = warp & 3;                 // TMEM lanes this warp may read
        const int q = q0 + quad * 32 + lane;
        bool ok = mbar_wait(done, 0, err);
        ok = __all_sync(0xffffffffu, ok);
        tc_fence_after();
        if (ok) {
            for (int c = 0; c < nbp; c += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c, v);
                if (q < P.B) {
                    double* dst = P.proj + ((size_t)sp * P.Bmax + q) * nbp + c;
#pragma unroll
                    for (int t = 0; t < 16; ++t) dst[t] = nk > 0 ? (double)v[t] : 0.0;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, tcols);
    }
}

// ---------------------------------------------------------------------------
// prolongation: ypro[q][i] = sum_k e[q][k] W[i][k]
// D (128 points x 128 queries) = W32r tile (points x K) * E tile (queries x K)^T:
// the TMEM lane is the point, so a warp's store for one query covers 32
// consecutive points (128 contiguous bytes).

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_prolong(const __grid_constant__ CUtensorMap tm_e, const __grid_constant__ CUtensorMap tm_wr, Params P,
                 int ctas_per_m, int stages, int ksub, int* err) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ int s_act[128];
    unsigned char* sm = align1024(smem_raw);
    constexpr uint32_t SUB = 128 * 128;   // one 128-row x 32-float swizzled sub-tile
    unsigned char* sE = sm;                                         // ksub sub-tiles (queries)
    unsigned char* sW = sm + (size_t)ksub * SUB;                    // stages x ksub sub-tiles (points)
    uint64_t* full = reinterpret_cast<uint64_t*>(sW + (size_t)stages * ksub * SUB);
    uint64_t* empty = full + stages;
    uint64_t* efull = empty + stages;
    uint64_t* tfull = efull + 1;     // [2]
    uint64_t* tempty = tfull + 2;    // [2]
    uint64_t* done = tempty + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    constexpr uint32_t TCOLS = 256;  // two 128-column accumulators

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mtile = blockIdx.x / ctas_per_m, c = blockIdx.x % ctas_per_m;
    const int q0 = mtile * 128;
    if (threadIdx.x < 128) {
        const int q = q0 + threadIdx.x;
        s_act[threadIdx.x] = (q < P.B && P.st[q].phase == PH_PREC) ? 1 : 0;
    }
    if (!__syncthreads_or(threadIdx.x < 128 ? s_act[threadIdx.x] : 0)) return;
    const long long n = P.g.n;
    const int nptiles = (int)((n + 127) / 128);
    const int per = (nptiles + ctas_per_m - 1) / ctas_per_m;
    const int p0 = c * per;
    const int p1 = p0 + per < nptiles ? p0 + per : nptiles;
    const int np = p1 > p0 ? p1 - p0 : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        mbar_init(efull, 1);
        mbar_init(tfull + 0, 1);
        mbar_init(tfull + 1, 1);
        mbar_init(tempty + 0, 4);
        mbar_init(tempty + 1, 4);
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tslot, TCOLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0 && np > 0) {
            int last_use[8];
            for (int s = 0; s < 8; ++s) last_use[s] = -1;
            mbar_expect_tx(efull, (uint32_t)ksub * SUB);
            for (int k = 0; k < ksub; ++k) tma2d(sE + (size_t)k * SUB, &tm_e, efull, 32 * k, q0);
            for (int i = 0; i < np; ++i) {
                const int s = i % stages;
                const int use = i / stages;
                if (use > 0 && !mbar_wait(empty + s, (use - 1) & 1, err)) break;
                mbar_expect_tx(full + s, (uint32_t)ksub * SUB);
                for (int k = 0; k < ksub; ++k)
                    tma2d(sW + ((size_t)s * ksub + k) * SUB, &tm_wr, full + s, 32 * k, (p0 + i) * 128);
                last_use[s] = use;
            }
            if (*(volatile int*)err) {
                mbar_drain(efull, 0);
                for (int s = 0; s < stages && s < 8; ++s)
                    if (last_use[s] >= 0) mbar_drain(full + s, last_use[s] & 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(128, 128);
            bool ok = np > 0 ? mbar_wait(efull, 0, err) : false;
            for (int i = 0; ok && i < np; ++i) {
                const int s = i % stages;
                const int use = i / stages;
                const int ab = i & 1;
                if (!mbar_wait(full + s, use & 1, err)) break;
                if (i >= 2 && !mbar_wait(tempty + ab, ((i >> 1) - 1) & 1, err)) break;
                tc_fence_after();
                for (int k = 0; k < ksub; ++k) {
                    const uint64_t ad = sdesc_sw128(s2u(sW + ((size_t)s * ksub + k) * SUB));
                    const uint64_t bd = sdesc_sw128(s2u(sE + (size_t)k * SUB));
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        umma_tf32(tmem + (uint32_t)(ab * 128), ad + 2 * j, bd + 2 * j, idesc,
                                  (k > 0 || j > 0) ? 1u : 0u);
                }
                umma_commit(empty + s);
                umma_commit(tfull + ab);
            }
            umma_commit(done);
        }
        __syncwarp();
    } else {
        const int quad = warp & 3;
        const int prow = quad * 32 + lane;          // point within the tile (TMEM lane)
        float* ybase = reinterpret_cast<float*>(P.ypro) + (size_t)q0 * n;
        __nv_bfloat16* hbase = reinterpret_cast<__nv_bfloat16*>(P.ypro) + (size_t)q0 * n;   // BF16 storage
        const bool bf = P.ybf16 != 0;
        for (int i = 0; i < np; ++i) {
            const int ab = i & 1;
            bool ok = mbar_wait(tfull + ab, (i >> 1) & 1, err);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            tc_fence_after();
            const long long pt = (long long)(p0 + i) * 128 + prow;
            const bool inside = pt < n;
            for (int cc = 0; cc < 128; cc += 16) {
                float v[16];
                tmem_ld16(tmem + (uint32_t)(ab * 128) + ((uint32_t)(quad * 32) << 16) + (uint32_t)cc, v);
                if (inside) {
                    if (bf) {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (s_act[cc + j])
                                __stcs(reinterpret_cast<unsigned short*>(hbase + (size_t)(cc + j) * n + pt),
                                       __bfloat16_as_ushort(__float2bfloat16_rn(v[j])));
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (s_act[cc + j]) __stcs(ybase + (size_t)(cc + j) * n + pt, v[j]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty + ab);
        }
        if (np > 0) {
            if (lane == 0) mbar_drain(done, 0);
            __syncwarp();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, TCOLS);
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

bool make_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t outer, uint32_t box_inner, uint32_t box_outer) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {inner * sizeof(float)};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

rb_status tc_init(TcPlan& t, const Geo& g, int Bmax, int nb_cap, int nbp, int nbp32, int num_sms, float* r32,
                  const float* W32c, float* e32, const float* W32r, int* d_err, std::string& err) {
    t = TcPlan{};
    t.Bmax = Bmax;
    t.nbp = nbp;
    t.nbp32 = nbp32;
    t.num_sms = num_sms;
    t.n = g.n;
    t.d_err = d_err;
    // the engine needs 16-byte aligned rows of whole 32-point blocks and at most 128 basis vectors
    if (g.n % 32 != 0 || nb_cap < 1 || nbp > 128 || nbp % 16 != 0 || nbp32 > 128 || nbp32 % 32 != 0) return RB_OK;
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10) return RB_OK;
    t.mtiles = (Bmax + 127) / 128;
    const uint64_t N = (uint64_t)g.n;
    if (!make_map(&t.tm_r, r32, N, (uint64_t)Bmax, 32, 128) || !make_map(&t.tm_wc, W32c, N, (uint64_t)nbp, 32, nbp) ||
        !make_map(&t.tm_e, e32, (uint64_t)nbp32, (uint64_t)Bmax, 32, 128) ||
        !make_map(&t.tm_wr, W32r, (uint64_t)nbp32, N, 32, 128)) {
        cudaGetLastError();
        return RB_OK;   // no tensor maps: stay on the CUDA-core engine
    }
    const size_t budget = 200 * 1024;
    const size_t pstage = 128 * 128 + (size_t)nbp * 128;
    t.proj_stages = (int)std::min<size_t>(6, budget / pstage);
    t.proj_smem = t.proj_stages * pstage + 1024 + 2 * 8 * 8 + 64;
    const int ksub = nbp32 / 32;
    const size_t sub = 128 * 128;
    t.prol_stages = (int)std::min<size_t>(4, (budget - ksub * sub) / (ksub * sub));
    t.prol_smem = (ksub + (size_t)t.prol_stages * ksub) * sub + 1024 + 8 * 8 + 8 * 8 + 64;
    if (t.proj_stages < 2 || t.prol_stages < 2) return RB_OK;
    t.proj_split = std::max(1, num_sms / t.mtiles);
    t.prol_ctas = std::max(1, num_sms / t.mtiles);
    if (cudaFuncSetAttribute(k_tc_project, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t.proj_smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_tc_prolong, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t.prol_smem) !=
            cudaSuccess) {
        cudaGetLastError();
        return RB_OK;
    }
    (void)err;
    t.ready = true;
    return RB_OK;
}

void tc_free(TcPlan& t) { t.ready = false; }

bool tc_usable(const TcPlan& t, int n) { return t.ready && n > 0; }

void tc_project(const TcPlan& t, const Params& P, const Launch& L) {
    const long long kblocks = (t.n + 31) / 32;
    k_tc_project<<<t.mtiles * t.proj_split, TC_THREADS, t.proj_smem, L.s>>>(t.tm_r, t.tm_wc, P, t.proj_split,
                                                                            t.proj_stages, kblocks, t.d_err);
}

void tc_prolong(const TcPlan& t, const Params& P, const Launch& L) {
    k_tc_prolong<<<t.mtiles * t.prol_ctas, TC_THREADS, t.prol_smem, L.s>>>(t.tm_e, t.tm_wr, P, t.prol_ctas,
                                                                           t.prol_stages, t.nbp32 / 32, t.d_err);
}

}  // namespace rbk
