// C interface of librb (include/rb.h): context set-up, the batched solve
// drivers, the offline greedy and the basis file.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "rb_common.cuh"
#include "rb_tc.cuh"

using namespace rbk;

namespace {

thread_local std::string g_create_error;

struct DevBuf {
    void* p = nullptr;
};

}  // namespace

namespace rbk {
// error text of calls that have no context (read back by rb_last_error(NULL))
void set_global_error(const std::string& m) { g_create_error = m; }

PtrKind pointer_kind(const void* p) {
    if (!p) return PTR_HOST;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return PTR_HOST;
    }
    if (a.type == cudaMemoryTypeManaged) return PTR_DEVICE;
    if (a.type != cudaMemoryTypeDevice) return PTR_HOST;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return PTR_OTHER_DEVICE;
    }
    return a.device == dev ? PTR_DEVICE : PTR_OTHER_DEVICE;
}

rb_status validate_problem(const rb_problem* prob, std::string& why) {
    if (!prob) { why = "problem is NULL"; return RB_EINVAL; }
    if (prob->dim != 2 && prob->dim != 3) { why = "dim must be 2 or 3"; return RB_EINVAL; }
    if (prob->n_fields < 0 || prob->n_fields > MAX_P || (prob->n_fields > 0 && !prob->fields)) {
        why = "n_fields must be in 0..64, with a field array when positive";
        return RB_EINVAL;
    }
    long long P = 1;
    for (int d = 0; d < 3; ++d) {
        if (prob->m[d] < 1 || prob->nb[d] < 1 || prob->nb[d] > prob->m[d]) {
            why = "grid sizes must be >= 1 and blocks must lie in 1..m per direction";
            return RB_EINVAL;
        }
        P *= prob->nb[d];
    }
    if (prob->dim == 2 && (prob->m[2] != 1 || prob->nb[2] != 1)) { why = "dim 2 needs m[2] = nb[2] = 1"; return RB_EINVAL; }
    if (P > MAX_P) { why = "too many blocks (max 64)"; return RB_EINVAL; }
    if (prob->n_fields > 0) {
        if (P != 1) { why = "a problem with coefficient fields has one block per direction"; return RB_EINVAL; }
        P = prob->n_fields;
    }
    if ((long long)prob->m[0] * prob->m[1] * prob->m[2] >= (1LL << 31)) { why = "grid too large (N_dof >= 2^31)"; return RB_EINVAL; }
    if (prob->n_loads < 1 || prob->n_loads > MAX_LOADS || !prob->loads) { why = "need 1..8 load terms"; return RB_EINVAL; }
    if (prob->n_mu < P || prob->n_mu > MAX_MU) { why = "n_mu must be in P..128"; return RB_EINVAL; }
    for (int r = 0; r < prob->n_loads; ++r) {
        const rb_load& l = prob->loads[r];
        if (l.kind < RB_LOAD_CONST || l.kind > RB_LOAD_BOUNDARY) { why = "unknown load kind"; return RB_EINVAL; }
        if (l.param >= prob->n_mu || l.param < -1) { why = "load parameter index out of range"; return RB_EINVAL; }
        if (l.kind == RB_LOAD_GAUSS && !(l.sigma > 0.0)) { why = "Gaussian load needs sigma > 0"; return RB_EINVAL; }
        if (l.kind >= RB_LOAD_ARRAY && !l.values) { why = "array and boundary loads need values"; return RB_EINVAL; }
        if (l.kind == RB_LOAD_BOUNDARY && (l.field < 0 || l.field >= P)) {
            why = "boundary load field index out of range";
            return RB_EINVAL;
        }
    }
    return RB_OK;
}

}  // namespace rbk

struct rb_ctx {
    // problem
    int dim = 2, m[3] = {1, 1, 1}, nbk[3] = {1, 1, 1}, P = 1, R = 1, n_mu = 1;
    long long N = 0;
    std::vector<rb_load> loads;                 // values point into load_vals
    std::vector<std::vector<double>> load_vals; // copies of the array / boundary loads' values
    int load_param[MAX_LOADS] = {0};
    int n_fields = 0;                           // coefficient fields (0: blocks)
    std::vector<double> h_fields;               // [Q][N] copy of the fields
    double* d_kf64 = nullptr;
    float* d_kf32 = nullptr;
    Geo geo{};
    int *d_bx = nullptr, *d_by = nullptr, *d_bz = nullptr, *d_rkey = nullptr;
    double* d_fr = nullptr;
    // basis
    int n = 0, n_cap = 0, nbp = 16, nbp32 = 32;
    double* d_W64c = nullptr;
    float* d_W32c = nullptr;
    float* d_W32r = nullptr;
    double* d_ANq = nullptr;
    double* d_fNr = nullptr;
    std::vector<double> h_ANq, h_fNr, h_Rsnap;
    std::vector<int> selected;
    // workspace
    int Bmax = 1;
    double* d_x64 = nullptr;
    double *d_r64 = nullptr, *d_p64 = nullptr, *d_y64 = nullptr, *d_ypro64 = nullptr, *d_tmp64 = nullptr;
    float *d_r32 = nullptr, *d_p32 = nullptr, *d_y32 = nullptr, *d_ypro32 = nullptr, *d_tmp32 = nullptr,
          *d_d32 = nullptr;
    double* d_e64 = nullptr;
    float* d_e32 = nullptr;
    double* d_L = nullptr;
    double* d_mu = nullptr;
    QState* d_st = nullptr;
    double* d_part = nullptr;
    int max_tiles = 1;
    double* d_proj = nullptr;
    int nsplit = 1;
    unsigned* d_tick = nullptr;
    int* d_lcnt = nullptr;
    int* d_lidx = nullptr;
    int* d_ndone = nullptr;
    int* d_done = nullptr;            // finished queries in finishing order
    double* d_scratch = nullptr;      // offline helpers
    size_t scratch_bytes = 0;
    TcPlan tc{};                      // tensor-core projection plans
    int* d_tcerr = nullptr;           // set by a tensor-core kernel whose wait expired
    int* d_flag = nullptr;            // breakdown flag of rb_warm_start
    int nsplit_max = 1;
    bool force_generic = false;       // testing: use the generic stencil kernels everywhere
    unsigned long long wait_ns = 2000000000ull;   // limit of the kernels' bounded waits (rb_debug_wait)
    long long dbg_skip = -1;                      // test hook of rb_debug_wait
    // error basis of the learned warm start (rb_error_basis): V [m_err][N], FP64 and FP32
    int m_err = 0;
    double* d_V64 = nullptr;
    float* d_V32 = nullptr;
    // the captured graph of the last solve (reused while its launch parameters stay the same)
    cudaGraphExec_t graph_exec = nullptr;
    std::vector<unsigned char> graph_key;
    cudaStream_t graph_stream = nullptr;
    // per-kernel timing (rb_profile)
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<std::pair<int, size_t>> prof_pending;   // (kernel kind, first event index)
    double prof_ms[32] = {0};
    long long prof_launches[32] = {0};
    // host
    QState* h_st = nullptr;
    int* h_ndone = nullptr;
    int* h_err = nullptr;             // device error flag polled with the done counter
    int* h_done = nullptr;
    cudaStream_t own_stream = nullptr;
    cudaStream_t copy_stream = nullptr;   // solutions of finished queries to host buffers
    int num_sms = 1;
    int grid = 1;
    std::string err;
    std::vector<void*> allocs;
};

namespace {

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);               \
            return RB_ECUDA;                                                             \
        }                                                                                \
    } while (0)

#define CK_GLOBAL(call)                                                                  \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            g_create_error = std::string(#call) + ": " + cudaGetErrorString(e_);         \
            return RB_ECUDA;                                                             \
        }                                                                                \
    } while (0)

template <typename T>
rb_status dalloc(rb_ctx* ctx, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->err = "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed: " + cudaGetErrorString(e);
        *p = nullptr;
        return RB_ENOMEM;
    }
    ctx->allocs.push_back((void*)*p);
    return RB_OK;
}

#define TRY(x)                        \
    do {                              \
        rb_status s_ = (x);           \
        if (s_ != RB_OK) return s_;   \
    } while (0)

// true for device (or managed) memory of the current device, false for host
// memory; a buffer on another device sets ctx->err and *bad
bool is_device_ptr(rb_ctx* ctx, const void* p, bool* bad) {
    const PtrKind k = pointer_kind(p);
    if (k == PTR_OTHER_DEVICE) {
        ctx->err = "a buffer lives on another device than the current one";
        *bad = true;
    }
    return k == PTR_DEVICE;
}

int pad_to(int v, int m) { return ((v + m - 1) / m) * m; }

// Allocate everything of a context for basis capacity n_cap and batch Bmax.
// f(i) = sum over the faces of node i to a boundary node j of F_q(i) g(j) / h_d^2 (the lift of the
// Dirichlet data g through field q); g on the grid extended by the boundary layer, x fastest.  In a
// block problem F_q is the indicator of block q.
void boundary_lift(const rb_ctx* ctx, int q, const double* gext, const std::vector<int> (&maps)[3],
                   std::vector<double>& f) {
    const int mx = ctx->m[0], my = ctx->m[1], mz = ctx->m[2], d3 = ctx->dim == 3;
    const long long N = ctx->N;
    f.assign(N, 0.0);
    const long long ex = mx + 2, exy = ex * (my + 2);
    auto G = [&](int ex_, int ey_, int ez_) { return gext[ex_ + ex * ey_ + exy * (d3 ? ez_ : 0)]; };
    auto F = [&](int ix, int iy, int iz) -> double {
        const long long i = ix + (long long)mx * (iy + (long long)my * iz);
        if (ctx->n_fields > 0) return ctx->h_fields[(size_t)q * N + i];
        const int p = maps[0][ix] + ctx->nbk[0] * (maps[1][iy] + ctx->nbk[1] * maps[2][iz]);
        return p == q ? 1.0 : 0.0;
    };
    const double ihx2 = (double)(mx + 1) * (mx + 1), ihy2 = (double)(my + 1) * (my + 1),
                 ihz2 = (double)(mz + 1) * (mz + 1);
    for (int iz = 0; iz < mz; ++iz)
        for (int iy = 0; iy < my; ++iy)
            for (int ix = 0; ix < mx; ++ix) {
                const bool bx0 = ix == 0, bx1 = ix == mx - 1, by0 = iy == 0, by1 = iy == my - 1;
                const bool bz0 = d3 && iz == 0, bz1 = d3 && iz == mz - 1;
                if (!(bx0 || bx1 || by0 || by1 || bz0 || bz1)) continue;
                const int ez = iz + 1;   // extended-grid indices of the node
                double s = 0.0;
                if (bx0) s += ihx2 * G(0, iy + 1, ez);
                if (bx1) s += ihx2 * G(mx + 1, iy + 1, ez);
                if (by0) s += ihy2 * G(ix + 1, 0, ez);
                if (by1) s += ihy2 * G(ix + 1, my + 1, ez);
                if (bz0) s += ihz2 * G(ix + 1, iy + 1, 0);
                if (bz1) s += ihz2 * G(ix + 1, iy + 1, mz + 1);
                f[ix + (long long)mx * (iy + (long long)my * iz)] = F(ix, iy, iz) * s;
            }
}

rb_status ctx_init(rb_ctx* ctx, const rb_problem* prob, int n_cap, int max_batch) {
    ctx->dim = prob->dim;
    for (int d = 0; d < 3; ++d) { ctx->m[d] = prob->m[d]; ctx->nbk[d] = prob->nb[d]; }
    ctx->n_fields = prob->n_fields;
    ctx->P = prob->n_fields > 0 ? prob->n_fields : prob->nb[0] * prob->nb[1] * prob->nb[2];
    ctx->R = prob->n_loads;
    ctx->n_mu = prob->n_mu;
    ctx->N = (long long)prob->m[0] * prob->m[1] * prob->m[2];
    ctx->loads.assign(prob->loads, prob->loads + prob->n_loads);
    ctx->load_vals.assign(prob->n_loads, std::vector<double>());
    for (int r = 0; r < ctx->R; ++r) {
        rb_load& l = ctx->loads[r];
        if (l.kind == RB_LOAD_ARRAY) {
            ctx->load_vals[r].assign(l.values, l.values + ctx->N);
        } else if (l.kind == RB_LOAD_BOUNDARY) {
            const size_t ext = (size_t)(prob->m[0] + 2) * (prob->m[1] + 2) * (prob->dim == 3 ? prob->m[2] + 2 : 1);
            ctx->load_vals[r].assign(l.values, l.values + ext);
        }
        l.values = l.kind >= RB_LOAD_ARRAY ? ctx->load_vals[r].data() : nullptr;
        if (l.kind != RB_LOAD_BOUNDARY) l.field = 0;
    }
    if (ctx->n_fields > 0) ctx->h_fields.assign(prob->fields, prob->fields + (size_t)ctx->n_fields * ctx->N);
    for (int r = 0; r < ctx->R; ++r) ctx->load_param[r] = prob->loads[r].param;
    ctx->n_cap = n_cap;
    ctx->nbp = std::max(16, pad_to(n_cap, 16));
    ctx->nbp32 = std::max(32, pad_to(n_cap, 32));
    ctx->Bmax = max_batch;
    const long long N = ctx->N;
    const int B = max_batch;

    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev));
    ctx->grid = ctx->num_sms * 8;
    CK(cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamDefault));

    // geometry and block maps
    std::vector<int> maps[3];
    for (int d = 0; d < 3; ++d) {
        maps[d].resize(ctx->m[d]);
        for (int i = 0; i < ctx->m[d]; ++i) maps[d][i] = (int)(((long long)i * ctx->nbk[d]) / ctx->m[d]);
    }
    TRY(dalloc(ctx, &ctx->d_bx, ctx->m[0]));
    TRY(dalloc(ctx, &ctx->d_by, ctx->m[1]));
    TRY(dalloc(ctx, &ctx->d_bz, ctx->m[2]));
    CK(cudaMemcpy(ctx->d_bx, maps[0].data(), ctx->m[0] * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_by, maps[1].data(), ctx->m[1] * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_bz, maps[2].data(), ctx->m[2] * sizeof(int), cudaMemcpyHostToDevice));
    {
        std::vector<int> rk(ctx->m[1]);
        const std::vector<int>& by = maps[1];
        for (int k = 0; k < ctx->m[1]; ++k)
            rk[k] = by[k] | ((k > 0 ? by[k - 1] : 0xFF) << 8) | ((k < ctx->m[1] - 1 ? by[k + 1] : 0xFF) << 16);
        TRY(dalloc(ctx, &ctx->d_rkey, ctx->m[1]));
        CK(cudaMemcpy(ctx->d_rkey, rk.data(), ctx->m[1] * sizeof(int), cudaMemcpyHostToDevice));
    }
    Geo& g = ctx->geo;
    g.dim = ctx->dim;
    g.mx = ctx->m[0]; g.my = ctx->m[1]; g.mz = ctx->m[2];
    g.nbx = ctx->nbk[0]; g.nby = ctx->nbk[1]; g.nbz = ctx->nbk[2];
    g.P = ctx->P;
    g.n = N;
    g.ihx2 = (double)(g.mx + 1) * (g.mx + 1);
    g.ihy2 = (double)(g.my + 1) * (g.my + 1);
    g.ihz2 = ctx->dim == 3 ? (double)(g.mz + 1) * (g.mz + 1) : 0.0;
    g.bx = ctx->d_bx; g.by = ctx->d_by; g.bz = ctx->d_bz; g.rkey = ctx->d_rkey;
    if (ctx->n_fields > 0) {
        const size_t QN = (size_t)ctx->n_fields * N;
        TRY(dalloc(ctx, &ctx->d_kf64, QN));
        TRY(dalloc(ctx, &ctx->d_kf32, QN));
        CK(cudaMemcpy(ctx->d_kf64, ctx->h_fields.data(), QN * sizeof(double), cudaMemcpyHostToDevice));
        std::vector<float> f32(ctx->h_fields.begin(), ctx->h_fields.end());
        CK(cudaMemcpy(ctx->d_kf32, f32.data(), QN * sizeof(float), cudaMemcpyHostToDevice));
        g.nf = ctx->n_fields;
        g.kf64 = ctx->d_kf64;
        g.kf32 = ctx->d_kf32;
        if (ctx->dim == 3) {   // per-query node coefficients for the 3D tile kernels
            double* k64;
            float* k32;
            TRY(dalloc(ctx, &k64, (size_t)B * N));
            TRY(dalloc(ctx, &k32, (size_t)B * N));
            g.kap64 = k64;
            g.kap32 = k32;
        }
    }

    // load terms
    TRY(dalloc(ctx, &ctx->d_fr, (size_t)ctx->R * N));
    {
        std::vector<int> kind(ctx->R);
        std::vector<double> center(3 * ctx->R), sigma(ctx->R);
        for (int r = 0; r < ctx->R; ++r) {
            kind[r] = ctx->loads[r].kind;
            for (int j = 0; j < 3; ++j) center[3 * r + j] = ctx->loads[r].center[j];
            sigma[r] = ctx->loads[r].sigma;
        }
        int* dk; double *dc, *ds;
        TRY(dalloc(ctx, &dk, ctx->R));
        TRY(dalloc(ctx, &dc, 3 * ctx->R));
        TRY(dalloc(ctx, &ds, ctx->R));
        CK(cudaMemcpy(dk, kind.data(), ctx->R * sizeof(int), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(dc, center.data(), 3 * ctx->R * sizeof(double), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ds, sigma.data(), ctx->R * sizeof(double), cudaMemcpyHostToDevice));
        launch_fill_loads(g, ctx->R, dk, dc, ds, ctx->d_fr, ctx->own_stream);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(ctx->own_stream));
        // array loads as given; boundary loads lifted on the host (only the nodes next to the
        // boundary are non-zero)
        for (int r = 0; r < ctx->R; ++r) {
            if (ctx->loads[r].kind == RB_LOAD_ARRAY) {
                CK(cudaMemcpy(ctx->d_fr + (size_t)r * N, ctx->load_vals[r].data(), N * sizeof(double),
                              cudaMemcpyHostToDevice));
            } else if (ctx->loads[r].kind == RB_LOAD_BOUNDARY) {
                std::vector<double> f;
                boundary_lift(ctx, ctx->loads[r].field, ctx->load_vals[r].data(), maps, f);
                CK(cudaMemcpy(ctx->d_fr + (size_t)r * N, f.data(), N * sizeof(double), cudaMemcpyHostToDevice));
            }
        }
    }

    // basis storage
    const int nbp = ctx->nbp;
    TRY(dalloc(ctx, &ctx->d_W64c, (size_t)nbp * N));
    TRY(dalloc(ctx, &ctx->d_W32c, (size_t)nbp * N));
    TRY(dalloc(ctx, &ctx->d_W32r, (size_t)ctx->nbp32 * N));
    CK(cudaMemset(ctx->d_W64c, 0, (size_t)nbp * N * sizeof(double)));
    CK(cudaMemset(ctx->d_W32c, 0, (size_t)nbp * N * sizeof(float)));
    CK(cudaMemset(ctx->d_W32r, 0, (size_t)ctx->nbp32 * N * sizeof(float)));
    TRY(dalloc(ctx, &ctx->d_ANq, (size_t)ctx->P * std::max(1, n_cap) * std::max(1, n_cap)));
    TRY(dalloc(ctx, &ctx->d_fNr, (size_t)ctx->R * std::max(1, n_cap)));

    // batch workspace
    const size_t BN = (size_t)B * N;
    TRY(dalloc(ctx, &ctx->d_x64, BN));
    TRY(dalloc(ctx, &ctx->d_r64, BN));
    TRY(dalloc(ctx, &ctx->d_p64, 2 * BN));
    TRY(dalloc(ctx, &ctx->d_y64, BN));
    TRY(dalloc(ctx, &ctx->d_ypro64, BN));
    TRY(dalloc(ctx, &ctx->d_tmp64, BN));
    TRY(dalloc(ctx, &ctx->d_r32, BN));
    TRY(dalloc(ctx, &ctx->d_p32, 2 * BN));
    TRY(dalloc(ctx, &ctx->d_y32, BN));
    TRY(dalloc(ctx, &ctx->d_ypro32, BN));
    TRY(dalloc(ctx, &ctx->d_tmp32, BN));
    TRY(dalloc(ctx, &ctx->d_d32, BN));
    CK(cudaMemset(ctx->d_p64, 0, 2 * BN * sizeof(double)));
    CK(cudaMemset(ctx->d_p32, 0, 2 * BN * sizeof(float)));
    CK(cudaMemset(ctx->d_r64, 0, BN * sizeof(double)));
    CK(cudaMemset(ctx->d_r32, 0, BN * sizeof(float)));
    TRY(dalloc(ctx, &ctx->d_e64, (size_t)B * nbp));
    TRY(dalloc(ctx, &ctx->d_e32, (size_t)B * ctx->nbp32));
    CK(cudaMemset(ctx->d_e32, 0, (size_t)B * ctx->nbp32 * sizeof(float)));
    TRY(dalloc(ctx, &ctx->d_L, (size_t)B * nbp * nbp));
    TRY(dalloc(ctx, &ctx->d_mu, (size_t)B * ctx->n_mu));
    TRY(dalloc(ctx, &ctx->d_st, B));
    ctx->max_tiles = std::max(tiles_flat(N), tiles_box(g));
    TRY(dalloc(ctx, &ctx->d_part, (size_t)B * ctx->max_tiles * 4));
    ctx->nsplit = (int)std::max<long long>(1, std::min<long long>(64, N / 4096));
    ctx->nsplit_max = std::max(ctx->nsplit, ctx->num_sms);
    TRY(dalloc(ctx, &ctx->d_proj, (size_t)ctx->nsplit_max * B * nbp));
    TRY(dalloc(ctx, &ctx->d_tick, B));
    CK(cudaMemset(ctx->d_tick, 0, B * sizeof(unsigned)));
    TRY(dalloc(ctx, &ctx->d_lcnt, N_LISTS));
    TRY(dalloc(ctx, &ctx->d_lidx, (size_t)N_LISTS * B));
    TRY(dalloc(ctx, &ctx->d_ndone, 1));
    TRY(dalloc(ctx, &ctx->d_done, B));
    ctx->scratch_bytes = std::max<size_t>((size_t)128 * 128 * 128 * sizeof(double), 4096);
    TRY(dalloc(ctx, &ctx->d_scratch, ctx->scratch_bytes / sizeof(double)));
    TRY(dalloc(ctx, &ctx->d_tcerr, 1));
    CK(cudaMemset(ctx->d_tcerr, 0, sizeof(int)));
    TRY(dalloc(ctx, &ctx->d_flag, 1));
    TRY(tc_init(ctx->tc, ctx->geo, B, n_cap, nbp, ctx->nbp32, ctx->num_sms, ctx->d_r32, ctx->d_W32c, ctx->d_e32,
                ctx->d_W32r, ctx->d_tcerr, ctx->err));

    if (cudaMallocHost((void**)&ctx->h_st, (size_t)B * sizeof(QState)) != cudaSuccess ||
        cudaMallocHost((void**)&ctx->h_ndone, sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void**)&ctx->h_err, sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void**)&ctx->h_done, (size_t)B * sizeof(int)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        ctx->err = "pinned host allocation failed";
        return RB_ENOMEM;
    }
    return RB_OK;
}

void ctx_destroy(rb_ctx* ctx) {
    if (!ctx) return;
    cudaDeviceSynchronize();
    tc_free(ctx->tc);
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    if (ctx->d_V64) cudaFree(ctx->d_V64);
    if (ctx->d_V32) cudaFree(ctx->d_V32);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    for (void* p : ctx->allocs) cudaFree(p);
    ctx->allocs.clear();
    if (ctx->h_st) cudaFreeHost(ctx->h_st);
    if (ctx->h_ndone) cudaFreeHost(ctx->h_ndone);
    if (ctx->h_err) cudaFreeHost(ctx->h_err);
    if (ctx->h_done) cudaFreeHost(ctx->h_done);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    delete ctx;
}

__global__ void k_w_copies(long long N, int nb, int nbp, int nbp32, const double* W64c, float* W32c, float* W32r) {
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < (long long)nbp32 * N;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long i = idx / nbp32;
        const int k = (int)(idx % nbp32);
        const double w = k < nb ? W64c[(size_t)k * N + i] : 0.0;
        W32r[idx] = (float)w;
        if (k < nbp) W32c[(size_t)k * N + i] = (float)w;
    }
}

// Upload the reduced data of the current n and refresh the FP32 copies of W.
rb_status ctx_refresh_basis(rb_ctx* ctx) {
    const int n = ctx->n;
    if (n > 0) {
        CK(cudaMemcpy(ctx->d_ANq, ctx->h_ANq.data(), ctx->h_ANq.size() * sizeof(double), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->d_fNr, ctx->h_fNr.data(), ctx->h_fNr.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    k_w_copies<<<4096, 256, 0, ctx->own_stream>>>(ctx->N, n, ctx->nbp, ctx->nbp32, ctx->d_W64c, ctx->d_W32c,
                                                  ctx->d_W32r);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(ctx->own_stream));
    return RB_OK;
}

// rows [r0, r0 + rows) of a row-major [N][n] basis into the column-major W64c
__global__ void k_scatter_rowmajor(long long N, long long r0, long long rows, int n, const double* Wrow,
                                   double* W64c) {
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < (long long)n * rows;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long i = idx / n;
        const int k = (int)(idx % n);
        W64c[(size_t)k * N + r0 + i] = Wrow[idx];
    }
}

rb_status upload_basis(rb_ctx* ctx, int n, const double* W, const double* ANq, const double* fNr) {
    ctx->n = n;
    const size_t Q = ctx->P, R = ctx->R;
    ctx->h_ANq.assign(ANq ? ANq : nullptr, ANq ? ANq + Q * n * n : nullptr);
    ctx->h_fNr.assign(fNr ? fNr : nullptr, fNr ? fNr + R * n : nullptr);
    ctx->h_Rsnap.assign((size_t)n * n, 0.0);
    ctx->selected.assign(n, -1);
    if (n > 0) {
        // stage the row-major host W through the device in slices
        const long long N = ctx->N;
        const long long rows_per = std::max<long long>(1, (long long)(ctx->scratch_bytes / sizeof(double)) / n);
        for (long long r0 = 0; r0 < N; r0 += rows_per) {
            const long long rows = std::min(rows_per, N - r0);
            CK(cudaMemcpy(ctx->d_scratch, W + r0 * n, (size_t)rows * n * sizeof(double), cudaMemcpyHostToDevice));
            k_scatter_rowmajor<<<1024, 256>>>(N, r0, rows, n, ctx->d_scratch, ctx->d_W64c);
            CK(cudaGetLastError());
            CK(cudaDeviceSynchronize());
        }
    }
    return ctx_refresh_basis(ctx);
}

}  // namespace

// ============================================================================
// solve drivers

namespace {

struct Mode {
    bool rbi;
    bool mixed;
};

// Kernel families a context may use.  Problems with coefficient fields run the generic
// kernels, except on 3D grids that the z-march tile kernels cover (those read kappa(mu)).
bool rowmarch_ok(const rb_ctx* ctx) { return use_rowmarch(ctx->geo) && !ctx->force_generic && ctx->n_fields == 0; }
bool zmarch_ok(const rb_ctx* ctx, bool fp64) {
    return use_zmarch_smoother(ctx->geo) && !ctx->force_generic &&
           (ctx->n_fields == 0 || (ctx->geo.kap64 && use_ztile(ctx->geo, fp64)));
}

Params make_params(rb_ctx* ctx, int B, double* x64, const rb_opts& o, Mode m, bool use_tc) {
    Params P{};
    P.g = ctx->geo;
    P.B = B;
    P.Bmax = ctx->Bmax;
    P.n_mu = ctx->n_mu;
    P.mu = ctx->d_mu;
    P.R = ctx->R;
    P.fr = ctx->d_fr;
    for (int r = 0; r < ctx->R; ++r) P.load_param[r] = ctx->load_param[r];
    P.nb = ctx->n;
    P.nbp = ctx->nbp;
    P.W64c = ctx->d_W64c;
    P.W32c = ctx->d_W32c;
    P.L = ctx->d_L;
    P.x64 = x64;
    if (m.mixed) {
        P.r = ctx->d_r32; P.p = ctx->d_p32; P.y = ctx->d_y32; P.ypro = ctx->d_ypro32;
        P.tmp = ctx->d_tmp32; P.d = ctx->d_d32; P.e = ctx->d_e32;
    } else {
        P.r = ctx->d_r64; P.p = ctx->d_p64; P.y = ctx->d_y64; P.ypro = ctx->d_ypro64;
        P.tmp = ctx->d_tmp64; P.d = x64; P.e = ctx->d_e64;
    }
    P.st = ctx->d_st;
    P.part = ctx->d_part;
    P.max_tiles = ctx->max_tiles;
    P.proj = ctx->d_proj;
    P.nsplit = use_tc ? ctx->tc.proj_split : ctx->nsplit;
    P.lde = (m.mixed && use_tc) ? ctx->nbp32 : ctx->nbp;
    P.tick = ctx->d_tick;
    P.lcnt = ctx->d_lcnt;
    P.lidx = ctx->d_lidx;
    P.ndone = ctx->d_ndone;
    P.done = ctx->d_done;
    P.err = ctx->d_tcerr;
    P.tol = o.tol;
    P.inner_tol = o.inner_tol;
    P.max_iter = o.max_iter;
    P.max_outer = o.max_outer;
    P.beta_form = o.beta_form;
    P.smoother = o.smoother;
    P.omega = o.omega;
    P.mixed = m.mixed ? 1 : 0;
    // BF16 iterates only where the staged red-black smoother runs (the mixed path)
    P.ybf16 = (m.mixed && o.store == RB_STORE_BF16 && o.smoother == RB_SMOOTH_RBGS && o.kernels == 0 &&
               rowmarch_ok(ctx) && use_tma_smoother(ctx->geo))
                  ? 1
                  : 0;
    P.adaptive = (!m.rbi && o.adaptive_n > 0 && ctx->n > 0) ? 1 : 0;
    P.gamma = o.gamma;
    P.wait_ns = ctx->wait_ns;
    P.dbg_skip = ctx->dbg_skip;
    return P;
}

// basis vectors of a query's first preconditioner application
int first_n_used(const rb_ctx* ctx, const rb_opts& o, Mode m) {
    return (!m.rbi && o.adaptive_n > 0) ? std::min(o.adaptive_n, ctx->n) : ctx->n;
}

enum KernelKind {
    KK_OUTER_UPDATE, KK_OUTER_RES, KK_RBI_RES, KK_PROJECT, KK_RSOLVE, KK_PROLONG, KK_SMOOTH, KK_CG_A, KK_CG_B,
    KK_TC_PROJECT, KK_TC_PROLONG, KK_COUNT
};
const char* const KK_NAMES[KK_COUNT] = {"outer_update", "outer_residual", "rbi_residual", "project",
                                        "reduced_solve", "prolong", "smooth", "cg_a", "cg_b",
                                        "tc_project", "tc_prolong"};

cudaEvent_t next_event(rb_ctx* ctx) {
    if (ctx->ev_used == ctx->ev_pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        ctx->ev_pool.push_back(e);
    }
    return ctx->ev_pool[ctx->ev_used++];
}

// Run f; while profiling, bracket it with events on the step's stream.
template <typename F>
void timed(rb_ctx* ctx, int kind, cudaStream_t s, F&& f) {
    if (!ctx->profiling) { f(); return; }
    const size_t first = ctx->ev_used;
    cudaEventRecord(next_event(ctx), s);
    f();
    cudaEventRecord(next_event(ctx), s);
    ctx->prof_pending.push_back({kind, first});
}

// Accumulate the recorded launches (the stream has been synchronised).
void flush_profile(rb_ctx* ctx) {
    for (auto& pr : ctx->prof_pending) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, ctx->ev_pool[pr.second], ctx->ev_pool[pr.second + 1]) == cudaSuccess) {
            ctx->prof_ms[pr.first] += ms;
            ctx->prof_launches[pr.first] += 1;
        }
    }
    cudaGetLastError();
    ctx->prof_pending.clear();
    ctx->ev_used = 0;
}

void enqueue_prec(rb_ctx* ctx, const Params& P, const Launch& L, const rb_opts& o, Mode m, bool use_tc);

// One step of the per-query state machine for every active query.
void enqueue_step(rb_ctx* ctx, const Params& P, const Launch& L, const rb_opts& o, Mode m, bool use_tc) {
    cudaStream_t s = L.s;
    const bool rm = rowmarch_ok(ctx);
    if (m.rbi) {
        timed(ctx, KK_RBI_RES, s, [&] { launch_rbi_residual(P, L); });
        cudaMemsetAsync(ctx->d_lcnt + L_OUT, 0, sizeof(int), s);
        timed(ctx, KK_PROJECT, s, [&] { launch_project<double>(P, L); });
        timed(ctx, KK_RSOLVE, s, [&] { launch_reduced_solve<double>(P, L); });
        timed(ctx, KK_PROLONG, s, [&] { launch_prolong<double>(P, L, true); });
        timed(ctx, KK_SMOOTH, s, [&] { launch_smoother<double>(P, L, o.nu, true); });
        cudaMemsetAsync(ctx->d_lcnt + L_PREC, 0, sizeof(int), s);
        return;
    }
    const bool staged_outer = rm && o.kernels != 2 && use_staged_outer(ctx->geo);
    const bool tile_outer = !ctx->force_generic && o.kernels == 0 && use_ztile_outer(ctx->geo);
    if (m.mixed) {
        timed(ctx, KK_OUTER_UPDATE, s, [&] { launch_outer_update(P, L); });
        timed(ctx, KK_OUTER_RES, s, [&] {
            if (staged_outer) launch2d_outer_residual_staged<float>(P, L);
            else if (!(tile_outer && launch3d_outer_tile<float>(P, L))) launch_outer_residual<float>(P, L);
        });
    } else {
        timed(ctx, KK_OUTER_RES, s, [&] {
            if (staged_outer) launch2d_outer_residual_staged<double>(P, L);
            else if (!(tile_outer && launch3d_outer_tile<double>(P, L))) launch_outer_residual<double>(P, L);
        });
    }
    cudaMemsetAsync(ctx->d_lcnt + L_OUT, 0, sizeof(int), s);
    enqueue_prec(ctx, P, L, o, m, use_tc);
    cudaMemsetAsync(ctx->d_lcnt + L_PREC, 0, sizeof(int), s);
    const bool staged = rm && o.kernels != 2 && use_staged_cg(ctx->geo);
    const bool z3 = zmarch_ok(ctx, !m.mixed) && o.kernels == 0;
    if (m.mixed) {
        timed(ctx, KK_CG_A, s, [&] {
            if (staged) launch2d_cg_a_staged<float>(P, L);
            else if (rm) launch2d_cg_a<float>(P, L);
            else if (z3) launch3d_cg_a<float>(P, L);
            else launch_cg_a<float>(P, L);
        });
        timed(ctx, KK_CG_B, s, [&] {
            if (staged) launch2d_cg_b_staged<float>(P, L);
            else if (rm) launch2d_cg_b<float>(P, L);
            else if (z3) launch3d_cg_b<float>(P, L);
            else launch_cg_b<float>(P, L);
        });
    } else {
        timed(ctx, KK_CG_A, s, [&] {
            if (staged) launch2d_cg_a_staged<double>(P, L);
            else if (rm) launch2d_cg_a<double>(P, L);
            else if (z3) launch3d_cg_a<double>(P, L);
            else launch_cg_a<double>(P, L);
        });
        timed(ctx, KK_CG_B, s, [&] {
            if (staged) launch2d_cg_b_staged<double>(P, L);
            else if (rm) launch2d_cg_b<double>(P, L);
            else if (z3) launch3d_cg_b<double>(P, L);
            else launch_cg_b<double>(P, L);
        });
    }
    cudaMemsetAsync(ctx->d_lcnt + L_ITER, 0, sizeof(int), s);
}

// The RBI preconditioner y = RBI(A, r, W, 1) for every query on the PREC list.
void enqueue_prec(rb_ctx* ctx, const Params& P, const Launch& L, const rb_opts& o, Mode m, bool use_tc) {
    cudaStream_t s = L.s;
    const bool rm = rowmarch_ok(ctx);
    const bool zm = zmarch_ok(ctx, !m.mixed);
    const bool blocks = ctx->n_fields == 0;   // the z-march kernels of kernels = 1 take blocks only
    if (m.mixed) {
        if (use_tc) {
            timed(ctx, KK_TC_PROJECT, s, [&] { tc_project(ctx->tc, P, L); });
            timed(ctx, KK_RSOLVE, s, [&] { launch_reduced_solve<float>(P, L); });
            timed(ctx, KK_TC_PROLONG, s, [&] { tc_prolong(ctx->tc, P, L); });
        } else {
            timed(ctx, KK_PROJECT, s, [&] { launch_project<float>(P, L); });
            timed(ctx, KK_RSOLVE, s, [&] { launch_reduced_solve<float>(P, L); });
            timed(ctx, KK_PROLONG, s, [&] { launch_prolong<float>(P, L, false); });
        }
        timed(ctx, KK_SMOOTH, s, [&] {
            if (o.smoother == RB_SMOOTH_RBGS && o.kernels == 1 && !ctx->force_generic && blocks &&
                use_fused_smoother(ctx->geo, o.nu))
                launch2d_smooth_fused(P, L, o.nu);
            else if (rm && o.smoother == RB_SMOOTH_RBGS && (o.kernels == 3 || o.kernels == 4) && !P.ybf16 &&
                     use_multi_smoother(ctx->geo))
                launch2d_smooth_multi(P, L, o.nu, o.kernels == 3 ? 3 : 2);
            else if (rm && o.smoother == RB_SMOOTH_RBGS && o.kernels == 0 && use_tma_smoother(ctx->geo))
                launch2d_smooth_tma<float>(P, L, o.nu);
            else if (rm && o.smoother == RB_SMOOTH_RBGS) launch2d_smooth<float>(P, L, o.nu);
            else if (zm && o.smoother == RB_SMOOTH_RBGS && o.kernels == 0) launch3d_smooth_staged<float>(P, L, o.nu);
            else if (zm && blocks && o.smoother == RB_SMOOTH_RBGS && o.kernels == 1)
                launch3d_smooth<float>(P, L, o.nu);
            else launch_smoother<float>(P, L, o.nu, false);
        });
    } else {
        timed(ctx, KK_PROJECT, s, [&] { launch_project<double>(P, L); });
        timed(ctx, KK_RSOLVE, s, [&] { launch_reduced_solve<double>(P, L); });
        timed(ctx, KK_PROLONG, s, [&] { launch_prolong<double>(P, L, false); });
        timed(ctx, KK_SMOOTH, s, [&] {
            if (rm && o.smoother == RB_SMOOTH_RBGS && o.kernels == 0 && use_tma_smoother(ctx->geo))
                launch2d_smooth_tma<double>(P, L, o.nu);
            else if (rm && o.smoother == RB_SMOOTH_RBGS) launch2d_smooth<double>(P, L, o.nu);
            else if (zm && o.smoother == RB_SMOOTH_RBGS && o.kernels == 0) launch3d_smooth_staged<double>(P, L, o.nu);
            else if (zm && blocks && o.smoother == RB_SMOOTH_RBGS && o.kernels == 1)
                launch3d_smooth<double>(P, L, o.nu);
            else launch_smoother<double>(P, L, o.nu, false);
        });
    }
}

rb_status validate_opts(rb_ctx* ctx, const rb_opts& o) {
    if (!(o.tol > 0.0) || o.max_iter < 1 || o.nu < 0 || o.max_outer < 1 || !(o.inner_tol > 0.0) ||
        (o.smoother < 0 || o.smoother > 2) || (o.beta_form != RB_BETA_FR && o.beta_form != RB_BETA_PR) ||
        (o.kernels < 0 || o.kernels > 4) || (o.store != RB_STORE_F32 && o.store != RB_STORE_BF16) ||
        (o.precision != RB_PREC_FP64 && o.precision != RB_PREC_MIXED) || o.adaptive_n < 0 ||
        !(o.gamma >= 0.0) || o.x0_mode < RB_X0_ZERO || o.x0_mode > RB_X0_RB) {
        ctx->err = "invalid options";
        return RB_EINVAL;
    }
    return RB_OK;
}

// One wave of B <= Bmax queries of a context in flight: set up by wave_begin, advanced
// by wave_launch (8 steps of the state machine, replayed as a CUDA graph) and
// wave_check (after the stream has been synchronised), closed by wave_end.
struct Wave {
    rb_ctx* ctx = nullptr;
    int B = 0;
    double* x64 = nullptr;      // device [B][N]
    double* x_host = nullptr;   // host [B][N] or null: finished solutions are copied there as they finish
    bool x_given = false;
    rb_opts o{};
    Mode m{false, false};
    cudaStream_t s = nullptr;
    Params P{};
    Launch L{};
    bool use_tc = false;
    cudaGraphExec_t exec = nullptr;
    long long steps = 0, max_steps = 0;
    int copied = 0;
    rb_status rs = RB_OK;
    bool finished = false;
};

constexpr int CHECK_EVERY = 8;   // state-machine steps per graph replay (between host polls)

// The captured graph of CHECK_EVERY steps is kept per context and reused while the launch
// parameters are the same (the usual case of repeated calls with the same buffers).
rb_status wave_graph(Wave& w) {
    rb_ctx* ctx = w.ctx;
    std::vector<unsigned char> key(sizeof(Params) + 6 * sizeof(int));
    std::memcpy(key.data(), &w.P, sizeof(Params));
    const int extra[6] = {w.o.nu, w.o.smoother, w.o.kernels, w.m.mixed ? 1 : 0, w.use_tc ? 1 : 0, w.m.rbi ? 1 : 0};
    std::memcpy(key.data() + sizeof(Params), extra, sizeof(extra));
    if (ctx->graph_exec && ctx->graph_stream == w.s && key == ctx->graph_key) {
        w.exec = ctx->graph_exec;
        return RB_OK;
    }
    if (ctx->graph_exec) {
        cudaGraphExecDestroy(ctx->graph_exec);
        ctx->graph_exec = nullptr;
    }
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(w.s, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < CHECK_EVERY; ++k) enqueue_step(ctx, w.P, w.L, w.o, w.m, w.use_tc);
    cudaError_t ce = cudaStreamEndCapture(w.s, &graph);
    if (ce != cudaSuccess) {
        ctx->err = std::string("graph capture failed: ") + cudaGetErrorString(ce);
        return RB_ECUDA;
    }
    ce = cudaGraphInstantiate(&ctx->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
        ctx->graph_exec = nullptr;
        ctx->err = std::string("graph instantiation failed: ") + cudaGetErrorString(ce);
        return RB_ECUDA;
    }
    ctx->graph_key.swap(key);
    ctx->graph_stream = w.s;
    w.exec = ctx->graph_exec;
    return RB_OK;
}

rb_status wave_begin(Wave& w, const double* mu_host) {
    rb_ctx* ctx = w.ctx;
    const int B = w.B;
    cudaStream_t s = w.s;
    const long long N = ctx->N;
    for (size_t i = 0; i < (size_t)B * ctx->n_mu; ++i) {
        if (!std::isfinite(mu_host[i])) {
            ctx->err = "parameter vector holds a non-finite value";
            return RB_EINVAL;
        }
    }
    CK(cudaMemcpyAsync(ctx->d_mu, mu_host, (size_t)B * ctx->n_mu * sizeof(double), cudaMemcpyHostToDevice, s));
    // RB_X0_RB: x_0 = W a_N(mu) (eqs. 2-3) in FP64; a query whose A_N(mu) is not positive definite
    // starts from it all the same and the solve's own Cholesky reports the breakdown
    const bool rb_start = w.o.x0_mode == RB_X0_RB && !w.x_given && ctx->n > 0;
    if (rb_start) {
        LoadMap lm{};
        for (int r = 0; r < ctx->R; ++r) lm.param[r] = ctx->load_param[r];
        CK(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), s));
        launch_galerkin(ctx->n, ctx->P, ctx->d_ANq, ctx->R, lm, ctx->d_fNr, ctx->n_mu, B, ctx->d_mu, ctx->d_e64,
                        ctx->d_flag, s);
        launch_lift64(N, ctx->n, ctx->d_W64c, B, ctx->d_e64, w.x64, ctx->grid, s);
        CK(cudaGetLastError());
    }
    for (int q = 0; q < B; ++q) {
        QState& st = ctx->h_st[q];
        std::memset(&st, 0, sizeof(QState));
        st.phase = PH_OUTER;
        st.start = 1;
        st.xzero = (w.x_given || rb_start) ? 0 : 1;
        st.n_used = first_n_used(ctx, w.o, w.m);
    }
    CK(cudaMemcpyAsync(ctx->d_st, ctx->h_st, (size_t)B * sizeof(QState), cudaMemcpyHostToDevice, s));
    std::vector<int> lc(N_LISTS, 0);
    lc[L_OUT] = B;
    std::vector<int> li(B);
    for (int q = 0; q < B; ++q) li[q] = q;
    CK(cudaMemcpyAsync(ctx->d_lcnt, lc.data(), N_LISTS * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->d_lidx + L_OUT * ctx->Bmax, li.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(ctx->d_ndone, 0, sizeof(int), s));
    CK(cudaMemsetAsync(ctx->d_tick, 0, (size_t)B * sizeof(unsigned), s));
    if (!w.x_given && !rb_start) CK(cudaMemsetAsync(w.x64, 0, (size_t)B * N * sizeof(double), s));
    if (w.m.mixed) CK(cudaMemsetAsync(ctx->d_d32, 0, (size_t)B * N * sizeof(float), s));
    // the host stages above are freed when the call returns: let them land first
    CK(cudaStreamSynchronize(s));

    w.use_tc = w.m.mixed && w.o.gemm != RB_GEMM_CUDA_CORES && tc_usable(ctx->tc, ctx->n);
    if (w.m.mixed && w.o.gemm == RB_GEMM_TENSOR && !w.use_tc) {
        ctx->err = "tensor-core engine unavailable for this problem (needs N_dof % 32 == 0, n >= 1, sm_10x)";
        return RB_EINVAL;
    }
    w.P = make_params(ctx, B, w.x64, w.o, w.m, w.use_tc);
    w.L = Launch{ctx->grid, s};
    launch_field_kappa(ctx->geo, B, ctx->n_mu, ctx->d_mu, s);
    launch_cholesky(w.P, s, ctx->d_ANq, ctx->P);
    CK(cudaGetLastError());
    w.exec = nullptr;
    if (w.o.graph && s != nullptr && !ctx->profiling) TRY(wave_graph(w));
    w.max_steps = (long long)w.o.max_iter + 2LL * w.o.max_outer + 64;
    return RB_OK;
}

// enqueue the next CHECK_EVERY steps and the copies of the done counter and error flag
rb_status wave_launch(Wave& w) {
    rb_ctx* ctx = w.ctx;
    if (w.exec) {
        cudaError_t e = cudaGraphLaunch(w.exec, w.s);
        if (e != cudaSuccess) { ctx->err = cudaGetErrorString(e); return RB_ECUDA; }
    } else {
        for (int k = 0; k < CHECK_EVERY; ++k) enqueue_step(ctx, w.P, w.L, w.o, w.m, w.use_tc);
    }
    w.steps += CHECK_EVERY;
    cudaMemcpyAsync(ctx->h_ndone, ctx->d_ndone, sizeof(int), cudaMemcpyDeviceToHost, w.s);
    cudaMemcpyAsync(ctx->h_err, ctx->d_tcerr, sizeof(int), cudaMemcpyDeviceToHost, w.s);
    if (w.x_host) cudaMemcpyAsync(ctx->h_done, ctx->d_done, (size_t)w.B * sizeof(int), cudaMemcpyDeviceToHost, w.s);
    return RB_OK;
}

// after wave_launch: wait for the stream, issue the copies of finished solutions, decide
void wave_check(Wave& w) {
    rb_ctx* ctx = w.ctx;
    const long long N = ctx->N;
    cudaError_t e = cudaStreamSynchronize(w.s);
    if (e != cudaSuccess) {
        ctx->err = std::string("solve failed: ") + cudaGetErrorString(e);
        w.rs = RB_ECUDA;
        w.finished = true;
        return;
    }
    if (ctx->profiling) flush_profile(ctx);
    if (*ctx->h_err) {
        // a kernel gave up waiting on an asynchronous copy: its work items are lost and some
        // query can no longer finish; stop here (the flag is cleared in wave_end)
        ctx->err = "a kernel gave up waiting on an asynchronous copy or MMA (device timeout)";
        w.rs = RB_ETIMEOUT;
        w.finished = true;
        return;
    }
    if (w.x_host) {
        const int upto = std::min(*ctx->h_ndone, w.B);
        for (; w.copied < upto; ++w.copied) {
            const int q = ctx->h_done[w.copied];
            if (q < 0 || q >= w.B) continue;
            cudaMemcpyAsync(w.x_host + (size_t)q * N, w.x64 + (size_t)q * N, (size_t)N * sizeof(double),
                            cudaMemcpyDeviceToHost, ctx->copy_stream);
        }
    }
    if (*ctx->h_ndone >= w.B) {
        w.finished = true;
        return;
    }
    if (w.steps > w.max_steps) {
        ctx->err = "solver state machine did not finish within its step budget";
        w.rs = RB_ETIMEOUT;
        w.finished = true;
    }
}

rb_status wave_end(Wave& w, rb_stats* stats) {
    rb_ctx* ctx = w.ctx;
    const int B = w.B;
    cudaStream_t s = w.s;
    const long long N = ctx->N;
    rb_status rs = w.rs;
    if (rs == RB_ETIMEOUT) {
        cudaStreamSynchronize(s);
        cudaMemsetAsync(ctx->d_tcerr, 0, sizeof(int), s);
        cudaStreamSynchronize(s);
    }
    if (w.x_host) {
        // queries that never reached PH_DONE (a failed wave) still get their current iterate
        if (rs != RB_OK) {
            std::vector<char> seen(B, 0);
            for (int i = 0; i < w.copied; ++i)
                if (ctx->h_done[i] >= 0 && ctx->h_done[i] < B) seen[ctx->h_done[i]] = 1;
            for (int q = 0; q < B; ++q)
                if (!seen[q])
                    cudaMemcpyAsync(w.x_host + (size_t)q * N, w.x64 + (size_t)q * N, (size_t)N * sizeof(double),
                                    cudaMemcpyDeviceToHost, s);
            cudaStreamSynchronize(s);
        }
        const cudaError_t ce = cudaStreamSynchronize(ctx->copy_stream);
        if (ce != cudaSuccess && rs == RB_OK) {
            ctx->err = std::string("solution copy failed: ") + cudaGetErrorString(ce);
            rs = RB_ECUDA;
        }
    }
    if (rs != RB_OK) return rs;
    {
        int derr = 0;
        CK(cudaMemcpyAsync(&derr, ctx->d_tcerr, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (derr) {
            cudaMemsetAsync(ctx->d_tcerr, 0, sizeof(int), s);
            ctx->err = "a kernel gave up waiting on an asynchronous copy or MMA (device timeout)";
            return RB_ETIMEOUT;
        }
    }
    CK(cudaMemcpyAsync(ctx->h_st, ctx->d_st, (size_t)B * sizeof(QState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    rb_status worst = RB_OK;
    for (int q = 0; q < B; ++q) {
        const QState& st = ctx->h_st[q];
        if (stats) {
            stats[q].iters = st.iters;
            stats[q].outer = st.outer;
            stats[q].restarts = st.restarts;
            stats[q].status = st.status;
            stats[q].rel_res = st.rel_res;
            stats[q].n_used = st.n_used;
        }
        if (st.status > (int)worst) worst = (rb_status)st.status;
    }
    return worst;
}

// Solve one wave of B <= Bmax queries; x64 is a device array [B][N].  With x_host
// (host [B][N]) the solution of every query is copied there as soon as the query
// finishes, on a side stream, while the others still iterate.
rb_status run_wave(rb_ctx* ctx, int B, const double* mu_host, double* x64, bool x_given, const rb_opts& o, Mode m,
                   rb_stats* stats, double* x_host) {
    Wave w;
    w.ctx = ctx;
    w.B = B;
    w.x64 = x64;
    w.x_host = x_host;
    w.x_given = x_given;
    w.o = o;
    w.m = m;
    w.s = o.stream ? (cudaStream_t)o.stream : ctx->own_stream;
    TRY(wave_begin(w, mu_host));
    while (!w.finished) {
        rb_status e = wave_launch(w);
        if (e != RB_OK) { w.rs = e; break; }
        wave_check(w);
    }
    return wave_end(w, stats);
}

rb_status run_batch(rb_ctx* ctx, int B, const double* mu, double* x, const rb_opts* opts, rb_stats* stats, Mode m) {
    if (!ctx) return RB_EINVAL;
    if (B < 0 || (B > 0 && (!mu || !x))) { ctx->err = "B < 0 or NULL mu / x"; return RB_EINVAL; }
    rb_opts o;
    rb_default_opts(&o);
    if (opts) o = *opts;
    TRY(validate_opts(ctx, o));
    if (m.rbi) m.mixed = false;
    else m.mixed = o.precision == RB_PREC_MIXED;
    bool bad = false;
    const bool dev_x = is_device_ptr(ctx, x, &bad);
    if (bad) return RB_EINVAL;
    const bool x_given = o.x0_mode == RB_X0_GIVEN;
    cudaStream_t s = o.stream ? (cudaStream_t)o.stream : ctx->own_stream;
    const long long N = ctx->N;
    rb_status worst = RB_OK;
    for (int b0 = 0; b0 < B; b0 += ctx->Bmax) {
        const int nbw = std::min(ctx->Bmax, B - b0);
        double* x64 = dev_x ? x + (size_t)b0 * N : ctx->d_x64;
        if (!dev_x && x_given)
            CK(cudaMemcpyAsync(x64, x + (size_t)b0 * N, (size_t)nbw * N * sizeof(double), cudaMemcpyHostToDevice, s));
        rb_status w = run_wave(ctx, nbw, mu + (size_t)b0 * ctx->n_mu, x64, x_given, o, m, stats ? stats + b0 : nullptr,
                               dev_x ? nullptr : x + (size_t)b0 * N);
        if (w == RB_EINVAL || w == RB_ECUDA || w == RB_ETIMEOUT) return w;
        if (w > worst) worst = w;
    }
    return worst;
}

}  // namespace

// ============================================================================
// public API

extern "C" {

void rb_default_opts(rb_opts* o) {
    if (!o) return;
    o->tol = 1e-10;
    o->max_iter = 20000;
    o->smoother = RB_SMOOTH_RBGS;
    o->nu = 1;
    o->omega = 2.0 / 3.0;
    o->precision = RB_PREC_FP64;
    o->beta_form = RB_BETA_PR;
    o->x0_mode = RB_X0_ZERO;
    o->inner_tol = 1e-5;
    o->max_outer = 12;
    o->gemm = RB_GEMM_AUTO;
    o->graph = 1;
    o->kernels = 0;
    o->store = RB_STORE_F32;
    o->adaptive_n = 0;
    o->gamma = 10.0;
    o->stream = nullptr;
}

void rb_default_build_opts(rb_build_opts* o) {
    if (!o) return;
    o->truth_tol = 1e-11;
    o->truth_max_iter = 200000;
    o->score = 0;
    o->drop_tol = 1e-10;
}

const char* rb_status_string(rb_status s) {
    switch (s) {
        case RB_OK: return "ok";
        case RB_EINVAL: return "invalid argument";
        case RB_ENOMEM: return "out of memory";
        case RB_EFORMAT: return "malformed basis file";
        case RB_ECUDA: return "CUDA error";
        case RB_EBREAKDOWN: return "numerical breakdown";
        case RB_ENOCONV: return "not converged";
        case RB_ETIMEOUT: return "timeout";
        case RB_EIO: return "I/O error";
    }
    return "unknown status";
}

const char* rb_last_error(const rb_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

void rb_free(rb_ctx* ctx) { ctx_destroy(ctx); }

rb_status rb_offline_load_arrays(rb_ctx** out, const rb_problem* prob, int n, const double* W, const double* ANq,
                                 const double* fNr, int max_batch) {
    if (!out) { g_create_error = "out is NULL"; return RB_EINVAL; }
    *out = nullptr;
    std::string why;
    rb_status v = validate_problem(prob, why);
    if (v != RB_OK) { g_create_error = why; return v; }
    if (n < 0 || n > MAX_N || max_batch < 1 || (n > 0 && (!W || !ANq || !fNr))) {
        g_create_error = "need 0 <= n <= 128, max_batch >= 1 and non-NULL W, ANq, fNr";
        return RB_EINVAL;
    }
    rb_ctx* ctx = new rb_ctx();
    rb_status s = ctx_init(ctx, prob, n, max_batch);
    if (s == RB_OK) s = upload_basis(ctx, n, W, ANq, fNr);
    if (s != RB_OK) {
        g_create_error = ctx->err;
        ctx_destroy(ctx);
        return s;
    }
    *out = ctx;
    return RB_OK;
}

rb_status rb_debug_wait(rb_ctx* ctx, double limit_s, long long skip_stage) {
    if (!ctx) return RB_EINVAL;
    if (!(limit_s > 0.0) || !(limit_s <= 2.0) || skip_stage < -1) {
        ctx->err = "need 0 < limit_s <= 2 and skip_stage >= -1";
        return RB_EINVAL;
    }
    ctx->wait_ns = (unsigned long long)(limit_s * 1e9);
    ctx->dbg_skip = skip_stage;
    return RB_OK;
}

rb_status rb_info(const rb_ctx* ctx, long long* n_dof, int* n, int* Q, int* R, int* n_mu) {
    if (!ctx) return RB_EINVAL;
    if (n_dof) *n_dof = ctx->N;
    if (n) *n = ctx->n;
    if (Q) *Q = ctx->P;
    if (R) *R = ctx->R;
    if (n_mu) *n_mu = ctx->n_mu;
    return RB_OK;
}

rb_status rb_profile(rb_ctx* ctx, int enable) {
    if (!ctx) return RB_EINVAL;
    ctx->profiling = enable != 0;
    if (enable) {
        for (int k = 0; k < 32; ++k) { ctx->prof_ms[k] = 0.0; ctx->prof_launches[k] = 0; }
        ctx->prof_pending.clear();
        ctx->ev_used = 0;
    }
    return RB_OK;
}

rb_status rb_profile_read(const rb_ctx* ctx, rb_kernel_time* out, int cap, int* count) {
    if (!ctx || (cap > 0 && !out)) return RB_EINVAL;
    int c = 0;
    for (int k = 0; k < KK_COUNT; ++k) {
        if (ctx->prof_launches[k] == 0) continue;
        if (c < cap) {
            std::memset(out[c].name, 0, sizeof(out[c].name));
            std::strncpy(out[c].name, KK_NAMES[k], sizeof(out[c].name) - 1);
            out[c].launches = ctx->prof_launches[k];
            out[c].ms = ctx->prof_ms[k];
        }
        ++c;
    }
    if (count) *count = c;
    return RB_OK;
}

rb_status rb_products(rb_ctx* ctx, int B, const float* R, double* WtR, const float* E, float* WE, int engine) {
    if (!ctx) return RB_EINVAL;
    if (B < 0 || B > ctx->Bmax) { ctx->err = "need 0 <= B <= max_batch"; return RB_EINVAL; }
    if (B == 0) return RB_OK;
    const int n = ctx->n;
    if (n == 0) { ctx->err = "the context has no basis"; return RB_EINVAL; }
    const bool can_tc = tc_usable(ctx->tc, n);
    if (engine == RB_GEMM_TENSOR && !can_tc) { ctx->err = "tensor-core engine unavailable for this problem"; return RB_EINVAL; }
    const bool use_tc = engine == RB_GEMM_TENSOR || (engine == RB_GEMM_AUTO && can_tc);
    rb_opts o;
    rb_default_opts(&o);
    o.precision = RB_PREC_MIXED;
    cudaStream_t s = ctx->own_stream;
    const long long N = ctx->N;
    Params P = make_params(ctx, B, ctx->d_x64, o, Mode{false, true}, use_tc);
    Launch L{ctx->grid, s};
    for (int q = 0; q < B; ++q) {
        std::memset(&ctx->h_st[q], 0, sizeof(QState));
        ctx->h_st[q].phase = PH_PREC;
        ctx->h_st[q].n_used = n;
    }
    CK(cudaMemcpyAsync(ctx->d_st, ctx->h_st, (size_t)B * sizeof(QState), cudaMemcpyHostToDevice, s));
    std::vector<int> lc(N_LISTS, 0), li(B);
    lc[L_PREC] = B;
    for (int q = 0; q < B; ++q) li[q] = q;
    CK(cudaMemcpyAsync(ctx->d_lcnt, lc.data(), N_LISTS * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->d_lidx + L_PREC * ctx->Bmax, li.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    if (R && WtR) {
        CK(cudaMemcpyAsync(ctx->d_r32, R, (size_t)B * N * sizeof(float), cudaMemcpyDefault, s));
        if (use_tc) tc_project(ctx->tc, P, L);
        else launch_project<float>(P, L);
        CK(cudaGetLastError());
        std::vector<double> part((size_t)P.nsplit * ctx->Bmax * ctx->nbp);
        CK(cudaMemcpyAsync(part.data(), ctx->d_proj, part.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int q = 0; q < B; ++q)
            for (int k = 0; k < n; ++k) {
                double acc = 0.0;
                for (int sp = 0; sp < P.nsplit; ++sp) acc += part[((size_t)sp * ctx->Bmax + q) * ctx->nbp + k];
                WtR[(size_t)q * n + k] = acc;
            }
    }
    if (E && WE) {
        std::vector<float> e((size_t)B * P.lde, 0.0f);
        for (int q = 0; q < B; ++q)
            for (int k = 0; k < n; ++k) e[(size_t)q * P.lde + k] = E[(size_t)q * n + k];
        CK(cudaMemcpyAsync(ctx->d_e32, e.data(), e.size() * sizeof(float), cudaMemcpyHostToDevice, s));
        if (use_tc) tc_prolong(ctx->tc, P, L);
        else launch_prolong<float>(P, L, false);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(WE, ctx->d_ypro32, (size_t)B * N * sizeof(float), cudaMemcpyDefault, s));
    }
    CK(cudaStreamSynchronize(s));
    int tcerr = 0;
    CK(cudaMemcpy(&tcerr, ctx->d_tcerr, sizeof(int), cudaMemcpyDeviceToHost));
    if (tcerr) {
        cudaMemset(ctx->d_tcerr, 0, sizeof(int));
        ctx->err = "a tensor-core kernel gave up waiting on its pipeline (device timeout)";
        return RB_ETIMEOUT;
    }
    return RB_OK;
}

rb_status rb_precondition(rb_ctx* ctx, int B, const double* mu, const void* r, void* y, const rb_opts* opts) {
    if (!ctx) return RB_EINVAL;
    if (B < 0 || B > ctx->Bmax || (B > 0 && (!mu || !r || !y))) {
        ctx->err = "need 0 <= B <= max_batch and non-NULL mu, r, y";
        return RB_EINVAL;
    }
    if (B == 0) return RB_OK;
    rb_opts o;
    rb_default_opts(&o);
    if (opts) o = *opts;
    TRY(validate_opts(ctx, o));
    for (size_t i = 0; i < (size_t)B * ctx->n_mu; ++i)
        if (!std::isfinite(mu[i])) { ctx->err = "non-finite parameter"; return RB_EINVAL; }
    const Mode m{false, o.precision == RB_PREC_MIXED};
    const bool use_tc = m.mixed && o.gemm != RB_GEMM_CUDA_CORES && tc_usable(ctx->tc, ctx->n);
    if (m.mixed && o.gemm == RB_GEMM_TENSOR && !use_tc) { ctx->err = "tensor-core engine unavailable"; return RB_EINVAL; }
    cudaStream_t s = o.stream ? (cudaStream_t)o.stream : ctx->own_stream;
    const long long N = ctx->N;
    const size_t es = m.mixed ? sizeof(float) : sizeof(double);
    CK(cudaMemcpyAsync(ctx->d_mu, mu, (size_t)B * ctx->n_mu * sizeof(double), cudaMemcpyHostToDevice, s));
    for (int q = 0; q < B; ++q) {
        std::memset(&ctx->h_st[q], 0, sizeof(QState));
        ctx->h_st[q].phase = PH_PREC;
        ctx->h_st[q].start = 1;
        ctx->h_st[q].n_used = first_n_used(ctx, o, m);
    }
    CK(cudaMemcpyAsync(ctx->d_st, ctx->h_st, (size_t)B * sizeof(QState), cudaMemcpyHostToDevice, s));
    std::vector<int> lc(N_LISTS, 0), li(B);
    lc[L_PREC] = B;
    for (int q = 0; q < B; ++q) li[q] = q;
    CK(cudaMemcpyAsync(ctx->d_lcnt, lc.data(), N_LISTS * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->d_lidx + L_PREC * ctx->Bmax, li.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(ctx->d_tick, 0, (size_t)B * sizeof(unsigned), s));
    CK(cudaMemsetAsync(ctx->d_ndone, 0, sizeof(int), s));
    Params P = make_params(ctx, B, ctx->d_x64, o, m, use_tc);
    Launch L{ctx->grid, s};
    launch_field_kappa(ctx->geo, B, ctx->n_mu, ctx->d_mu, s);
    launch_cholesky(P, s, ctx->d_ANq, ctx->P);
    CK(cudaMemcpyAsync(P.r, r, (size_t)B * N * es, cudaMemcpyDefault, s));
    if (ctx->n == 0) CK(cudaMemsetAsync(P.ypro, 0, (size_t)B * N * es, s));
    enqueue_prec(ctx, P, L, o, m, use_tc);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(y, P.y, (size_t)B * N * es, cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(ctx->h_st, ctx->d_st, (size_t)B * sizeof(QState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int q = 0; q < B; ++q)
        if (ctx->h_st[q].status == RB_EBREAKDOWN) return RB_EBREAKDOWN;
    return RB_OK;
}

rb_status rb_autotune(rb_ctx* ctx, int B, const double* mu, double* x, rb_opts* opts, rb_tune_result* res) {
    if (!ctx || !opts || B < 1 || !mu || !x) {
        if (ctx) ctx->err = "rb_autotune needs opts, B >= 1, mu and x";
        return RB_EINVAL;
    }
    TRY(validate_opts(ctx, *opts));
    cudaStream_t s = opts->stream ? (cudaStream_t)opts->stream : ctx->own_stream;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    std::vector<rb_stats> st(B);
    int trials = 0;
    // time of one batch (after one untimed run); +inf if a query does not converge
    auto trial = [&](const rb_opts& t) -> double {
        ++trials;
        if (rb_pcg(ctx, B, mu, x, &t, st.data()) != RB_OK) return 1e300;
        cudaEventRecord(e0, s);
        const rb_status r = rb_pcg(ctx, B, mu, x, &t, st.data());
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        return r == RB_OK ? (double)ms : 1e300;
    };
    rb_opts best = *opts;
    double best_ms = trial(best);
    // the start: zero or the RB approximation (a basis that resolves the solutions makes the RB
    // start converge in a step or two; a rougher one can make it slower than zero)
    const bool try_start = opts->x0_mode != RB_X0_GIVEN && ctx->n > 0;
    auto other_start = [&]() {
        if (!try_start) return;
        rb_opts t = best;
        t.x0_mode = best.x0_mode == RB_X0_RB ? RB_X0_ZERO : RB_X0_RB;
        const double ms = trial(t);
        if (ms < best_ms) { best_ms = ms; best = t; }
    };
    other_start();
    // sweep count, for each storage of the smoother's iterates that applies (BF16
    // makes a sweep cheaper and may move the best nu)
    const bool bf16_ok = opts->precision == RB_PREC_MIXED && opts->smoother == RB_SMOOTH_RBGS &&
                         rowmarch_ok(ctx) && use_tma_smoother(ctx->geo);
    const rb_opts start = best;
    for (int store = RB_STORE_F32; store <= (bf16_ok ? RB_STORE_BF16 : RB_STORE_F32); ++store) {
        for (int nu = 1; nu <= 6; ++nu) {
            if (nu == start.nu && store == start.store) continue;
            rb_opts t = start;
            t.nu = nu;
            t.store = store;
            if (store == RB_STORE_BF16) t.kernels = 0;
            const double ms = trial(t);
            if (ms < best_ms) { best_ms = ms; best = t; }
        }
    }
    if (best.precision == RB_PREC_MIXED) {
        const double tols[3] = {1e-4, 1e-5, 1e-6};
        const rb_opts base = best;
        for (double it : tols) {
            if (it == base.inner_tol) continue;
            rb_opts t = base;
            t.inner_tol = it;
            const double ms = trial(t);
            if (ms < best_ms) { best_ms = ms; best = t; }
        }
        if (tc_usable(ctx->tc, ctx->n)) {
            rb_opts t = best;
            t.gemm = best.gemm == RB_GEMM_CUDA_CORES ? RB_GEMM_TENSOR : RB_GEMM_CUDA_CORES;
            const double ms = trial(t);
            if (ms < best_ms) { best_ms = ms; best = t; }
        }
        if (best.smoother == RB_SMOOTH_RBGS && ctx->n_fields == 0 && (rowmarch_ok(ctx) || zmarch_ok(ctx, false))) {
            const rb_opts base = best;
            for (int kk = 0; kk <= 4; ++kk) {
                if (kk == base.kernels || (kk == 1 && ctx->geo.dim == 2 && !use_fused_smoother(ctx->geo, base.nu)))
                    continue;
                if (kk >= 3 && (ctx->geo.dim != 2 || !use_multi_smoother(ctx->geo))) continue;
                rb_opts t = base;
                t.kernels = kk;
                // BF16 iterates need kernels = 0: the other families are tried with FP32 storage (a
                // local optimum of the storage must not hide them)
                if (kk != 0 && t.store == RB_STORE_BF16) t.store = RB_STORE_F32;
                const double ms = trial(t);
                if (ms < best_ms) { best_ms = ms; best = t; }
            }
            // a smoother that makes several sweeps per pass moves the best sweep count up
            if (best.kernels >= 3) {
                const rb_opts b2 = best;
                for (int nu = 2; nu <= 9; ++nu) {
                    if (nu == b2.nu) continue;
                    rb_opts t = b2;
                    t.nu = nu;
                    const double ms = trial(t);
                    if (ms < best_ms) { best_ms = ms; best = t; }
                }
            }
        }
    }
    other_start();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_ms >= 1e299) { ctx->err = "no candidate configuration converged on the sample"; return RB_ENOCONV; }
    *opts = best;
    if (res) {
        res->nu = best.nu;
        res->inner_tol = best.inner_tol;
        res->gemm = best.gemm;
        res->ms_per_solve = best_ms / B;
        res->trials = trials;
        res->kernels = best.kernels;
        res->store = best.store;
        res->x0_mode = best.x0_mode;
    }
    return RB_OK;
}

rb_status rb_solve(rb_ctx* ctx, int B, const double* mu, double* x, const rb_opts* opts, rb_stats* stats) {
    return run_batch(ctx, B, mu, x, opts, stats, Mode{true, false});
}

rb_status rb_pcg(rb_ctx* ctx, int B, const double* mu, double* x, const rb_opts* opts, rb_stats* stats) {
    return run_batch(ctx, B, mu, x, opts, stats, Mode{false, false});
}

rb_status rb_pcg_ragged(rb_ctx* const* ctxs, int nctx, const int* B, const double* const* mu, double* const* x,
                        const rb_opts* opts, rb_stats* const* stats) {
    if (!ctxs || !B || !mu || !x || nctx < 1 || nctx > 16) {
        g_create_error = "rb_pcg_ragged needs 1..16 contexts and their B, mu and x";
        return RB_EINVAL;
    }
    rb_opts o;
    rb_default_opts(&o);
    if (opts) o = *opts;
    std::vector<Wave> waves(nctx);
    for (int c = 0; c < nctx; ++c) {
        rb_ctx* ctx = ctxs[c];
        if (!ctx) { g_create_error = "a context is NULL"; return RB_EINVAL; }
        for (int d = 0; d < c; ++d)
            if (ctxs[d] == ctx) { g_create_error = "a context appears twice"; return RB_EINVAL; }
        TRY(validate_opts(ctx, o));
        if (B[c] < 0 || B[c] > ctx->Bmax || (B[c] > 0 && (!mu[c] || !x[c]))) {
            ctx->err = "need 0 <= B <= max_batch of the context and non-NULL mu, x";
            return RB_EINVAL;
        }
        bool bad = false;
        if (B[c] > 0 && !is_device_ptr(ctx, x[c], &bad)) {
            if (!bad) ctx->err = "rb_pcg_ragged needs x in device memory";
            return RB_EINVAL;
        }
        Wave& w = waves[c];
        w.ctx = ctx;
        w.B = B[c];
        w.x64 = x[c];
        w.x_given = o.x0_mode == RB_X0_GIVEN;
        w.o = o;
        w.o.stream = nullptr;   // every context advances on its own stream
        w.m = Mode{false, o.precision == RB_PREC_MIXED};
        w.s = ctx->own_stream;
        w.finished = B[c] == 0;
    }
    // every context's setup, then one launch sequence: each round enqueues CHECK_EVERY steps of
    // every unfinished context on its own stream (the kernels of the contexts run side by
    // side on the GPU), then polls them all
    if (o.stream) CK_GLOBAL(cudaStreamSynchronize((cudaStream_t)o.stream));
    for (int c = 0; c < nctx; ++c)
        if (!waves[c].finished) TRY(wave_begin(waves[c], mu[c]));
    for (;;) {
        bool any = false;
        for (Wave& w : waves)
            if (!w.finished) {
                rb_status e = wave_launch(w);
                if (e != RB_OK) { w.rs = e; w.finished = true; }
                any = true;
            }
        if (!any) break;
        for (Wave& w : waves)
            if (!w.finished) wave_check(w);
    }
    rb_status worst = RB_OK;
    for (int c = 0; c < nctx; ++c) {
        rb_status r = B[c] > 0 ? wave_end(waves[c], stats ? stats[c] : nullptr) : RB_OK;
        if (r > worst) worst = r;
    }
    return worst;
}

rb_status rb_apply(rb_ctx* ctx, int B, const double* mu, const double* x, double* y, void* stream) {
    if (!ctx) return RB_EINVAL;
    if (B < 0 || (B > 0 && (!mu || !x || !y))) { ctx->err = "B < 0 or NULL argument"; return RB_EINVAL; }
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->own_stream;
    const long long N = ctx->N;
    bool bad = false;
    const bool dx = is_device_ptr(ctx, x, &bad), dy = is_device_ptr(ctx, y, &bad);
    if (bad) return RB_EINVAL;
    for (int b0 = 0; b0 < B; b0 += ctx->Bmax) {
        const int nbw = std::min(ctx->Bmax, B - b0);
        for (size_t i = 0; i < (size_t)nbw * ctx->n_mu; ++i)
            if (!std::isfinite(mu[(size_t)b0 * ctx->n_mu + i])) { ctx->err = "non-finite parameter"; return RB_EINVAL; }
        CK(cudaMemcpyAsync(ctx->d_mu, mu + (size_t)b0 * ctx->n_mu, (size_t)nbw * ctx->n_mu * sizeof(double),
                           cudaMemcpyHostToDevice, s));
        const double* xs = dx ? x + (size_t)b0 * N : ctx->d_x64;
        double* ys = dy ? y + (size_t)b0 * N : ctx->d_y64;
        if (!dx) CK(cudaMemcpyAsync(ctx->d_x64, x + (size_t)b0 * N, (size_t)nbw * N * sizeof(double),
                                    cudaMemcpyHostToDevice, s));
        launch_apply(ctx->geo, nbw, ctx->n_mu, ctx->d_mu, xs, ys, s);
        CK(cudaGetLastError());
        if (!dy) CK(cudaMemcpyAsync(y + (size_t)b0 * N, ys, (size_t)nbw * N * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return RB_OK;
}

rb_status rb_warm_start(rb_ctx* ctx, rb_mlp* net, int B, const double* mu, double* x, double* coef, void* stream) {
    if (!ctx) return RB_EINVAL;
    if (B < 0 || (B > 0 && (!mu || !x))) { ctx->err = "B < 0 or NULL mu / x"; return RB_EINVAL; }
    if (net && (mlp_n_in(net) != ctx->n_mu || mlp_n_out(net) != ctx->n)) {
        ctx->err = "the network must map n_mu parameters to n coefficients of this context";
        return RB_EINVAL;
    }
    if (net && !mlp_ready(net)) { ctx->err = "the network has not been fitted"; return RB_EINVAL; }
    if (pointer_kind(mu) != PTR_HOST) { ctx->err = "mu must be host memory"; return RB_EINVAL; }
    for (size_t i = 0; i < (size_t)B * ctx->n_mu; ++i) {
        if (!std::isfinite(mu[i]) || ((int)(i % ctx->n_mu) < ctx->P && !(mu[i] > 0.0))) {
            ctx->err = "parameter vectors must be finite, with positive diffusion coefficients";
            return RB_EINVAL;
        }
    }
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->own_stream;
    const long long N = ctx->N;
    const int n = ctx->n;
    bool bad = false;
    const bool dx = is_device_ptr(ctx, x, &bad), dc = coef && is_device_ptr(ctx, coef, &bad);
    if (bad) return RB_EINVAL;
    LoadMap lm{};
    for (int r = 0; r < ctx->R; ++r) lm.param[r] = ctx->load_param[r];
    const int chunk = std::max(1, std::min<int>(ctx->Bmax, (int)(ctx->scratch_bytes / sizeof(double)) / std::max(1, n)));
    CK(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), s));
    for (int b0 = 0; b0 < B; b0 += chunk) {
        const int nbw = std::min(chunk, B - b0);
        CK(cudaMemcpyAsync(ctx->d_mu, mu + (size_t)b0 * ctx->n_mu, (size_t)nbw * ctx->n_mu * sizeof(double),
                           cudaMemcpyHostToDevice, s));
        double* c = dc ? coef + (size_t)b0 * n : ctx->d_scratch;
        if (n > 0) {
            if (net) {
                rb_status st = mlp_predict_device(net, nbw, ctx->d_mu, ctx->n_mu, c, s);
                if (st != RB_OK) { ctx->err = "network evaluation failed"; return st; }
            } else {
                launch_galerkin(n, ctx->P, ctx->d_ANq, ctx->R, lm, ctx->d_fNr, ctx->n_mu, nbw, ctx->d_mu, c,
                                ctx->d_flag, s);
            }
        }
        double* xs = dx ? x + (size_t)b0 * N : ctx->d_x64;
        launch_lift(N, n, ctx->d_W32c, nbw, c, xs, ctx->grid, s);
        CK(cudaGetLastError());
        if (!dx) CK(cudaMemcpyAsync(x + (size_t)b0 * N, xs, (size_t)nbw * N * sizeof(double), cudaMemcpyDeviceToHost, s));
        if (coef && !dc && n > 0)
            CK(cudaMemcpyAsync(coef + (size_t)b0 * n, c, (size_t)nbw * n * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    int notspd = 0;
    CK(cudaMemcpyAsync(&notspd, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (notspd) { ctx->err = "A_N(mu) is not positive definite for some query"; return RB_EBREAKDOWN; }
    return RB_OK;
}

namespace {

// Galerkin coefficients a_N(mu_b) of eq. 2 for B <= Bmax host parameter vectors into coef
// (device [B][n]); RB_EBREAKDOWN when some A_N(mu_b) is not SPD
rb_status galerkin_device(rb_ctx* ctx, int B, const double* mu, double* coef, cudaStream_t s) {
    LoadMap lm{};
    for (int r = 0; r < ctx->R; ++r) lm.param[r] = ctx->load_param[r];
    CK(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), s));
    CK(cudaMemcpyAsync(ctx->d_mu, mu, (size_t)B * ctx->n_mu * sizeof(double), cudaMemcpyHostToDevice, s));
    launch_galerkin(ctx->n, ctx->P, ctx->d_ANq, ctx->R, lm, ctx->d_fNr, ctx->n_mu, B, ctx->d_mu, coef, ctx->d_flag, s);
    CK(cudaGetLastError());
    int notspd = 0;
    CK(cudaMemcpyAsync(&notspd, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (notspd) { ctx->err = "A_N(mu) is not positive definite for some query"; return RB_EBREAKDOWN; }
    return RB_OK;
}

rb_status check_mu_positive(rb_ctx* ctx, int B, const double* mu) {
    if (pointer_kind(mu) != PTR_HOST) { ctx->err = "mu must be host memory"; return RB_EINVAL; }
    for (size_t i = 0; i < (size_t)B * ctx->n_mu; ++i)
        if (!std::isfinite(mu[i]) || ((int)(i % ctx->n_mu) < ctx->P && !(mu[i] > 0.0))) {
            ctx->err = "parameter vectors must be finite, with positive diffusion coefficients";
            return RB_EINVAL;
        }
    return RB_OK;
}

// E = X - W a_N(mu) for B <= Bmax solutions X (host or device) into ctx->d_r64
rb_status errors_device(rb_ctx* ctx, int B, const double* mu, const double* X, cudaStream_t s) {
    const long long N = ctx->N;
    bool bad = false;
    const bool dx = is_device_ptr(ctx, X, &bad);
    if (bad) return RB_EINVAL;
    const double* Xd = X;
    if (!dx) {
        CK(cudaMemcpyAsync(ctx->d_x64, X, (size_t)B * N * sizeof(double), cudaMemcpyHostToDevice, s));
        Xd = ctx->d_x64;
    }
    double* a = ctx->d_scratch;   // [B][n]
    TRY(galerkin_device(ctx, B, mu, a, s));
    launch_eb_errors(N, ctx->n, ctx->d_W64c, B, a, Xd, ctx->d_r64, ctx->grid, s);
    CK(cudaGetLastError());
    return RB_OK;
}

}  // namespace

rb_status rb_error_basis(rb_ctx* ctx, int S, const double* mu, const double* X, int m, double* Z, double* sigma,
                         void* stream) {
    if (!ctx) return RB_EINVAL;
    if (S < 1 || S > ctx->Bmax || S > 512 || m < 1 || m > 64 || m > S || !mu || !X || ctx->n == 0) {
        ctx->err = "need 1 <= m <= min(S, 64), 1 <= S <= min(max_batch, 512), mu, X and a basis";
        return RB_EINVAL;
    }
    TRY(check_mu_positive(ctx, S, mu));
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->own_stream;
    const long long N = ctx->N;
    if ((size_t)2 * ctx->Bmax * N < eb_gram_part_elems(S) || ctx->scratch_bytes / sizeof(double) < (size_t)S * S) {
        ctx->err = "grid too small for the Gram partial sums of this many snapshots";
        return RB_EINVAL;
    }
    TRY(errors_device(ctx, S, mu, X, s));
    // Gram matrix E^T E: partial sums in the (idle) FP64 direction workspace, the sum in scratch
    double* G = ctx->d_scratch;
    launch_eb_gram(N, S, ctx->d_r64, ctx->d_p64, G, ctx->grid, s);
    CK(cudaGetLastError());
    std::vector<double> Gh((size_t)S * S), lam, Phi;
    CK(cudaMemcpyAsync(Gh.data(), G, Gh.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    jacobi_eigen(S, Gh, lam, Phi);
    // modes whose singular value is below 1e-12 of the largest carry nothing: zero columns
    std::vector<double> C((size_t)S * m, 0.0), sig(m, 0.0);
    for (int k = 0; k < m; ++k) {
        const double l = lam[k] > 0.0 ? lam[k] : 0.0;
        sig[k] = std::sqrt(l);
        if (!(sig[k] > 1e-12 * std::sqrt(std::max(lam[0], 0.0)))) { sig[k] = 0.0; continue; }
        for (int i = 0; i < S; ++i) C[(size_t)i * m + k] = Phi[(size_t)i * S + k] / sig[k];
    }
    if (ctx->m_err != m) {
        if (ctx->d_V64) cudaFree(ctx->d_V64);
        if (ctx->d_V32) cudaFree(ctx->d_V32);
        ctx->d_V64 = nullptr;
        ctx->d_V32 = nullptr;
        ctx->m_err = 0;
        if (cudaMalloc((void**)&ctx->d_V64, (size_t)m * N * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void**)&ctx->d_V32, (size_t)m * N * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            ctx->err = "allocation of the error basis failed";
            return RB_ENOMEM;
        }
    }
    double* dC = ctx->d_scratch;   // G is no longer needed
    CK(cudaMemcpyAsync(dC, C.data(), C.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    launch_eb_modes(N, S, m, ctx->d_r64, dC, ctx->d_V64, ctx->d_V32, ctx->grid, s);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    ctx->m_err = m;
    // Z = V^T E = diag(sigma) Phi_m^T, [S][m]
    if (Z) {
        std::vector<double> Zh((size_t)S * m);
        for (int i = 0; i < S; ++i)
            for (int k = 0; k < m; ++k) Zh[(size_t)i * m + k] = sig[k] * Phi[(size_t)i * S + k];
        CK(cudaMemcpyAsync(Z, Zh.data(), Zh.size() * sizeof(double), cudaMemcpyDefault, s));
        CK(cudaStreamSynchronize(s));
    }
    if (sigma) std::copy(sig.begin(), sig.end(), sigma);
    return RB_OK;
}

rb_status rb_error_coefficients(rb_ctx* ctx, int B, const double* mu, const double* X, double* Z, void* stream) {
    if (!ctx) return RB_EINVAL;
    if (B < 0 || (B > 0 && (!mu || !X || !Z))) { ctx->err = "B < 0 or NULL mu / X / Z"; return RB_EINVAL; }
    if (ctx->m_err == 0) { ctx->err = "the context has no error basis (rb_error_basis)"; return RB_EINVAL; }
    TRY(check_mu_positive(ctx, B, mu));
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->own_stream;
    const long long N = ctx->N;
    const int m = ctx->m_err;
    bool bad = false;
    const bool dX = is_device_ptr(ctx, X, &bad), dZ = is_device_ptr(ctx, Z, &bad);
    if (bad) return RB_EINVAL;
    const size_t sd = ctx->scratch_bytes / sizeof(double);
    int chunk = std::min(ctx->Bmax, 256);
    while (chunk > 1 && (size_t)coef_splits(chunk, ctx->num_sms) * chunk * m + (size_t)chunk * (ctx->n + m) > sd)
        chunk /= 2;
    for (int b0 = 0; b0 < B; b0 += chunk) {
        const int nbw = std::min(chunk, B - b0);
        TRY(errors_device(ctx, nbw, mu + (size_t)b0 * ctx->n_mu, dX ? X + (size_t)b0 * N : X + (size_t)b0 * N, s));
        double* zc = dZ ? Z + (size_t)b0 * m : ctx->d_scratch + (size_t)chunk * ctx->n;
        launch_coefficients(N, m, ctx->d_V32, nbw, ctx->d_r64, zc, ctx->d_scratch + (size_t)chunk * (ctx->n + m),
                            ctx->num_sms, s);
        CK(cudaGetLastError());
        if (!dZ) CK(cudaMemcpyAsync(Z + (size_t)b0 * m, zc, (size_t)nbw * m * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return RB_OK;
}

rb_status rb_warm_start_error(rb_ctx* ctx, rb_mlp* net, int B, const double* mu, double* x, const double* z,
                              void* stream) {
    if (!ctx) return RB_EINVAL;
    if (B < 0 || (B > 0 && (!mu || !x))) { ctx->err = "B < 0 or NULL mu / x"; return RB_EINVAL; }
    if (ctx->m_err == 0) { ctx->err = "the context has no error basis (rb_error_basis)"; return RB_EINVAL; }
    if ((net == nullptr) == (z == nullptr)) { ctx->err = "give exactly one of a network and coefficients z"; return RB_EINVAL; }
    if (net && (mlp_n_in(net) != ctx->n_mu || mlp_n_out(net) != ctx->m_err)) {
        ctx->err = "the network must map n_mu parameters to the m coefficients of the error basis";
        return RB_EINVAL;
    }
    if (net && !mlp_ready(net)) { ctx->err = "the network has not been fitted"; return RB_EINVAL; }
    TRY(check_mu_positive(ctx, B, mu));
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->own_stream;
    const long long N = ctx->N;
    const int n = ctx->n, m = ctx->m_err;
    bool bad = false;
    const bool dx = is_device_ptr(ctx, x, &bad);
    const bool dz = z && is_device_ptr(ctx, z, &bad);
    if (bad) return RB_EINVAL;
    const int chunk = std::max(1, std::min<int>(ctx->Bmax, (int)(ctx->scratch_bytes / sizeof(double)) / (n + m)));
    for (int b0 = 0; b0 < B; b0 += chunk) {
        const int nbw = std::min(chunk, B - b0);
        double* a = ctx->d_scratch;
        double* zc = ctx->d_scratch + (size_t)chunk * n;
        TRY(galerkin_device(ctx, nbw, mu + (size_t)b0 * ctx->n_mu, a, s));
        if (net) {
            rb_status st = mlp_predict_device(net, nbw, ctx->d_mu, ctx->n_mu, zc, s);
            if (st != RB_OK) { ctx->err = "network evaluation failed"; return st; }
        } else {
            CK(cudaMemcpyAsync(zc, z + (size_t)b0 * m, (size_t)nbw * m * sizeof(double),
                               dz ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        }
        double* xs = dx ? x + (size_t)b0 * N : ctx->d_x64;
        launch_lift(N, n, ctx->d_W32c, nbw, a, xs, ctx->grid, s);
        launch_eb_lift_add(N, m, ctx->d_V32, nbw, zc, xs, ctx->grid, s);
        CK(cudaGetLastError());
        if (!dx) CK(cudaMemcpyAsync(x + (size_t)b0 * N, xs, (size_t)nbw * N * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return RB_OK;
}

rb_status rb_coefficients(rb_ctx* ctx, int B, const double* x, double* coef, void* stream) {
    if (!ctx) return RB_EINVAL;
    if (B < 0 || (B > 0 && (!x || !coef))) { ctx->err = "B < 0 or NULL x / coef"; return RB_EINVAL; }
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->own_stream;
    const long long N = ctx->N;
    const int n = ctx->n;
    if (n == 0 || B == 0) return RB_OK;
    bool bad = false;
    const bool dx = is_device_ptr(ctx, x, &bad), dc = is_device_ptr(ctx, coef, &bad);
    if (bad) return RB_EINVAL;
    const size_t sd = ctx->scratch_bytes / sizeof(double);
    int chunk = std::min(ctx->Bmax, 256);
    while (chunk > 1 && (size_t)coef_splits(chunk, ctx->num_sms) * chunk * n > sd) chunk /= 2;
    for (int b0 = 0; b0 < B; b0 += chunk) {
        const int nbw = std::min(chunk, B - b0);
        const double* xs = dx ? x + (size_t)b0 * N : ctx->d_x64;
        if (!dx) CK(cudaMemcpyAsync(ctx->d_x64, x + (size_t)b0 * N, (size_t)nbw * N * sizeof(double),
                                    cudaMemcpyHostToDevice, s));
        double* c = dc ? coef + (size_t)b0 * n : ctx->d_e64;
        launch_coefficients(N, n, ctx->d_W32c, nbw, xs, c, ctx->d_scratch, ctx->num_sms, s);
        CK(cudaGetLastError());
        if (!dc) CK(cudaMemcpyAsync(coef + (size_t)b0 * n, c, (size_t)nbw * n * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return RB_OK;
}

}  // extern "C"

#include "rb_offline.inl"
