// rb_residual_noalloc: relative residuals ||f(mu) - A(mu) x|| / ||f(mu)|| of a
// batch of device vectors, computed without allocating any device memory.
//
// Why it exists: some callers cannot call cudaMalloc.  A framework that keeps
// the device's memory in its own caching allocator may have reserved nearly
// all of it, so a fresh cudaMalloc can fail.  A latency-sensitive caller also
// cannot accept the device-wide synchronisation that cudaMalloc / cudaFree may
// imply.  Such a caller can still check its solutions with this entry point: it
// needs no context (a context allocates its workspace), and its only scratch
// memory is the file-scope array below.
//
// The scratch is a fixed 1 MiB array that every GPU which loads the library
// holds until the process exits.  The kernel is a variant of the outer-residual
// kernel of the solvers: per-tile partial sums of ||r||^2 and ||f||^2 go to
// the scratch instead of a context workspace, then one warp per query adds
// them in a fixed order.  Block indices and load terms are computed on the
// fly, so no table of the context is needed either.
#include <cuda.h>   // driver types only (entry points are looked up through the runtime)
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "rb_common.cuh"

namespace rbk {
void set_global_error(const std::string& m);
}

namespace {

constexpr size_t NA_SCRATCH_BYTES = size_t(1) << 20;
constexpr int NA_THREADS = 256;
constexpr int NA_TILE = 1024;
constexpr int NA_MAX_DEVICES = 64;

// Host code must not take this symbol's address directly: there it names a
// host-side stand-in, not device memory.  The device address comes from
// cudaGetSymbolAddress (see na_scratch_address).
static __device__ __align__(256) unsigned char g_na_scratch[NA_SCRATCH_BYTES];

std::mutex g_na_mutex;
// per device: the CUDA context the address was looked up in (its process-unique id) and the address
struct NaSlot {
    unsigned long long ctx_id;
    void* addr;
};
NaSlot g_na_slot[NA_MAX_DEVICES] = {};

// error text is reported through rb_last_error(NULL)
struct NaError {
    void clear() { rbk::set_global_error(std::string()); }
    NaError& operator=(const std::string& m) { rbk::set_global_error(m); return *this; }
    NaError& operator=(const char* m) { rbk::set_global_error(m ? std::string(m) : std::string()); return *this; }
};
NaError g_na_error;

struct NaProblem {
    int dim, mx, my, mz, nbx, nby, nbz, n_mu, R;
    long long n;
    double ihx2, ihy2, ihz2;
    int kind[rbk::MAX_LOADS], param[rbk::MAX_LOADS];
    double cx[rbk::MAX_LOADS], cy[rbk::MAX_LOADS], cz[rbk::MAX_LOADS], sigma[rbk::MAX_LOADS];
};

__device__ __forceinline__ int na_block(int i, int nb, int m) { return (int)(((long long)i * nb) / m); }

__device__ __forceinline__ double na_mu(const NaProblem& g, const double* mus, int ix, int iy, int iz) {
    return mus[na_block(ix, g.nbx, g.mx) + g.nbx * (na_block(iy, g.nby, g.my) + g.nby * na_block(iz, g.nbz, g.mz))];
}

// r = f - A x at every point of a flat tile of one query; partial sums of r^2 and f^2.
__global__ void __launch_bounds__(NA_THREADS) k_na_partials(NaProblem g, const double* __restrict__ mu_all,
                                                           const double* __restrict__ x_all, double* part,
                                                           int ntiles) {
    __shared__ double mus[rbk::MAX_MU];
    __shared__ double red[2][NA_THREADS / 32];
    const int q = blockIdx.y, tile = blockIdx.x;
    if (threadIdx.x < g.n_mu) mus[threadIdx.x] = mu_all[(size_t)q * g.n_mu + threadIdx.x];
    __syncthreads();
    const double* x = x_all + (size_t)q * g.n;
    double rr = 0.0, ff = 0.0;
    for (int j = 0; j < NA_TILE / NA_THREADS; ++j) {
        const long long i = (long long)tile * NA_TILE + j * NA_THREADS + threadIdx.x;
        if (i >= g.n) continue;
        const int ix = (int)(i % g.mx);
        const int iy = (int)((i / g.mx) % g.my);
        const int iz = (int)(i / ((long long)g.mx * g.my));
        // f(mu) at the node
        double b = 0.0;
        for (int r = 0; r < g.R; ++r) {
            const double phi = g.param[r] < 0 ? 1.0 : mus[g.param[r]];
            double v = 1.0;
            if (g.kind[r] == RB_LOAD_GAUSS) {
                const double px = (ix + 1.0) / (g.mx + 1.0), py = (iy + 1.0) / (g.my + 1.0);
                double d2 = (px - g.cx[r]) * (px - g.cx[r]) + (py - g.cy[r]) * (py - g.cy[r]);
                if (g.dim == 3) {
                    const double pz = (iz + 1.0) / (g.mz + 1.0);
                    d2 += (pz - g.cz[r]) * (pz - g.cz[r]);
                }
                v = exp(-d2 / (2.0 * g.sigma[r] * g.sigma[r]));
            }
            b += phi * v;
        }
        // A x at the node: faces to the neighbours (value 0 outside the grid)
        // same association as the solvers' residual: diag = ((kxm + kxp) + kym) + kyp [+ (kzm + kzp)],
        // off-diagonal terms added in the order x-, x+, y-, y+, z-, z+
        const double m = na_mu(g, mus, ix, iy, iz);
        const double kxm = g.ihx2 * (ix > 0 ? 0.5 * (m + na_mu(g, mus, ix - 1, iy, iz)) : m);
        const double kxp = g.ihx2 * (ix < g.mx - 1 ? 0.5 * (m + na_mu(g, mus, ix + 1, iy, iz)) : m);
        const double kym = g.ihy2 * (iy > 0 ? 0.5 * (m + na_mu(g, mus, ix, iy - 1, iz)) : m);
        const double kyp = g.ihy2 * (iy < g.my - 1 ? 0.5 * (m + na_mu(g, mus, ix, iy + 1, iz)) : m);
        double diag = kxm + kxp + kym + kyp;
        double off = 0.0;
        if (ix > 0) off += kxm * x[i - 1];
        if (ix < g.mx - 1) off += kxp * x[i + 1];
        if (iy > 0) off += kym * x[i - g.mx];
        if (iy < g.my - 1) off += kyp * x[i + g.mx];
        if (g.dim == 3) {
            const long long pl = (long long)g.mx * g.my;
            const double kzm = g.ihz2 * (iz > 0 ? 0.5 * (m + na_mu(g, mus, ix, iy, iz - 1)) : m);
            const double kzp = g.ihz2 * (iz < g.mz - 1 ? 0.5 * (m + na_mu(g, mus, ix, iy, iz + 1)) : m);
            diag += kzm + kzp;
            if (iz > 0) off += kzm * x[i - pl];
            if (iz < g.mz - 1) off += kzp * x[i + pl];
        }
        const double rv = b - (diag * x[i] - off);
        rr += rv * rv;
        ff += b * b;
    }
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_down_sync(0xffffffffu, rr, o);
        ff += __shfl_down_sync(0xffffffffu, ff, o);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { red[0][w] = rr; red[1][w] = ff; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int k = 0; k < NA_THREADS / 32; ++k) { a += red[0][k]; c += red[1][k]; }
        part[((size_t)q * ntiles + tile) * 2 + 0] = a;
        part[((size_t)q * ntiles + tile) * 2 + 1] = c;
    }
}

// one warp per query: fixed-order sum of the tile partials
__global__ void k_na_finish(int B, int ntiles, const double* part, double* out) {
    const int q = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (q >= B) return;
    double rr = 0.0, ff = 0.0;
    for (int t = lane; t < ntiles; t += 32) {
        rr += part[((size_t)q * ntiles + t) * 2 + 0];
        ff += part[((size_t)q * ntiles + t) * 2 + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_down_sync(0xffffffffu, rr, o);
        ff += __shfl_down_sync(0xffffffffu, ff, o);
    }
    if (lane == 0) out[q] = ff > 0.0 ? sqrt(rr) / sqrt(ff) : sqrt(rr);
}

size_t round256(size_t v) { return (v + 255) & ~size_t(255); }

// Id of the current CUDA context (0 when it cannot be had).  A device reset, or a release and
// re-creation of the primary context, reloads the module, and the scratch array may then live at
// another address; the id tells the two contexts apart.  The driver entry points are looked up
// through the runtime, so the library needs no link to libcuda.
unsigned long long na_context_id() {
    typedef CUresult (*GetCurrent)(CUcontext*);
    typedef CUresult (*GetId)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        cudaGetLastError();
        looked_up = true;
    }
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&c) == CUDA_SUCCESS && c && get_id(c, &id) == CUDA_SUCCESS) return id;
    return 0;
}

// Device address of the scratch array on the current device, looked up with that device
// current on the first call in each context (once per device unless the device is reset).
rb_status na_scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { g_na_error = cudaGetErrorString(e); return RB_ECUDA; }
    if (dev < 0 || dev >= NA_MAX_DEVICES) { g_na_error = "device index out of range"; return RB_EINVAL; }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    NaSlot& slot = g_na_slot[dev];
    const unsigned long long id = na_context_id();
    if (!slot.addr || id == 0 || id != slot.ctx_id) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess || !p) {
            g_na_error = std::string("cudaGetSymbolAddress of the scratch array failed: ") + cudaGetErrorString(e);
            return RB_ECUDA;
        }
        slot.addr = p;
        slot.ctx_id = na_context_id();   // the lookup has made the context current if it was not
    }
    *out = slot.addr;
    return RB_OK;
}

}  // namespace

extern "C" rb_status rb_residual_noalloc(const rb_problem* prob, int B, const double* mu, const double* x,
                                         double* rel_res, void* stream) {
    g_na_error.clear();
    if (B < 0 || (B > 0 && (!mu || !x || !rel_res))) { g_na_error = "NULL argument or B < 0"; return RB_EINVAL; }
    std::string why;
    if (rbk::validate_problem(prob, why) != RB_OK) { g_na_error = why; return RB_EINVAL; }
    bool needs_ctx = prob->n_fields > 0;
    for (int r = 0; r < prob->n_loads; ++r) needs_ctx |= prob->loads[r].kind >= RB_LOAD_ARRAY;
    if (needs_ctx) {
        g_na_error = "coefficient fields and array or boundary loads need a context";
        return RB_EINVAL;
    }
    const long long n = (long long)prob->m[0] * prob->m[1] * prob->m[2];
    if (B == 0) return RB_OK;
    for (size_t i = 0; i < (size_t)B * prob->n_mu; ++i)
        if (!std::isfinite(mu[i])) { g_na_error = "non-finite parameter"; return RB_EINVAL; }
    const rbk::PtrKind xk = rbk::pointer_kind(x);
    if (xk != rbk::PTR_DEVICE) {
        g_na_error = xk == rbk::PTR_OTHER_DEVICE ? "x lives on another device than the current one"
                                                 : "x must be device memory";
        return RB_EINVAL;
    }
    const int ntiles = (int)((n + NA_TILE - 1) / NA_TILE);
    const size_t mu_bytes = round256((size_t)B * prob->n_mu * sizeof(double));
    const size_t part_bytes = round256((size_t)B * ntiles * 2 * sizeof(double));
    const size_t out_bytes = round256((size_t)B * sizeof(double));
    if (mu_bytes + part_bytes + out_bytes > NA_SCRATCH_BYTES) {
        g_na_error = "batch too large for the 1 MiB scratch of rb_residual_noalloc: need " +
                     std::to_string(mu_bytes + part_bytes + out_bytes) + " bytes";
        return RB_EINVAL;
    }
    void* base = nullptr;
    rb_status st = na_scratch_address(&base);
    if (st != RB_OK) return st;
    unsigned char* sb = static_cast<unsigned char*>(base);
    double* d_mu = reinterpret_cast<double*>(sb);
    double* d_part = reinterpret_cast<double*>(sb + mu_bytes);
    double* d_out = reinterpret_cast<double*>(sb + mu_bytes + part_bytes);

    NaProblem g{};
    g.dim = prob->dim;
    g.mx = prob->m[0]; g.my = prob->m[1]; g.mz = prob->m[2];
    g.nbx = prob->nb[0]; g.nby = prob->nb[1]; g.nbz = prob->nb[2];
    g.n_mu = prob->n_mu;
    g.R = prob->n_loads;
    g.n = n;
    g.ihx2 = (double)(g.mx + 1) * (g.mx + 1);
    g.ihy2 = (double)(g.my + 1) * (g.my + 1);
    g.ihz2 = g.dim == 3 ? (double)(g.mz + 1) * (g.mz + 1) : 0.0;
    for (int r = 0; r < g.R; ++r) {
        const rb_load& l = prob->loads[r];
        g.kind[r] = l.kind;
        g.param[r] = l.param;
        g.cx[r] = l.center[0]; g.cy[r] = l.center[1]; g.cz[r] = l.center[2];
        g.sigma[r] = l.sigma;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(d_mu, mu, (size_t)B * prob->n_mu * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_na_partials<<<dim3(ntiles, B), NA_THREADS, 0, s>>>(g, d_mu, x, d_part, ntiles);
        k_na_finish<<<(B + 7) / 8, 256, 0, s>>>(B, ntiles, d_part, d_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(rel_res, d_out, (size_t)B * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { g_na_error = cudaGetErrorString(e); return RB_ECUDA; }
    return RB_OK;
}
