// Tensor-core (tcgen05, TF32 operands, FP32 accumulation in TMEM) engine for the
// batched projection r_N = W^T r (eq. 5) and prolongation y = W e_N (eq. 7) of
// the mixed-precision RBI preconditioner.
#pragma once

#include <cuda.h>

#include <string>

#include "rb_common.cuh"

namespace rbk {

struct TcPlan {
    bool ready = false;
    int Bmax = 0;
    int nbp = 0;          // projection N (basis rows of W32c), multiple of 16
    int nbp32 = 0;        // prolongation K (columns of W32r / e32), multiple of 32
    int num_sms = 0;
    long long n = 0;      // grid points
    int mtiles = 0;       // ceil(Bmax / 128)
    int proj_split = 0;   // split-K factor of the projection
    int prol_ctas = 0;    // CTAs per query tile of the prolongation
    size_t proj_smem = 0, prol_smem = 0;
    int proj_stages = 0, prol_stages = 0;
    CUtensorMap tm_r;     // r32 [Bmax][N], box {32, 128}
    CUtensorMap tm_wc;    // W32c [nbp][N], box {32, nbp}
    CUtensorMap tm_e;     // e32 [Bmax][nbp32], box {32, 128}
    CUtensorMap tm_wr;    // W32r [N][nbp32], box {32, 128}
    int* d_err = nullptr; // device flag: a bounded wait gave up
};

// Sets up the plan (tensor maps over the context's buffers).  Leaves t.ready
// false (CUDA-core engine is used) when the sizes do not fit the kernels.
rb_status tc_init(TcPlan& t, const Geo& g, int Bmax, int nb_cap, int nbp, int nbp32, int num_sms, float* r32,
                  const float* W32c, float* e32, const float* W32r, int* d_err, std::string& err);
void tc_free(TcPlan& t);
bool tc_usable(const TcPlan& t, int n);
void tc_project(const TcPlan& t, const Params& P, const Launch& L);
void tc_prolong(const TcPlan& t, const Params& P, const Launch& L);

}  // namespace rbk
