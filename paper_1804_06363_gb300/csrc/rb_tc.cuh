// Tensor-core (tcgen05, TF32) engine for the batched projection W^T R and
// prolongation W E of the mixed-precision preconditioner.
#pragma once

#include <string>

#include "rb_common.cuh"

namespace rbk {

struct TcPlan {
    bool ready = false;
    int Bmax = 0;
    int nbp32 = 0;
    int num_sms = 0;
};

rb_status tc_init(TcPlan& t, const Geo& g, int Bmax, int nbp32, int num_sms, std::string& err);
void tc_free(TcPlan& t);
bool tc_usable(const TcPlan& t, int n);
void tc_project(const TcPlan& t, const Params& P, const Launch& L);
void tc_prolong(const TcPlan& t, const Params& P, const Launch& L, const float* W32r);

}  // namespace rbk
