// Tensor-core engine of the mixed-precision preconditioner (see rb_tc.cuh).
#include "rb_tc.cuh"

namespace rbk {

rb_status tc_init(TcPlan& t, const Geo& g, int Bmax, int nbp32, int num_sms, std::string& err) {
    (void)g;
    (void)err;
    t.Bmax = Bmax;
    t.nbp32 = nbp32;
    t.num_sms = num_sms;
    t.ready = false;
    return RB_OK;
}

void tc_free(TcPlan& t) { t.ready = false; }

bool tc_usable(const TcPlan& t, int n) { return t.ready && n > 0; }

void tc_project(const TcPlan& t, const Params& P, const Launch& L) {
    (void)t;
    launch_project<float>(P, L);
}

void tc_prolong(const TcPlan& t, const Params& P, const Launch& L, const float* W32r) {
    (void)t;
    (void)W32r;
    launch_prolong<float>(P, L, false);
}

}  // namespace rbk
