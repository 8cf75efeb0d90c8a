// Source-plane chi^2 plans (Eq. chi2_src, Sec. 3.1) -- under construction.
#include "lf_internal.h"

struct lf_plan { int dummy; };

extern "C" lf_status lf_plan_create(lf_plan** out, const lf_cluster*, int32_t, int32_t, int32_t,
                                    int32_t) {
  if (out) *out = nullptr;
  return lf::fail(LF_EUNSUPPORTED, "chi^2 plans are not built yet");
}
extern "C" lf_status lf_chi2_batch(lf_plan*, const double*, int32_t, double*, void*) {
  return lf::fail(LF_EUNSUPPORTED, "chi^2 plans are not built yet");
}
extern "C" lf_status lf_chi2_grad_batch(lf_plan*, const double*, int32_t, double*, double*, void*) {
  return lf::fail(LF_EUNSUPPORTED, "chi^2 plans are not built yet");
}
extern "C" lf_status lf_plan_destroy(lf_plan*) { return LF_OK; }
extern "C" lf_status lf_plan_info(const lf_plan*, int32_t*, int32_t*, int32_t*) {
  return lf::fail(LF_EUNSUPPORTED, "chi^2 plans are not built yet");
}
