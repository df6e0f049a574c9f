// Serving: continuous batching of k-point requests.
#include "plan.h"

struct ServeState {};

void hs_plan_s::serve_shutdown() {}

extern "C" int hs_submit(hs_plan_t, const hs_z*, const hs_z*, int, const double*, int, hs_z*,
                         hs_z*, int64_t*) {
  return HS_ENOTSUP;
}
extern "C" int hs_poll(hs_plan_t, int64_t, int64_t, hs_info*) { return HS_ENOTSUP; }
