// Split-precision (Ozaki-style) contractions on BF16 tensor cores.
#include "plan.h"

struct SplitWork {};

size_t hs_plan_s::split_bytes(int) const { return 0; }
int hs_plan_s::split_alloc() { return HS_OK; }
void hs_plan_s::split_release() {}
int hs_plan_s::split_enqueue(const SegList&, const SegList&, int, double2*, double2*,
                             cudaStream_t, bool) {
  return HS_ENOTSUP;
}
