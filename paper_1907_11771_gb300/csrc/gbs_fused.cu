// Time-blocked FP32 macro-step kernels (not yet available: the plain path is used).
#include "gbs_internal.h"

namespace gbs {

bool fused_supported(const StepPlan&) { return false; }
int64_t fused_scratch_bytes(const StepPlan&) { return 0; }
int fused_macro_step(const StepPlan&, const void*, void*, cudaStream_t, int*, void*, int64_t) { return -1; }

}  // namespace gbs
