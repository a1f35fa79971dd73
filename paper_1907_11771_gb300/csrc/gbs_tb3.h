// Time-blocked leap-frog passes for 3D acoustics with FP32 states (gbs_tb3.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "gbs_internal.h"

namespace gbs {

struct Tb3Work;
Tb3Work* tb3_create();
void tb3_destroy(Tb3Work* w);
// 3D acoustics, FP32 states, every step count of the slots in use even (a pass advances two
// leap-frog levels)
bool tb3_supported(const StepPlan& p, const ProbDev* probs_h, const SlotDev* slots_h, int n_slots);
// Tiles, z-segments of zseg planes and the second level-buffer pair (set-up time: allocates).
// Returns 0, -2 when the allocation failed, -1 otherwise (msg says why).
int tb3_prepare(Tb3Work* w, const StepPlan& p, const ProbDev* probs_h, const SlotDev* slots_h, int zseg,
                char* msg, size_t msglen);
// Bytes of device memory tb3_prepare allocates for a state of state_elems FP32 scalars.
size_t tb3_workspace_bytes(int64_t state_elems);
// One macro-step (or, with p.partial, the combine share of p.seq_mask's sequences in p.acc):
// f0, then every sequence's passes.  Returns the number of kernels launched, or -1.
int tb3_macro_step(const Tb3Work* w, const StepPlan& p, const void* y_in, void* y_out, cudaStream_t s);

}  // namespace gbs
