// Sequence-fused one-level step (gbs_plain.cu): FP32 2D/3D acoustics, every sequence of the
// scheme with its own pair of level buffers, so that one launch per leap-frog level n advances
// all sequences that have level n, the blocks of one tile for all of them side by side; their
// shared operands (f0 and the media) then come from DRAM about once per level instead of once
// per sequence.  Needs distinct step counts within a weight slot (at most one sequence finishes
// at a level, so the combine updates of a launch never meet).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gbs_internal.h"

namespace gbs {

struct SeqLevels {
  void* base;          // [2 m][state]: sequence k's levels at buffers 2k (even n) and 2k + 1
  int64_t stride;      // elements between two level buffers (the state size)
  const void* tmap;    // host pointer to the tensor map over base, the fields of all level
                       // buffers merged into its fourth dimension (k_lf_tiled's staging), or NULL
  int group;           // most sequences per launch (0: all of a level's); 3D grids read
                       // z-neighbour planes of the level from the cache, whose window grows with it
};

// One macro-step with the sequence-fused launches where they apply (FP32 acoustics, 2D/3D,
// lv.base set), otherwise plain_macro_step.  Returns the number of kernels launched, or -1.
int plain_macro_step_seqfused(const StepPlan& p, const SeqLevels& lv, const void* y_in, void* y_out, cudaStream_t s);

// The adjoint macro-step of a GBS_F32X2 handle in FP32-pair arithmetic (the adjoint kernels
// instantiated for pairs): y_in, kappa, b and lam_out (FP64) are converted to pairs, lam_in is
// written in FP64 and the gradient accumulated in FP64 as on the FP64 path.  lam_pairs: a
// scratch state of pairs (8 bytes per element).  Returns the number of kernels launched, or -1.
int plain_adjoint_step_pairs(const AdjPlan& a, void* lam_pairs, const void* y_in, const void* lam_out, void* lam_in,
                             double* grad_kappa, const int64_t* rcv_idx, int n_rcv, const void* rcv_resid,
                             cudaStream_t s);

}  // namespace gbs
