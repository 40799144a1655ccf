// Scratch-slot assignment of the plan and internal entry points shared by
// the C-ABI translation units.
#pragma once

#include "common.cuh"

namespace bdg {

enum ScratchSlot {
  SLOT_GRAM_WS = 0,  // Gram partial sums
  SLOT_SMALL = 1,    // small FP64 matrices
  SLOT_VEC_A = 2,    // one or more block vectors
  SLOT_VEC_B = 3,
  SLOT_SOLVER = 4,   // solver arena
  SLOT_SOLVER2 = 5,
  SLOT_SOLVER3 = 6,
  SLOT_AUX = 7,
  SLOT_PHASE = 8,   // phase tables of the perturbed densities
  SLOT_COUNT = 9,
};
static_assert(sizeof(bdg_plan_s::scratch) / sizeof(Buffer) == SLOT_COUNT, "one scratch buffer per slot");

// y = M x with the plan's chemical potentials, or mu_override if non-NULL.
bdg_status apply_internal(bdg_plan_t plan, int mode, int dtype, const void* x, void* y, int nvec,
                          cudaStream_t s, const double* mu_override);

}  // namespace bdg
