// inplace.h -- launchers of the single-buffer (in-place) step (inplace.cu).
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace mhd {

// One time step on the single buffer s.dst (s.src must equal s.dst; periodic
// x axis).  phase 0 takes the canonical state to the streamed state, phase 1
// the streamed state back to the canonical one.
cudaError_t launch_aa_step(const StepLaunch& s, int phase, cudaStream_t st);
// streamed -> canonical layout of the same time step, without a collision
cudaError_t launch_aa_unstream(const Layout& L, int prec, void* buf, int wall_y, cudaStream_t st);

}  // namespace mhd
