// lbcm_internal.h -- declarations shared by the translation units of the library.
#pragma once
#include <cuda_runtime.h>
#include "lbcm_device.cuh"

namespace lbcm {
// One time step (boundary planes, phase field, collision) on stream s, for population
// storage STORE_FP32 or STORE_FP16.  When ev is not
// NULL, ev[0..3] are recorded before the boundary kernel, before the phase-field kernel,
// before the collision kernel and after it.  *launches is increased by the number of
// kernels launched.
cudaError_t launch_step(const StepArgs &a, int storage, cudaStream_t s, cudaEvent_t *ev, long long *launches);
}  // namespace lbcm
