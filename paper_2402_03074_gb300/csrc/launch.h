// launch.h -- host-side declarations shared by the engine and the kernel translation units.
#pragma once
#include <cuda_runtime.h>

#include "hweno_device.cuh"

namespace hw {

// One stage of the modified SSP-RK3 over a whole grid (1D / 2D), asynchronous on st.
cudaError_t launch_stage1d(int eq, bool characteristic, bool mixed, const KProblem& P,
                           const KStage& S, cudaStream_t st);
cudaError_t launch_stage2d(int eq, bool characteristic, bool mixed, const KProblem& P,
                           const KStage& S, cudaStream_t st);
// Wave speeds of a state (raises alpha_out[0..1]).
cudaError_t launch_alpha(int eq, int dim, const KProblem& P, const double* U, double* alpha_out,
                         cudaStream_t st);

}  // namespace hw
