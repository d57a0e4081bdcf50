// launch.h -- host-side declarations shared by the engine and the kernel translation units.
#pragma once
#include <cuda_runtime.h>

#include "hweno_device.cuh"

namespace hw {

// Device-resident scalars of a solve.
struct DevScal {
  double alpha[4][2];  // [3]: LF speeds of U^n (previous step / open); [0..2]: stage inputs
  double dt;
  double t;
  double t_end;
  double dt_fixed;
  double cfl;
  long long steps;
  long long step_limit;
  int active;
  uint32_t status;
};

// Start of a time step (one thread): Delta t from the LF speeds of U^n (CFL rule) or the
// fixed step, clipped to t_end; clears the speed slots the three stages raise; sets `active`
// (0 once t_end, the step limit or a non-physical state is reached; the informational status
// bits do not stop the solve).
__device__ __forceinline__ void dt_update(DevScal* s, double inv_dx, double inv_dy, int dim) {
  const double a0 = s->alpha[3][0], a1 = s->alpha[3][1];
  s->alpha[0][0] = a0;
  s->alpha[0][1] = a1;
  s->alpha[1][0] = s->alpha[1][1] = 0.0;
  s->alpha[2][0] = s->alpha[2][1] = 0.0;
  s->alpha[3][0] = s->alpha[3][1] = 0.0;
  const double t = s->t, te = s->t_end;
  if (!(t < te) || s->steps >= s->step_limit || (s->status & kStatusNonphysical) != 0u) {
    s->active = 0;
    s->dt = 0.0;
    s->alpha[3][0] = a0;  // the state is unchanged: keep its speeds
    s->alpha[3][1] = a1;
    return;
  }
  double dt;
  if (s->dt_fixed > 0.0) {
    dt = s->dt_fixed;
  } else {
    const double rate = a0 * inv_dx + (dim == 2 ? a1 * inv_dy : 0.0);
    dt = (rate > 0.0) ? s->cfl / rate : te - t;
  }
  double tn = t + dt;
  if (!(tn < te)) {  // clip the last step onto t_end
    dt = te - t;
    tn = te;
  }
  s->dt = dt;
  s->t = tn;
  s->steps += 1;
  s->active = 1;
}

// Tile shape of the 2D single-solve launch: rows per chunk (tile height; < -1: segments of
// -rows band-rows, geometry.h) and number of bands (tile width = ceil(nx / bands) output
// columns); 0 = the default for that dimension (one wave of blocks over the resident slots, in
// chunks or segments; the widest bands).
struct TileShape {
  int rows = 0;
  int bands = 0;
  // block width: 2D 64, 96, 128 or 192 threads (0 = default_width2d); 1D 0 = the default rule,
  // else 32, 64 or 128 threads.  1D threads per cell (0 or 1: one thread per cell; 4: one lane per
  // characteristic field, 1D Euler with the characteristic decomposition)
  int width = 0;
  int lanes = 0;
};
// Default block width of the 2D single-solve launch: 96 threads for characteristic FP64
// Euler (the kernel that keeps the conserved coefficients in shared memory), 192 for
// characteristic FP32-bulk Euler (two blocks per SM: fewer idle lanes and ring columns than
// three of 128; 8.3 ms instead of 9.1 ms per 2048^2 stage), else 128.
constexpr int default_width2d(int eq, bool characteristic, bool mixed) {
  return eq == EQ_EULER && characteristic ? (mixed ? 192 : 96) : 128;
}
// Tuning table keyed by (equation, characteristic, precision, nx, ny); all zero = not tuned.
TileShape tuning_shape(int eq, int characteristic, int mixed, int nx, int ny);
void tuning_set_shape(int eq, int characteristic, int mixed, int nx, int ny, TileShape t);
// Shape override for the next 2D launches of this thread (autotuner): rows / bands > 0 fix
// them, -1 the default geometry ignoring the table, {0, 0} no override.
void tuning_force_shape(TileShape t);
// The same for 1D launches (block width and threads per cell); all zero = no override.
void tuning_force_shape1d(TileShape t);

// Device pointers of a 1D solve for the multi-step cooperative launch: U[0] = U^n (stage 3
// writes it in place), U[1], U[2] the stage buffers, Vh the first-moment modifications.
struct Step1D {
  KProblem P;
  DevScal* sc;
  double* U[3];
  double* Vh;
};
// Up to nsteps SSP-RK3 steps of a 1D solve in one cooperative launch (fewer when the solve
// reaches its target); asynchronous on st.  steps1d_supported(): the device can launch
// cooperative kernels.
cudaError_t launch_steps1d(int eq, bool characteristic, bool mixed, const Step1D& A,
                           int nsteps, cudaStream_t st);
bool steps1d_supported();

// One stage of the modified SSP-RK3 over a whole grid (1D / 2D), asynchronous on st.
cudaError_t launch_stage1d(int eq, bool characteristic, bool mixed, const KProblem& P,
                           const KStage& S, cudaStream_t st);
cudaError_t launch_stage2d(int eq, bool characteristic, bool mixed, const KProblem& P,
                           const KStage& S, cudaStream_t st);
// Set the launch attributes of every kernel instantiation and report the largest per-thread
// local memory (stack frame) any of them uses; called before any launch or graph capture.
cudaError_t prepare_stage1d(size_t* max_local);
cudaError_t prepare_stage2d(size_t* max_local);
cudaError_t prepare_batch(size_t* max_local);
cudaError_t prepare_kernels(int device);

// Wave speeds of a state (raises alpha_out[0..1]).
cudaError_t launch_alpha(int eq, int dim, const KProblem& P, const double* U, double* alpha_out,
                         cudaStream_t st);

}  // namespace hw
