// batch.h -- device work lists of the batched persistent stage launches (batch.cu).
#pragma once
#include <cuda_runtime.h>

#include "geometry.h"
#include "launch.h"

namespace hw {

// Threads per block of the batched stage kernels, every class.  The characteristic FP64 class
// keeps the 128-thread kernel that forms the coefficients from each pass's projected stencil:
// its 96-thread counterpart (coefficients once per cell, 111 KB of shared memory per block),
// faster for a solve alone, shares the SMs worse with the FP32-bulk class's blocks of a mixed
// stream (the configured served stream: 0.163 instead of 0.171 solves/s).  The FP32-bulk
// class's 192-thread blocks, faster for a solve alone, have not been measured here.
constexpr int kBatchBW = 128;
inline int batch_bw2d(int, int, int) { return kBatchBW; }
constexpr int kBatchClasses = 16;  // {2D, 1D} x {advection, Burgers, Euler comp.-wise,
                                   // Euler char.} x {FP64, mixed}

// One solve in a batch (device-resident array, rewritten on admission / retirement).
struct BatchSolve {
  KProblem P;
  double* U[3];        // U^n, U^(1), U^(2)
  double* Vh;
  DevScal* sc;
  int mixed;           // 1: FP32 bulk / FP64 weights
  int bands, wout, rows, chunks;  // 1D: bands = blocks of kBatchBW - 2 cells, chunks = 1
  int item_base;       // first work item of the solve
};

// Control block of one class's launches.
struct BatchCtl {
  int n_solves;
  int n_items;
  unsigned int next[3];  // work counters of the three stage launches of a step
};

// Per-solve step scalars of every solve in the batch (all classes).
constexpr int kBatchCap = 1024;
struct BatchDt {
  int n;       // solves whose step starts here (the batched ones, first in the list)
  int n_all;   // all live solves (the gather of their scalars)
  DevScal* sc[kBatchCap];
  double inv_dx[kBatchCap], inv_dy[kBatchCap];
  int dim[kBatchCap];
};

int batch_class(int equation, int characteristic, int mixed, int dim = 2);
// bands (of at most bw - 2 columns for blocks of bw threads; lane_aware: of at most bw - 34
// columns when that leaves fewer idle lanes, for the FP64 classes) and row chunks of `rows`
// rows
void batch_geometry(int nx, int ny, int rows, int bw, int* bands, int* wout, int* chunks,
                    bool lane_aware = false);
void batch_geometry1d(int nx, int* blocks);
int batch_slots(int cls);  // resident blocks of the class's persistent launch
cudaError_t launch_batch_dt(BatchDt* d, BatchCtl* ctl, int nctl, int cap, cudaStream_t st);
cudaError_t launch_batch_stage(int cls, const BatchSolve* bs, BatchCtl* ctl, int k,
                               cudaStream_t st);

}  // namespace hw
