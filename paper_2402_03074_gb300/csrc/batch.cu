// batch.cu -- batched, persistent HWENO-U stage launches over many solves.
//
// All live solves of one kernel class (dimension, equation, characteristic decomposition,
// precision) are advanced by one launch per RK stage.  The launch is persistent (one block
// per resident slot); its blocks take work items from a device counter.  An item is exactly
// the unit of the single-solve kernel -- one (band, row chunk) of a 2D solve, one block of
// kBatchBW - 2 cells of a 1D solve -- so uneven grids share the GPU and the load balances at
// item granularity.  FP64 and FP32-bulk solves are separate classes (one
// instantiation each, so every kernel keeps the register, shared-memory and stack footprint
// of the single-solve kernel of its width).  Every solve keeps its own scalars (dt, t, LF speeds,
// status); one thread per solve advances them at the start of each step, so each solve
// steps with its own dt.  The work lists live in device memory: admission and retirement
// rewrite them between steps and the captured step graph stays valid.
#include "batch.h"
#include "stage1d_item.cuh"
#include "stage2d_item.cuh"

namespace hw {

// the owning solve of a work item: the last solve with item_base <= item
__device__ __forceinline__ int batch_owner(const BatchSolve* bs, int n_solves, int item) {
  int lo = 0, hi = n_solves - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bs[mid].item_base <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void batch_dt_kernel(BatchDt* d, BatchCtl* ctl, int nctl) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < d->n) dt_update(d->sc[s], d->inv_dx[s], d->inv_dy[s], d->dim[s]);
  if (s < nctl) {
    ctl[s].next[0] = 0u;
    ctl[s].next[1] = 0u;
    ctl[s].next[2] = 0u;
  }
}

template <int EQ, bool CHAR, typename R, int BW>
__global__ void __launch_bounds__(BW, kMinBlocks2D<R, BW>)
    batch_stage_kernel(const BatchSolve* bs, BatchCtl* ctl, int k) {
  extern __shared__ double smem[];
  __shared__ double red[2][BW / 32];
  __shared__ int item_s;
  const int n_items = ctl->n_items, n_solves = ctl->n_solves;
#pragma unroll 1
  for (;;) {
    if (threadIdx.x == 0) item_s = (int)atomicAdd(&ctl->next[k - 1], 1u);
    __syncthreads();
    const int item = item_s;
    __syncthreads();
    if (item >= n_items) break;
    const BatchSolve& B = bs[batch_owner(bs, n_solves, item)];
    if (*(volatile const int*)&B.sc->active == 0) continue;  // uniform over the block
    const int local = item - B.item_base;
    const int band = local % B.bands, chunk = local / B.bands;
    KStage S;
    S.Uin = B.U[k - 1];
    S.Un = B.U[0];
    S.Vh = B.Vh;
    S.Uout = B.U[k % 3];
    S.alpha_in = B.sc->alpha[k - 1];
    S.alpha_out = B.sc->alpha[k];
    S.dt = &B.sc->dt;
    S.status = &B.sc->status;
    S.active = &B.sc->active;
    S.k = k;
    const int j0 = chunk * B.rows;
    stage2d_item<EQ, CHAR, R, BW>(B.P, S, band, j0, min(B.P.ny, j0 + B.rows), B.wout, smem, red);
  }
}

template <int EQ, bool CHAR, typename R, int BW>
__global__ void __launch_bounds__(BW) batch1d_stage_kernel(const BatchSolve* bs, BatchCtl* ctl,
                                                           int k) {
  __shared__ int item_s;
  const int n_items = ctl->n_items, n_solves = ctl->n_solves;
#pragma unroll 1
  for (;;) {
    if (threadIdx.x == 0) item_s = (int)atomicAdd(&ctl->next[k - 1], 1u);
    __syncthreads();
    const int item = item_s;
    __syncthreads();
    if (item >= n_items) break;
    const BatchSolve& B = bs[batch_owner(bs, n_solves, item)];
    if (*(volatile const int*)&B.sc->active == 0) continue;  // uniform over the block
    KStage S;
    S.Uin = B.U[k - 1];
    S.Un = B.U[0];
    S.Vh = B.Vh;
    S.Uout = B.U[k % 3];
    S.alpha_in = B.sc->alpha[k - 1];
    S.alpha_out = B.sc->alpha[k];
    S.dt = &B.sc->dt;
    S.status = &B.sc->status;
    S.active = &B.sc->active;
    S.k = k;
    stage1d_item<EQ, CHAR, R, BW>(B.P, S, item - B.item_base);
  }
}

template <int EQ, bool CHAR, typename R>
static cudaError_t init_batch1d_t(int* slots_out, size_t* local_out) {
  constexpr int BW = kBatchBW;
  auto kern = batch1d_stage_kernel<EQ, CHAR, R, BW>;
  static int slots = 0;
  static size_t local = 0;
  if (slots == 0) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    local = fa.localSizeBytes;
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, BW, 0);
    if (e != cudaSuccess) return e;
    slots = (per > 0 ? per : 1) * (nsm > 0 ? nsm : 1);
  }
  if (slots_out) *slots_out = slots;
  if (local_out) *local_out = local;
  return cudaSuccess;
}

template <int EQ, bool CHAR, typename R>
static cudaError_t launch_batch1d_t(const BatchSolve* bs, BatchCtl* ctl, int k, cudaStream_t st) {
  constexpr int BW = kBatchBW;
  int slots = 0;
  cudaError_t e = init_batch1d_t<EQ, CHAR, R>(&slots, nullptr);
  if (e != cudaSuccess) return e;
  batch1d_stage_kernel<EQ, CHAR, R, BW><<<slots, BW, 0, st>>>(bs, ctl, k);
  return cudaGetLastError();
}

template <int EQ, bool CHAR, typename R>
static cudaError_t init_batch_t(int* slots_out, size_t* local_out) {
  constexpr int BW = kBatchBW;
  const size_t smem = smem_bytes2d<EQ, CHAR, R, BW>();
  auto kern = batch_stage_kernel<EQ, CHAR, R, BW>;
  static int slots = 0;
  static size_t local = 0;
  if (slots == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    local = fa.localSizeBytes;
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, BW, smem);
    if (e != cudaSuccess) return e;
    slots = (per > 0 ? per : 1) * (nsm > 0 ? nsm : 1);
  }
  if (slots_out) *slots_out = slots;
  if (local_out) *local_out = local;
  return cudaSuccess;
}

template <int EQ, bool CHAR, typename R>
static cudaError_t launch_batch_t(const BatchSolve* bs, BatchCtl* ctl, int k, cudaStream_t st) {
  constexpr int BW = kBatchBW;
  int slots = 0;
  cudaError_t e = init_batch_t<EQ, CHAR, R>(&slots, nullptr);
  if (e != cudaSuccess) return e;
  batch_stage_kernel<EQ, CHAR, R, BW><<<slots, BW, smem_bytes2d<EQ, CHAR, R, BW>(), st>>>(bs, ctl, k);
  return cudaGetLastError();
}

// class = 8 * (1D) + 2 * (0 advection, 1 Burgers, 2 Euler component-wise,
// 3 Euler characteristic) + mixed
cudaError_t launch_batch_stage(int cls, const BatchSolve* bs, BatchCtl* ctl, int k,
                               cudaStream_t st) {
  switch (cls) {
    case 8: return launch_batch1d_t<EQ_ADV, false, double>(bs, ctl, k, st);
    case 9: return launch_batch1d_t<EQ_ADV, false, float>(bs, ctl, k, st);
    case 10: return launch_batch1d_t<EQ_BURG, false, double>(bs, ctl, k, st);
    case 11: return launch_batch1d_t<EQ_BURG, false, float>(bs, ctl, k, st);
    case 12: return launch_batch1d_t<EQ_EULER, false, double>(bs, ctl, k, st);
    case 13: return launch_batch1d_t<EQ_EULER, false, float>(bs, ctl, k, st);
    case 14: return launch_batch1d_t<EQ_EULER, true, double>(bs, ctl, k, st);
    case 15: return launch_batch1d_t<EQ_EULER, true, float>(bs, ctl, k, st);
    case 0: return launch_batch_t<EQ_ADV, false, double>(bs, ctl, k, st);
    case 1: return launch_batch_t<EQ_ADV, false, float>(bs, ctl, k, st);
    case 2: return launch_batch_t<EQ_BURG, false, double>(bs, ctl, k, st);
    case 3: return launch_batch_t<EQ_BURG, false, float>(bs, ctl, k, st);
    case 4: return launch_batch_t<EQ_EULER, false, double>(bs, ctl, k, st);
    case 5: return launch_batch_t<EQ_EULER, false, float>(bs, ctl, k, st);
    case 6: return launch_batch_t<EQ_EULER, true, double>(bs, ctl, k, st);
    default: return launch_batch_t<EQ_EULER, true, float>(bs, ctl, k, st);
  }
}

cudaError_t prepare_batch(size_t* max_local) {
  size_t m = 0, l = 0;
  cudaError_t e = cudaSuccess;
#define HW_PREP(EQ, CH, R)                                            \
  if (e == cudaSuccess) {                                             \
    e = init_batch_t<EQ, CH, R>(nullptr, &l);                         \
    m = l > m ? l : m;                                                \
  }
  HW_PREP(EQ_ADV, false, double) HW_PREP(EQ_ADV, false, float)
  HW_PREP(EQ_BURG, false, double) HW_PREP(EQ_BURG, false, float)
  HW_PREP(EQ_EULER, false, double) HW_PREP(EQ_EULER, false, float)
  HW_PREP(EQ_EULER, true, double) HW_PREP(EQ_EULER, true, float)
#undef HW_PREP
#define HW_PREP1(EQ, CH, R)                                           \
  if (e == cudaSuccess) {                                             \
    e = init_batch1d_t<EQ, CH, R>(nullptr, &l);                       \
    m = l > m ? l : m;                                                \
  }
  HW_PREP1(EQ_ADV, false, double) HW_PREP1(EQ_ADV, false, float)
  HW_PREP1(EQ_BURG, false, double) HW_PREP1(EQ_BURG, false, float)
  HW_PREP1(EQ_EULER, false, double) HW_PREP1(EQ_EULER, false, float)
  HW_PREP1(EQ_EULER, true, double) HW_PREP1(EQ_EULER, true, float)
#undef HW_PREP1
  if (max_local) *max_local = m;
  return e;
}

int batch_class(int equation, int characteristic, int mixed, int dim) {
  const int base = (equation == EQ_ADV) ? 0 : (equation == EQ_BURG ? 1 : (characteristic ? 3 : 2));
  return (dim == 1 ? 8 : 0) + 2 * base + (mixed ? 1 : 0);
}

cudaError_t launch_batch_dt(BatchDt* d, BatchCtl* ctl, int nctl, int cap, cudaStream_t st) {
  const int n = cap > nctl ? cap : nctl;
  batch_dt_kernel<<<(n + 127) / 128, 128, 0, st>>>(d, ctl, nctl);
  return cudaGetLastError();
}

int batch_slots(int cls) {
  int slots = 0;
  cudaError_t e;
  switch (cls) {
    case 0: e = init_batch_t<EQ_ADV, false, double>(&slots, nullptr); break;
    case 1: e = init_batch_t<EQ_ADV, false, float>(&slots, nullptr); break;
    case 2: e = init_batch_t<EQ_BURG, false, double>(&slots, nullptr); break;
    case 3: e = init_batch_t<EQ_BURG, false, float>(&slots, nullptr); break;
    case 4: e = init_batch_t<EQ_EULER, false, double>(&slots, nullptr); break;
    case 5: e = init_batch_t<EQ_EULER, false, float>(&slots, nullptr); break;
    case 6: e = init_batch_t<EQ_EULER, true, double>(&slots, nullptr); break;
    case 7: e = init_batch_t<EQ_EULER, true, float>(&slots, nullptr); break;
    case 8: e = init_batch1d_t<EQ_ADV, false, double>(&slots, nullptr); break;
    case 9: e = init_batch1d_t<EQ_ADV, false, float>(&slots, nullptr); break;
    case 10: e = init_batch1d_t<EQ_BURG, false, double>(&slots, nullptr); break;
    case 11: e = init_batch1d_t<EQ_BURG, false, float>(&slots, nullptr); break;
    case 12: e = init_batch1d_t<EQ_EULER, false, double>(&slots, nullptr); break;
    case 13: e = init_batch1d_t<EQ_EULER, false, float>(&slots, nullptr); break;
    case 14: e = init_batch1d_t<EQ_EULER, true, double>(&slots, nullptr); break;
    default: e = init_batch1d_t<EQ_EULER, true, float>(&slots, nullptr); break;
  }
  return e == cudaSuccess ? slots : 0;
}

void batch_geometry1d(int nx, int* blocks) { *blocks = (nx + (kBatchBW - 2) - 1) / (kBatchBW - 2); }

void batch_geometry(int nx, int ny, int rows, int bw, int* bands, int* wout, int* chunks,
                    bool lane_aware) {
  split_bands(nx, default_bands(nx, bw, lane_aware), bands, wout);
  if (rows < 1) rows = 1;
  *chunks = (ny + rows - 1) / rows;
}

}  // namespace hw
