// static_batch.cu -- one batched stage over caller-owned device buffers that allocates nothing.
//
// Some callers cannot allocate device memory: applications whose device memory is owned by
// a pool allocator of their own (every byte must come from the pool), and latency-critical
// loops that cannot afford cudaMalloc / cudaFree, which may synchronise the whole device.
// For them hweno_stage_batch_static runs the batched persistent stage kernel with its work
// list and work counter in a fixed-size array of this file instead of allocated scratch.
// The caller still passes every input and output buffer.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "../../include/hweno.h"
#include "batch.h"
#include "stage2d_item.cuh"

namespace hw {

struct StaticItem {
  KProblem P;
  const double* Uin;
  const double* Un;
  double* Vh;
  double* Uout;
  const double* alpha_in;
  double* alpha_out;
  const double* dt;
  uint32_t* status;
  int bands, wout, rows, chunks, item_base;
};

struct StaticScratch {
  unsigned int next;  // work counter of the launch
  int n;              // solves
  int n_items;        // work items
  int pad;
  StaticItem item[HWENO_STATIC_BATCH_MAX];
};

// It is passed by value to static_setup_kernel: keep it within the 4 KB kernel-parameter
// limit that holds on every CUDA version.
static_assert(sizeof(StaticScratch) <= 4096, "StaticScratch must fit a kernel parameter");

// The scratch of hweno_stage_batch_static.  Every GPU that loads the library holds it (a few
// KB) until the process exits; every call overwrites it, so calls that overlap on the GPU
// race on it.
static __device__ __align__(256) unsigned char g_static_scratch[sizeof(StaticScratch)];

// writes the call's work list into the scratch and clears the work counter
__global__ void static_setup_kernel(StaticScratch* dst, StaticScratch src) {
  const int nw = (int)(sizeof(StaticScratch) / sizeof(unsigned int));
  const unsigned int* s = reinterpret_cast<const unsigned int*>(&src);
  unsigned int* d = reinterpret_cast<unsigned int*>(dst);
  for (int q = threadIdx.x; q < nw; q += blockDim.x) d[q] = s[q];
  __syncthreads();
  if (threadIdx.x == 0) dst->next = 0u;
}

template <int EQ, bool CHAR, typename R, int BW>
__global__ void __launch_bounds__(BW, kMinBlocks2D<R, BW>)
    static_batch_kernel(StaticScratch* sc, int k) {
  extern __shared__ double smem[];
  __shared__ double red[2][BW / 32];
  __shared__ int item_s;
  const int n_items = sc->n_items, n = sc->n;
#pragma unroll 1
  for (;;) {
    if (threadIdx.x == 0) item_s = (int)atomicAdd(&sc->next, 1u);
    __syncthreads();
    const int item = item_s;
    __syncthreads();
    if (item >= n_items) break;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sc->item[mid].item_base <= item) lo = mid;
      else hi = mid - 1;
    }
    const StaticItem& B = sc->item[lo];
    const int local = item - B.item_base;
    KStage S;
    S.Uin = B.Uin;
    S.Un = B.Un;
    S.Vh = B.Vh;
    S.Uout = B.Uout;
    S.alpha_in = B.alpha_in;
    S.alpha_out = B.alpha_out;
    S.dt = B.dt;
    S.status = B.status;
    S.active = nullptr;
    S.k = k;
    const int j0 = (local / B.bands) * B.rows;
    stage2d_item<EQ, CHAR, R, BW>(B.P, S, local % B.bands, j0, min(B.P.ny, j0 + B.rows), B.wout,
                                  smem, red);
  }
}

// per device: the scratch address (cudaGetSymbolAddress) and per class the launch setup
struct StaticSetup {
  StaticScratch* ptr = nullptr;
  int slots[kBatchClasses] = {};
  size_t local[kBatchClasses] = {};
};
static std::mutex g_static_mu;
static StaticSetup g_static[64];
static bool g_static_ready[64];

template <int EQ, bool CHAR, typename R>
static cudaError_t static_class_setup(int* slots, size_t* local) {
  constexpr int BW = kBatchBW;
  auto kern = static_batch_kernel<EQ, CHAR, R, BW>;
  const size_t smem = smem_bytes2d<EQ, CHAR, R, BW>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  *local = fa.localSizeBytes;
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, BW, smem);
  if (e != cudaSuccess) return e;
  *slots = (per > 0 ? per : 1) * (nsm > 0 ? nsm : 1);
  return cudaSuccess;
}

template <int EQ, bool CHAR, typename R>
static void static_launch(int slots, StaticScratch* ptr, int k, cudaStream_t st) {
  constexpr int BW = kBatchBW;
  static_batch_kernel<EQ, CHAR, R, BW><<<slots, BW, smem_bytes2d<EQ, CHAR, R, BW>(), st>>>(ptr, k);
}

// set-up of one device (the current one): scratch address and every class's launch setup
static int static_device_setup(int dev) {
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (dev < 0 || dev >= 64) return HWENO_ERR_ARG;
  if (g_static_ready[dev]) return HWENO_OK;
  StaticSetup& S = g_static[dev];
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return HWENO_ERR_CUDA;
  S.ptr = static_cast<StaticScratch*>(p);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = static_class_setup<EQ_ADV, false, double>(&S.slots[0], &S.local[0]);
  if (e == cudaSuccess) e = static_class_setup<EQ_ADV, false, float>(&S.slots[1], &S.local[1]);
  if (e == cudaSuccess) e = static_class_setup<EQ_BURG, false, double>(&S.slots[2], &S.local[2]);
  if (e == cudaSuccess) e = static_class_setup<EQ_BURG, false, float>(&S.slots[3], &S.local[3]);
  if (e == cudaSuccess) e = static_class_setup<EQ_EULER, false, double>(&S.slots[4], &S.local[4]);
  if (e == cudaSuccess) e = static_class_setup<EQ_EULER, false, float>(&S.slots[5], &S.local[5]);
  if (e == cudaSuccess) e = static_class_setup<EQ_EULER, true, double>(&S.slots[6], &S.local[6]);
  if (e == cudaSuccess) e = static_class_setup<EQ_EULER, true, float>(&S.slots[7], &S.local[7]);
  if (e != cudaSuccess) return HWENO_ERR_CUDA;
  g_static_ready[dev] = true;
  return HWENO_OK;
}

int problem_check(const hweno_problem* p, std::string* why);
KProblem kproblem_of(const hweno_problem* p);

}  // namespace hw

using namespace hw;

extern "C" int hweno_stage_batch_static(int n, const hweno_problem* problems, int k,
                                        const double* const* U_in, const double* const* U_n,
                                        double* const* Vh, double* const* U_out,
                                        const double* const* alpha_in, double* const* alpha_out,
                                        const double* const* dt, uint32_t* const* status,
                                        void* stream) {
  if (n < 1 || n > HWENO_STATIC_BATCH_MAX) return HWENO_ERR_ARG;  // the scratch holds at most
                                                                   // HWENO_STATIC_BATCH_MAX solves
  if (!problems || k < 1 || k > 3 || !U_in || !U_n || !Vh || !U_out || !alpha_in || !alpha_out ||
      !dt || !status)
    return HWENO_ERR_ARG;
  const hweno_problem& p0 = problems[0];
  const int ch0 = p0.equation == HWENO_EULER ? p0.characteristic : 0;
  for (int s = 0; s < n; ++s) {
    const hweno_problem& p = problems[s];
    if (problem_check(&p, nullptr) != HWENO_OK || p.dim != 2) return HWENO_ERR_ARG;
    const int ch = p.equation == HWENO_EULER ? p.characteristic : 0;
    if (p.equation != p0.equation || ch != ch0 || p.precision != p0.precision) return HWENO_ERR_ARG;
    if (!U_in[s] || !U_n[s] || !Vh[s] || !U_out[s] || !alpha_in[s] || !alpha_out[s] || !dt[s] ||
        !status[s] || U_out[s] == U_in[s])
      return HWENO_ERR_ARG;
  }
  // one launch reads every solve's inputs while it writes every solve's outputs: an output
  // that is another solve's input, base state, first-moment array or output would race
  for (int s = 0; s < n; ++s)
    for (int t = 0; t < n; ++t) {
      const void* o = U_out[s];
      if (o == U_in[t] || o == Vh[t] || (t != s && (o == U_n[t] || o == U_out[t])) ||
          (t != s && ((const void*)Vh[s] == U_in[t] || (const void*)Vh[s] == U_n[t] ||
                      Vh[s] == Vh[t])))
        return HWENO_ERR_ARG;
    }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HWENO_ERR_CUDA;
  const int rc = static_device_setup(dev);
  if (rc) return rc;
  const StaticSetup& D = g_static[dev];
  const int cls = batch_class(p0.equation, ch0, p0.precision == HWENO_MIXED32);
  // the kernel's stack frame must fit the context's per-thread stack limit (raising the
  // limit can allocate device memory, so this entry point does not)
  size_t limit = 0;
  if (cudaDeviceGetLimit(&limit, cudaLimitStackSize) != cudaSuccess) return HWENO_ERR_CUDA;
  if (D.local[cls] > limit) return HWENO_ERR_STATE;
  // work list: one item per (band, row chunk); the rows per chunk give the launch the fewest
  // waves of items over the resident block slots for its length
  StaticScratch host;
  std::memset(&host, 0, sizeof(host));
  int bands[HWENO_STATIC_BATCH_MAX], wout[HWENO_STATIC_BATCH_MAX], chunks[HWENO_STATIC_BATCH_MAX];
  int nys[HWENO_STATIC_BATCH_MAX];
  for (int s = 0; s < n; ++s) {
    batch_geometry(problems[s].nx, problems[s].ny, 1,
                   batch_bw2d(problems[s].equation, problems[s].characteristic,
                              problems[s].precision == HWENO_MIXED32),
                   &bands[s], &wout[s], &chunks[s]);
    nys[s] = problems[s].ny;
  }
  const int rows = batch_rows(bands, nys, n, D.slots[cls]);
  int items = 0;
  for (int s = 0; s < n; ++s) {
    StaticItem& it = host.item[s];
    it.P = kproblem_of(&problems[s]);
    it.Uin = U_in[s];
    it.Un = U_n[s];
    it.Vh = Vh[s];
    it.Uout = U_out[s];
    it.alpha_in = alpha_in[s];
    it.alpha_out = alpha_out[s];
    it.dt = dt[s];
    it.status = status[s];
    it.bands = bands[s];
    it.wout = wout[s];
    it.rows = rows;
    it.chunks = (problems[s].ny + it.rows - 1) / it.rows;
    it.item_base = items;
    items += it.bands * it.chunks;
  }
  host.n = n;
  host.n_items = items;
  cudaStream_t st = (cudaStream_t)stream;
  static_setup_kernel<<<1, 128, 0, st>>>(D.ptr, host);
  switch (cls) {
    case 0: static_launch<EQ_ADV, false, double>(D.slots[cls], D.ptr, k, st); break;
    case 1: static_launch<EQ_ADV, false, float>(D.slots[cls], D.ptr, k, st); break;
    case 2: static_launch<EQ_BURG, false, double>(D.slots[cls], D.ptr, k, st); break;
    case 3: static_launch<EQ_BURG, false, float>(D.slots[cls], D.ptr, k, st); break;
    case 4: static_launch<EQ_EULER, false, double>(D.slots[cls], D.ptr, k, st); break;
    case 5: static_launch<EQ_EULER, false, float>(D.slots[cls], D.ptr, k, st); break;
    case 6: static_launch<EQ_EULER, true, double>(D.slots[cls], D.ptr, k, st); break;
    default: static_launch<EQ_EULER, true, float>(D.slots[cls], D.ptr, k, st); break;
  }
  return cudaGetLastError() == cudaSuccess ? HWENO_OK : HWENO_ERR_CUDA;
}
