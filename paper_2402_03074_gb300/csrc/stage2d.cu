// stage2d.cu -- single-solve launch of the fused 2D HWENO-U stage (one block per band x
// row chunk; the work item itself is in stage2d_item.cuh).
#include "geometry.h"
#include "launch.h"
#include "stage2d_item.cuh"

namespace hw {

// single-solve kernel (geometry.h): chunks (seg = 0), one block per (band, row chunk); or
// segments, block b sweeping the band-rows [b seg, (b + 1) seg) of the `bands` bands taken one
// after another, in one piece per band it touches
template <int EQ, bool CHAR, typename R, int BW>
__global__ void __launch_bounds__(BW, kMinBlocks2D<R, BW>)
    stage2d_kernel(KProblem P, KStage S, int rows, int wout, int seg, int bands) {
  if (S.active && *S.active == 0) return;
  extern __shared__ double smem[];
  __shared__ double red[2][BW / 32];
  const int ny = P.ny;
  if (seg == 0) {
    const int j0 = blockIdx.y * rows;
    stage2d_item<EQ, CHAR, R, BW>(P, S, blockIdx.x, j0, min(ny, j0 + rows), wout, smem, red);
    return;
  }
  long long q = (long long)blockIdx.x * seg;
  const long long qend = min(q + seg, (long long)bands * ny);
#pragma unroll 1
  while (q < qend) {  // uniform over the block
    const int band = (int)(q / ny), j0 = (int)(q - (long long)band * ny);
    const int j1 = (int)min((long long)ny, (long long)j0 + (qend - q));
    stage2d_item<EQ, CHAR, R, BW>(P, S, band, j0, j1, wout, smem, red);
    q += j1 - j0;
  }
}

static thread_local TileShape g_force_shape;
void tuning_force_shape(TileShape t) { g_force_shape = t; }

template <int EQ, bool CHAR, typename R, int BW>
static cudaError_t init2d_t(int* slots_out, size_t* local_out) {
  const size_t smem = smem_bytes2d<EQ, CHAR, R, BW>();
  auto kern = stage2d_kernel<EQ, CHAR, R, BW>;
  static int slots = 0;  // resident blocks per GPU for this instantiation
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

template <int EQ, bool CHAR, typename R, int BW>
static cudaError_t launch2d_w(const KProblem& P, const KStage& S, TileShape t, cudaStream_t st) {
  int slots = 0;
  cudaError_t e = init2d_t<EQ, CHAR, R, BW>(&slots, nullptr);
  if (e != cudaSuccess) return e;
  // bands of equal width, swept in row chunks or segments filling the resident block slots
  // once, unless the tuning table (or the autotuner) fixes the tile shape (geometry.h)
  const Geom2D g = geom2d(P.nx, P.ny, BW, slots, (t.rows > 0 || t.rows < -1) ? t.rows : 0,
                          t.bands > 0 ? t.bands : 0, sizeof(R) == sizeof(double));
  const dim3 grid = g.seg > 0 ? dim3(g.blocks) : dim3(g.bands, g.chunks);
  stage2d_kernel<EQ, CHAR, R, BW><<<grid, BW, smem_bytes2d<EQ, CHAR, R, BW>(), st>>>(
      P, S, g.rows, g.wout, g.seg, g.bands);
  return cudaGetLastError();
}

template <int EQ, bool CHAR, typename R>
static cudaError_t launch2d_t(const KProblem& P, const KStage& S, cudaStream_t st) {
  TileShape t = g_force_shape;  // > 0 fixed, -1 default geometry, {0, 0} consult the table
  if (t.rows == 0 && t.bands == 0 && t.width == 0)
    t = tuning_shape(EQ, CHAR ? 1 : 0, sizeof(R) == 4 ? 1 : 0, P.nx, P.ny);
  const int w = t.width > 0 ? t.width : default_width2d(EQ, CHAR, sizeof(R) == 4);
  if (w == 64) return launch2d_w<EQ, CHAR, R, 64>(P, S, t, st);
  if (w == 96) return launch2d_w<EQ, CHAR, R, 96>(P, S, t, st);
  return launch2d_w<EQ, CHAR, R, 128>(P, S, t, st);
}

cudaError_t prepare_stage2d(size_t* max_local) {
  size_t m = 0, l = 0;
  cudaError_t e = cudaSuccess;
#define HW_PREP(EQ, CH, R)                                            \
  if (e == cudaSuccess) {                                             \
    e = init2d_t<EQ, CH, R, 128>(nullptr, &l);                        \
    m = l > m ? l : m;                                                \
    if (e == cudaSuccess) e = init2d_t<EQ, CH, R, 96>(nullptr, &l);   \
    m = l > m ? l : m;                                                \
    if (e == cudaSuccess) e = init2d_t<EQ, CH, R, 64>(nullptr, &l);   \
    m = l > m ? l : m;                                                \
  }
  HW_PREP(EQ_ADV, false, double) HW_PREP(EQ_ADV, false, float)
  HW_PREP(EQ_BURG, false, double) HW_PREP(EQ_BURG, false, float)
  HW_PREP(EQ_EULER, false, double) HW_PREP(EQ_EULER, false, float)
  HW_PREP(EQ_EULER, true, double) HW_PREP(EQ_EULER, true, float)
#undef HW_PREP
  if (max_local) *max_local = m;
  return e;
}

cudaError_t launch_stage2d(int eq, bool characteristic, bool mixed, const KProblem& P,
                           const KStage& S, cudaStream_t st) {
  if (eq == EQ_ADV) return mixed ? launch2d_t<EQ_ADV, false, float>(P, S, st)
                                 : launch2d_t<EQ_ADV, false, double>(P, S, st);
  if (eq == EQ_BURG) return mixed ? launch2d_t<EQ_BURG, false, float>(P, S, st)
                                  : launch2d_t<EQ_BURG, false, double>(P, S, st);
  if (characteristic) return mixed ? launch2d_t<EQ_EULER, true, float>(P, S, st)
                                   : launch2d_t<EQ_EULER, true, double>(P, S, st);
  return mixed ? launch2d_t<EQ_EULER, false, float>(P, S, st)
               : launch2d_t<EQ_EULER, false, double>(P, S, st);
}

}  // namespace hw
