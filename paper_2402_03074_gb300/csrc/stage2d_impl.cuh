// stage2d_impl.cuh -- the single-solve 2D stage kernel and its launch for one block width,
// instantiated per width in stage2d.cu (128 threads), stage2d_w96.cu, stage2d_w64.cu and
// stage2d_w192.cu so the widths compile in parallel; the dispatch over widths and classes is
// in stage2d.cu.
#pragma once
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
  // the block's pieces: one (band, row chunk), or the pieces of its segment; one call site of
  // the (large, inlined) work item
  int band, j0, j1;
  long long q = 0, qend = 0;
  if (seg == 0) {
    band = blockIdx.x;
    j0 = blockIdx.y * rows;
    j1 = min(ny, j0 + rows);
  } else {
    q = (long long)blockIdx.x * seg;
    qend = min(q + seg, (long long)bands * ny);
    band = (int)(q / ny);
    j0 = (int)(q - (long long)band * ny);
    j1 = (int)min((long long)ny, (long long)j0 + (qend - q));
    q += j1 - j0;
  }
#pragma unroll 1
  for (;;) {  // uniform over the block
    stage2d_item<EQ, CHAR, R, BW>(P, S, band, j0, j1, wout, smem, red);
    if (q >= qend) break;
    band = (int)(q / ny);
    j0 = (int)(q - (long long)band * ny);
    j1 = (int)min((long long)ny, (long long)j0 + (qend - q));
    q += j1 - j0;
  }
}

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

// The launch and the set-up of every class (equation, characteristic decomposition,
// precision) in blocks of BW threads, one specialisation per width translation unit.
template <int BW>
cudaError_t launch2d_width(int eq, bool characteristic, bool mixed, const KProblem& P,
                           const KStage& S, TileShape t, cudaStream_t st);
template <int BW>
cudaError_t prepare2d_width(size_t* max_local);
#define HW_STAGE2D_DECLARE(BW)                                                                \
  template <>                                                                                 \
  cudaError_t launch2d_width<BW>(int eq, bool characteristic, bool mixed, const KProblem& P,  \
                                 const KStage& S, TileShape t, cudaStream_t st);              \
  template <>                                                                                 \
  cudaError_t prepare2d_width<BW>(size_t* max_local);
HW_STAGE2D_DECLARE(128)
HW_STAGE2D_DECLARE(96)
HW_STAGE2D_DECLARE(64)
HW_STAGE2D_DECLARE(192)
#undef HW_STAGE2D_DECLARE

#define HW_STAGE2D_WIDTH(BW)                                                                  \
  template <>                                                                                 \
  cudaError_t launch2d_width<BW>(int eq, bool characteristic, bool mixed, const KProblem& P,  \
                                 const KStage& S, TileShape t, cudaStream_t st) {             \
    if (eq == EQ_ADV) return mixed ? launch2d_w<EQ_ADV, false, float, BW>(P, S, t, st)        \
                                   : launch2d_w<EQ_ADV, false, double, BW>(P, S, t, st);      \
    if (eq == EQ_BURG) return mixed ? launch2d_w<EQ_BURG, false, float, BW>(P, S, t, st)      \
                                    : launch2d_w<EQ_BURG, false, double, BW>(P, S, t, st);    \
    if (characteristic) return mixed ? launch2d_w<EQ_EULER, true, float, BW>(P, S, t, st)     \
                                     : launch2d_w<EQ_EULER, true, double, BW>(P, S, t, st);   \
    return mixed ? launch2d_w<EQ_EULER, false, float, BW>(P, S, t, st)                        \
                 : launch2d_w<EQ_EULER, false, double, BW>(P, S, t, st);                      \
  }                                                                                           \
  template <>                                                                                 \
  cudaError_t prepare2d_width<BW>(size_t* max_local) {                                        \
    size_t m = 0, l = 0;                                                                      \
    cudaError_t e = cudaSuccess;                                                              \
    if (e == cudaSuccess && (e = init2d_t<EQ_ADV, false, double, BW>(nullptr, &l)) == cudaSuccess) m = l > m ? l : m;    \
    if (e == cudaSuccess && (e = init2d_t<EQ_ADV, false, float, BW>(nullptr, &l)) == cudaSuccess) m = l > m ? l : m;     \
    if (e == cudaSuccess && (e = init2d_t<EQ_BURG, false, double, BW>(nullptr, &l)) == cudaSuccess) m = l > m ? l : m;   \
    if (e == cudaSuccess && (e = init2d_t<EQ_BURG, false, float, BW>(nullptr, &l)) == cudaSuccess) m = l > m ? l : m;    \
    if (e == cudaSuccess && (e = init2d_t<EQ_EULER, false, double, BW>(nullptr, &l)) == cudaSuccess) m = l > m ? l : m;  \
    if (e == cudaSuccess && (e = init2d_t<EQ_EULER, false, float, BW>(nullptr, &l)) == cudaSuccess) m = l > m ? l : m;   \
    if (e == cudaSuccess && (e = init2d_t<EQ_EULER, true, double, BW>(nullptr, &l)) == cudaSuccess) m = l > m ? l : m;   \
    if (e == cudaSuccess && (e = init2d_t<EQ_EULER, true, float, BW>(nullptr, &l)) == cudaSuccess) m = l > m ? l : m;    \
    if (max_local) *max_local = m;                                                            \
    return e;                                                                                 \
  }

}  // namespace hw
