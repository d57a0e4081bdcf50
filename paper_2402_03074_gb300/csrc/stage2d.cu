// stage2d.cu -- single-solve launch of the fused 2D HWENO-U stage (one block per band x
// row chunk; the work item itself is in stage2d_item.cuh).
#include "launch.h"
#include "stage2d_item.cuh"

namespace hw {

// single-solve kernel: one block per (band, chunk)
template <int EQ, bool CHAR, typename R, int BW>
__global__ void __launch_bounds__(BW, 1) stage2d_kernel(KProblem P, KStage S, int rows, int wout) {
  if (S.active && *S.active == 0) return;
  extern __shared__ double smem[];
  __shared__ double red[2][BW / 32];
  stage2d_item<EQ, CHAR, R, BW>(P, S, blockIdx.x, blockIdx.y, rows, wout, smem, red);
}

// Launch geometry: bands of equal width (<= BW-2 output columns) and row chunks sized so
// that bands x chunks fills the resident block slots of the GPU once.
struct Geom2D {
  int bands, wout, chunks, rows;
};
static Geom2D geom2d(int nx, int ny, int bw, int slots) {
  Geom2D g;
  g.bands = (nx + (bw - 2) - 1) / (bw - 2);
  g.wout = (nx + g.bands - 1) / g.bands;
  int ch = slots / g.bands;
  if (ch < 1) ch = 1;
  if (ch > ny) ch = ny;
  g.rows = (ny + ch - 1) / ch;
  g.chunks = (ny + g.rows - 1) / g.rows;
  return g;
}

template <int EQ, bool CHAR, typename R>
static cudaError_t launch2d_t(const KProblem& P, const KStage& S, cudaStream_t st) {
  constexpr int BW = 128;
  const size_t smem = smem_bytes2d<EQ, R, BW>();
  auto kern = stage2d_kernel<EQ, CHAR, R, BW>;
  static int slots = 0;  // resident blocks per GPU for this instantiation
  if (slots == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, BW, smem);
    if (e != cudaSuccess) return e;
    slots = (per > 0 ? per : 1) * (nsm > 0 ? nsm : 1);
  }
  const Geom2D g = geom2d(P.nx, P.ny, BW, slots);
  dim3 grid(g.bands, g.chunks);
  kern<<<grid, BW, smem, st>>>(P, S, g.rows, g.wout);
  return cudaGetLastError();
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
