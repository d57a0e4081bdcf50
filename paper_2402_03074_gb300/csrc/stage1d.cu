// stage1d.cu -- single-solve launch of the fused 1D HWENO-U stage (one block per BW-2 cells;
// the block's work is in stage1d_item.cuh).
#include "launch.h"
#include "stage1d_item.cuh"

namespace hw {

template <int EQ, bool CHAR, typename R, int BW>
__global__ void __launch_bounds__(BW) stage1d_kernel(KProblem P, KStage S) {
  if (S.active && *S.active == 0) return;
  stage1d_item<EQ, CHAR, R, BW>(P, S, blockIdx.x);
}

template <int EQ, bool CHAR, typename R>
static cudaError_t launch1d_t(const KProblem& P, const KStage& S, cudaStream_t st) {
  constexpr int BW = 128;
  const int blocks = (P.nx + (BW - 2) - 1) / (BW - 2);
  stage1d_kernel<EQ, CHAR, R, BW><<<blocks, BW, 0, st>>>(P, S);
  return cudaGetLastError();
}

template <int EQ, bool CHAR, typename R>
static size_t local1d_t() {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, stage1d_kernel<EQ, CHAR, R, 128>) != cudaSuccess) return 0;
  return fa.localSizeBytes;
}

cudaError_t prepare_stage1d(size_t* max_local) {
  size_t m = 0;
  const size_t l[8] = {local1d_t<EQ_ADV, false, double>(), local1d_t<EQ_ADV, false, float>(),
                       local1d_t<EQ_BURG, false, double>(), local1d_t<EQ_BURG, false, float>(),
                       local1d_t<EQ_EULER, false, double>(), local1d_t<EQ_EULER, false, float>(),
                       local1d_t<EQ_EULER, true, double>(), local1d_t<EQ_EULER, true, float>()};
  for (size_t x : l) m = x > m ? x : m;
  if (max_local) *max_local = m;
  return cudaGetLastError();
}

cudaError_t launch_stage1d(int eq, bool characteristic, bool mixed, const KProblem& P,
                           const KStage& S, cudaStream_t st) {
  if (eq == EQ_ADV) return mixed ? launch1d_t<EQ_ADV, false, float>(P, S, st)
                                 : launch1d_t<EQ_ADV, false, double>(P, S, st);
  if (eq == EQ_BURG) return mixed ? launch1d_t<EQ_BURG, false, float>(P, S, st)
                                  : launch1d_t<EQ_BURG, false, double>(P, S, st);
  if (characteristic) return mixed ? launch1d_t<EQ_EULER, true, float>(P, S, st)
                                   : launch1d_t<EQ_EULER, true, double>(P, S, st);
  return mixed ? launch1d_t<EQ_EULER, false, float>(P, S, st)
               : launch1d_t<EQ_EULER, false, double>(P, S, st);
}

}  // namespace hw
