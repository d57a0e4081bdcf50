// stage2d.cu -- single-solve launch of the fused 2D HWENO-U stage: the dispatch over block
// widths (the tuning table's or the class default) and the 128-thread instantiations; the
// kernel and its launch are in stage2d_impl.cuh, the work item in stage2d_item.cuh.
#include "stage2d_impl.cuh"

namespace hw {

HW_STAGE2D_WIDTH(128)

static thread_local TileShape g_force_shape;
void tuning_force_shape(TileShape t) { g_force_shape = t; }

cudaError_t launch_stage2d(int eq, bool characteristic, bool mixed, const KProblem& P,
                           const KStage& S, cudaStream_t st) {
  TileShape t = g_force_shape;  // > 0 fixed, -1 default geometry, {0, 0} consult the table
  const bool ch = eq == EQ_EULER && characteristic;
  if (t.rows == 0 && t.bands == 0 && t.width == 0)
    t = tuning_shape(eq, ch ? 1 : 0, mixed ? 1 : 0, P.nx, P.ny);
  const int w = t.width > 0 ? t.width : default_width2d(eq, ch, mixed);
  if (w == 64) return launch2d_width<64>(eq, ch, mixed, P, S, t, st);
  if (w == 96) return launch2d_width<96>(eq, ch, mixed, P, S, t, st);
  if (w == 192) return launch2d_width<192>(eq, ch, mixed, P, S, t, st);
  return launch2d_width<128>(eq, ch, mixed, P, S, t, st);
}

cudaError_t prepare_stage2d(size_t* max_local) {
  size_t m = 0, l = 0;
  cudaError_t e = prepare2d_width<128>(&l);
  m = l > m ? l : m;
  if (e == cudaSuccess) e = prepare2d_width<96>(&l);
  m = l > m ? l : m;
  if (e == cudaSuccess) e = prepare2d_width<64>(&l);
  m = l > m ? l : m;
  if (e == cudaSuccess) e = prepare2d_width<192>(&l);
  m = l > m ? l : m;
  if (max_local) *max_local = m;
  return e;
}

}  // namespace hw
