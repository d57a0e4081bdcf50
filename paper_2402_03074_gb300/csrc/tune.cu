// tune.cu -- launch-geometry autotuner and its tuning table.
//
// The 2D stage kernel's blocks sweep row chunks of a band.  The tile shape trades redundant
// work against balance and latency hiding: taller chunks waste fewer ring rows, narrower
// bands more ring columns and lanes, the tile count sets how evenly the blocks fill the SMs,
// and the block width (64, 96, 128 or 192 threads) sets the resident warps per SM and the idle
// lanes of a band (the 96-thread characteristic FP64 kernel also forms the coefficients once
// per cell).  The autotuner times one stage launch of a problem for each candidate shape
// (block width x band count x chunk height) on a scratch copy of the caller's moments (with
// dt = 0, so the copy does not evolve), times the closest few again over whole three-stage
// sequences, and keeps the fastest in a process-wide table keyed by (equation,
// characteristic decomposition, precision, grid); the table is consulted by every later
// single-solve launch of such a problem (the batched launches size their work items from the
// load instead).  The table can be saved and loaded as text; entries carry the GPU name.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/hweno.h"
#include "launch.h"
#include "server.h"

namespace hw {

using TuneKey = std::tuple<int, int, int, int, int>;
static std::mutex g_tune_mu;
static std::map<TuneKey, TileShape> g_tune;

TileShape tuning_shape(int eq, int characteristic, int mixed, int nx, int ny) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(TuneKey(eq, characteristic, mixed, nx, ny));
  return it == g_tune.end() ? TileShape() : it->second;
}

void tuning_set_shape(int eq, int characteristic, int mixed, int nx, int ny, TileShape t) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[TuneKey(eq, characteristic, mixed, nx, ny)] = t;
}

static std::string device_name() {
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
    return "unknown";
  std::string n = prop.name;
  for (char& c : n)
    if (c == ' ') c = '_';
  return n;
}

// scratch-solve accessors implemented in engine.cu
KStage solve_stage(Solve* s, int k);
const hweno_problem* solve_problem(Solve* s);
KProblem solve_kproblem(Solve* s);

}  // namespace hw

using namespace hw;

// 1D: block width x threads per cell.  Candidates: 128- and 32-thread blocks of one thread per
// cell, and for Euler with the characteristic decomposition 128-, 64- and 32-thread blocks of
// one lane per characteristic field; each timed over eight stage launches (a 1D stage lasts
// microseconds), the fastest kept.  *best_rows = block width, *best_bands = threads per cell.
static int tune1d(const hweno_problem* p, Solve* s, cudaStream_t st, int* best_rows,
                  int* best_bands, double* best_ms) {
  const bool ch = p->equation == HWENO_EULER && p->characteristic;
  const int cand[5][2] = {{128, 1}, {32, 1}, {128, 4}, {64, 4}, {32, 4}};
  const int ncand = ch ? 5 : 2;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const KStage S = solve_stage(s, 1);
  const KProblem kp = solve_kproblem(s);
  int rc = HWENO_OK;
  float best_t = 1e30f;
  TileShape best;
  for (int c = 0; c < ncand && rc == HWENO_OK; ++c) {
    TileShape t;
    t.width = cand[c][0];
    t.lanes = cand[c][1];
    tuning_force_shape1d(t);
    float tmin = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      cudaEventRecord(a, st);
      cudaError_t e = cudaSuccess;
      for (int l = 0; l < 8 && e == cudaSuccess; ++l)
        e = launch_stage1d(p->equation, ch, p->precision == HWENO_MIXED32, kp, S, st);
      cudaEventRecord(b, st);
      if (e != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess) {
        rc = HWENO_ERR_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      if (rep > 0 && ms / 8.f < tmin) tmin = ms / 8.f;
    }
    if (rc == HWENO_OK && tmin < best_t) {
      best_t = tmin;
      best = t;
    }
  }
  tuning_force_shape1d(TileShape());
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  tuning_set_shape(p->equation, ch ? 1 : 0, p->precision == HWENO_MIXED32, p->nx, 1, best);
  if (best_rows) *best_rows = best.width;
  if (best_bands) *best_bands = best.lanes;
  if (best_ms) *best_ms = best_t;
  return HWENO_OK;
}

extern "C" {

int hweno_autotune(hweno_engine* e, const hweno_problem* p, const double* host, int* best_rows,
                   int* best_bands, double* best_ms) {
  if (!e || !p || !host) return HWENO_ERR_ARG;
  std::lock_guard<std::recursive_mutex> lk(engine_mutex(e));
  cudaSetDevice(engine_device(e));
  Solve* s = nullptr;
  int rc = engine_alloc_solve(e, p, &s);
  if (rc) return rc;
  cudaStream_t st = engine_stream(e);
  rc = engine_load_state(e, s, host, 0.0, st);
  if (rc) {
    engine_release_solve(e, s);
    return rc;
  }
  if (p->dim == 1) {
    rc = tune1d(p, s, st, best_rows, best_bands, best_ms);
    engine_release_solve(e, s);
    if (rc) engine_set_error(e, "autotune launch failed");
    return rc;
  }
  // candidates: block widths (128, 96, 64 and 192 threads) x band counts (0 = the default bands; then
  // 1.25, 1.5 and 2 times as many as the widest bands of that width) x chunk heights (0 = one
  // wave over the resident slots).  Screened on stage 1 (the fastest of three launches after
  // one untimed); the finalists -- at most four, within 3 % of the fastest -- are then timed
  // over whole three-stage sequences (stages 2 and 3 also read U^n and V-hat), and the fastest
  // sequence decides.
  const int rows_c[] = {0, 8, 16, 32, 64, 128, 256};
  const int widths[] = {128, 96, 64, 192};
  constexpr int kWidths = sizeof(widths) / sizeof(widths[0]);
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const KStage S3[3] = {solve_stage(s, 1), solve_stage(s, 2), solve_stage(s, 3)};
  const KProblem kp = solve_kproblem(s);
  const bool ch = p->equation == HWENO_EULER && p->characteristic;
  const bool mixed = p->precision == HWENO_MIXED32;
  // the fastest of reps - 1 timed runs (after one untimed) of the stages k0 .. k1 in shape t,
  // per stage; < 0 on a launch error
  auto time_shape = [&](const TileShape& t, int k0, int k1, int reps) -> float {
    tuning_force_shape(t);
    float tmin = 1e30f;
    for (int rep = 0; rep < reps; ++rep) {
      cudaEventRecord(a, st);
      cudaError_t c = cudaSuccess;
      for (int k = k0; k <= k1 && c == cudaSuccess; ++k)
        c = launch_stage2d(p->equation, ch, mixed, kp, S3[k - 1], st);
      cudaEventRecord(b, st);
      if (c != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess) return -1.f;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      ms /= (float)(k1 - k0 + 1);
      if (rep > 0 && ms < tmin) tmin = ms;
    }
    return tmin;
  };
  std::vector<std::pair<float, TileShape>> screened;
  for (int wi = 0; wi < kWidths && rc == HWENO_OK; ++wi) {
    const int bw = widths[wi];
    const int bmin = (p->nx + bw - 3) / (bw - 2);
    const int bands_c[4] = {0, (5 * bmin + 3) / 4, (3 * bmin + 1) / 2, 2 * bmin};
    for (int bi = 0; bi < 4 && rc == HWENO_OK; ++bi) {
      const int bc = bands_c[bi];
      if (bi > 0 && (bc <= bmin || bc > p->nx || bc == bands_c[bi - 1])) continue;
      for (int r : rows_c) {
        if (r > 0 && r >= p->ny && r != rows_c[1]) continue;
        TileShape t;
        t.rows = r > 0 ? r : -1;
        t.bands = bc > 0 ? bc : -1;
        t.width = bw;
        const float ms = time_shape(t, 1, 1, 4);
        if (ms < 0.f) {
          rc = HWENO_ERR_CUDA;
          break;
        }
        screened.push_back({ms, t});
      }
    }
  }
  TileShape best;
  float best_t = 1e30f;
  if (rc == HWENO_OK && !screened.empty()) {
    std::stable_sort(screened.begin(), screened.end(),
                     [](const std::pair<float, TileShape>& x,
                        const std::pair<float, TileShape>& y) { return x.first < y.first; });
    const float lim = screened[0].first * 1.03f;
    for (size_t i = 0; i < screened.size() && i < 4 && rc == HWENO_OK; ++i) {
      if (i > 0 && screened[i].first > lim) break;
      const float ms = time_shape(screened[i].second, 1, 3, 5);
      if (ms < 0.f) {
        rc = HWENO_ERR_CUDA;
        break;
      }
      if (ms < best_t) {
        best_t = ms;
        best = screened[i].second;
      }
    }
  }
  tuning_force_shape(TileShape());
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  engine_release_solve(e, s);
  if (rc) {
    engine_set_error(e, "autotune launch failed");
    return rc;
  }
  TileShape keep;
  keep.rows = best.rows > 0 ? best.rows : -1;
  keep.bands = best.bands > 0 ? best.bands : -1;
  keep.width = best.width;
  tuning_set_shape(p->equation, p->equation == HWENO_EULER ? p->characteristic : 0,
                   p->precision == HWENO_MIXED32, p->nx, p->ny, keep);
  if (best_rows) *best_rows = best.rows > 0 ? best.rows : 0;
  if (best_bands) *best_bands = best.bands > 0 ? best.bands : 0;
  if (best_ms) *best_ms = best_t;
  return HWENO_OK;
}

int hweno_tuning_query(const hweno_problem* p, int* rows, int* bands, int* width, int* lanes) {
  if (!p || (p->dim != 1 && p->dim != 2)) return HWENO_ERR_ARG;
  const int ch = p->equation == HWENO_EULER ? p->characteristic : 0;
  const TileShape t = tuning_shape(p->equation, ch, p->precision == HWENO_MIXED32, p->nx,
                                   p->dim == 1 ? 1 : p->ny);
  if (rows) *rows = t.rows;
  if (bands) *bands = t.bands;
  if (width) *width = t.width;
  if (lanes) *lanes = t.lanes;
  return (t.rows | t.bands | t.width | t.lanes) ? 1 : 0;
}

int hweno_tuning_save(const char* path) {
  if (!path) return HWENO_ERR_ARG;
  FILE* f = std::fopen(path, "w");
  if (!f) return HWENO_ERR_ARG;
  const std::string dev = device_name();
  std::lock_guard<std::mutex> lk(g_tune_mu);
  std::fprintf(f, "# hweno tuning table: gpu equation characteristic mixed nx ny rows bands "
                 "width lanes\n");
  for (auto& kv : g_tune)
    std::fprintf(f, "%s %d %d %d %d %d %d %d %d %d\n", dev.c_str(), std::get<0>(kv.first),
                 std::get<1>(kv.first), std::get<2>(kv.first), std::get<3>(kv.first),
                 std::get<4>(kv.first), kv.second.rows, kv.second.bands, kv.second.width,
                 kv.second.lanes);
  std::fclose(f);
  return HWENO_OK;
}

int hweno_tuning_load(const char* path) {
  if (!path) return HWENO_ERR_ARG;
  FILE* f = std::fopen(path, "r");
  if (!f) return HWENO_ERR_ARG;
  const std::string dev = device_name();
  char line[512], name[256];
  int n = 0;
  while (std::fgets(line, sizeof line, f)) {
    if (line[0] == '#') continue;
    int eq, ch, mx, nx, ny;
    TileShape t;
    const int got = std::sscanf(line, "%255s %d %d %d %d %d %d %d %d %d", name, &eq, &ch, &mx,
                                &nx, &ny, &t.rows, &t.bands, &t.width, &t.lanes);
    if ((got == 8 || got == 10) && dev == name) {
      tuning_set_shape(eq, ch, mx, nx, ny, t);
      ++n;
    }
  }
  std::fclose(f);
  return n;
}

}  // extern "C"
