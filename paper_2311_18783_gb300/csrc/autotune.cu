// Autotuner of the streaming SYMV launch configuration.
//
// The knob space (dense.cu, SymvCands): bulk-copy stages in flight, tiles
// consumed per barrier pair, warps sharing a tile and persistent CTAs per
// SM.  For every tile batch the solve path applies (the local factors in
// float32 and float64, the float64 S_j^-1 blocks of the split and of the
// GenEO operator), each candidate is timed with CUDA events on the set-up
// stream over a few launches on the batch's real tiles, and the fastest one
// is kept.  Results are cached per process, keyed by the target, the storage
// precision, the number of right-hand sides (1: the SYMV applies one column
// per launch), the mean matrix size bucket (n_i rounded to a power of two)
// and the stored-tile bucket; with options.autotune_cache set, the cache is
// read from and appended to that text file ("key index milliseconds" per
// line), so later set-ups of the same shapes skip the timing.  The same
// cache holds the choice between the two shapes of the sparse coarse solve
// (autotune_coarse).
#include <cmath>
#include <cstdio>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>

#include "setup.hpp"

namespace geneo {
namespace {

std::mutex g_tune_mu;
std::map<std::string, int> g_tune_cache;
std::map<std::string, bool> g_tune_loaded;

int pow2_bucket(double v) { return v < 1 ? 0 : (int)std::lround(std::log2(v)); }

std::string tune_key(const char *target, int prec, const TileBatch &b) {
  double mean = 0;
  for (int m = 0; m < b.nmat; ++m) mean += (double)b.dim[m];
  mean /= std::max(1, b.nmat);
  std::ostringstream k;
  k << "symv/" << target << "/" << (prec == GENEO_PREC_FP32 ? "f32" : "f64") << "/nrhs1/ni2^"
    << pow2_bucket(mean) << "/tiles2^" << pow2_bucket((double)b.ntiles);
  return k.str();
}

void load_cache_file(const char *path) {
  if (!path || !*path || g_tune_loaded[path]) return;
  g_tune_loaded[path] = true;
  std::ifstream f(path);
  std::string key;
  int idx;
  double ms;
  while (f >> key >> idx >> ms) g_tune_cache[key] = idx;
}

void append_cache_file(const char *path, const std::string &key, int idx, double ms) {
  if (!path || !*path) return;
  std::ofstream f(path, std::ios::app);
  f << key << " " << idx << " " << ms << "\n";
}

// mean milliseconds of `reps` applications of the batch with candidate idx
template <typename T>
double time_candidate(geneo_ctx *c, TileBatch &b, const T *data, int idx, const double *x,
                      double *y, int reps) {
  cudaStream_t s = c->stream;
  const int slot = sizeof(T) == 8 ? 1 : 0;
  const int keep = b.symv_cfg[slot];
  b.symv_cfg[slot] = idx;
  cudaEvent_t e0, e1;
  GENEO_CUDA(cudaEventCreate(&e0));
  GENEO_CUDA(cudaEventCreate(&e1));
  float ms = 0;
  try {
    symv_batch<T>(b, data, x, y, c->d_err.p, s);  // warm-up (attributes, schedule)
    GENEO_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r) symv_batch<T>(b, data, x, y, c->d_err.p, s);
    GENEO_CUDA(cudaEventRecord(e1, s));
    GENEO_CUDA(cudaEventSynchronize(e1));
    GENEO_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b.symv_cfg[slot] = keep;
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b.symv_cfg[slot] = keep;
  check_device_error(c, s);
  return ms / reps;
}

template <typename T>
void tune_one(geneo_ctx *c, const char *target, int prec, TileBatch &b, const T *data) {
  if (!data || b.ntiles == 0) return;
  const int slot = sizeof(T) == 8 ? 1 : 0;
  const std::string key = tune_key(target, prec, b);
  const char *path = c->opt.autotune_cache;
  TuneRecord rec;
  rec.target = target;
  rec.key = key;
  rec.precision = prec;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    load_cache_file(path);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end() && it->second >= 0 && it->second < symv_candidates<T>()) {
      b.symv_cfg[slot] = it->second;
      rec.chosen = it->second;
      rec.from_cache = true;
      c->tune.push_back(rec);
      return;
    }
  }
  // timing buffers: padded local vectors of the batch (values do not matter)
  DevBuf<double> x, y;
  x.alloc(b.vlen);
  y.alloc(b.vlen);
  x.zero(c->stream);
  // enough launches for about 20 ms per candidate, between 3 and 50
  const double t0 = time_candidate<T>(c, b, data, 0, x.p, y.p, 1);
  const int reps = std::max(3, std::min(50, (int)(20.0 / std::max(t0, 1e-3))));
  int best = 0;
  double best_ms = 1e300;
  for (int i = 0; i < symv_candidates<T>(); ++i) {
    const double ms = time_candidate<T>(c, b, data, i, x.p, y.p, reps);
    rec.ms.push_back(ms);
    if (ms < best_ms) {
      best_ms = ms;
      best = i;
    }
  }
  b.symv_cfg[slot] = best;
  rec.chosen = best;
  c->tune.push_back(rec);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[key] = best;
  append_cache_file(path, key, best, best_ms);
}

}  // namespace

void autotune_symv(geneo_ctx *c) {
  if (c->loc_f32.p) tune_one<float>(c, "local", GENEO_PREC_FP32, c->loc, c->loc_f32.p);
  if (c->loc_f64.p) tune_one<double>(c, "local", GENEO_PREC_FP64, c->loc, c->loc_f64.p);
  if (c->xi && c->xi->s_inv.p) tune_one<double>(c, "gradient", GENEO_PREC_FP64, c->xi->sb,
                                                c->xi->s_inv.p);
  if (c->xi && c->xi->s_inv32.p) tune_one<float>(c, "gradient", GENEO_PREC_FP32, c->xi->sb,
                                                 c->xi->s_inv32.p);
}

void autotune_coarse(geneo_ctx *c) {
  if (!mf_single_launch_available(c)) return;
  std::ostringstream k;
  k << "coarse/f64/nrhs1/n0_2^" << pow2_bucket((double)c->n0) << "/bytes2^"
    << pow2_bucket((double)mf_solve_bytes(c));
  TuneRecord rec;
  rec.target = "coarse";
  rec.key = k.str();
  rec.precision = GENEO_PREC_FP64;
  const char *path = c->opt.autotune_cache;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    load_cache_file(path);
    auto it = g_tune_cache.find(rec.key);
    if (it != g_tune_cache.end() && (it->second == 0 || it->second == 1)) {
      c->mf_persist = it->second == 1;
      rec.chosen = it->second;
      rec.from_cache = true;
      c->tune.push_back(rec);
      return;
    }
  }
  // candidate 0: one launch per level and phase, 1: one cooperative launch;
  // five solves each on the context's own factor (right-hand side values do
  // not change the work)
  cudaStream_t s = c->stream;
  cudaEvent_t e0, e1;
  GENEO_CUDA(cudaEventCreate(&e0));
  GENEO_CUDA(cudaEventCreate(&e1));
  int best = 0;
  double best_ms = 1e300;
  try {
    for (int cand = 0; cand < 2; ++cand) {
      c->mf_persist = cand == 1;
      mf_solve(c, c->crs_x.p, c->crs_y.p, s, 1);  // warm-up
      GENEO_CUDA(cudaEventRecord(e0, s));
      for (int r = 0; r < 5; ++r) mf_solve(c, c->crs_x.p, c->crs_y.p, s, 1);
      GENEO_CUDA(cudaEventRecord(e1, s));
      GENEO_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      GENEO_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      rec.ms.push_back(ms / 5);
      if (ms / 5 < best_ms) {
        best_ms = ms / 5;
        best = cand;
      }
    }
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->mf_persist = false;
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  check_device_error(c, s);
  c->mf_persist = best == 1;
  rec.chosen = best;
  c->tune.push_back(rec);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[rec.key] = best;
  append_cache_file(path, rec.key, best, best_ms);
}

void autotune_clear_cache() {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache.clear();
  g_tune_loaded.clear();
}

}  // namespace geneo
