// Autotuning of the ingest's launch shape: the group size (how many device columns one sketch
// launch reads; one HBM read of each column sketches all s + h rows for the whole group) and the
// number of CTAs per sketch launch.  Larger groups spread the on-chip generation of Omega and the
// fill of each launch's pipeline over more columns; smaller groups start earlier.  Fewer CTAs
// leave more SMs to the batch step that runs beside the ingest on its own streams; more CTAs
// read faster.  Which wins depends on m, s + h, k, the precision and the device, so it is
// measured: each candidate runs the caller's columns through a handle of its own (public entry
// points only; nothing here touches device memory directly), and the wall time of a whole pass
// -- the ingest and the batch steps it triggers, up to the synchronization -- is compared.
// Host code only.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <string>
#include <vector>

#include "rid.h"
#include "rid_internal.cuh"
#include "tune_cache.h"

namespace {

int fail_global(int code, const char* msg) {
  rid::set_global_error(msg);
  return code;
}

// Cache key: the device and every configuration field the pass's cost depends on.
std::string tune_key(const rid_config* c, int dev, int* n_sm) {
  cudaDeviceProp p;
  memset(&p, 0, sizeof(p));
  cudaGetDeviceProperties(&p, dev);
  *n_sm = p.multiProcessorCount;
  std::string name(p.name);
  for (char& ch : name)
    if (ch == ' ' || ch == '\t' || ch == '|') ch = '_';
  char buf[512];
  snprintf(buf, sizeof(buf), "%s|sm%d|cc%d.%d|m%lld|k%d|s%d|h%d|dt%d|sp%d|om%d|gd%d|rl%d|gc%d",
           name.c_str(), p.multiProcessorCount, p.major, p.minor, (long long)c->m, c->k, c->s, c->h,
           c->data_dtype, c->sketch_prec, c->omega_kind, c->grad_dims, c->right_l, c->grad_coeff);
  return std::string(buf);
}

// Wall time (microseconds per column) of a whole pass over the columns -- reset, ingest with
// groups of at most g columns and `ctas` CTAs per sketch launch (0: automatic), the batch steps
// the columns trigger, synchronization -- the fastest of three passes after one untimed pass.
int time_config(const rid_config* base, int g, int ctas, const void* cols, int64_t ld, int32_t ncols,
                double* us) {
  rid_config c = *base;
  c.group_max = g;
  c.ingest_ctas = ctas;
  c.defer_device_input = 1;
  if (c.n_max < ncols) c.n_max = ncols;
  rid_handle* h = nullptr;
  int rc = rid_init(&h, &c);
  if (rc != RID_OK) return rc;
  double best = 0.0;
  for (int pass = 0; pass < 4 && rc == RID_OK; ++pass) {
    rc = rid_reset(h);
    if (rc == RID_OK) rc = rid_sync(h);
    const auto t0 = std::chrono::steady_clock::now();
    if (rc == RID_OK) rc = rid_ingest(h, cols, ld, ncols, 1);
    if (rc == RID_OK) rc = rid_sync(h);
    const double dt = std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
    if (pass > 0 && (best == 0.0 || dt < best)) best = dt;
  }
  if (rc != RID_OK) {
    const char* e = rid_last_error(h);
    rid::set_global_error(e ? e : "autotune measurement failed");
  }
  rid_destroy(h);
  if (rc == RID_OK) *us = best / ncols;
  return rc;
}

// The index of the last (prefer_last) or the first entry within 2 % of the fastest time.
size_t pick(const std::vector<double>& ts, bool prefer_last) {
  double lo = ts[0];
  for (double t : ts) lo = t < lo ? t : lo;
  size_t best = 0;
  bool found = false;
  for (size_t i = 0; i < ts.size(); ++i)
    if (ts[i] <= 1.02 * lo && (prefer_last || !found)) {
      best = i;
      found = true;
    }
  return best;
}

}  // namespace

extern "C" int rid_autotune(rid_config* cfg, const void* cols, int64_t ld, int32_t ncols, double* us_per_col) {
  if (!cfg || !cols) return fail_global(RID_EINVAL, "NULL argument");
  int rc = rid_config_check(cfg);
  if (rc != RID_OK) return rc;
  if (ncols < 1) return fail_global(RID_EINVAL, "ncols must be >= 1");
  if (ld < cfg->m) return fail_global(RID_EINVAL, "ld < m");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail_global(RID_ENOLIB, "no CUDA device");
  }
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, cols) != cudaSuccess ||
      (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)) {
    cudaGetLastError();
    return fail_global(RID_EINVAL, "cols must be device memory");
  }
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  const std::string key = tune_key(cfg, dev, &n_sm);
  const bool tc = cfg->sketch_prec != RID_SKETCH_NATIVE;
  const int gmax = tc ? rid::kMaxGroup : rid::kMaxB;
  const char* path = getenv("RID_AUTOTUNE_CACHE");
  {
    int g = 0, ctas = 0;
    double us = 0.0;
    if (path && *path && rid::tune_cache_lookup(path, key, gmax, &g, &ctas, &us)) {
      cfg->group_max = g;
      cfg->ingest_ctas = ctas;
      if (us_per_col) *us_per_col = us;
      return RID_OK;
    }
  }
  // 1. Group size, with the automatic CTA count.  Groups never span a batch (t = k columns) nor
  // exceed the columns given, so every candidate above the first power of two >= min(ncols, k)
  // forms the same groups.  Ties go to the larger group (fewer launches, less host work).
  const int cap = ncols < cfg->k ? ncols : cfg->k;
  std::vector<int> gs;
  std::vector<double> ts;
  for (int g = 1; g <= gmax; g *= 2) {
    double us = 0.0;
    rc = time_config(cfg, g, 0, cols, ld, ncols, &us);
    if (rc != RID_OK) return rc;
    gs.push_back(g);
    ts.push_back(us);
    if (g >= cap) break;
  }
  size_t ib = pick(ts, true);
  const int gbest = gs[ib];
  double us_best = ts[ib];
  // 2. CTAs per sketch launch for that group size: the automatic count first (kept on a tie),
  // then fractions of the SMs (tensor cores; clamped by rid_init to the buffers it sizes) or
  // multiples of them (native path, at most its automatic four per SM).
  std::vector<int> cs = {0};
  if (tc) {
    for (int num : {1, 2, 3, 4, 5, 6}) cs.push_back(n_sm * num / 6 > 0 ? n_sm * num / 6 : 1);
  } else {
    for (int mul : {1, 2, 3}) cs.push_back(n_sm * mul);
  }
  std::vector<double> tc_times = {us_best};
  for (size_t i = 1; i < cs.size(); ++i) {
    double us = 0.0;
    rc = time_config(cfg, gbest, cs[i], cols, ld, ncols, &us);
    if (rc != RID_OK) return rc;
    tc_times.push_back(us);
  }
  const size_t ic = pick(tc_times, false);
  cfg->group_max = gbest;
  cfg->ingest_ctas = cs[ic];
  us_best = tc_times[ic];
  if (us_per_col) *us_per_col = us_best;
  if (path && *path) rid::tune_cache_store(path, key, gbest, cs[ic], us_best);
  return RID_OK;
}
