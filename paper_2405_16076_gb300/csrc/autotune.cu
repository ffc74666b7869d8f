// Autotuning of the ingest's group size: the number of device columns that one sketch launch
// reads (one HBM read of each column sketches all s + h rows for the whole group).  Larger groups
// spread the on-chip generation of Omega and the fill of each launch's pipeline over more
// columns; smaller groups start earlier and, beside a batch step running on its own streams,
// hold the SMs for shorter stretches.  Which wins depends on m, s + h, the precision and the
// device, so it is measured: each candidate runs the caller's columns through a handle of its own
// (public entry points only, nothing here touches device memory directly) and the device time of
// the ingest phases per column is compared.  Host code only.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <vector>

#include "rid.h"
#include "rid_internal.cuh"

namespace {

int fail_global(int code, const char* msg) {
  rid::set_global_error(msg);
  return code;
}

// Cache key: the device and every configuration field the ingest's cost depends on.
std::string tune_key(const rid_config* c, int dev) {
  cudaDeviceProp p;
  memset(&p, 0, sizeof(p));
  cudaGetDeviceProperties(&p, dev);
  std::string name(p.name);
  for (char& ch : name)
    if (ch == ' ' || ch == '\t' || ch == '|') ch = '_';
  char buf[512];
  snprintf(buf, sizeof(buf), "%s|sm%d|cc%d.%d|m%lld|k%d|s%d|h%d|dt%d|sp%d|om%d|gd%d|rl%d",
           name.c_str(), p.multiProcessorCount, p.major, p.minor, (long long)c->m, c->k, c->s, c->h,
           c->data_dtype, c->sketch_prec, c->omega_kind, c->grad_dims, c->right_l);
  return std::string(buf);
}

// The last entry of the cache file for this key, if any.  Lines: "<key> <group> <us per column>".
bool cache_lookup(const char* path, const std::string& key, int gmax, int* g, double* us) {
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[1024];
  char k[1024];
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    int gv = 0;
    double uv = 0.0;
    if (sscanf(line, "%1023s %d %lf", k, &gv, &uv) == 3 && key == k && gv >= 1 && gv <= gmax) {
      *g = gv;
      *us = uv;
      found = true;
    }
  }
  fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& key, int g, double us) {
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %.6g\n", key.c_str(), g, us);
  fclose(f);
}

// Device time (microseconds per column) of the ingest phases -- sketch launch, reduction, copy
// into the buffer slots, norms, SS^T -- for groups of at most g columns: one untimed pass, then
// one pass bracketed by the handle's own event pairs.  Batch steps that the columns trigger run
// on their own streams and are not counted.
int time_group(const rid_config* base, int g, const void* cols, int64_t ld, int32_t ncols, double* us) {
  rid_config c = *base;
  c.group_max = g;
  c.defer_device_input = 1;
  if (c.n_max < ncols) c.n_max = ncols;
  rid_handle* h = nullptr;
  int rc = rid_init(&h, &c);
  if (rc != RID_OK) return rc;
  for (int pass = 0; pass < 2 && rc == RID_OK; ++pass) {
    rc = rid_reset(h);
    if (rc == RID_OK) rc = rid_profile(h, pass);
    if (rc == RID_OK) rc = rid_ingest(h, cols, ld, ncols, 1);
    if (rc == RID_OK) rc = rid_sync(h);
  }
  double ms[3] = {0.0, 0.0, 0.0};
  if (rc == RID_OK) rc = rid_profile_read(h, ms, nullptr, nullptr);
  if (rc != RID_OK) {
    const char* e = rid_last_error(h);
    rid::set_global_error(e ? e : "autotune measurement failed");
  }
  rid_destroy(h);
  if (rc == RID_OK) *us = (ms[0] + ms[1]) * 1e3 / ncols;
  return rc;
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
  int dev = 0;
  cudaGetDevice(&dev);
  const std::string key = tune_key(cfg, dev);
  const int gmax = cfg->sketch_prec != RID_SKETCH_NATIVE ? rid::kMaxGroup : rid::kMaxB;
  const char* path = getenv("RID_AUTOTUNE_CACHE");
  int g_hit = 0;
  double us_hit = 0.0;
  if (path && *path && cache_lookup(path, key, gmax, &g_hit, &us_hit)) {
    cfg->group_max = g_hit;
    if (us_per_col) *us_per_col = us_hit;
    return RID_OK;
  }
  // Groups never span a batch boundary (t = k columns) nor exceed the columns given, so every
  // candidate above the first power of two >= min(ncols, k) forms the same groups.
  const int cap = ncols < cfg->k ? ncols : cfg->k;
  std::vector<int> gs;
  std::vector<double> ts;
  for (int g = 1; g <= gmax; g *= 2) {
    double us = 0.0;
    rc = time_group(cfg, g, cols, ld, ncols, &us);
    if (rc != RID_OK) return rc;
    gs.push_back(g);
    ts.push_back(us);
    if (g >= cap) break;
  }
  // the largest group within 2 % of the fastest: fewer launches and less host work per column
  double best_us = ts[0];
  for (double t : ts) best_us = t < best_us ? t : best_us;
  int best = gs[0];
  double chosen_us = ts[0];
  for (size_t i = 0; i < gs.size(); ++i)
    if (ts[i] <= 1.02 * best_us) {
      best = gs[i];
      chosen_us = ts[i];
    }
  cfg->group_max = best;
  if (us_per_col) *us_per_col = chosen_us;
  if (path && *path) cache_store(path, key, best, chosen_us);
  return RID_OK;
}
