// Host side of the C ABI declared in include/rid.h: validation, device
// allocation, and the column-counting state machine of Algorithm 3 that
// issues the ingest launches and, every t columns, the device batch step.
// The host never reads device state while ingesting, so a whole stream can
// be enqueued (or captured) without synchronization.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "fault_inject.h"
#include "rid.h"
#include "rid_internal.cuh"

using rid::Dev;

struct rid_handle {
  rid_config cfg;
  Dev d;
  cudaStream_t st;        // the caller's stream: ingest, and a snapshot of SS^T and ||A||^2 per batch
  cudaStream_t stl[2];    // lambda streams: the lambda part of batch b on stl[b % 2], from the snapshot
  cudaStream_t sts;       // the select stream: ridge scores, uniforms and prune/refill of each step
  cudaStream_t stb;       // the batch stream: the tail of each batch step (basis Gram .. commit)
  cudaStream_t stg;       // the tail's Gram side, forked from and joined to stb within a step
  cudaEvent_t ev_fork;
  // per batch b, slot b % kEv (recorded once per step; the slot of step b is reused by step
  // b + kEv, long after every wait on it was enqueued)
  static constexpr int kEv = 8;
  cudaEvent_t ev_snap[kEv], ev_lambda[kEv], ev_scores[kEv], ev_select[kEv], ev_gram[kEv], ev_tail[kEv];
  int* dslot_buf;         // la x t: buffer-slot lists of the batches b .. b + la - 1 (batch b at b % la)
  double* snap;           // 2 x (s*s + 2): SS^T and ||A||^2 as of the end of a batch, by parity
  // selection records of the steps in flight, by batch parity: the previous and the new basis
  // (indices and pool slots) and the index lists of the tail
  int64_t* rec_i64;       // 2 x 2t
  int* rec_i32;           // 2 x (10t + META_LEN)
  int count;          // columns buffered since the last batch step
  int64_t n_obs;      // columns ingested
  int64_t n_prev;     // columns covered by the last batch step
  int batch;          // batch steps run
  bool finalized;
  rid_rcss* rcss = nullptr;       // Algorithm 1 as the selector (rid_attach_rcss), or NULL
  bool joined;            // the caller's stream already waits for every batch step issued
  bool kg_ready;          // d.Kg holds Omega G^p Omega^T / s
  size_t esize;
  void* staging;          // host-input staging: two areas of group_max columns of m_pad
  cudaStream_t stc;       // host-to-device copies of host columns into the staging areas
  cudaEvent_t ev_cfork;   // on st: the ingest of the previous group has been enqueued before this point
  cudaEvent_t ev_cfull;   // on stc: the copies of the group being flushed are complete
  bool cfork_valid;       // ev_cfork has been recorded
  int stage_area;         // staging area the current group's host columns go to
  int pend_host;          // host columns in the pending group
  std::vector<const void*> pend;   // columns recorded but not yet sketched
  int group_max;
  bool tc;                // tensor-core ingest (FP32 data, BF16 / BF16x2 sketch)
  int tc_blocks;          // CTAs of the basis Gram (and the bound of the partial buffers)
  int ingest_blocks;      // CTAs of the tensor-core ingest
  int first_blocks;       // CTAs of the first batch's ingest (no batch step beside it)
  float* tc_part;
  double* tc_npart;
  std::string err;
  int n_sm;
  // measurement (rid_profile)
  bool prof;
  std::vector<cudaEvent_t> evpool;
  size_t evused;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> spans[3];
  int64_t kernels[3];
  // per-batch phase timeline (rid_profile_timeline): base event, then (batch, phase, start, end)
  cudaEvent_t tl_base;
  struct TlRec { int batch, phase; cudaEvent_t a, b; };
  std::vector<TlRec> tl;
  float* tg_part;
  // SM partition (cfg.batch_sms > 0): green contexts of the batch steps' streams (stl, sts, stb,
  // stg) and of the ingest stream sti, which takes every group after the first batch's
  CUgreenCtx green_b;
  CUgreenCtx green_i;
  cudaStream_t sti;
  cudaEvent_t ev_ing0;    // on st: the caller's work before an ingest group
  cudaEvent_t ev_ing1;    // on sti: the ingest group
  int part_b, part_i;     // SMs of the two partitions
  // per-batch log (rid_log_enable): log_cap slots of kLogSlot bytes on the device, batch b in
  // slot b % log_cap; log_first = the first batch step it covers
  char* log_dev;
  int log_cap;
  int log_first;
};

// A log slot: the step's scal[] at 0 (after its tail), lambda and ||A_obs||^2 at 128 (after its
// lambda part, before the next step's lambda part overwrites them), meta[] at 144.
constexpr size_t kLogSlot = 256;
static_assert(144 + sizeof(int) * rid::META_LEN <= kLogSlot && sizeof(double) * rid::SCAL_LOG <= 128,
              "log slot layout");

static thread_local std::string g_init_err;

namespace rid {
void set_global_error(const char* msg) { g_init_err = msg ? msg : ""; }
}  // namespace rid

namespace {

// NVTX range over a host-side phase (the enqueue of an ingest call, a sketch group or a batch
// step), so that profilers can attribute and filter the kernels it launches; a no-op unless a
// tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

int fail(rid_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg; else g_init_err = msg;
  return code;
}

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(h, e_ == cudaErrorMemoryAllocation ? RID_ENOMEM : RID_ECUDA,         \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                 \
  } while (0)

// Allocation-failure injection, for tests of the error paths (no device fault is involved): with
// RID_FAULT_INJECT=alloc:<n> in the environment when rid_init starts, the n-th device allocation
// of the handles from then on -- inside that rid_init or in a later capacity growth -- reports
// cudaErrorMemoryAllocation without calling cudaMalloc.  Every rid_init re-reads the variable
// (unset: off).
rid::AllocCountdown g_alloc_countdown;

void arm_fault_injection() { g_alloc_countdown.arm(rid::parse_fault_inject(getenv("RID_FAULT_INJECT"))); }

template <typename T>
cudaError_t dalloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  if (g_alloc_countdown.next_fails()) return cudaErrorMemoryAllocation;
  return cudaMalloc((void**)p, n * sizeof(T));
}

void free_all(Dev& d, void* staging) {
  void* ptrs[] = {d.pool, d.omegaT, d.omegagT, d.S, d.SSt, d.fro2, d.JC, d.JC_prev, d.slotC,
                  d.slotC_prev, d.dslot_all, d.JD, d.tau_old, d.tauC, d.tauD, d.meta, d.act,
                  d.pact, d.isnew, d.posof, d.newpos, d.gnew, d.gtgt, d.scal, d.Gp, d.gpart,
                  d.P, d.cand, d.work, d.hpart, d.spart, d.npart, d.err, d.gbar, d.Y, d.Wr, d.zq, d.Sg,
                  d.Kg, d.gnorm, d.xbuf, d.gfield, d.glev, d.gnorm2, staging};
  for (void* p : ptrs) if (p) cudaFree(p);
  if (d.Slev && d.Slev != d.S) cudaFree(d.Slev);
}

// Driver entry points of the green-context calls (SM partition), fetched through the runtime so
// that the library needs no link against the driver library; ok = all of them were found.
struct GreenApi {
  CUresult (*dev_get)(CUdevice*, int) = nullptr;
  CUresult (*dev_res)(CUdevice, CUdevResource*, CUdevResourceType) = nullptr;
  CUresult (*split)(CUdevResource*, unsigned int*, const CUdevResource*, CUdevResource*, unsigned int,
                    unsigned int) = nullptr;
  CUresult (*gen_desc)(CUdevResourceDesc*, CUdevResource*, unsigned int) = nullptr;
  CUresult (*create)(CUgreenCtx*, CUdevResourceDesc, CUdevice, unsigned int) = nullptr;
  CUresult (*destroy)(CUgreenCtx) = nullptr;
  CUresult (*to_ctx)(CUcontext*, CUgreenCtx) = nullptr;
  CUresult (*stream_create)(CUstream*, CUgreenCtx, unsigned int, int) = nullptr;
  CUresult (*stream_destroy)(CUstream) = nullptr;
  CUresult (*ctx_get)(CUcontext*) = nullptr;
  CUresult (*ctx_set)(CUcontext) = nullptr;
  bool ok = false;
};

const GreenApi& green_api() {
  static const GreenApi api = [] {
    GreenApi a;
    auto get = [](const char* name, void** fn) {
      cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
      const bool found = cudaGetDriverEntryPointByVersion(name, fn, 13000, cudaEnableDefault, &q) == cudaSuccess &&
                         q == cudaDriverEntryPointSuccess && *fn != nullptr;
      cudaGetLastError();
      return found;
    };
    a.ok = get("cuDeviceGet", (void**)&a.dev_get) && get("cuDeviceGetDevResource", (void**)&a.dev_res) &&
           get("cuDevSmResourceSplitByCount", (void**)&a.split) &&
           get("cuDevResourceGenerateDesc", (void**)&a.gen_desc) && get("cuGreenCtxCreate", (void**)&a.create) &&
           get("cuGreenCtxDestroy", (void**)&a.destroy) && get("cuCtxFromGreenCtx", (void**)&a.to_ctx) &&
           get("cuGreenCtxStreamCreate", (void**)&a.stream_create) &&
           get("cuStreamDestroy", (void**)&a.stream_destroy) && get("cuCtxGetCurrent", (void**)&a.ctx_get) &&
           get("cuCtxSetCurrent", (void**)&a.ctx_set);
    return a;
  }();
  return api;
}

// The SM partition: a green context of at least cfg.batch_sms SMs (a group of the device's SM
// resource, split so that it keeps the largest thread-block clusters) with the batch steps'
// streams, and one of the remaining SMs with the ingest stream.  The events stay in the primary
// context (a green context's stream records them and waits on them like any other).
int create_partition(rid_handle* h, int prio_hi) {
  const GreenApi& g = green_api();
  if (!g.ok) return fail(h, RID_ECUDA, "SM partition: the CUDA driver offers no green contexts");
  int dev = 0;
  cudaGetDevice(&dev);
  CUdevice cd = 0;
  CUdevResource all = {}, grp = {}, rest = {};
  unsigned int nb = 1;
  if (g.dev_get(&cd, dev) != CUDA_SUCCESS || g.dev_res(cd, &all, CU_DEV_RESOURCE_TYPE_SM) != CUDA_SUCCESS)
    return fail(h, RID_ECUDA, "SM partition: cannot read the device's SM resource");
  if ((unsigned int)h->cfg.batch_sms >= all.sm.smCount)
    return fail(h, RID_EINVAL, "batch_sms must be below the device's SM count");
  if (g.split(&grp, &nb, &all, &rest, CU_DEV_SM_RESOURCE_SPLIT_MAX_POTENTIAL_CLUSTER_SIZE,
              (unsigned int)h->cfg.batch_sms) != CUDA_SUCCESS ||
      nb != 1 || grp.sm.smCount == 0 || rest.sm.smCount == 0)
    return fail(h, RID_EINVAL, "SM partition: cannot split the SMs at batch_sms");
  CUdevResourceDesc db = nullptr, di = nullptr;
  if (g.gen_desc(&db, &grp, 1) != CUDA_SUCCESS || g.gen_desc(&di, &rest, 1) != CUDA_SUCCESS ||
      g.create(&h->green_b, db, cd, CU_GREEN_CTX_DEFAULT_STREAM) != CUDA_SUCCESS ||
      g.create(&h->green_i, di, cd, CU_GREEN_CTX_DEFAULT_STREAM) != CUDA_SUCCESS)
    return fail(h, RID_ECUDA, "SM partition: green-context creation failed");
  for (cudaStream_t* sp : {&h->stb, &h->stl[0], &h->stl[1], &h->sts, &h->stg}) {
    CUstream x = nullptr;
    if (g.stream_create(&x, h->green_b, CU_STREAM_NON_BLOCKING, prio_hi) != CUDA_SUCCESS)
      return fail(h, RID_ECUDA, "SM partition: stream creation failed");
    *sp = (cudaStream_t)x;
  }
  {
    CUstream x = nullptr;
    if (g.stream_create(&x, h->green_i, CU_STREAM_NON_BLOCKING, 0) != CUDA_SUCCESS)
      return fail(h, RID_ECUDA, "SM partition: stream creation failed");
    h->sti = (cudaStream_t)x;
  }
  h->part_b = (int)grp.sm.smCount;
  h->part_i = (int)rest.sm.smCount;
  // the batch step's cluster kernels must be schedulable inside their partition
  CUcontext prev = nullptr, cb = nullptr;
  if (g.ctx_get(&prev) != CUDA_SUCCESS || g.to_ctx(&cb, h->green_b) != CUDA_SUCCESS || g.ctx_set(cb) != CUDA_SUCCESS)
    return fail(h, RID_ECUDA, "SM partition: cannot enter the batch partition's context");
  const bool fits = rid::batch_clusters_fit(h->d.s, h->d.t);
  g.ctx_set(prev);
  if (!fits) return fail(h, RID_EINVAL, "SM partition: batch_sms SMs cannot co-schedule the batch step's clusters");
  return RID_OK;
}

void destroy_sync_objects(rid_handle* h) {
  const bool part = h->green_b != nullptr || h->green_i != nullptr;
  for (cudaStream_t* sp : {&h->stb, &h->stl[0], &h->stl[1], &h->sts, &h->stg, &h->sti}) {
    if (*sp) {
      if (part) green_api().stream_destroy((CUstream)*sp);
      else cudaStreamDestroy(*sp);
    }
    *sp = nullptr;
  }
  if (h->stc) cudaStreamDestroy(h->stc);
  h->stc = nullptr;
  for (CUgreenCtx* gp : {&h->green_b, &h->green_i}) {
    if (*gp) green_api().destroy(*gp);
    *gp = nullptr;
  }
  for (cudaEvent_t* e : {&h->ev_fork, &h->ev_cfork, &h->ev_cfull, &h->ev_ing0, &h->ev_ing1}) {
    if (*e) cudaEventDestroy(*e);
    *e = nullptr;
  }
  for (int i = 0; i < rid_handle::kEv; ++i)
    for (cudaEvent_t* e : {&h->ev_snap[i], &h->ev_lambda[i], &h->ev_scores[i], &h->ev_select[i], &h->ev_gram[i],
                           &h->ev_tail[i]}) {
      if (*e) cudaEventDestroy(*e);
      *e = nullptr;
    }
}

int create_sync_objects(rid_handle* h) {
  int prio_lo = 0, prio_hi = 0;
  // The batch-step streams get the device's highest priority: their kernels are short and on
  // the critical path, and each of the ingest's CTAs holds a whole SM for its chunk range, so
  // freed SMs should go to them first.
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (h->cfg.batch_sms > 0) {
    const int rc = create_partition(h, prio_hi);
    if (rc != RID_OK) return rc;
  } else {
    for (cudaStream_t* sp : {&h->stb, &h->stl[0], &h->stl[1], &h->sts, &h->stg})
      if (cudaStreamCreateWithPriority(sp, cudaStreamNonBlocking, prio_hi) != cudaSuccess)
        return fail(h, RID_ECUDA, "stream creation failed");
  }
  if (cudaStreamCreateWithFlags(&h->stc, cudaStreamNonBlocking) != cudaSuccess)
    return fail(h, RID_ECUDA, "stream creation failed");
  for (cudaEvent_t* e : {&h->ev_fork, &h->ev_cfork, &h->ev_cfull, &h->ev_ing0, &h->ev_ing1})
    if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess)
      return fail(h, RID_ECUDA, "event creation failed");
  for (int i = 0; i < rid_handle::kEv; ++i)
    for (cudaEvent_t* e : {&h->ev_snap[i], &h->ev_lambda[i], &h->ev_scores[i], &h->ev_select[i], &h->ev_gram[i],
                           &h->ev_tail[i]})
      if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess)
        return fail(h, RID_ECUDA, "event creation failed");
  return RID_OK;
}

// The device view for batch b: its buffer-slot list and the next batch's.
Dev dev_for(const rid_handle* h, int b) {
  Dev d = h->d;
  const int t = d.t;
  d.dslot = h->dslot_buf + (size_t)(b % d.la) * t;
  return d;
}

// The selection record of step b (copy b % 2) as the device view its tail reads: JC / slotC the
// new basis, JC_prev / slotC_prev the previous one, the index lists and the step's counts.
Dev rec_view(const rid_handle* h, int b) {
  Dev r = dev_for(h, b);
  const int t = r.t;
  int64_t* i64 = h->rec_i64 + (size_t)(b & 1) * 2 * t;
  int* i32 = h->rec_i32 + (size_t)(b & 1) * (10 * (size_t)t + rid::META_LEN);
  r.JC = i64;
  r.JC_prev = i64 + t;
  r.slotC = i32;
  r.slotC_prev = i32 + t;
  r.act = i32 + 2 * t;
  r.pact = i32 + 3 * t;
  r.isnew = i32 + 4 * t;
  r.posof = i32 + 5 * t;
  r.newpos = i32 + 6 * t;
  r.gnew = i32 + 7 * t;
  r.gtgt = i32 + 8 * t;                 // 2t
  r.meta = i32 + 10 * t;
  return r;
}

// Make the caller's stream wait for the tail of the latest batch step (after this, work on
// h->st and a synchronization of h->st cover everything the handle has launched).
// Make the caller's stream wait for the last batch step (once per batch step issued: a handle
// whose stream already waits -- e.g. after an asynchronous finalize captured into a CUDA graph,
// whose events must not be waited on outside the graph -- adds no second wait).
void join(rid_handle* h) {
  if (h->batch >= 1 && !h->joined) cudaStreamWaitEvent(h->st, h->ev_tail[(h->batch - 1) % rid_handle::kEv], 0);
  h->joined = true;
}

int64_t hpart_len(const Dev& d, int64_t ncap) {
  const int64_t hh = d.h1 + d.h2 + d.h3;
  return 4 * ((ncap + 31) / 32) * rid::hpart_stride(hh, d.t);
}

// (Re)allocate the arrays whose size follows the column capacity, keeping S, Slev and P.
int grow(rid_handle* h, int64_t need) {
  Dev& d = h->d;
  if (need <= d.n_cap && d.S) return RID_OK;
  int64_t cap = d.n_cap > 0 ? d.n_cap : 1;
  while (cap < need) cap *= 2;
  join(h);
  CK(cudaStreamSynchronize(h->st));
  // New arrays first; on any failure they are released and the handle keeps its current ones.
  double *S = nullptr, *Slev = nullptr, *P = nullptr, *cand = nullptr, *hpart = nullptr, *zq = nullptr,
         *Sg = nullptr;
  cudaError_t e = dalloc(&S, (size_t)d.rows * cap);
  if (e == cudaSuccess && d.grad) e = dalloc(&Slev, (size_t)d.s * cap);
  if (e == cudaSuccess) e = dalloc(&P, (size_t)d.t * cap);
  if (e == cudaSuccess) e = dalloc(&cand, (size_t)4 * d.t * cap);
  if (e == cudaSuccess) e = dalloc(&hpart, (size_t)hpart_len(d, cap));
  if (e == cudaSuccess) e = dalloc(&zq, (size_t)2 * d.t * cap);
  if (e == cudaSuccess && d.grad_coeff) e = dalloc(&Sg, (size_t)2 * d.s * cap);
  if (e == cudaSuccess) e = cudaMemsetAsync(P, 0, sizeof(double) * (size_t)d.t * cap, h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(cand, 0, sizeof(double) * (size_t)4 * d.t * cap, h->st);
  if (e == cudaSuccess && d.S) {
    e = cudaMemcpyAsync(S, d.S, sizeof(double) * (size_t)d.rows * d.n_cap, cudaMemcpyDeviceToDevice, h->st);
    if (e == cudaSuccess && d.grad)
      e = cudaMemcpyAsync(Slev, d.Slev, sizeof(double) * (size_t)d.s * d.n_cap, cudaMemcpyDeviceToDevice, h->st);
    if (e == cudaSuccess && d.grad_coeff)
      e = cudaMemcpyAsync(Sg, d.Sg, sizeof(double) * 2 * (size_t)d.s * d.n_cap, cudaMemcpyDeviceToDevice, h->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(P, d.P, sizeof(double) * (size_t)d.t * d.n_cap, cudaMemcpyDeviceToDevice, h->st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(h->st);
    for (double* p : {S, Slev, P, cand, hpart, zq, Sg})
      if (p) cudaFree(p);
    return fail(h, e == cudaErrorMemoryAllocation ? RID_ENOMEM : RID_ECUDA,
                std::string("capacity growth: ") + cudaGetErrorString(e));
  }
  if (d.S) {
    cudaFree(d.S);
    if (d.grad) cudaFree(d.Slev);
    cudaFree(d.P);
    cudaFree(d.cand);
    cudaFree(d.hpart);
    cudaFree(d.zq);
    if (d.Sg) cudaFree(d.Sg);
  }
  d.S = S;
  d.Slev = d.grad ? Slev : S;
  d.P = P;
  d.cand = cand;
  d.hpart = hpart;
  d.zq = zq;
  d.Sg = Sg;
  d.n_cap = cap;
  return RID_OK;
}

cudaEvent_t next_event(rid_handle* h) {
  if (h->evused == h->evpool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    h->evpool.push_back(e);
  }
  return h->evpool[h->evused++];
}

// Batch step b.  The caller's stream snapshots SS^T and ||A||^2 (buffer b % 2, free once
// the lambda part of step b-2 has run) and goes on ingesting; the lambda part runs on lambda
// stream b % 2 from the snapshot into output copy b % 2 (after step b-2's scores, the last
// reader of that copy); the select part runs on the select stream after it (writing selection
// record b % 2 once the tail of step b-2, its last reader, has ended); the tail runs on the
// batch stream after the select.
int run_batch(rid_handle* h) {
  NvtxRange nvtx("rid_batch_step");
  const int b = h->batch;
  constexpr int E = rid_handle::kEv;
  h->joined = false;
  const Dev db = dev_for(h, b);
  const Dev rv = rec_view(h, b);
  cudaStream_t stl = h->stl[b & 1];
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (h->prof) { e0 = next_event(h); e1 = next_event(h); cudaEventRecord(e0, h->st); }
  const size_t ss = (size_t)db.s * db.s;
  double* snap = h->snap + (size_t)(b & 1) * (ss + 2);
  if (b >= 2) CK(cudaStreamWaitEvent(h->st, h->ev_lambda[(b - 2) % E], 0));
  CK(cudaMemcpyAsync(snap, db.SSt, ss * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  CK(cudaMemcpyAsync(snap + ss, db.fro2, 2 * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  CK(cudaEventRecord(h->ev_snap[b % E], h->st));
  CK(cudaStreamWaitEvent(stl, h->ev_snap[b % E], 0));
  // the lambda outputs of batch b share their copy (b % 2) with the scores of batch b-2; its
  // ||A_obs||^2 slot (b % 4) was last read by the tail of batch b-4, which ended before the
  // select of batch b-2 wrote the buffer slots of this batch (whose ingest preceded the snapshot)
  if (b >= 2) CK(cudaStreamWaitEvent(stl, h->ev_scores[(b - 2) % E], 0));
  Dev dl = db;
  dl.SSt = snap;
  dl.fro2 = snap + ss;
  cudaEvent_t tle[rid::kTlEvents] = {};
  if (h->prof) {
    for (auto& e : tle) e = next_event(h);
    cudaEventRecord(tle[rid::TL_SNAP], h->st);
    cudaEventRecord(tle[rid::TL_LAMBDA0], stl);
  }
  const int nl = rid::launch_batch_lambda(dl, b, stl);
  if (h->prof) cudaEventRecord(tle[rid::TL_LAMBDA1], stl);
  if (nl && h->log_cap > 0) {
    char* slot = h->log_dev + (size_t)(b % h->log_cap) * kLogSlot;
    CK(cudaMemcpyAsync(slot + 128, dl.scal + rid::SCAL_LAMBDA + (b & 1), sizeof(double), cudaMemcpyDeviceToDevice,
                       stl));
    CK(cudaMemcpyAsync(slot + 136, dl.scal + rid::SCAL_FRO0 + (b & 7), sizeof(double), cudaMemcpyDeviceToDevice,
                       stl));
  }
  CK(cudaEventRecord(h->ev_lambda[b % E], stl));
  CK(cudaStreamWaitEvent(h->sts, h->ev_lambda[b % E], 0));
  const int ns = nl ? rid::launch_batch_select(db, rv, h->count, h->n_obs, b, h->sts, h->ev_scores[b % E],
                                               b >= 2 ? h->ev_tail[(b - 2) % E] : nullptr, h->prof ? tle : nullptr)
                    : 0;
  CK(cudaEventRecord(h->ev_select[b % E], h->sts));
  CK(cudaStreamWaitEvent(h->stb, h->ev_select[b % E], 0));
  const int nt = ns ? rid::launch_batch_tail(rv, h->count, h->n_obs, h->n_prev, b, h->stb, h->stg, h->ev_fork,
                                             h->ev_gram[b % E], db.meta, db.JC_prev, db.slotC_prev,
                                             h->prof ? tle : nullptr)
                    : 0;
  if (nl == 0 || ns == 0 || nt == 0) {
    cudaGetLastError();
    return fail(h, RID_ECUDA, "batch step launch failed (cooperative or cluster launch refused)");
  }
  if (h->log_cap > 0) {
    char* slot = h->log_dev + (size_t)(b % h->log_cap) * kLogSlot;
    CK(cudaMemcpyAsync(slot, db.scal, sizeof(double) * rid::SCAL_LOG, cudaMemcpyDeviceToDevice, h->stb));
    CK(cudaMemcpyAsync(slot + 144, db.meta, sizeof(int) * rid::META_LEN, cudaMemcpyDeviceToDevice, h->stb));
  }
  CK(cudaEventRecord(h->ev_tail[b % E], h->stb));
  const int nk = nl + ns + nt;
  if (h->prof) {
    cudaEventRecord(e1, h->stb);
    h->spans[2].push_back({e0, e1});
    h->kernels[2] += nk;
    // phases of the step: lambda part, scores, select, Gram side, QR side, coefficients..commit
    const int pairs[][3] = {{rid::TLP_LAMBDA, rid::TL_LAMBDA0, rid::TL_LAMBDA1},
                            {rid::TLP_SCORES, rid::TL_TAIL0, rid::TL_SCORES},
                            {rid::TLP_SELECT, rid::TL_SCORES, rid::TL_SELECT},
                            {rid::TLP_GRAM, rid::TL_GRAM0, rid::TL_GRAM1},
                            {rid::TLP_QR, rid::TL_QR0, rid::TL_QR1},
                            {rid::TLP_COEFF, rid::TL_QR1, rid::TL_TAIL1}};
    for (const auto& pr : pairs) h->tl.push_back({b, pr[0], tle[pr[1]], tle[pr[2]]});
  }
  h->n_prev = h->n_obs;
  h->batch += 1;
  h->count = 0;
  CK(cudaGetLastError());
  return RID_OK;
}

int check_device_error(rid_handle* h) {
  join(h);
  int e = 0;
  CK(cudaMemcpyAsync(&e, h->d.err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (e & rid::ERR_TIMEOUT) return fail(h, RID_ETIMEOUT, "a bounded device wait gave up");
  if (e & rid::ERR_NONFINITE) return fail(h, RID_ENONFINITE, "a non-finite snapshot was ingested");
  return RID_OK;
}

// Sketch the pending columns (one read of each), append them, and run the batch step
// when the t-th buffered column has arrived.
int flush(rid_handle* h) {
  NvtxRange nvtx("rid_sketch_group");
  const int G = (int)h->pend.size();
  if (G == 0) return RID_OK;
  int rc = grow(h, h->n_obs + G);
  if (rc != RID_OK) return rc;
  // Host columns of this group were copied into staging area stage_area on the copy stream; the
  // copies of the next group (into the other area) may start once the caller's stream has passed
  // the ingest of the previous group, the last reader of that area: ev_cfork marks that point,
  // before the waits below, so that the copies overlap this group's ingest.
  if (h->pend_host > 0) CK(cudaEventRecord(h->ev_cfull, h->stc));
  CK(cudaEventRecord(h->ev_cfork, h->st));
  h->cfork_valid = true;
  // The batch's buffer slots were chosen by the select of step batch - la among the slots holding
  // neither its previous nor its new basis nor the columns of the batches in between; they may
  // still hold basis columns of step batch - la - 1, which the Gram side of that step's tail
  // reads (it may still run).
  {
    const int la = h->d.la;
    if (h->count == 0 && h->batch >= la) {
      CK(cudaStreamWaitEvent(h->st, h->ev_select[(h->batch - la) % rid_handle::kEv], 0));
      if (h->batch >= la + 1) CK(cudaStreamWaitEvent(h->st, h->ev_gram[(h->batch - la - 1) % rid_handle::kEv], 0));
    }
  }
  if (h->pend_host > 0) {
    CK(cudaStreamWaitEvent(h->st, h->ev_cfull, 0));
    h->pend_host = 0;
    h->stage_area ^= 1;
  }
  const Dev db = dev_for(h, h->batch);
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  if (h->prof) for (auto& e : ev) e = next_event(h);
  int nk0 = 0, nk1 = 0;
  // With an SM partition every group after the first batch's runs on the ingest stream, in the
  // SMs the batch steps do not use; the caller's stream hands over to it and waits for it.
  cudaStream_t sg = h->st;
  if (h->sti && h->batch >= 1) {
    CK(cudaEventRecord(h->ev_ing0, h->st));
    CK(cudaStreamWaitEvent(h->sti, h->ev_ing0, 0));
    sg = h->sti;
  }
  if (h->tc) {
    const int split = (h->cfg.sketch_prec == RID_SKETCH_BF16X2 || h->cfg.sketch_prec == RID_SKETCH_FP8X2) ? 1 : 0;
    const int fp8 = (h->cfg.sketch_prec == RID_SKETCH_FP8 || h->cfg.sketch_prec == RID_SKETCH_FP8X2) ? 1 : 0;
    // no batch step can run beside the first batch's ingest: it takes the whole grid
    const int nblk = h->batch >= 1 ? h->ingest_blocks : h->first_blocks;
    if (rid::launch_tc_ingest(db, h->pend.data(), G, split, h->count, h->n_obs, nblk,
                              h->tc_part, h->tc_npart, sg, h->prof ? ev : nullptr, fp8) != 0)
      return fail(h, RID_ECUDA, "tensor-core ingest launch failed");
    if (db.allreduce && rid::shard_exchange_sketch(db, G, h->n_obs, sg) != 0)
      return fail(h, RID_ECUDA, "row-shard exchange (allreduce) of the sketch failed");
    rid::launch_gram_update(db, G, h->n_obs, sg);
    nk0 = 1;
    nk1 += 2;
  } else {
    for (int q0 = 0; q0 < G; q0 += rid::kMaxB) {
      const int nb = G - q0 < rid::kMaxB ? G - q0 : rid::kMaxB;
      cudaEvent_t* e = (h->prof && q0 == 0) ? ev : nullptr;
      nk1 += rid::launch_ingest(db, h->pend.data() + q0, nb, h->count + q0, h->n_obs + q0, sg, e) - 1;
      if (db.allreduce && rid::shard_exchange_sketch(db, nb, h->n_obs + q0, sg) != 0)
        return fail(h, RID_ECUDA, "row-shard exchange (allreduce) of the sketch failed");
      if (db.grad) nk1 += rid::launch_grad(db, h->pend.data() + q0, nb, h->n_obs + q0, sg);
      rid::launch_gram_update(db, nb, h->n_obs + q0, sg);
      nk0 += 1;
      nk1 += 1;
    }
  }
  // the optional right sketch over the same columns (not part of the paper's method)
  if (db.right_l > 0) {
    const int nr = rid::launch_right_sketch(db, h->pend.data(), G, h->n_obs, sg);
    if (nr < 0) return fail(h, RID_ECUDA, "right-sketch launch failed");
    nk1 += nr;
  }
  if (h->prof) cudaEventRecord(ev[2], sg);
  if (sg != h->st) {
    CK(cudaEventRecord(h->ev_ing1, sg));
    CK(cudaStreamWaitEvent(h->st, h->ev_ing1, 0));
  }
  if (h->prof) {
    h->spans[0].push_back({ev[0], ev[1]});
    h->spans[1].push_back({ev[1], ev[2]});
    h->tl.push_back({h->batch, rid::TLP_INGEST, ev[0], ev[2]});
    h->kernels[0] += nk0;
    h->kernels[1] += nk1;
  }
  CK(cudaGetLastError());
  h->count += G;
  h->n_obs += G;
  h->pend.clear();
  if (h->count == h->d.t) return run_batch(h);
  return RID_OK;
}

// Host-side checks of a configuration, before any device call (the message goes to the calling
// thread's error text).
int check_config(const rid_config* c) {
  rid_handle* h = nullptr;
  if (c->m < 1) return fail(h, RID_EINVAL, "m must be >= 1");
  if (c->k < 1 || c->k > 1024) return fail(h, RID_EINVAL, "k must be in [1, 1024]");
  if (c->s <= c->k || c->s > 4096) return fail(h, RID_EINVAL, "s must satisfy k < s <= 4096");
  if (c->h < 0 || c->h > 1024 || (c->h > 0 && c->h < 3)) return fail(h, RID_EINVAL, "h must be 0 or in [3, 1024]");
  if (!(c->c1 > 0.0) || !(c->c2 > c->c1) || !(c->c1 + c->c2 < 1.0))
    return fail(h, RID_EINVAL, "need 0 < c1 < c2 and c1 + c2 < 1");
  if (!(c->eps > 0.0) || !(c->delta > 0.0 && c->delta < 1.0) || !(c->c_const > 0.0))
    return fail(h, RID_EINVAL, "need eps > 0, 0 < delta < 1, c_const > 0");
  if (c->lambda_mode != RID_LAMBDA_STREAMING && c->lambda_mode != RID_LAMBDA_FIXED)
    return fail(h, RID_EINVAL, "unknown lambda_mode");
  if (c->lambda_mode == RID_LAMBDA_FIXED && !(c->lambda_fixed >= 0.0))
    return fail(h, RID_EINVAL, "lambda_fixed must be >= 0");
  if (c->omega_kind != RID_OMEGA_GAUSSIAN && c->omega_kind != RID_OMEGA_RADEMACHER)
    return fail(h, RID_EINVAL, "unknown omega_kind");
  if (c->data_dtype != RID_F64 && c->data_dtype != RID_F32) return fail(h, RID_EINVAL, "unknown data_dtype");
  if (c->sketch_prec != RID_SKETCH_NATIVE && c->sketch_prec != RID_SKETCH_BF16 &&
      c->sketch_prec != RID_SKETCH_BF16X2 && c->sketch_prec != RID_SKETCH_FP8 && c->sketch_prec != RID_SKETCH_FP8X2)
    return fail(h, RID_EINVAL, "unknown sketch_prec");
  if ((c->sketch_prec == RID_SKETCH_FP8 || c->sketch_prec == RID_SKETCH_FP8X2) && c->s + c->h > 480)
    return fail(h, RID_EINVAL, "FP8 sketches support s + h <= 480 (TMEM holds the block scales beside the sums)");
  if (c->sketch_prec != RID_SKETCH_NATIVE) {
    if (c->data_dtype != RID_F32) return fail(h, RID_EINVAL, "tensor-core sketches need FP32 data");
    if (c->omega_kind != RID_OMEGA_RADEMACHER) return fail(h, RID_EINVAL, "tensor-core sketches need a Rademacher Omega");
    if (c->s + c->h > 4096) return fail(h, RID_EINVAL, "tensor-core sketches support s + h <= 4096");
  }
  if (c->group_max < 0 || c->group_max > rid::kMaxGroup) return fail(h, RID_EINVAL, "group_max must be in [0, 64]");
  if (c->right_l < 0 || c->right_l > 4096) return fail(h, RID_EINVAL, "right_l must be in [0, 4096]");
  if (c->ingest_ctas < 0) return fail(h, RID_EINVAL, "ingest_ctas must be >= 0");
  if (c->batch_sms < 0) return fail(h, RID_EINVAL, "batch_sms must be >= 0");
  if (c->refill_mode != RID_REFILL_FIRST && c->refill_mode != RID_REFILL_PROPORTIONAL)
    return fail(h, RID_EINVAL, "unknown refill_mode");
  if (c->lookahead != 0 && (c->lookahead < 2 || c->lookahead > 4))
    return fail(h, RID_EINVAL, "lookahead must be 0 (default 3) or in [2, 4]");
  if (c->allreduce) {
    if (c->row_offset < 0 || c->row_offset % 128 != 0)
      return fail(h, RID_EINVAL, "row sharding needs row_offset >= 0, a multiple of 128");
    if (c->m_global < c->row_offset + c->m) return fail(h, RID_EINVAL, "row sharding needs m_global >= row_offset + m");
    if (c->grad_dims != 0 || c->grad_coeff != 0) return fail(h, RID_EINVAL, "row sharding does not support gradient mode");
  } else if (c->row_offset != 0) {
    return fail(h, RID_EINVAL, "row_offset needs an allreduce (row sharding)");
  }
  if (c->grad_coeff != 0 && c->grad_dims != 2)
    return fail(h, RID_EINVAL, "grad_coeff needs gradient mode (grad_dims = 2)");
  if (c->grad_dims != 0) {
    if (c->grad_dims != 2) return fail(h, RID_EINVAL, "grad_dims must be 0 or 2 (2-D grids)");
    if (c->nx < 2 || c->ny < 2 || c->nfields < 1)
      return fail(h, RID_EINVAL, "gradient mode needs nx >= 2, ny >= 2, nfields >= 1");
    if ((int64_t)c->nx * c->ny * c->nfields != c->m) return fail(h, RID_EINVAL, "gradient mode needs m = nx ny nfields");
    if (c->sketch_prec == RID_SKETCH_FP8 || c->sketch_prec == RID_SKETCH_FP8X2)
      return fail(h, RID_EINVAL, "gradient mode runs the native or the BF16 sketches");
    if (c->grad_coeff != 0 && c->sketch_prec != RID_SKETCH_NATIVE)
      return fail(h, RID_EINVAL, "grad_coeff needs the native-precision sketch (sketch_prec NATIVE)");
  }
  {
    const int nprobe = c->h > 0 ? c->h : c->s;
    if (nprobe - (int)floor(c->c1 * nprobe) - (int)floor(c->c2 * nprobe) < 1)
      return fail(h, RID_EINVAL, "empty Omega_3 split");
  }
  return RID_OK;
}

}  // namespace

extern "C" {

int rid_config_default(rid_config* cfg) {
  if (!cfg) return RID_EINVAL;
  memset(cfg, 0, sizeof(*cfg));
  cfg->c1 = 1.0 / 6.0;
  cfg->c2 = 1.0 / 3.0;
  cfg->eps = 0.5;
  cfg->delta = 0.05;
  cfg->c_const = 1.0;
  cfg->lambda_mode = RID_LAMBDA_STREAMING;
  cfg->omega_kind = RID_OMEGA_RADEMACHER;
  cfg->data_dtype = RID_F32;
  cfg->sketch_prec = RID_SKETCH_NATIVE;
  cfg->n_max = 1024;
  return RID_OK;
}

int rid_config_check(const rid_config* cfg) {
  if (!cfg) return fail(nullptr, RID_EINVAL, "NULL argument");
  return check_config(cfg);
}

int rid_init(rid_handle** out, const rid_config* c) {
  rid_handle* h = nullptr;
  if (!out || !c) return fail(h, RID_EINVAL, "NULL argument");
  *out = nullptr;
  cudaGetLastError();                          // an error left by other code is not this handle's
  {
    const int vrc = check_config(c);
    if (vrc != RID_OK) return vrc;
  }
  arm_fault_injection();
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(h, RID_ENOLIB, "no CUDA device");
  }
  h = new (std::nothrow) rid_handle();
  if (!h) return fail(nullptr, RID_ENOMEM, "host allocation failed");
  h->cfg = *c;
  h->st = (cudaStream_t)c->cuda_stream;
  h->esize = c->data_dtype == RID_F64 ? 8 : 4;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, dev);
  Dev& d = h->d;
  memset(&d, 0, sizeof(d));
  d.m = c->m;
  d.m_pad = (c->m + 63) / 64 * 64;
  d.t = c->k;
  d.s = c->s;
  d.h = c->h;
  d.rows = c->s + c->h;
  const int nprobe = c->h > 0 ? c->h : c->s;
  d.hbase = c->h > 0 ? c->s : 0;
  d.h1 = (int)floor(c->c1 * nprobe);
  d.h2 = (int)floor(c->c2 * nprobe);
  d.h3 = nprobe - d.h1 - d.h2;
  if (d.h3 < 1) { delete h; return fail(nullptr, RID_EINVAL, "empty Omega_3 split"); }
  d.dtype = c->data_dtype == RID_F64 ? 0 : 1;
  d.omega_kind = c->omega_kind == RID_OMEGA_RADEMACHER ? 1 : 0;
  d.lambda_mode = c->lambda_mode == RID_LAMBDA_FIXED ? 1 : 0;
  d.lambda_fixed = c->lambda_fixed;
  const double k = (double)c->k;
  d.refill_scale = c->c_const * (k * log(k) + k * log(1.0 / c->delta) / c->eps) / (double)c->k;
  d.refill_mode = c->refill_mode;
  d.row_offset = c->allreduce ? c->row_offset : 0;
  d.allreduce = (void*)c->allreduce;
  d.allreduce_user = c->allreduce_user;
  {
    const uint32_t wl = rid::parse_wait_inject(getenv("RID_FAULT_INJECT"));
    d.ring_wait_limit = wl ? wl : rid::kRingWaitLimit;
  }
  d.la = c->lookahead > 0 ? c->lookahead : 3;
  d.seed = c->seed;
  d.grad = c->grad_dims != 0 ? 1 : 0;
  d.nx = c->nx;
  d.ny = c->ny;
  d.nfields = c->nfields;
  d.lev_ld = d.grad ? d.s : d.rows;     // gradient mode: a separate s x n leverage sketch
  d.right_l = c->right_l;
  d.grad_coeff = c->grad_coeff != 0 ? 1 : 0;
  const int64_t nchunks = (d.m + rid::kChunk - 1) / rid::kChunk;
  d.n_sketch_blocks = (int)(nchunks < 4 * h->n_sm ? nchunks : 4 * h->n_sm);
  if (c->ingest_ctas > 0 && c->ingest_ctas < d.n_sketch_blocks) d.n_sketch_blocks = c->ingest_ctas;
  int64_t gs = (d.m + 16383) / 16384;
  d.gram_split = (int)(gs < 1 ? 1 : (gs > 256 ? 256 : gs));
  const int t = d.t;
  h->tc = c->sketch_prec != RID_SKETCH_NATIVE;
  // Accuracy of the sketch entries and of the basis Gram (about ten times their relative
  // rounding): no rank tolerance of the coefficient solves or of the Hutch++ pseudo-inverse
  // goes below them, so that directions the rounding decides are dropped, not amplified.
  if (d.dtype == 0) {                       // FP64 sums
    d.sk_rel = 0.0;
    d.gram_rho0 = 1e-11;
  } else if (!h->tc) {                      // FP32 products summed in FP32 over short runs
    d.sk_rel = 1e-6;
    d.gram_rho0 = 1e-6;
  } else {                                  // tensor cores; the Gram always takes the BF16x2 split
    // relative accuracy of a sketch entry: BF16x2 ~2^-16, BF16 and E4M3x2 ~2^-8, E4M3 ~2^-4
    d.sk_rel = c->sketch_prec == RID_SKETCH_BF16X2 ? 2e-5
             : c->sketch_prec == RID_SKETCH_FP8 ? 6e-2 : 4e-3;
    d.gram_rho0 = 3e-5;
  }
  h->group_max = c->group_max > 0 ? c->group_max : (h->tc ? rid::kMaxGroup : rid::kMaxB);
  {
    const int64_t tc_chunks = (d.m + 63) / 64;
    const int64_t want_blocks = (tc_chunks + 1) / 2;
    // leave 16 SMs to the lambda part's 16-CTA cluster, which runs beside the ingest
    const int avail = h->n_sm >= 64 ? h->n_sm - 16 : h->n_sm;
    h->tc_blocks = (int)(want_blocks < avail ? want_blocks : avail);
    if (h->tc_blocks < 1) h->tc_blocks = 1;
    // The ingest is off the critical path (it runs a batch ahead of the batch step), and each of
    // its CTAs holds a whole SM for its chunk range: it leaves a third of the SMs to the batch
    // step's kernels, which run beside it.
    const int ingest_avail = h->n_sm >= 96 ? h->n_sm - h->n_sm / 3 : avail;
    h->ingest_blocks = (int)(want_blocks < ingest_avail ? want_blocks : ingest_avail);
    if (h->ingest_blocks < 1) h->ingest_blocks = 1;
    // nothing runs beside the first batch's ingest: it takes every SM
    h->first_blocks = (int)(want_blocks < h->n_sm ? want_blocks : h->n_sm);
    if (h->first_blocks < 1) h->first_blocks = 1;
    // a chosen count (rid_autotune) stays within the partial buffers sized below
    if (c->ingest_ctas > 0) h->ingest_blocks = c->ingest_ctas < h->first_blocks ? c->ingest_ctas : h->first_blocks;
  }
  int rc = RID_OK;
#define AL(ptr, n) do { if (dalloc(&(ptr), (size_t)(n)) != cudaSuccess) { rc = RID_ENOMEM; goto fail_alloc; } } while (0)
  if (h->tc) {
    const int nrows16 = (d.rows + 15) / 16 * 16;
    // ingest partials (one pass: at most 512 rows) or Gram partials (256 rows)
    const int prow = nrows16 > 256 ? (nrows16 > 512 ? 512 : nrows16) : 256;
    const int pblk = h->first_blocks > h->tc_blocks ? h->first_blocks : h->tc_blocks;
    AL(h->tc_part, (size_t)pblk * prow * 128);
    AL(h->tg_part, (size_t)h->tc_blocks * 512 * 128);     // basis-Gram partials: 512 rows per CTA
    AL(h->tc_npart, (size_t)pblk * 128);
    d.tc_blocks = h->tc_blocks;
    d.tc_part = h->tc_part;
    d.tg_part = h->tg_part;
    if (d.grad) {
      // gradient mode on tensor cores: the group's 2m-long gradient fields and their sketches
      d.gfield_ld = (2 * d.m + 63) / 64 * 64;
      const int gmax = h->group_max;
      AL(d.gfield, (size_t)gmax * d.gfield_ld);
      AL(d.glev, (size_t)gmax * d.s);
      AL(d.gnorm2, (size_t)gmax);
    }
  }
  {
    char* pool = nullptr;
    // (la + 2) t slots: the previous and the new basis of the latest step (at most 2t together
    // with its batch), and the la batches after it, ingested while steps are in flight (t each)
    d.npool = (d.la + 2) * t;
    AL(pool, (size_t)d.npool * d.m_pad * h->esize);
    d.pool = pool;
    if (cudaMemset(d.pool, 0, (size_t)d.npool * d.m_pad * h->esize) != cudaSuccess) { rc = RID_ECUDA; goto fail_alloc; }
  }
  if (d.omega_kind == 0) AL(d.omegaT, (size_t)d.m_pad * d.rows);
  AL(d.SSt, (size_t)d.s * d.s);
  AL(h->snap, (size_t)2 * ((size_t)d.s * d.s + 2));
  AL(d.fro2, 2);
  AL(d.JC, t); AL(d.JC_prev, t); AL(d.JD, t);
  AL(d.slotC, t); AL(d.slotC_prev, t); AL(d.dslot_all, (size_t)d.la * t);
  AL(d.tau_old, t); AL(d.tauC, t); AL(d.tauD, t);
  AL(d.meta, rid::META_LEN); AL(d.scal, rid::SCAL_LEN);
  AL(d.act, t); AL(d.pact, t); AL(d.isnew, t); AL(d.posof, t); AL(d.newpos, t);
  AL(d.gnew, t); AL(d.gtgt, 2 * t);
  if (d.allreduce) {
    AL(d.gnorm, rid::kMaxGroup);
    AL(d.xbuf, 2 * (size_t)t * t);
  }
  AL(h->rec_i64, 4 * (size_t)t);
  AL(h->rec_i32, 2 * (10 * (size_t)t + rid::META_LEN));
  AL(d.Gp, (size_t)d.npool * d.npool);
  AL(d.gpart, (size_t)d.gram_split * t * 2 * t);
  AL(d.spart, (size_t)d.n_sketch_blocks * rid::kMaxB * d.rows);
  AL(d.npart, (size_t)d.n_sketch_blocks * rid::kMaxB);
  AL(d.err, 1);
  AL(d.gbar, 12);                      // [0, 4) lambda part of even batches, [4, 8) QRs, [8, 12) odd batches
  if (d.grad_coeff) AL(d.Kg, (size_t)2 * d.s * d.s);
  if (d.right_l > 0) {
    char* y = nullptr;
    char* wr = nullptr;
    AL(y, (size_t)d.m_pad * d.right_l * h->esize);
    d.Y = y;
    AL(wr, rid::right_w_bytes(d));
    d.Wr = wr;
    // tensor-core handles with FP32 data and a +-1 test matrix take the right sketch on tcgen05
    // (BF16x2: ~2^-16 of each value, the accuracy of the FP32 sums), the others the FP32/FP64 pipe
    d.tc_right = (h->tc && d.dtype == 1 && d.omega_kind == 1) ? 1 : 0;
    if (cudaMemset(d.Y, 0, (size_t)d.m_pad * d.right_l * h->esize) != cudaSuccess) { rc = RID_ECUDA; goto fail_alloc; }
  }
  d.gbar2 = d.gbar + 4;
  d.n_sm = h->n_sm;
  d.work_len = rid::work_doubles(d);
  AL(d.work, d.work_len);
  {
    char* stg = nullptr;
    AL(stg, 2 * (size_t)h->group_max * d.m_pad * h->esize);
    h->staging = stg;
  }
#undef AL
  {
    int64_t want = c->n_max > 0 ? c->n_max : 1024;
    rc = grow(h, want);
    if (rc != RID_OK) goto fail_alloc;
  }
  h->dslot_buf = d.dslot_all;
  d.dslot = d.dslot_all;
  rc = create_sync_objects(h);
  if (rc != RID_OK) goto fail_alloc;
  if (h->sti) {
    // one ingest CTA per SM of its partition (fewer if ingest_ctas asks), the basis Gram on the
    // batch partition's SMs; the partial buffers were sized for the larger whole-device counts
    h->ingest_blocks = c->ingest_ctas > 0 && c->ingest_ctas < h->part_i ? c->ingest_ctas : h->part_i;
    if (h->ingest_blocks > h->first_blocks) h->ingest_blocks = h->first_blocks;
    if (h->tc_blocks > h->part_b) h->tc_blocks = h->part_b;
    d.tc_blocks = h->tc_blocks;
  }
  if (d.omega_kind == 0) rid::launch_materialize_omega(d, h->st);
  rid::launch_reset_state(d, h->st);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(h->st) != cudaSuccess) {
    rc = RID_ECUDA;
    goto fail_alloc;
  }
  *out = h;
  return RID_OK;
fail_alloc:
  {
    std::string msg = rc == RID_ENOMEM ? "device allocation failed" : (h->err.empty() ? "CUDA error during init" : h->err);
    free_all(h->d, h->staging);
    if (h->tc_part) cudaFree(h->tc_part);
    if (h->tg_part) cudaFree(h->tg_part);
    if (h->tc_npart) cudaFree(h->tc_npart);
    if (h->snap) cudaFree(h->snap);
    if (h->rec_i64) cudaFree(h->rec_i64);
    if (h->rec_i32) cudaFree(h->rec_i32);
    destroy_sync_objects(h);
    delete h;
    return fail(nullptr, rc, msg);
  }
}

int rid_ingest(rid_handle* h, const void* cols, int64_t ld, int32_t ncols, int32_t on_device) {
  NvtxRange nvtx("rid_ingest");
  if (!h) return RID_EINVAL;
  if (h->finalized) return fail(h, RID_ESTATE, "rid_ingest after rid_finalize (call rid_reset first)");
  if (ncols < 0) return fail(h, RID_EINVAL, "ncols < 0");
  if (ncols == 0) return RID_OK;
  if (!cols) return fail(h, RID_EINVAL, "cols is NULL");
  if (ld < h->d.m) return fail(h, RID_EINVAL, "ld < m");
  if (h->rcss) {
    // the attached selector decides these columns first, on the handle's stream, so that its list
    // holds them before the batch step that reads it is queued
    const int rc = rid_rcss_ingest(h->rcss, cols, ld, ncols, on_device);
    if (rc != RID_OK) return fail(h, rc, std::string("selector: ") + rid_last_error(nullptr));
  }
  const size_t cbytes = (size_t)h->d.m * h->esize;
  for (int32_t q = 0; q < ncols; ++q) {
    const char* src = (const char*)cols + (size_t)q * ld * h->esize;
    if (!on_device) {
      // Host columns go through a staging area on the copy stream: the group's columns into area
      // stage_area, while the caller's stream ingests the previous group from the other area.
      // (The pool slot a column lands in is chosen on the device, so the copy cannot go there
      // directly.)  The first copy of a group waits until the ingest that last read the area has
      // been passed (ev_cfork, recorded by the previous flush, or here when none was).
      if (h->pend_host == 0) {
        if (!h->cfork_valid) {
          CK(cudaEventRecord(h->ev_cfork, h->st));
          h->cfork_valid = true;
        }
        CK(cudaStreamWaitEvent(h->stc, h->ev_cfork, 0));
      }
      char* dst = (char*)h->staging + ((size_t)h->stage_area * h->group_max + h->pend.size()) *
                                           (size_t)h->d.m_pad * h->esize;
      CK(cudaMemcpyAsync(dst, src, cbytes, cudaMemcpyHostToDevice, h->stc));
      h->pend_host += 1;
      src = dst;
    }
    h->pend.push_back(src);
    const bool full = (int)h->pend.size() == h->group_max;
    const bool batch_end = h->count + (int)h->pend.size() == h->d.t;
    if (full || batch_end) {
      const int rc = flush(h);
      if (rc != RID_OK) return rc;
    }
  }
  // device columns are read before the call returns unless the caller opted into deferral
  if (on_device && !h->cfg.defer_device_input) return flush(h);
  return RID_OK;
}

int rid_batch_ingest(rid_handle* const* hs, int32_t nh, const void* const* cols, const int64_t* ld,
                     const int32_t* ncols, int32_t on_device) {
  if (nh < 0 || (nh > 0 && (!hs || !cols || !ld || !ncols))) return fail(nullptr, RID_EINVAL, "rid_batch_ingest: NULL array or nh < 0");
  for (int32_t i = 0; i < nh; ++i)
    if (!hs[i]) return fail(nullptr, RID_EINVAL, "rid_batch_ingest: NULL handle");
  for (int32_t i = 0; i < nh; ++i) {
    const int rc = rid_ingest(hs[i], cols[i], ld[i], ncols[i], on_device);
    if (rc != RID_OK) return rc;
  }
  return RID_OK;
}

int rid_finalize(rid_handle* h, int64_t* J_out, double* P_out, int64_t ldp, int32_t on_device) {
  NvtxRange nvtx("rid_finalize");
  if (!h) return RID_EINVAL;
  const int t = h->d.t;
  if (P_out && ldp < t) return fail(h, RID_EINVAL, "ldp < t");
  if (!h->finalized) {
    int rc = flush(h);
    if (rc != RID_OK) return rc;
    if (h->count > 0) {
      rc = run_batch(h);
      if (rc != RID_OK) return rc;
    }
  }
  h->finalized = true;
  const bool async = on_device == RID_OUT_DEVICE_ASYNC;
  if (async) {
    join(h);                                     // the batch streams rejoin the caller's stream
  } else {
    const int rc = check_device_error(h);
    if (rc != RID_OK) return rc;
  }
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (J_out) CK(cudaMemcpyAsync(J_out, h->d.JC, sizeof(int64_t) * t, kind, h->st));
  if (P_out && h->n_obs > 0)
    CK(cudaMemcpy2DAsync(P_out, sizeof(double) * ldp, h->d.P, sizeof(double) * t, sizeof(double) * t,
                         (size_t)h->n_obs, kind, h->st));
  if (!async) CK(cudaStreamSynchronize(h->st));
  return RID_OK;
}

int rid_error_estimate(rid_handle* h, double est_sq[5], double est_fro[5], int32_t* q_star) {
  if (!h) return RID_EINVAL;
  {
    const int rc = flush(h);
    if (rc != RID_OK) return rc;
  }
  if (h->batch == 0) return fail(h, RID_ESTATE, "no batch step has run yet");
  join(h);
  double e[4];
  int meta[rid::META_LEN];
  CK(cudaMemcpyAsync(e, h->d.scal + rid::SCAL_EST, sizeof(e), cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(meta, h->d.meta, sizeof(meta), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  const int q = meta[rid::META_QSTAR];
  double out[5] = {e[q - 4], e[0], e[1], e[2], e[3]};
  for (int i = 0; i < 5; ++i) {
    if (est_sq) est_sq[i] = out[i];
    if (est_fro) est_fro[i] = sqrt(out[i] > 0.0 ? out[i] : 0.0);
  }
  if (q_star) *q_star = q;
  return RID_OK;
}

int64_t rid_n_obs(const rid_handle* h) { return h ? h->n_obs + (int64_t)h->pend.size() : -1; }

int rid_get_basis(rid_handle* h, void* out, int64_t ld, int32_t on_device) {
  if (!h || !out) return RID_EINVAL;
  if (ld < h->d.m) return fail(h, RID_EINVAL, "ld < m");
  {
    const int rc = flush(h);
    if (rc != RID_OK) return rc;
  }
  join(h);
  const int t = h->d.t;
  std::vector<int> slot(t);
  std::vector<int64_t> jc(t);
  CK(cudaMemcpyAsync(slot.data(), h->d.slotC, sizeof(int) * t, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int i = 0; i < t; ++i) {
    char* dst = (char*)out + (size_t)i * ld * h->esize;
    if (slot[i] >= 0) {
      CK(cudaMemcpyAsync(dst, (const char*)h->d.pool + (size_t)slot[i] * h->d.m_pad * h->esize,
                         (size_t)h->d.m * h->esize, kind, h->st));
    } else if (on_device) {
      CK(cudaMemsetAsync(dst, 0, (size_t)h->d.m * h->esize, h->st));
    } else {
      CK(cudaStreamSynchronize(h->st));
      memset(dst, 0, (size_t)h->d.m * h->esize);
    }
  }
  CK(cudaStreamSynchronize(h->st));
  return RID_OK;
}

int rid_get_right_sketch(rid_handle* h, void* out, int64_t ld, int32_t on_device) {
  if (!h || !out) return RID_EINVAL;
  if (h->d.right_l <= 0) return fail(h, RID_ESTATE, "no right sketch (right_l = 0)");
  if (ld < h->d.m) return fail(h, RID_EINVAL, "ld < m");
  {
    const int rc = flush(h);
    if (rc != RID_OK) return rc;
  }
  join(h);
  const size_t es = h->esize;
  CK(cudaMemcpy2DAsync(out, es * (size_t)ld, h->d.Y, es * (size_t)h->d.m_pad, es * (size_t)h->d.m,
                       (size_t)h->d.right_l, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return RID_OK;
}

int rid_gradient_coefficients(rid_handle* h, double* P_out, int64_t ldp, int32_t on_device, double* lambda_out,
                              double* gcv_out) {
  if (!h || !P_out) return RID_EINVAL;
  if (!h->d.grad_coeff) return fail(h, RID_ESTATE, "gradient sketches were not kept (grad_coeff = 0)");
  if (ldp < h->d.t) return fail(h, RID_EINVAL, "ldp < t");
  if (!h->finalized) {
    const int rc = rid_finalize(h, nullptr, nullptr, h->d.t, RID_OUT_DEVICE);
    if (rc != RID_OK) return rc;
  }
  join(h);
  const int t = h->d.t;
  std::vector<int64_t> jc(t);
  CK(cudaMemcpyAsync(jc.data(), h->d.JC, sizeof(int64_t) * t, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  std::vector<int64_t> jact;
  std::vector<int> slot;
  for (int i = 0; i < t; ++i)
    if (jc[i] >= 0) { jact.push_back(jc[i]); slot.push_back(i); }
  if (jact.empty()) return fail(h, RID_ESTATE, "empty basis");
  if (rid::gradient_coefficients(h->d, h->st, h->n_obs, jact.data(), slot.data(), (int)jact.size(), -3.0, 3.0, 1e-3,
                                 P_out, ldp, on_device, &h->kg_ready, lambda_out, gcv_out) != 0)
    return fail(h, RID_ECUDA, "gradient-coefficient computation failed");
  return RID_OK;
}

int rid_get_state(rid_handle* h, int32_t item, void* out, int64_t count) {
  if (!h || !out) return RID_EINVAL;
  {
    const int rc = flush(h);
    if (rc != RID_OK) return rc;
  }
  join(h);
  const Dev& d = h->d;
  const int64_t n = h->n_obs;
  const void* src = nullptr;
  size_t bytes = 0;
  std::vector<double> tmp;
  switch (item) {
    case RID_STATE_SKETCH: src = d.S; bytes = sizeof(double) * d.rows * n; break;
    case RID_STATE_SKETCH_LEV:
      if (d.lev_ld == d.s) { src = d.Slev; bytes = sizeof(double) * d.s * n; }
      else {
        if (count < (int64_t)d.s * n) return fail(h, RID_EINVAL, "buffer too small");
        CK(cudaMemcpy2DAsync(out, sizeof(double) * d.s, d.Slev, sizeof(double) * d.lev_ld,
                             sizeof(double) * d.s, (size_t)n, cudaMemcpyDeviceToHost, h->st));
        CK(cudaStreamSynchronize(h->st));
        return RID_OK;
      }
      break;
    case RID_STATE_SST: src = d.SSt; bytes = sizeof(double) * d.s * d.s; break;
    case RID_STATE_FRO2: src = d.fro2; bytes = sizeof(double) * 2; break;
    case RID_STATE_JC: src = d.JC; bytes = sizeof(int64_t) * d.t; break;
    case RID_STATE_TAU_OLD: src = d.tau_old; bytes = sizeof(double) * d.t; break;
    case RID_STATE_LAMBDA:
      if (h->batch < 1) return fail(h, RID_ESTATE, "no batch step has run yet");
      src = d.scal + rid::SCAL_LAMBDA + ((h->batch - 1) & 1);
      bytes = sizeof(double);
      break;
    case RID_STATE_GRAM_SHIFT: src = d.scal + rid::SCAL_GSHIFT; bytes = sizeof(double); break;
    case RID_STATE_GRAD_SKETCH:
      if (!d.grad_coeff) return fail(h, RID_ESTATE, "no gradient sketches (grad_coeff = 0)");
      src = d.Sg;
      bytes = sizeof(double) * 2 * (size_t)d.s * n;
      break;
    case RID_STATE_CAND: {
      if (count < 4 * (int64_t)d.t * h->n_prev) return fail(h, RID_EINVAL, "buffer too small");
      for (int q = 0; q < 4; ++q)
        CK(cudaMemcpyAsync((double*)out + (size_t)q * d.t * h->n_prev, d.cand + (size_t)q * d.t * d.n_cap,
                           sizeof(double) * d.t * h->n_prev, cudaMemcpyDeviceToHost, h->st));
      CK(cudaStreamSynchronize(h->st));
      return RID_OK;
    }
    case RID_STATE_BATCHES: {
      if (count < 1) return fail(h, RID_EINVAL, "buffer too small");
      *(int64_t*)out = h->batch;
      return RID_OK;
    }
    default: return fail(h, RID_EINVAL, "unknown state item");
  }
  const size_t esz = (item == RID_STATE_JC) ? sizeof(int64_t) : sizeof(double);
  if ((size_t)count * esz < bytes) return fail(h, RID_EINVAL, "buffer too small");
  if (bytes) CK(cudaMemcpyAsync(out, src, bytes, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return RID_OK;
}

// ---------------------------------------------------------------- checkpoint / resume
// Layout (host bytes): header | config | counters | arrays, each array as stored on the device.
// Between batch steps the previous basis equals the current one, so the pool slots still in
// use are the basis slots and the buffer slots of the count columns buffered so far.
namespace {

constexpr uint64_t kCkptMagic = 0x31545043444952ull;   // "RIDCPT1"

struct CkptCounters {
  int64_t n_obs, n_prev;
  int32_t count, batch, finalized, nslots;
};

bool same_config(const rid_config& a, const rid_config& b) {
  return a.m == b.m && a.k == b.k && a.s == b.s && a.h == b.h && a.lambda_mode == b.lambda_mode &&
         a.c1 == b.c1 && a.c2 == b.c2 && a.eps == b.eps && a.delta == b.delta && a.c_const == b.c_const &&
         a.lambda_fixed == b.lambda_fixed && a.omega_kind == b.omega_kind && a.data_dtype == b.data_dtype &&
         a.sketch_prec == b.sketch_prec && a.grad_dims == b.grad_dims && a.nx == b.nx && a.ny == b.ny &&
         a.nfields == b.nfields && a.seed == b.seed && a.right_l == b.right_l && a.grad_coeff == b.grad_coeff &&
         a.refill_mode == b.refill_mode && a.lookahead == b.lookahead && a.row_offset == b.row_offset &&
         a.m_global == b.m_global;
}

struct CkptPlan {
  std::vector<std::pair<void*, size_t>> arrays;   // device pointer, bytes
  std::vector<int> slots;                         // pool slots saved, in order
  size_t total;
};

// The device arrays of the stream state for n observed columns, in their fixed order (device
// pointer, bytes); the list depends only on the configuration and n.
std::vector<std::pair<void*, size_t>> ckpt_arrays(rid_handle* h, int64_t n) {
  Dev& d = h->d;
  const int t = d.t;
  std::vector<std::pair<void*, size_t>> a = {
      {d.S, sizeof(double) * (size_t)d.rows * n},
      {d.SSt, sizeof(double) * (size_t)d.s * d.s},
      {d.fro2, 2 * sizeof(double)},
      {d.JC, sizeof(int64_t) * t}, {d.JC_prev, sizeof(int64_t) * t},
      {d.slotC, sizeof(int) * t}, {d.slotC_prev, sizeof(int) * t},
      {h->dslot_buf, sizeof(int) * (size_t)d.la * t},
      {d.tau_old, sizeof(double) * t},
      {d.meta, sizeof(int) * rid::META_LEN}, {d.scal, sizeof(double) * rid::SCAL_LEN},
      {d.P, sizeof(double) * (size_t)t * n},
      {d.Gp, sizeof(double) * (size_t)d.npool * d.npool},
  };
  if (d.grad) a.push_back({d.Slev, sizeof(double) * (size_t)d.s * n});
  if (d.right_l > 0) a.push_back({d.Y, (size_t)d.m_pad * d.right_l * h->esize});
  if (d.grad_coeff) a.push_back({d.Sg, sizeof(double) * 2 * (size_t)d.s * n});
  return a;
}

// The device arrays of the stream state and the pool slots in use.
int ckpt_plan(rid_handle* h, CkptPlan& pl) {
  Dev& d = h->d;
  const int t = d.t;
  pl.arrays = ckpt_arrays(h, h->n_obs);
  std::vector<int> slotc(t), dsl((size_t)d.la * t);
  CK(cudaMemcpyAsync(slotc.data(), d.slotC, sizeof(int) * t, cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(dsl.data(), h->dslot_buf, sizeof(int) * (size_t)d.la * t, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  pl.slots.clear();
  for (int i = 0; i < t; ++i) if (slotc[i] >= 0) pl.slots.push_back(slotc[i]);
  const int* cur = dsl.data() + (size_t)(h->batch % d.la) * t;
  for (int q = 0; q < h->count; ++q) pl.slots.push_back(cur[q]);
  size_t tot = sizeof(uint64_t) + sizeof(rid_config) + sizeof(CkptCounters);
  for (auto& a : pl.arrays) tot += a.second;
  tot += sizeof(int) * pl.slots.size() + pl.slots.size() * (size_t)d.m * h->esize;
  pl.total = tot;
  return RID_OK;
}

// Checks of a checkpoint's counters against the handle's configuration, before anything of the
// handle changes: between batch steps 0 <= count < t columns are buffered since the last step,
// which covered n_prev = n_obs - count columns; the saved pool slots are the occupied basis slots
// and the count buffer slots.  Returns an empty string when the counters are consistent.
const char* ckpt_counters_invalid(const CkptCounters& cn, int t, int npool) {
  if (cn.n_obs < 0 || cn.n_obs > ((int64_t)1 << 40)) return "checkpoint counter n_obs out of range";
  if (cn.count < 0 || cn.count >= t) return "checkpoint counter count out of range (0 <= count < t)";
  if (cn.n_prev < 0 || cn.n_prev > cn.n_obs || cn.n_obs - cn.n_prev != cn.count)
    return "checkpoint counters n_prev, n_obs and count disagree";
  if (cn.batch < 0 || (int64_t)cn.batch > cn.n_obs) return "checkpoint counter batch out of range";
  if (cn.finalized != 0 && cn.finalized != 1) return "checkpoint flag finalized is not 0 or 1";
  if (cn.nslots < 0 || cn.nslots > t + cn.count || cn.nslots > npool)
    return "checkpoint counter nslots out of range";
  return "";
}

}  // namespace

int rid_checkpoint_size(rid_handle* h, int64_t* bytes) {
  if (!h || !bytes) return RID_EINVAL;
  if (h->rcss) return fail(h, RID_ESTATE, "a checkpoint does not cover an attached selector");
  int rc = flush(h);
  if (rc != RID_OK) return rc;
  join(h);
  CkptPlan pl;
  rc = ckpt_plan(h, pl);
  if (rc != RID_OK) return rc;
  *bytes = (int64_t)pl.total;
  return RID_OK;
}

int rid_checkpoint(rid_handle* h, void* buf, int64_t bytes) {
  if (!h || !buf) return RID_EINVAL;
  if (h->rcss) return fail(h, RID_ESTATE, "a checkpoint does not cover an attached selector");
  int rc = flush(h);
  if (rc != RID_OK) return rc;
  rc = check_device_error(h);                   // joins the batch streams and synchronizes
  if (rc != RID_OK) return rc;
  CkptPlan pl;
  rc = ckpt_plan(h, pl);
  if (rc != RID_OK) return rc;
  if ((size_t)bytes < pl.total) return fail(h, RID_EINVAL, "checkpoint buffer too small (see rid_checkpoint_size)");
  char* p = (char*)buf;
  const uint64_t magic = kCkptMagic;
  memcpy(p, &magic, sizeof(magic)); p += sizeof(magic);
  memcpy(p, &h->cfg, sizeof(rid_config)); p += sizeof(rid_config);
  CkptCounters cn{h->n_obs, h->n_prev, h->count, h->batch, h->finalized ? 1 : 0, (int32_t)pl.slots.size()};
  memcpy(p, &cn, sizeof(cn)); p += sizeof(cn);
  for (auto& a : pl.arrays) {
    if (a.second) CK(cudaMemcpyAsync(p, a.first, a.second, cudaMemcpyDeviceToHost, h->st));
    p += a.second;
  }
  memcpy(p, pl.slots.data(), sizeof(int) * pl.slots.size()); p += sizeof(int) * pl.slots.size();
  const size_t cb = (size_t)h->d.m * h->esize;
  for (int sl : pl.slots) {
    CK(cudaMemcpyAsync(p, (const char*)h->d.pool + (size_t)sl * h->d.m_pad * h->esize, cb, cudaMemcpyDeviceToHost, h->st));
    p += cb;
  }
  CK(cudaStreamSynchronize(h->st));
  return RID_OK;
}

int rid_restore(rid_handle* h, const void* buf, int64_t bytes) {
  if (!h || !buf) return RID_EINVAL;
  if (bytes < 0) return fail(h, RID_EINVAL, "checkpoint size < 0");
  const char* p = (const char*)buf;
  const size_t head = sizeof(uint64_t) + sizeof(rid_config) + sizeof(CkptCounters);
  if ((size_t)bytes < head) return fail(h, RID_EINVAL, "checkpoint truncated");
  uint64_t magic;
  memcpy(&magic, p, sizeof(magic)); p += sizeof(magic);
  if (magic != kCkptMagic) return fail(h, RID_EINVAL, "not a checkpoint of this library");
  rid_config cf;
  memcpy(&cf, p, sizeof(cf)); p += sizeof(cf);
  if (!same_config(cf, h->cfg)) return fail(h, RID_EINVAL, "checkpoint of a different configuration");
  CkptCounters cn;
  memcpy(&cn, p, sizeof(cn)); p += sizeof(cn);
  // Everything is checked before the handle changes: a rejected checkpoint leaves the handle's
  // stream as it was.
  {
    const char* why = ckpt_counters_invalid(cn, h->d.t, h->d.npool);
    if (*why) return fail(h, RID_EINVAL, why);
  }
  const size_t cb = (size_t)h->d.m * h->esize;
  size_t need = head;
  for (auto& a : ckpt_arrays(h, cn.n_obs)) need += a.second;     // sizes only
  need += (size_t)cn.nslots * (sizeof(int) + cb);
  if ((size_t)bytes < need) return fail(h, RID_EINVAL, "checkpoint truncated");
  size_t arr_bytes = 0;
  for (auto& a : ckpt_arrays(h, cn.n_obs)) arr_bytes += a.second;
  std::vector<int> slots((size_t)cn.nslots);
  memcpy(slots.data(), p + arr_bytes, sizeof(int) * slots.size());
  for (int sl : slots)
    if (sl < 0 || sl >= h->d.npool) return fail(h, RID_EINVAL, "checkpoint holds an invalid pool slot");
  int rc = rid_reset(h);                       // joins, clears pending columns and counters
  if (rc != RID_OK) return rc;
  rc = grow(h, cn.n_obs > 0 ? cn.n_obs : 1);
  if (rc != RID_OK) return rc;
  h->n_obs = cn.n_obs;
  h->n_prev = cn.n_prev;
  h->count = cn.count;
  h->batch = cn.batch;
  h->log_first = h->batch;
  h->finalized = cn.finalized != 0;
  for (auto& a : ckpt_arrays(h, h->n_obs)) {
    if (a.second) CK(cudaMemcpyAsync(a.first, p, a.second, cudaMemcpyHostToDevice, h->st));
    p += a.second;
  }
  p += sizeof(int) * slots.size();
  for (int sl : slots) {
    CK(cudaMemcpyAsync((char*)h->d.pool + (size_t)sl * h->d.m_pad * h->esize, p, cb, cudaMemcpyHostToDevice, h->st));
    p += cb;
  }
  CK(cudaStreamSynchronize(h->st));
  return RID_OK;
}

int rid_profile(rid_handle* h, int32_t enable) {
  if (!h) return RID_EINVAL;
  join(h);
  CK(cudaStreamSynchronize(h->st));
  h->prof = enable != 0;
  h->evused = 0;
  for (auto& v : h->spans) v.clear();
  h->tl.clear();
  if (h->prof) {
    if (!h->tl_base) CK(cudaEventCreate(&h->tl_base));
    CK(cudaEventRecord(h->tl_base, h->st));
  }
  for (auto& k : h->kernels) k = 0;
  return RID_OK;
}

int rid_profile_read(rid_handle* h, double ms[3], int64_t kernels[3], int64_t groups[3]) {
  if (!h) return RID_EINVAL;
  join(h);
  CK(cudaStreamSynchronize(h->st));
  for (int p = 0; p < 3; ++p) {
    double tot = 0.0;
    for (auto& sp : h->spans[p]) {
      float e = 0.f;
      CK(cudaEventElapsedTime(&e, sp.first, sp.second));
      tot += e;
    }
    if (ms) ms[p] = tot;
    if (kernels) kernels[p] = h->kernels[p];
    if (groups) groups[p] = (int64_t)h->spans[p].size();
  }
  return RID_OK;
}

int rid_profile_timeline(rid_handle* h, double* out, int32_t max_records, int32_t* n_out) {
  if (!h) return RID_EINVAL;
  if (n_out) *n_out = 0;
  if (max_records < 0 || (max_records > 0 && !out)) return fail(h, RID_EINVAL, "bad output buffer");
  if (!h->prof || !h->tl_base) return fail(h, RID_ESTATE, "profiling is off (rid_profile)");
  join(h);
  CK(cudaStreamSynchronize(h->st));
  const int32_t n = (int32_t)h->tl.size() < max_records ? (int32_t)h->tl.size() : max_records;
  for (int32_t i = 0; i < n; ++i) {
    const auto& r = h->tl[(size_t)i];
    float a = 0.f, b = 0.f;
    CK(cudaEventElapsedTime(&a, h->tl_base, r.a));
    CK(cudaEventElapsedTime(&b, h->tl_base, r.b));
    out[4 * (size_t)i + 0] = r.batch;
    out[4 * (size_t)i + 1] = r.phase;
    out[4 * (size_t)i + 2] = a;
    out[4 * (size_t)i + 3] = b;
  }
  if (n_out) *n_out = max_records == 0 ? (int32_t)h->tl.size() : n;
  return RID_OK;
}

int rid_sync(rid_handle* h) {
  if (!h) return RID_EINVAL;
  const int rc = flush(h);
  if (rc != RID_OK) return rc;
  return check_device_error(h);
}

int rid_attach_rcss(rid_handle* h, rid_rcss* g) {
  if (!h) return RID_EINVAL;
  if (h->n_obs > 0 || !h->pend.empty()) return fail(h, RID_ESTATE, "attach the selector before the first ingest");
  if (!g) {
    h->rcss = nullptr;
    h->d.ext_sel = nullptr;
    h->d.ext_nsel = nullptr;
    return RID_OK;
  }
  const int64_t* sel = nullptr;
  const int* nsel = nullptr;
  int64_t m = 0;
  int cap = 0, stop = 0, dtype = 0;
  cudaStream_t gst = nullptr;
  rid::rcss_selection_view(g, &sel, &nsel, &m, &cap, &stop, &dtype, &gst);
  if (m != h->d.m || dtype != h->d.dtype || cap > h->d.t || !stop || gst != h->st || h->d.allreduce ||
      h->d.grad)
    return fail(h, RID_EINVAL,
                "selector: needs the handle's m, data type and stream, cap <= t with stop_at_cap, and a handle "
                "without row shards or gradient mode");
  h->rcss = g;
  h->d.ext_sel = sel;
  h->d.ext_nsel = nsel;
  return RID_OK;
}

int rid_reset(rid_handle* h) {
  if (!h) return RID_EINVAL;
  join(h);
  h->rcss = nullptr;                      // a selector serves one stream: attach a new one
  h->d.ext_sel = nullptr;
  h->d.ext_nsel = nullptr;
  const int nk = rid::launch_reset_state(h->d, h->st);
  if (h->prof) h->kernels[1] += nk;
  if (h->d.right_l > 0) CK(cudaMemsetAsync(h->d.Y, 0, (size_t)h->d.m_pad * h->d.right_l * h->esize, h->st));
  CK(cudaGetLastError());
  h->pend.clear();
  h->pend_host = 0;
  h->count = 0;
  h->n_obs = 0;
  h->n_prev = 0;
  h->batch = 0;
  h->log_first = 0;
  h->finalized = false;
  return RID_OK;
}

int rid_log_enable(rid_handle* h, int32_t capacity) {
  if (!h) return RID_EINVAL;
  if (capacity < 0 || capacity > (1 << 20)) return fail(h, RID_EINVAL, "capacity must be in [0, 1048576]");
  join(h);
  CK(cudaStreamSynchronize(h->st));
  if (h->log_dev) cudaFree(h->log_dev);
  h->log_dev = nullptr;
  h->log_cap = 0;
  h->log_first = h->batch;
  if (capacity > 0) {
    char* p = nullptr;
    CK(dalloc(&p, (size_t)capacity * kLogSlot));
    h->log_dev = p;
    CK(cudaMemsetAsync(p, 0, (size_t)capacity * kLogSlot, h->st));
    h->log_cap = capacity;
  }
  return RID_OK;
}

int rid_get_log(rid_handle* h, rid_log_record* out, int32_t max_records, int32_t* n_out) {
  if (!h) return RID_EINVAL;
  if (n_out) *n_out = 0;
  if (max_records < 0 || (max_records > 0 && !out)) return fail(h, RID_EINVAL, "bad output buffer");
  if (h->log_cap == 0) return fail(h, RID_ESTATE, "the log is off (rid_log_enable)");
  join(h);
  int64_t nrec = h->batch - h->log_first;
  if (nrec > h->log_cap) nrec = h->log_cap;
  if (nrec < 0) nrec = 0;
  if (max_records == 0) {                      // a size query
    if (n_out) *n_out = (int32_t)nrec;
    return RID_OK;
  }
  if (nrec > max_records) nrec = max_records;
  std::vector<char> buf((size_t)h->log_cap * kLogSlot);
  CK(cudaMemcpyAsync(buf.data(), h->log_dev, buf.size(), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  for (int64_t i = 0; i < nrec; ++i) {
    const int64_t b = h->batch - nrec + i;
    const char* slot = buf.data() + (size_t)(b % h->log_cap) * kLogSlot;
    double sc[rid::SCAL_LOG], lf[2];
    int mt[rid::META_LEN];
    memcpy(sc, slot, sizeof(sc));
    memcpy(lf, slot + 128, sizeof(lf));
    memcpy(mt, slot + 144, sizeof(mt));
    rid_log_record& r = out[i];
    r.batch = mt[rid::META_BATCH] - 1;
    r.n_obs = mt[rid::META_NPREV];
    r.lambda = lf[0];
    r.fro2 = lf[1];
    for (int q = 0; q < 4; ++q) {
      r.est_sq[q] = sc[rid::SCAL_EST + q];
      r.est_unc[q] = sc[rid::SCAL_UNC + q];
    }
    r.gram_shift = sc[rid::SCAL_GSHIFT];
    r.q_star = mt[rid::META_QSTAR];
    r.n_active = mt[rid::META_NACT];
    r.n_kept = mt[rid::META_NKEPT];
    r.n_new = mt[rid::META_NNEW];
  }
  if (n_out) *n_out = (int32_t)nrec;
  return RID_OK;
}

const char* rid_last_error(const rid_handle* h) {
  return h ? h->err.c_str() : g_init_err.c_str();
}

void rid_destroy(rid_handle* h) {
  if (!h) return;
  join(h);
  cudaStreamSynchronize(h->st);
  for (cudaStream_t x : {h->stb, h->stl[0], h->stl[1], h->sts, h->stg, h->stc, h->sti})
    if (x) cudaStreamSynchronize(x);
  for (auto e : h->evpool) cudaEventDestroy(e);
  if (h->tl_base) cudaEventDestroy(h->tl_base);
  free_all(h->d, h->staging);
  if (h->tc_part) cudaFree(h->tc_part);
  if (h->tg_part) cudaFree(h->tg_part);
  if (h->tc_npart) cudaFree(h->tc_npart);
  if (h->snap) cudaFree(h->snap);
  if (h->rec_i64) cudaFree(h->rec_i64);
  if (h->rec_i32) cudaFree(h->rec_i32);
  if (h->log_dev) cudaFree(h->log_dev);
  destroy_sync_objects(h);
  delete h;
}

}  // extern "C"
