// Device-state layout and kernel launchers shared by the CUDA translation units.
//
// HBM layout (all column-major):
//   pool   : 2t slots of m_pad elements (data dtype).  Basis columns C and
//            buffered columns D both live here; a selection only moves slot
//            indices, never data.
//   S      : (s+h) x n_cap doubles, S(:, j) = Omega a_j (unit-variance rows;
//            rows [0, s) are the left sketch, [s, s+h) the Hutch++ probes).
//   Slev   : sketch used by the ridge scores (= S rows [0,s) with stride s+h,
//            or an s x n_cap buffer of Omega a + Omega_g G a in gradient mode).
//   SSt    : s x s doubles, Slev Slev^T.
//   P      : t x n_cap doubles (slot rows); cand: 4 candidates t x n_cap
//            (active-slot rows).
//   Gp     : 2t x 2t doubles, Gram of pool slots (entries are valid for pairs
//            whose slots have not been overwritten since they were computed).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

struct rid_rcss;

namespace rid {

constexpr int kMaxB = 16;          // columns per ingest launch
constexpr int kSketchThreads = 256;
constexpr int kChunk = 256;        // coordinates staged per CTA iteration

struct Dev {
  // sizes
  int64_t m, m_pad;
  int t, s, h, rows;              // rows = s + h
  int hbase, h1, h2, h3;          // probe rows [hbase, hbase+h1+h2+h3) split into Omega_1/2/3
  int64_t n_cap;
  int dtype;                      // 0 f64, 1 f32
  double sk_rel;                  // relative accuracy of a sketch entry (0 for FP64 sketches)
  double gram_rho0;               // pivot threshold and Tikhonov shift of the basis Gram
  int omega_kind;                 // 0 gaussian, 1 rademacher
  int lambda_mode;
  double lambda_fixed;
  double refill_scale;            // c (k ln k + k ln(1/delta)/eps) / t
  int refill_mode;                // 0 first success (R7), 1 proportional draw (R7p)
  const int64_t* ext_sel;         // Algorithm 1 as the selector: its selection list (NULL: Algorithm 3)
  const int* ext_nsel;            // and its length, both in the attached selector's device state
  uint32_t ring_wait_limit;       // polls of a tensor-core pipeline wait before it gives up
  // row sharding: global row of local row 0 (a multiple of 128; Omega is keyed by the global row);
  // with an exchange (allreduce non-null) the sketch reductions leave the group's squared norms in
  // gnorm instead of adding them to fro2, and xbuf holds a step's partial basis-Gram block
  int64_t row_offset;
  void* allreduce;                // rid_allreduce_fn, host-side only
  void* allreduce_user;
  double* gnorm;                  // kMaxGroup doubles (sharded only)
  // gradient mode on tensor cores: the group's gradient fields (FP32, column q at gfield + q
  // gfield_ld, 2m entries), the gradient part of its leverage sketch (s x group) and ||G a_q||^2
  float* gfield;
  int64_t gfield_ld;
  double* glev;
  double* gnorm2;
  double* xbuf;                   // t x 2t doubles (sharded only)
  uint64_t seed;
  int grad;                       // gradient mode
  int nx, ny, nfields;
  int lev_ld;                     // leading dimension of Slev
  // data
  void* pool;
  double* omegaT;                 // Gaussian mode: m_pad x rows (entry (i, r) at i*rows + r)
  double* omegagT;                // Gaussian gradient sketch: (2 m_pad) x s
  double* S;
  double* Slev;
  double* SSt;
  double* fro2;                   // [0] ||A_obs||^2, [1] leverage norm
  // selection state (device)
  int64_t* JC; int64_t* JC_prev;  // t
  int* slotC; int* slotC_prev;    // t, pool slot of each basis slot (-1 empty)
  int* dslot;                     // t, pool slot receiving the q-th buffered column of this batch
  int* dslot_all;                 // la x t: the lists of batches b .. b + la - 1, batch b at (b % la) t
  int la;                         // lookahead: the select of step b picks the slots of batch b + la
  int npool;                      // pool slots: (la + 2) t (previous and new basis, la batches)
  int64_t* JD;                    // t, global index of the q-th buffered column
  double* tau_old;                // t
  double* tauC; double* tauD;     // t each
  int* meta;                      // small ints, see META_*
  int* act; int* pact;            // active slots now / before (ordered by slot)
  int* isnew;                     // per active position: 1 if new basis element
  int* posof;                     // per slot: active position or -1
  int* newpos;                    // active positions of the new basis elements
  int* gnew; int* gtgt;           // pool slots: new entries, Gram targets
  double* scal;                   // small doubles, see SCAL_*
  // batch-step work
  double* Gp;                     // 2t x 2t
  double* gpart;                  // gram split-K partials
  double* P;                      // t x n_cap
  double* cand;                   // 4 x t x n_cap
  double* zq;                     // 2 x t x n_cap: Q4^T (Omega A_obs) and Q6^T (Omega A_obs) / sqrt(s)
  double* work;                   // linear-algebra scratch
  double* hpart;                  // Hutch++ partials
  double* spart;                  // sketch partials
  double* npart;                  // norm partials
  int* err;                       // device error word
  unsigned int* gbar;             // grid-barrier words of the cooperative kernels
  int n_sm;
  int tc_blocks;                  // CTAs of the tensor-core kernels
  int tc_right;                   // 1: the right sketch runs on tensor cores (FP32 data, +-1 W)
  float* tc_part;                 // ingest partial accumulators (tc_blocks x max(rows16, 256) x 128 floats)
  float* tg_part;                 // basis-Gram partial accumulators (tc_blocks x 512 x 128 floats)
  unsigned int* gbar2;            // grid-barrier words of the batch-step stream's cooperative kernels
  int n_sketch_blocks;
  int gram_split;
  int64_t work_len;
  int grad_coeff;                 // keep Omega G^p a (Sec. 3.4's gradient-augmented coefficients)
  double* Sg;                     // 2 s x n_cap: column j = [Omega G^1 a_j; Omega G^2 a_j] (unit variance)
  double* Kg;                     // 2 s x s: Omega G^p Omega^T / s, formed on first use (gcv.cu)
  int right_l;                    // columns of the optional right sketch (0: off)
  void* Y;                        // right sketch, m_pad x right_l, data dtype
  void* Wr;                       // the group's right-sketch vectors (see right.cu)
};

// meta[] indices
enum {
  META_NACT = 0, META_NPACT = 1, META_NNEW = 2, META_NTGT = 3, META_COUNT = 4,
  META_NOBS = 5, META_NPREV = 6, META_BATCH = 7, META_QSTAR = 8, META_NKEPT = 9, META_LEN = 16
};
// scal[] indices
// SCAL_FRO0 + (batch & 7): ||A_obs||^2 as the batch's step saw it, written by its lambda part and
// read at the end of its tail (eight slots: the lambda parts of the next steps may run while this
// step's tail still reads it; the lambda part of step b + 8 follows the ingest of its batch, which
// follows the select of step b + 8 - la, which follows the tail of step b + 6 - la >= b)
// SCAL_GSHIFT: the Tikhonov shift of the basis Gram in the last batch step, relative to its
// largest diagonal entry (0 when the Gram was factored as is).
// SCAL_UNC + q: rounding uncertainty of candidate q's estimate relative to ||A_obs||^2 (see
// hutch_finish_kernel); 0 for FP64 sketches.
// SCAL_LAMBDA + (batch & 1): lambda of the step (two slots: consecutive steps' lambda parts run
// concurrently on two streams).
// Entries [0, SCAL_LOG) are the step's decision quantities copied into the per-batch log.
enum {
  SCAL_LAMBDA = 5 /* 2 slots */, SCAL_EST = 1 /* 4 signed estimates */, SCAL_FRO0 = 16 /* 8 slots */,
  SCAL_GSHIFT = 7, SCAL_UNC = 8 /* 4 values */, SCAL_LOG = 16, SCAL_LEN = 24
};

// Per (candidate, column chunk) partials of the Hutch++ step: H P_q^T (hh x t), tr(G P P^T) and
// sum_j sum_a G_aa P_aj^2.
inline __host__ __device__ int64_t hpart_stride(int64_t hh, int64_t t) { return hh * t + 2; }

// device error bits
enum { ERR_NONFINITE = 1, ERR_CHOL = 2, ERR_EIG = 4, ERR_TIMEOUT = 8 };

constexpr int kMaxGroup = 64;      // columns per tensor-core ingest launch
constexpr uint32_t kRingWaitLimit = 1u << 22;   // default polls of a tensor-core pipeline wait

// ingest.cu: SIMT path (FP64 or FP32, native precision), nb <= kMaxB columns given by
// pointer.  Returns the number of kernels launched; ev[0..2] (may be null) are recorded
// before the sketch kernel, after it, and after the reductions.
int launch_ingest(const Dev& d, const void* const* cols, int nb, int count, int64_t n_obs,
                  cudaStream_t st, cudaEvent_t* ev);
// Gradient mode (Sec. 3.4): the leverage sketch of nb columns given by pointer, after their
// sketch has been reduced; returns the number of kernels launched.
int launch_grad(const Dev& d, const void* const* cols, int nb, int64_t n_obs, cudaStream_t st);
// Gradient stencil of Sec. 3.4 on each field's nx x ny grid (x fastest): entry j of the
// stacked d m = 2 m gradient vector, direction p = j / m at coordinate i = j mod m, is
// wm a[i - st] + wc a[i] + wp a[i + st]: central difference inside, one-sided at the boundary
// (spacing 1; fields independent).
struct GradStencil {
  int64_t i, st;
  double wm, wc, wp;
};
__device__ __forceinline__ GradStencil grad_stencil(int64_t j, int64_t m, int nx, int ny) {
  GradStencil g;
  const int p = j >= m ? 1 : 0;                // d = 2
  g.i = j - (p ? m : 0);
  const int64_t ql = g.i % ((int64_t)nx * ny);
  const int c = p == 0 ? (int)(ql % nx) : (int)(ql / nx);
  const int len = p == 0 ? nx : ny;
  g.st = p == 0 ? 1 : nx;
  if (c == 0) { g.wm = 0.0; g.wc = -1.0; g.wp = 1.0; }
  else if (c == len - 1) { g.wm = -1.0; g.wc = 1.0; g.wp = 0.0; }
  else { g.wm = -0.5; g.wc = 0.0; g.wp = 0.5; }
  return g;
}

// Optional right sketch Y += sum_q a_q omega_{j0+q}^T over ncols ingested columns (right.cu).
int launch_right_sketch(const Dev& d, const void* const* cols, int ncols, int64_t j0, cudaStream_t st);
size_t right_w_bytes(const Dev& d);

// Sec. 3.4's gradient-augmented coefficients for the final basis with lambda chosen by the
// sketched GCV function (gcv.cu).  jact: the na active basis columns (global indices, slot
// order) and slot: their slots; P_out rows are slots (ldp >= t), empty slots zero.  kg_ready:
// whether d.Kg already holds Omega G^p Omega^T / s (set on return).  Returns 0 or a CUDA error.
int gradient_coefficients(const Dev& d, cudaStream_t st, int64_t n, const int64_t* jact, const int* slot, int na,
                          double lo, double hi, double tol, double* P_out, int64_t ldp, int on_device,
                          bool* kg_ready, double* lambda_out, double* gcv_out);
// SS^T update for nb new columns (shared by both ingest paths).
void launch_gram_update(const Dev& d, int nb, int64_t n_obs, cudaStream_t st);

// tc_ingest.cu: tensor-core path for FP32 data (ncols <= kMaxGroup); records ev[0], ev[1]
// around the sketch kernel and launches the reduction.  Returns 0 on success.
int launch_tc_ingest(const Dev& d, const void* const* cols, int ncols, int split, int count,
                     int64_t n_obs, int nblk, float* part, double* npart, cudaStream_t st,
                     cudaEvent_t* ev, int fp8);
int tc_smem_bytes();
// Basis Gram of the new x target pool slots on tensor cores (FP32 pool); returns the
// number of kernels launched, or -1.  part holds nblk x 512 x 128 floats.
int launch_tc_gram(const Dev& d, int nblk, float* part, cudaStream_t st);
// The optional right sketch of a group of <= 64 FP32 columns on tensor cores (BF16x2, +-1 W given
// as G x lw FP32 values in W); returns the kernels launched, or -1.
int launch_tc_right(const Dev& d, const void* const* cols, int ncols, const float* W, int lw, cudaStream_t st);
// Whether the current context can co-schedule the batch step's cluster kernels (coop.cu).
bool batch_clusters_fit(int s, int t);
void launch_materialize_omega(const Dev& d, cudaStream_t st);

// Timeline events of one batch step (recorded only while profiling; tl may be null).
enum { TL_SNAP = 0, TL_LAMBDA0, TL_LAMBDA1, TL_TAIL0, TL_SCORES, TL_SELECT, TL_GRAM0, TL_GRAM1, TL_QR0, TL_QR1,
       TL_TAIL1, kTlEvents };
// Phases reported by rid_profile_timeline.
enum { TLP_INGEST = 0, TLP_LAMBDA = 1, TLP_SCORES = 2, TLP_SELECT = 3, TLP_GRAM = 4, TLP_QR = 5, TLP_COEFF = 6 };
// A batch step runs in three parts on their own streams; events order them and the host never
// waits.  The lambda part (tridiagonalization of the sketch Gram, its top-k eigenvalues, lambda
// and the LDL^T of T + lambda I; it also snapshots ||A_obs||^2) reads only the sketch: batch b's
// runs on lambda stream b % 2 with scratch copy b % 2, so that consecutive batches' lambda parts
// overlap.  The select part (ridge scores, uniforms, prune/refill) runs on the select stream:
// it reads and updates the live selection state of d and writes the step's selection record r
// (previous and new basis, index lists); ev_scores (may be null) is recorded after the scores,
// and the select waits for ev_wait_rec (the end of the tail that last read the record).  The
// tail (basis Gram, Algorithms 4-8, commit) reads only the record (d of launch_batch_tail is
// the record view): its Gram side (basis Gram, G and its factor, T) runs on stg between ev_fork
// and ev_gram, beside the sketch side's QRs on st; finish_kernel copies its counts and basis to
// the reporting state (gmeta, gjcp, gslotp).  Each returns the number of kernels launched (0 on
// failure).
int launch_batch_lambda(const Dev& d, int batch, cudaStream_t st);
int launch_batch_select(const Dev& d, const Dev& r, int count, int64_t n_obs, int batch, cudaStream_t st,
                        cudaEvent_t ev_scores, cudaEvent_t ev_wait_rec, cudaEvent_t* tl);
int launch_batch_tail(const Dev& d, int count, int64_t n_obs, int64_t n_prev, int batch,
                      cudaStream_t st, cudaStream_t stg, cudaEvent_t ev_fork, cudaEvent_t ev_gram,
                      int* gmeta, int64_t* gjcp, int* gslotp, cudaEvent_t* tl);
// Row sharding: sum the group's partial sketch columns (S(:, n_obs .. n_obs + ncols)) and squared
// norms over the shards with d.allreduce, then add the norms to ||A_obs||^2 in column order.
// Returns 0, or -1 if the exchange failed.
int shard_exchange_sketch(const Dev& d, int ncols, int64_t n_obs, cudaStream_t st);
int launch_reset_state(const Dev& d, cudaStream_t st);

// coop.cu: lambda (Eq. 23) through a tridiagonalization of the sketch Gram (cluster or
// grid), and the sketched ridge scores of C and D from its reflectors; 0 on failure.
int launch_lambda(const Dev& d, int batch, double* work_base, int64_t off_A, int64_t off_R, int64_t off_d,
                  int64_t off_e, int64_t off_beta, int64_t off_vhead, int64_t off_p, int64_t off_mu,
                  int64_t off_ldld, int64_t off_ldll, unsigned int* bar_mem, int n_sm, cudaStream_t st);
int launch_scores(const Dev& d, int count, int64_t jd0, double* work_base, int64_t off_R, int64_t off_beta,
                  int64_t off_vhead, int64_t off_ldld, int64_t off_ldll, int64_t off_vec, int vstride,
                  cudaStream_t st);
// coop.cu: Householder QR of Omega A_J (s x n_act) and of its new-element columns
// (s x n_new) on every SM; R's diagonal goes to r4 / r6.  Returns 1, or 0 on failure.
int launch_qr_coop(const Dev& d, double* Q4, double* b4, double* h4, double* r4, double* Q6,
                   double* b6, double* h6, double* r6, unsigned int* bar_mem, cudaStream_t st);
int64_t work_doubles(const Dev& d);

// The device view of a residual-CSS selector (csrc/rcss.cu): its selection list and length, its
// sizes, capacity, cap mode, data type and stream.
void rcss_selection_view(const rid_rcss* g, const int64_t** sel, const int** nsel, int64_t* m, int* cap,
                         int* stop_at_cap, int* dtype, cudaStream_t* st);

// Message returned by rid_last_error(NULL) for failures outside a handle.
void set_global_error(const char* msg);

}  // namespace rid
