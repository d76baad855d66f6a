// Host engine and C ABI: restarted, adaptively restarted BFOM / BGMRES with a
// low-synchronization block Arnoldi skeleton (arXiv 2208.09899, Sec. 2.4 and 4).
//
// Each restart cycle is enqueued on the handle's stream as one batch: the
// CholQR of the start block, then every loop iteration the cycle may need
// (SpMM, one-pass Gram, small step kernel, basis update).  The small kernel
// clears the device-side `active` flag when the cycle ends (estimate below tol,
// a Cholesky NaN-flag, or the basis size limit), which turns the remaining
// launches of the batch into no-ops; the host then reads the 100-byte control
// record once per cycle and enqueues the cycle end (X and U update) with the
// next cycle.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lsba.h"
#include "lsba_internal.cuh"

using namespace lsba;

enum { MODE_FP64 = 0, MODE_DF = 1, MODE_F32 = 2 };

struct lsba_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  lsba_options opt;
  int num_sms = 0;
  // workspace capacity
  int64_t cap_n = 0;
  int cap_s = 0, cap_m = 0;
  double* basis = nullptr;     // (m+1) blocks
  double* Wb = nullptr;        // n x s
  double* Ub = nullptr;        // n x s
  double* partials = nullptr;
  size_t partials_cap = 0;
  double* Gbuf = nullptr;
  size_t G_cap = 0;
  double* small = nullptr;     // all small matrices
  size_t small_cap = 0;
  int* ismall = nullptr;
  size_t ismall_cap = 0;
  Ctl* d_ctl = nullptr;
  Ctl* h_ctl = nullptr;        // pinned mirror
  unsigned long long* d_range = nullptr;   // magnitude ranges of A and B (k_absrange)
  unsigned long long* h_range = nullptr;   // pinned mirror
  SmallWs ws;
  // host-buffer solve
  int32_t* hA_rowptr = nullptr;
  int32_t* hA_colidx = nullptr;
  double* hA_vals = nullptr;
  double* hB = nullptr;
  double* hX = nullptr;
  int64_t host_n = 0, host_nnz = 0;
  int host_s = 0;
  // results
  lsba_stats stats;
  std::vector<double> h_est;
  std::vector<int32_t> h_est_cycle, h_est_j, h_cycle_m, h_cycle_flag, h_cycle_mcur;
  std::vector<double> h_first_H, h_first_beta, h_gram_data;
  std::vector<int32_t> h_gram_rows, h_gram_cols;
  int first_j = 0;
  // profiling: CUDA event pairs around launches, collected at each host sync
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_class;
  size_t ev_used = 0;
  // side stream for the off-critical-path small kernel, and its events
  cudaStream_t side = nullptr;
  std::vector<cudaEvent_t> ev_main, ev_side;
  // working precision of the bandwidth-shaped passes
  int mode = 0;
  float2* A_df = nullptr;      // CSR values as hi + lo pairs
  size_t A_df_cap = 0;
  double* Bdf = nullptr;       // n x s float2 (as raw 8-byte words)
  double* Xdf = nullptr;
  float2* cdf = nullptr;       // converted update coefficients
  size_t cdf_cap = 0;
  // stored digit planes of the basis (tensor-core Gram, s = 8): block i at
  // dig + i * digit_block_bytes(n, s), exponents at dexp + i * digit_exp_count(n, s)
  unsigned char* dig = nullptr;
  int* dexp = nullptr;
  bool use_tcs = false;
  // FP64 on the tensor cores (exact digit products, kernels_f64tc.cu): lagged
  // skeletons, s = 8.  Per-(tile, column) exponents of the basis blocks
  // (block i at fexp + i * f64tc_exp_count(n, s)), of U, W and the cycle's
  // start block, their digit planes (block i at fpl + i * f64tc_plane_bytes(n),
  // then U, W, the start block), and the folded FP64 update coefficients.
  bool use_ftc = false;
  int* fexp = nullptr;
  int* fexp_U = nullptr;
  int* fexp_W = nullptr;
  int* fexp_R0 = nullptr;
  unsigned char* fpl = nullptr;
  unsigned char* fpl_U = nullptr;
  unsigned char* fpl_W = nullptr;
  unsigned char* fpl_R0 = nullptr;
  double* cf64 = nullptr;
  double prof_ms[LSBA_K_NCLASS] = {0, 0, 0, 0};
  int64_t prof_n[LSBA_K_NCLASS] = {0, 0, 0, 0};
  // captured restart cycles (see run_cycle_body)
  uint64_t ws_gen = 1;         // bumped whenever workspace buffers move
  std::vector<struct CycleGraph> graphs;
  uint64_t graph_clock = 0;
  std::vector<uint8_t> side_recorded;  // side events recorded in the current cycle
  bool own_stream = false;     // stream created by the handle (caller passed NULL)
  // lsba_autotune: measured kernel shapes per lagged iteration k for one (n, s)
  int64_t tune_n = 0;
  int tune_s = 0;
  std::vector<lsba_tune_entry> tune;   // indexed by k; gram_kernel < 0: no choice
  int tune_gen = 0;
};

// The launch sequence of one restart cycle is fixed by these values; a cycle
// graph is reused only when all of them match.
struct CycleKey {
  const void* rowptr;
  const void* colidx;
  const void* vals;
  const void* a_lowprec;
  const double* rstart;
  int64_t n;
  int s, m_cur, start_flags, skel, modification, mode, tensor_cores, global_ip, col_muscle, pad;
  uint64_t ws_gen;
  bool operator==(const CycleKey& o) const { return memcmp(this, &o, sizeof(*this)) == 0; }
};
struct CycleGraph {
  CycleKey key;
  cudaGraphExec_t exec;   // null until the key is seen a second time
  uint64_t last_use;
  bool failed;            // capture failed: issue this cycle directly
};
static const size_t LSBA_MAX_CYCLE_GRAPHS = 8;

// Record the start event of a launch of kernel class `cls` (no-op unless profiling).
static void prof_begin(lsba_ctx* h, int cls, cudaStream_t st) {
  if (!h->opt.profile) return;
  if (h->ev_used + 2 > h->ev.size()) {
    for (int i = 0; i < 2; ++i) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      h->ev.push_back(e);
    }
    h->ev_class.resize(h->ev.size() / 2);
  }
  h->ev_class[h->ev_used / 2] = cls;
  cudaEventRecord(h->ev[h->ev_used], st);
}
static void prof_begin(lsba_ctx* h, int cls) { prof_begin(h, cls, h->stream); }
static void prof_end(lsba_ctx* h, cudaStream_t st) {
  if (!h->opt.profile) return;
  cudaEventRecord(h->ev[h->ev_used + 1], st);
  h->ev_used += 2;
}
static void prof_end(lsba_ctx* h) { prof_end(h, h->stream); }
// Accumulate the recorded pairs (the stream must be synchronized).
static void prof_collect(lsba_ctx* h) {
  for (size_t i = 0; i + 1 < h->ev_used; i += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev[i], h->ev[i + 1]) == cudaSuccess) {
      h->prof_ms[h->ev_class[i / 2]] += ms;
      h->prof_n[h->ev_class[i / 2]] += 1;
    }
  }
  h->ev_used = 0;
}

#define CK(x)                                         \
  do {                                                \
    cudaError_t e_ = (x);                             \
    if (e_ != cudaSuccess) {                          \
      fprintf(stderr, "lsba: CUDA error %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
      return LSBA_CUDA_ERROR;                         \
    }                                                 \
  } while (0)

// Workspace memory is stream-ordered (cudaMallocAsync / cudaFreeAsync on the
// handle's stream, from the device's default memory pool): growing or
// releasing one handle's workspace never synchronises the device, so solves on
// other streams keep running.
static cudaError_t ws_alloc(lsba_ctx* h, void* pp, size_t bytes) {
  return cudaMallocAsync((void**)pp, bytes, h->stream);
}
static void ws_free(lsba_ctx* h, void* p) {
  if (p) cudaFreeAsync(p, h->stream);
}

static void clear_graphs(lsba_ctx* h) {
  for (auto& g : h->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
}

static void free_ws(lsba_ctx* h) {
  clear_graphs(h);
  ++h->ws_gen;
  ws_free(h, h->dig);
  ws_free(h, h->dexp);
  h->dig = nullptr;
  h->dexp = nullptr;
  ws_free(h, h->fexp);
  ws_free(h, h->cf64);
  ws_free(h, h->fpl);
  h->fexp = h->fexp_U = h->fexp_W = h->fexp_R0 = nullptr;
  h->fpl = h->fpl_U = h->fpl_W = h->fpl_R0 = nullptr;
  h->cf64 = nullptr;
  ws_free(h, h->basis);
  ws_free(h, h->Wb);
  ws_free(h, h->Ub);
  ws_free(h, h->partials);
  ws_free(h, h->Gbuf);
  ws_free(h, h->small);
  ws_free(h, h->ismall);
  ws_free(h, h->Bdf);
  ws_free(h, h->Xdf);
  ws_free(h, h->cdf);
  h->Bdf = h->Xdf = nullptr;
  h->cdf = nullptr;
  h->cdf_cap = 0;
  h->basis = h->Wb = h->Ub = h->partials = h->Gbuf = h->small = nullptr;
  h->ismall = nullptr;
  h->cap_n = 0;
  h->cap_s = h->cap_m = 0;
  h->partials_cap = h->G_cap = h->small_cap = h->ismall_cap = 0;
}

static size_t max_partials(int64_t n, int s, int mmax, int sms, size_t* qmax_out) {
  size_t best = 0, qmax = 0;
  for (int a = 1; a <= mmax + 2; ++a)
    for (int b = 1; b <= 2; ++b) {
      GramPlan p = plan_gram(n, s, a, b, sms);
      size_t v = (size_t)p.grid_x * p.q;
      if (v > best) best = v;
      if ((size_t)p.q > qmax) qmax = p.q;
      for (int tc = 0; tc < 3; tc += 2) {
        GramPlan pd = plan_gram_df(n, s, a, b, sms, tc);
        v = (size_t)pd.grid_x * pd.q;
        if (v > best) best = v;
      }
      {
        // the autotuner's largest FP32-pipe grid
        GramPlan pd = plan_gram_df(n, s, a, b, sms, 0, LSBA_TUNE_MAX_CPS, 1);
        v = (size_t)pd.grid_x * pd.q;
        if (v > best) best = v;
      }
      if (gram_tcs_eligible(s, a, b)) {
        GramPlan pt = plan_gram_tcs(n, s, a, b, sms);
        v = (size_t)pt.grid_x * pt.q;
        if (v > best) best = v;
      }
      if (gram_f64tc_eligible(s, a, b, false)) {
        GramPlan pt = plan_gram_f64tc(n, s, a, b, sms);
        v = (size_t)pt.grid_x * pt.q;
        if (v > best) best = v;
      }
      if (s % 4 == 0) {
        GramPlan pf = plan_gram_f32(n, s, a, b, sms);
        v = (size_t)pf.grid_x * pf.q;
        if (v > best) best = v;
      }
    }
  *qmax_out = qmax;
  return best;
}

// Offsets (in doubles, 256-byte aligned) of the small matrices of one handle
// in its single small-matrix allocation.  The restart history holds at most
// LSBA_HIST_RESTARTS cycles.
#define LSBA_HIST_RESTARTS 4096
struct SmallLayout {
  size_t oH, oT, oJ, oc1, oc2, och, ot1, ot2, oRb, orf, otau, otw, og, oTf, ogf, ocf, ouf, oC,
      oBc, oXi, oMv, owk, osz, osy, osr, ohe, ogh, omu, opr;
  size_t hist_cap, gram_hist_cap, total;
};

static SmallLayout small_layout(int s, int m, int max_restarts) {
  SmallLayout L;
  const size_t ldH = (size_t)(m + 2) * s, ldR = (size_t)(m + 1) * s;
  const size_t ss = (size_t)s * s;
  const int restarts = max_restarts < LSBA_HIST_RESTARTS ? max_restarts : LSBA_HIST_RESTARTS;
  L.hist_cap = (size_t)(restarts + 3) * (m + 2) + 16;
  L.gram_hist_cap = (size_t)(m + 3) * (m + 3) * 2 * ss + 64;
  size_t off = 0;
  auto take = [&](size_t count) {
    size_t o = off;
    off += (count + 31) & ~(size_t)31;
    return o;
  };
  L.oH = take(ldH * (m + 1) * s);
  L.oT = take(ldH * ldH);
  L.oJ = take(ldH * s);
  L.oc1 = take((size_t)(m + 4) * ss);
  L.oc2 = take((size_t)(m + 4) * ss);
  L.och = take(ss);
  L.ot1 = take(ss);
  L.ot2 = take(ss);
  L.oRb = take(ldR * ldR);
  L.orf = take((size_t)(m + 1) * 2 * ss);
  L.otau = take((size_t)(m + 1) * s);
  L.otw = take((size_t)(m + 1) * ss);
  L.og = take(ldH * s);
  L.oTf = take(ss);
  L.ogf = take(ss);
  L.ocf = take(ss);
  L.ouf = take(ldH * s);
  L.oC = take(ss);
  L.oBc = take(ss);
  L.oXi = take(ldH * s);
  L.oMv = take(ldH * s);
  L.owk = take(6 * ldH * s + 16 * ss);
  L.osz = take(ldH * s);
  L.osy = take(ldH * s);
  L.osr = take(ss);
  L.ohe = take(L.hist_cap);
  L.ogh = take(L.gram_hist_cap);
  L.omu = take(muscle_area_doubles(s));
  L.opr = take((size_t)LSBA_LS_PROD_CTAS * 2 * ss);
  L.total = off;
  return L;
}

// Allocate (or grow) the workspace for n x s blocks and basis size m.
static int ensure_ws(lsba_ctx* h, int64_t n, int s, int m) {
  if (n <= h->cap_n && s == h->cap_s && m <= h->cap_m && h->basis) return LSBA_OK;
  free_ws(h);
  const size_t blk = (size_t)n * s;
  if (ws_alloc(h, &h->basis, sizeof(double) * blk * (m + 1)) != cudaSuccess ||
      ws_alloc(h, &h->Wb, sizeof(double) * blk) != cudaSuccess ||
      ws_alloc(h, &h->Ub, sizeof(double) * blk) != cudaSuccess) {
    cudaGetLastError();
    free_ws(h);
    return LSBA_OUT_OF_MEMORY;
  }
  size_t qmax = 0;
  h->partials_cap = max_partials(n, s, m, h->num_sms, &qmax);
  h->G_cap = qmax;
  const int ldH = (m + 2) * s, ldR = (m + 1) * s;
  const SmallLayout L = small_layout(s, m, h->opt.max_restarts);
  const size_t hist_cap = L.hist_cap, gram_hist_cap = L.gram_hist_cap;
  const size_t oH = L.oH, oT = L.oT, oJ = L.oJ, oc1 = L.oc1, oc2 = L.oc2, och = L.och, ot1 = L.ot1,
               ot2 = L.ot2, oRb = L.oRb, orf = L.orf, otau = L.otau, otw = L.otw, og = L.og,
               oTf = L.oTf, ogf = L.ogf, ocf = L.ocf, ouf = L.ouf, oC = L.oC, oBc = L.oBc,
               oXi = L.oXi, oMv = L.oMv, owk = L.owk, osz = L.osz, osy = L.osy, osr = L.osr,
               ohe = L.ohe, ogh = L.ogh;
  const size_t off = L.total;
  h->small_cap = off;
  if (ws_alloc(h, &h->small, sizeof(double) * off) != cudaSuccess ||
      ws_alloc(h, &h->partials, sizeof(double) * h->partials_cap) != cudaSuccess ||
      ws_alloc(h, &h->Gbuf, sizeof(double) * h->G_cap) != cudaSuccess) {
    cudaGetLastError();
    free_ws(h);
    return LSBA_OUT_OF_MEMORY;
  }
  h->ismall_cap = 2 * hist_cap + 2 * (m + 4);
  h->cdf_cap = coef_df_count(m + 3, s, true);
  if (ws_alloc(h, &h->Bdf, sizeof(double) * blk) != cudaSuccess ||
      ws_alloc(h, &h->Xdf, sizeof(double) * blk) != cudaSuccess ||
      ws_alloc(h, &h->cdf, sizeof(float2) * h->cdf_cap) != cudaSuccess) {
    cudaGetLastError();
    free_ws(h);
    return LSBA_OUT_OF_MEMORY;
  }
  if (ws_alloc(h, &h->ismall, sizeof(int) * h->ismall_cap) != cudaSuccess) {
    cudaGetLastError();
    free_ws(h);
    return LSBA_OUT_OF_MEMORY;
  }
  cudaMemsetAsync(h->small, 0, sizeof(double) * off, h->stream);
  SmallWs& w = h->ws;
  w.s = s;
  w.m = m;
  w.ldH = ldH;
  w.ldT = ldH;
  w.ldR = ldR;
  double* b = h->small;
  w.H = b + oH;
  w.T = b + oT;
  w.J = b + oJ;
  w.G = h->Gbuf;
  w.coef1 = b + oc1;
  w.coef2 = b + oc2;
  w.chain = b + och;
  w.tri1 = b + ot1;
  w.tri2 = b + ot2;
  w.Rbar = b + oRb;
  w.refl = b + orf;
  w.tau = b + otau;
  w.Twy = b + otw;
  w.g = b + og;
  w.Tfom = b + oTf;
  w.gfom = b + ogf;
  w.cfom = b + ocf;
  w.ufom = b + ouf;
  w.Cfac = b + oC;
  w.Bcyc = b + oBc;
  w.Xi = b + oXi;
  w.Mvec = b + oMv;
  w.work = b + owk;
  w.saveZP = b + osz;
  w.saveY = b + osy;
  w.saveR = b + osr;
  w.hist_est = b + ohe;
  w.gram_hist = b + ogh;
  w.mus = b + L.omu;
  w.prod = b + L.opr;
  w.hist_cycle = h->ismall;
  w.hist_j = h->ismall + hist_cap;
  w.gram_dims = h->ismall + 2 * hist_cap;
  w.ctl = h->d_ctl;
  h->h_ctl->hist_cap = (int)hist_cap;
  h->h_ctl->gram_hist_cap = (int)gram_hist_cap;
  if (!h->side) {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, hi) != cudaSuccess) {
      cudaGetLastError();
      h->side = nullptr;
      free_ws(h);
      return LSBA_CUDA_ERROR;
    }
  }
  while ((int)h->ev_main.size() < m + 3) {
    cudaEvent_t a, b;
    if (cudaEventCreateWithFlags(&a, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      free_ws(h);
      return LSBA_CUDA_ERROR;
    }
    h->ev_main.push_back(a);
    h->ev_side.push_back(b);
  }
  h->cap_n = n;
  h->cap_s = s;
  h->cap_m = m;
  return LSBA_OK;
}

// Digit planes for the m + 1 basis blocks (allocated on first use, within the
// workspace's capacity n <= cap_n, m <= cap_m).
static int ensure_digits(lsba_ctx* h) {
  if (h->dig) return LSBA_OK;
  const size_t nb = (size_t)h->cap_m + 1;
  if (ws_alloc(h, &h->dig, nb * digit_block_bytes(h->cap_n, h->cap_s)) != cudaSuccess ||
      ws_alloc(h, &h->dexp, sizeof(int) * nb * digit_exp_count(h->cap_n, h->cap_s)) != cudaSuccess) {
    cudaGetLastError();
    ws_free(h, h->dig);
    ws_free(h, h->dexp);
    h->dig = nullptr;
    h->dexp = nullptr;
    return LSBA_OUT_OF_MEMORY;
  }
  return LSBA_OK;
}

// Exponent arrays and FP64 coefficient buffer of the FP64 tensor-core path
// (allocated on first use, within the workspace's capacity).
static int ensure_f64tc(lsba_ctx* h) {
  if (h->fexp) return LSBA_OK;
  const size_t ec = f64tc_exp_count(h->cap_n, h->cap_s);
  const size_t nb = (size_t)h->cap_m + 1 + 3;
  const size_t pb = f64tc_plane_bytes(h->cap_n);
  if (ws_alloc(h, &h->fexp, sizeof(int) * nb * ec) != cudaSuccess ||
      ws_alloc(h, &h->cf64, sizeof(double) * 2 * 8 * (size_t)(h->cap_m + 3) * 8) != cudaSuccess ||
      ws_alloc(h, &h->fpl, pb * nb) != cudaSuccess) {
    cudaGetLastError();
    ws_free(h, h->fexp);
    ws_free(h, h->cf64);
    ws_free(h, h->fpl);
    h->fexp = nullptr;
    h->cf64 = nullptr;
    h->fpl = nullptr;
    return LSBA_OUT_OF_MEMORY;
  }
  h->fexp_U = h->fexp + (size_t)(h->cap_m + 1) * ec;
  h->fexp_W = h->fexp_U + ec;
  h->fexp_R0 = h->fexp_W + ec;
  h->fpl_U = h->fpl + (size_t)(h->cap_m + 1) * pb;
  h->fpl_W = h->fpl_U + pb;
  h->fpl_R0 = h->fpl_W + pb;
  return LSBA_OK;
}

static BlockPtrs basis_list(const lsba_ctx* h, int64_t n, int s, int count) {
  BlockPtrs p;
  memset(&p, 0, sizeof(p));
  for (int i = 0; i < count; ++i) p.p[i] = h->basis + (size_t)i * n * s;
  return p;
}

static int push_ctl(lsba_ctx* h) {
  CK(cudaMemcpyAsync(h->d_ctl, h->h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, h->stream));
  return LSBA_OK;
}
static int pull_ctl(lsba_ctx* h) {
  CK(cudaMemcpyAsync(h->h_ctl, h->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  prof_collect(h);
  return LSBA_OK;
}

// Profiled launch wrappers.
#define PROF(cls, call)     \
  do {                      \
    prof_begin(h, cls);     \
    call;                   \
    prof_end(h);            \
  } while (0)

enum { SK_BCGS = 0, SK_PIP = 1, SK_LS = 2, SK_ICWY = 3, SK_CWY = 4, SK_BMGS = 5, SK_PIO = 6,
       SK_SVL = 7, SK_LTS = 8 };
static bool lagged(int skel) { return skel == SK_LS || skel == SK_ICWY || skel == SK_CWY; }

// Precision dispatch of the three bandwidth-shaped passes (profiled).  In the
// double-float mode every block vector buffer holds float2 (hi, lo) pairs.
static void do_gram(lsba_ctx* h, const BlockPtrs& L, int a, const BlockPtrs& R, int b, int64_t n,
                    int s, const Ctl* ctl, int guard, const lsba_tune_entry* tk = nullptr) {
  prof_begin(h, LSBA_K_GRAM);
  if (h->mode == MODE_DF) {
    // a tuned shape: kernel 1 the split-digit tensor-core Gram, 0 the FP32-pipe
    // Gram with the tuned CTAs per SM and chunk rows
    GramPlan p = tk ? plan_gram_df(n, s, a, b, h->num_sms, tk->gram_kernel == 1 ? 2 : 0, tk->gram_ctas_per_sm,
                                   tk->gram_rows)
                    : plan_gram_df(n, s, a, b, h->num_sms, h->opt.tensor_cores);
    launch_gram_df(h->stream, p, L, a, R, b, n, s, (float2*)h->partials, h->Gbuf, ctl, guard,
                   &h->d_ctl->error);
  } else if (h->mode == MODE_F32) {
    GramPlan p = plan_gram_f32(n, s, a, b, h->num_sms);
    launch_gram_f32(h->stream, p, L, a, R, b, n, s, (float*)h->partials, h->Gbuf, ctl, guard,
                    &h->d_ctl->error);
  } else {
    GramPlan p = plan_gram(n, s, a, b, h->num_sms);
    launch_gram(h->stream, p, L, a, R, b, n, s, h->partials, h->Gbuf, ctl, guard);
  }
  prof_end(h);
}

static void do_spmm(lsba_ctx* h, const lsba_csr* A, const double* V, double* W, int s,
                    const Ctl* ctl, int guard) {
  prof_begin(h, LSBA_K_SPMM);
  if (h->mode == MODE_DF)
    launch_spmm_df(h->stream, A->n, A->d_rowptr, A->d_colidx, h->A_df, (const float2*)V,
                   (float2*)W, s, ctl, guard);
  else if (h->mode == MODE_F32)
    launch_spmm_f32(h->stream, A->n, A->d_rowptr, A->d_colidx, (const float*)h->A_df,
                    (const float*)V, (float*)W, s, ctl, guard);
  else
    launch_spmm(h->stream, A->n, A->d_rowptr, A->d_colidx, A->d_vals, V, W, s, ctl, guard);
  prof_end(h);
}

static void do_update(lsba_ctx* h, const BlockPtrs& in, int nin, int64_t n, int s, double* out1,
                      const double* coef1, const double* tri1, double* out2, const double* coef2,
                      const double* chain, const double* tri2, const Ctl* ctl, int step, int cps = 0) {
  prof_begin(h, LSBA_K_UPDATE);
  if (h->mode == MODE_DF)
    launch_update_df(h->stream, in, nin, n, s, (float2*)out1, coef1, tri1, (float2*)out2, coef2,
                     chain, tri2, h->cdf, ctl, step, h->num_sms, cps);
  else if (h->mode == MODE_F32)
    launch_update_f32(h->stream, in, nin, n, s, (float*)out1, coef1, tri1, (float*)out2, coef2,
                      chain, tri2, (float*)h->cdf, ctl, step, h->num_sms);
  else
    launch_update(h->stream, in, nin, n, s, out1, coef1, tri1, out2, coef2, chain, tri2, ctl, step);
  prof_end(h);
}

// The Gram of a lagged skeleton's iteration k >= 2 on the stored digit planes:
// [V_1..V_{k-1}, U]^T [U, W].
static void do_gram_tcs(lsba_ctx* h, int k, int64_t n, int s, const Ctl* ctl) {
  prof_begin(h, LSBA_K_GRAM);
  GramPlan p = plan_gram_tcs(n, s, k, 2, h->num_sms);
  launch_gram_tcs(h->stream, p, h->dig, h->dexp, n, s, k, (const float2*)h->Ub,
                  (const float2*)h->Wb, (float2*)h->partials, h->Gbuf, ctl, 1, &h->d_ctl->error);
  prof_end(h);
}
// Digit planes of basis block i, written by the update of iteration `step`.
static void split_basis(lsba_ctx* h, int i, int64_t n, int s, const Ctl* ctl, int step) {
  prof_begin(h, LSBA_K_UPDATE);
  launch_split_digits(h->stream, (const float2*)(h->basis + (size_t)i * n * s), n, s,
                      h->dig + (size_t)i * digit_block_bytes(n, s),
                      h->dexp + (size_t)i * digit_exp_count(n, s), ctl, step, h->num_sms);
  prof_end(h);
}

// FP64 tensor-core passes.  Block i of the basis and its exponents:
static int* basis_exp(const lsba_ctx* h, int64_t n, int s, int i) {
  return h->fexp + (size_t)i * f64tc_exp_count(n, s);
}
static unsigned char* basis_planes(const lsba_ctx* h, int64_t n, int i) {
  return h->fpl + (size_t)i * f64tc_plane_bytes(n);
}
static void do_block_digits(lsba_ctx* h, const double* V, int* ex, unsigned char* planes, int64_t n,
                            const Ctl* ctl, int guard) {
  prof_begin(h, LSBA_K_SPMM);
  launch_block_digits(h->stream, V, n, ex, planes, ctl, guard);
  prof_end(h);
}
static void do_gram_ftc(lsba_ctx* h, const unsigned char* const* L, const int* const* Le, int a,
                        const unsigned char* const* R, const int* const* Re, int b, bool shared,
                        int64_t n, int s, const Ctl* ctl, int guard) {
  prof_begin(h, LSBA_K_GRAM);
  GramPlan p = plan_gram_f64tc(n, s, a, b, h->num_sms);
  launch_gram_f64tc(h->stream, p, L, Le, a, R, Re, b, shared, n, h->partials, h->Gbuf, ctl, guard,
                    &h->d_ctl->error);
  prof_end(h);
}
static void do_update_ftc(lsba_ctx* h, const unsigned char* const* in, const int* const* ein,
                          int nin, const double* X, int64_t n, double* out1, int* e1,
                          unsigned char* p1, double* out2, int* e2, unsigned char* p2,
                          const double* coef1, const double* tri1, const double* coef2,
                          const double* chain, const double* tri2, const Ctl* ctl, int step) {
  prof_begin(h, LSBA_K_UPDATE);
  launch_update_f64tc(h->stream, in, ein, nin, X, n, out1, e1, p1, out2, e2, p2, coef1, tri1, coef2,
                      chain, tri2, h->cf64, ctl, step, &h->d_ctl->error, h->num_sms);
  prof_end(h);
}

// After the small kernel of loop iteration k: run its side kernel on the side
// stream (it overlaps the next iteration's SpMM and Gram).  The next small
// kernel, and the end of the batch, wait for it.
static void enqueue_side(lsba_ctx* h, int k) {
  cudaEventRecord(h->ev_main[k], h->stream);
  cudaStreamWaitEvent(h->side, h->ev_main[k], 0);
  prof_begin(h, LSBA_K_SMALL, h->side);
  launch_small_side(h->side, h->ws, k);
  prof_end(h, h->side);
  cudaEventRecord(h->ev_side[k], h->side);
  h->side_recorded[k] = 1;
}
// Join the side kernel of iteration k (if this cycle launched one).
static void wait_side(lsba_ctx* h, int k) {
  if (k >= 1 && h->side_recorded[k]) cudaStreamWaitEvent(h->stream, h->ev_side[k], 0);
}

// One cycle of a lagged skeleton (Alg. 6, 7) on the FP64 tensor-core passes
// (s = 8): CholQR of R_start, iteration 1, iterations k = 2..kmax.  The same
// launches as the generic path; every block's per-tile exponents and digit
// planes are written by the pass that writes the block (the update for the
// basis blocks and U, the digit kernel after the SpMM for W).
static void enqueue_cycle_ftc(lsba_ctx* h, const lsba_csr* A, const double* Rstart, int64_t n,
                              int s, int kmax, int start_flags) {
  cudaStream_t st = h->stream;
  const SmallWs& w = h->ws;
  const int skel = w.skel;
  Ctl* ctl = h->d_ctl;
  const size_t blk = (size_t)n * s;
  const int* Le[LSBA_MAXB];
  const unsigned char* Lp[LSBA_MAXB];
  const unsigned char* Rp[2];
  const int* Re[2];
  do_block_digits(h, Rstart, h->fexp_R0, h->fpl_R0, n, ctl, 0);
  Le[0] = h->fexp_R0;
  Lp[0] = h->fpl_R0;
  do_gram_ftc(h, Lp, Le, 1, Lp, Le, 1, true, n, s, ctl, 0);
  PROF(LSBA_K_SMALL, launch_small_start(st, w, start_flags));
  do_update_ftc(h, Lp, Le, 1, nullptr, n, h->basis, h->fexp, h->fpl, nullptr, nullptr, nullptr,
                w.coef1, w.tri1, nullptr, nullptr, nullptr, ctl, 0);
  if (!lagged(skel)) {
    // BCGS-PIP / BCGS-PIO (Alg. 3: one Gram [V_1..V_k, W]^T W, one update) and
    // BCGS (Sec. 3.1: Gram V^T W, W' = W - V H, CholQR of W'), the same
    // launch sequence as the FP64 kernels with every pass on digit planes
    // (W' kept in U's buffers, which these skeletons use only at the cycle end)
    for (int k = 1; k <= kmax; ++k) {
      const double* Vk = h->basis + (size_t)(k - 1) * blk;
      prof_begin(h, LSBA_K_SPMM);
      launch_spmm_digits(st, A->n, A->d_rowptr, A->d_colidx, A->d_vals, Vk, h->Wb, h->fexp_W, h->fpl_W,
                         ctl, 1);
      prof_end(h);
      for (int i = 0; i < k; ++i) {
        Le[i] = basis_exp(h, n, s, i);
        Lp[i] = basis_planes(h, n, i);
      }
      Le[k] = h->fexp_W;
      Lp[k] = h->fpl_W;
      double* Vnext = h->basis + (size_t)k * blk;
      if (skel == SK_PIP || skel == SK_PIO) {
        // R = [W], the last block of L
        do_gram_ftc(h, Lp, Le, k + 1, Lp + k, Le + k, 1, true, n, s, ctl, 1);
        wait_side(h, k - 1);
        PROF(LSBA_K_SMALL, launch_small_step(st, w, k, 0));
        enqueue_side(h, k);
        do_update_ftc(h, Lp, Le, k + 1, nullptr, n, Vnext, basis_exp(h, n, s, k), basis_planes(h, n, k),
                      nullptr, nullptr, nullptr, w.coef1, w.tri1, nullptr, nullptr, nullptr, ctl, k);
      } else {
        Rp[0] = h->fpl_W;
        Re[0] = h->fexp_W;
        do_gram_ftc(h, Lp, Le, k, Rp, Re, 1, false, n, s, ctl, 1);
        wait_side(h, k - 1);
        PROF(LSBA_K_SMALL, launch_small_step(st, w, k, 0));
        do_update_ftc(h, Lp, Le, k + 1, nullptr, n, h->Ub, h->fexp_U, h->fpl_U, nullptr, nullptr, nullptr,
                      w.coef1, nullptr, nullptr, nullptr, nullptr, ctl, k);
        Rp[0] = h->fpl_U;
        Re[0] = h->fexp_U;
        do_gram_ftc(h, Rp, Re, 1, Rp, Re, 1, true, n, s, ctl, 1);
        PROF(LSBA_K_SMALL, launch_small_step(st, w, k, 1));
        enqueue_side(h, k);
        do_update_ftc(h, Rp, Re, 1, nullptr, n, Vnext, basis_exp(h, n, s, k), basis_planes(h, n, k), nullptr,
                      nullptr, nullptr, w.coef1, w.tri1, nullptr, nullptr, nullptr, ctl, k);
      }
    }
    wait_side(h, kmax);
    return;
  }
  for (int k = 1; k <= kmax; ++k) {
    const double* U = (k == 1) ? h->basis : h->Ub;
    prof_begin(h, LSBA_K_SPMM);
    launch_spmm_digits(st, A->n, A->d_rowptr, A->d_colidx, A->d_vals, U, h->Wb, h->fexp_W, h->fpl_W,
                       ctl, 1);
    prof_end(h);
    if (k == 1) {
      Le[0] = h->fexp;
      Lp[0] = h->fpl;
      Rp[0] = h->fpl_W;
      Re[0] = h->fexp_W;
      do_gram_ftc(h, Lp, Le, 1, Rp, Re, 1, false, n, s, ctl, 1);
      PROF(LSBA_K_SMALL, launch_small_step(st, w, 1, 0));
      Le[1] = h->fexp_W;
      Lp[1] = h->fpl_W;
      do_update_ftc(h, Lp, Le, 2, nullptr, n, h->Ub, h->fexp_U, h->fpl_U, nullptr, nullptr, nullptr,
                    w.coef1, nullptr, nullptr, nullptr, nullptr, ctl, 1);
    } else {
      for (int i = 0; i < k - 1; ++i) {
        Le[i] = basis_exp(h, n, s, i);
        Lp[i] = basis_planes(h, n, i);
      }
      Le[k - 1] = h->fexp_U;
      Lp[k - 1] = h->fpl_U;
      Rp[0] = h->fpl_U;
      Re[0] = h->fexp_U;
      Rp[1] = h->fpl_W;
      Re[1] = h->fexp_W;
      do_gram_ftc(h, Lp, Le, k, Rp, Re, 2, true, n, s, ctl, 1);
      wait_side(h, k - 1);
      PROF(LSBA_K_SMALL, launch_small_step(st, w, k, 0));
      enqueue_side(h, k);
      Le[k] = h->fexp_W;
      Lp[k] = h->fpl_W;
      do_update_ftc(h, Lp, Le, k + 1, nullptr, n, h->basis + (size_t)(k - 1) * blk,
                    basis_exp(h, n, s, k - 1), basis_planes(h, n, k - 1), h->Ub, h->fexp_U, h->fpl_U,
                    w.coef1, w.tri1, w.coef2, w.chain, skel == SK_LS ? w.tri2 : nullptr, ctl, k);
    }
  }
  wait_side(h, kmax);
}

// Enqueue the CholQR of R_start and every loop iteration of one cycle.
static void enqueue_cycle(lsba_ctx* h, const lsba_csr* A, const double* Rstart, int64_t n, int s,
                          int m_cur, int start_flags) {
  cudaStream_t st = h->stream;
  const SmallWs& w = h->ws;
  const int skel = w.skel;
  Ctl* ctl = h->d_ctl;
  h->side_recorded.assign(h->ev_side.size(), 0);
  if (h->use_ftc) {
    enqueue_cycle_ftc(h, A, Rstart, n, s, lagged(skel) ? m_cur + 1 : m_cur, start_flags);
    return;
  }
  BlockPtrs one;
  memset(&one, 0, sizeof(one));
  one.p[0] = Rstart;
  if (w.col_muscle) {
    // V_1 from R_start by the column muscle, in place in the first basis block
    const size_t esz = h->mode == MODE_F32 ? sizeof(float) : sizeof(double);
    cudaMemcpyAsync(h->basis, Rstart, esz * (size_t)n * s, cudaMemcpyDeviceToDevice, st);
    PROF(LSBA_K_GRAM, launch_col_muscle(st, h->basis, h->mode, n, s, skel == SK_LTS, w.mus, ctl,
                                        -1, h->num_sms));
    PROF(LSBA_K_SMALL, launch_small_start(st, w, start_flags));
  } else {
    do_gram(h, one, 1, one, 1, n, s, ctl, 0);
    PROF(LSBA_K_SMALL, launch_small_start(st, w, start_flags));
    do_update(h, one, 1, n, s, h->basis, w.coef1, w.tri1, nullptr, nullptr, nullptr, nullptr, ctl,
              0);
  }
  if (h->use_tcs) split_basis(h, 0, n, s, ctl, 0);
  const int kmax = lagged(skel) ? m_cur + 1 : m_cur;
  const size_t blk = (size_t)n * s;
  for (int k = 1; k <= kmax; ++k) {
    if (skel == SK_SVL || skel == SK_LTS) {
      // Alg. 5: Y = <V_k, W>, H = T^T Y or T^{-T} Y, W <- W - V_k H in place;
      // CholQR of W; Z = <V_k, V_{k+1}> updates T's new block column.
      const double* Vk = h->basis + (size_t)(k - 1) * blk;
      double* Vnext = h->basis + (size_t)k * blk;
      do_spmm(h, A, Vk, h->Wb, s, ctl, 1);
      BlockPtrs L = basis_list(h, n, s, k);
      BlockPtrs R;
      memset(&R, 0, sizeof(R));
      R.p[0] = h->Wb;
      do_gram(h, L, k, R, 1, n, s, ctl, 1);
      wait_side(h, k - 1);
      PROF(LSBA_K_SMALL, launch_small_step(st, w, k, 0));
      BlockPtrs in = basis_list(h, n, s, k);
      in.p[k] = h->Wb;
      do_update(h, in, k + 1, n, s, h->Wb, w.coef1, nullptr, nullptr, nullptr, nullptr, nullptr,
                ctl, k);
      if (w.col_muscle) {
        // MGS-SVL / MGS-LTS on W in place, then V_{k+1} = W
        PROF(LSBA_K_GRAM, launch_col_muscle(st, h->Wb, h->mode, n, s, skel == SK_LTS, w.mus, ctl,
                                            k, h->num_sms));
        PROF(LSBA_K_SMALL, launch_small_step(st, w, k, 1));
        do_update(h, R, 1, n, s, Vnext, w.coef1, nullptr, nullptr, nullptr, nullptr, nullptr, ctl,
                  k);
      } else {
        do_gram(h, R, 1, R, 1, n, s, ctl, 1);
        PROF(LSBA_K_SMALL, launch_small_step(st, w, k, 1));
        do_update(h, R, 1, n, s, Vnext, w.coef1, w.tri1, nullptr, nullptr, nullptr, nullptr, ctl,
                  k);
      }
      BlockPtrs Rn;
      memset(&Rn, 0, sizeof(Rn));
      Rn.p[0] = Vnext;
      do_gram(h, L, k, Rn, 1, n, s, ctl, 1);
      PROF(LSBA_K_SMALL, launch_small_step(st, w, k, 2));
      enqueue_side(h, k);
    } else if (skel == SK_BMGS) {
      // Alg. 2: one Gram and one in-place update per earlier basis block, then CholQR.
      const double* Vk = h->basis + (size_t)(k - 1) * blk;
      do_spmm(h, A, Vk, h->Wb, s, ctl, 1);
      BlockPtrs R;
      memset(&R, 0, sizeof(R));
      R.p[0] = h->Wb;
      for (int jb = 1; jb <= k; ++jb) {
        BlockPtrs L;
        memset(&L, 0, sizeof(L));
        L.p[0] = h->basis + (size_t)(jb - 1) * blk;
        do_gram(h, L, 1, R, 1, n, s, ctl, 1);
        if (jb == 1) wait_side(h, k - 1);
        PROF(LSBA_K_SMALL, launch_small_step(st, w, k, jb - 1));
        BlockPtrs in = L;
        in.p[1] = h->Wb;
        do_update(h, in, 2, n, s, h->Wb, w.coef1, nullptr, nullptr, nullptr, nullptr, nullptr,
                  ctl, k);
      }
      do_gram(h, R, 1, R, 1, n, s, ctl, 1);
      PROF(LSBA_K_SMALL, launch_small_step(st, w, k, k));
      enqueue_side(h, k);
      do_update(h, R, 1, n, s, h->basis + (size_t)k * blk, w.coef1, w.tri1, nullptr, nullptr,
                nullptr, nullptr, ctl, k);
    } else if (skel == SK_PIP || skel == SK_PIO || skel == SK_BCGS) {
      const double* Vk = h->basis + (size_t)(k - 1) * blk;
      do_spmm(h, A, Vk, h->Wb, s, ctl, 1);
      BlockPtrs L = basis_list(h, n, s, k);
      BlockPtrs R;
      memset(&R, 0, sizeof(R));
      R.p[0] = h->Wb;
      BlockPtrs in = basis_list(h, n, s, k);
      in.p[k] = h->Wb;
      double* Vnext = h->basis + (size_t)k * blk;
      if (skel == SK_PIP || skel == SK_PIO) {
        // one fused Gram [V_k W]^T W (for PIO it also gives the muscle's <W, W>)
        L.p[k] = h->Wb;
        do_gram(h, L, k + 1, R, 1, n, s, ctl, 1);
        wait_side(h, k - 1);
        PROF(LSBA_K_SMALL, launch_small_step(st, w, k, 0));
        enqueue_side(h, k);
        do_update(h, in, k + 1, n, s, Vnext, w.coef1, w.tri1, nullptr, nullptr, nullptr, nullptr,
                  ctl, k);
      } else {
        do_gram(h, L, k, R, 1, n, s, ctl, 1);
        wait_side(h, k - 1);
        PROF(LSBA_K_SMALL, launch_small_step(st, w, k, 0));
        do_update(h, in, k + 1, n, s, h->Wb, w.coef1, nullptr, nullptr, nullptr, nullptr, nullptr,
                  ctl, k);
        do_gram(h, R, 1, R, 1, n, s, ctl, 1);
        PROF(LSBA_K_SMALL, launch_small_step(st, w, k, 1));
        enqueue_side(h, k);
        do_update(h, R, 1, n, s, Vnext, w.coef1, w.tri1, nullptr, nullptr, nullptr, nullptr, ctl, k);
      }
    } else {
      const double* U = (k == 1) ? h->basis : h->Ub;
      do_spmm(h, A, U, h->Wb, s, ctl, 1);
      if (k == 1) {
        BlockPtrs L = basis_list(h, n, s, 1);
        BlockPtrs R;
        memset(&R, 0, sizeof(R));
        R.p[0] = h->Wb;
        do_gram(h, L, 1, R, 1, n, s, ctl, 1);
        PROF(LSBA_K_SMALL, launch_small_step(st, w, 1, 0));
        BlockPtrs in = basis_list(h, n, s, 1);
        in.p[1] = h->Wb;
        do_update(h, in, 2, n, s, h->Ub, w.coef1, nullptr, nullptr, nullptr, nullptr, nullptr, ctl,
                  1);
      } else {
        BlockPtrs L = basis_list(h, n, s, k - 1);
        L.p[k - 1] = h->Ub;
        BlockPtrs R;
        memset(&R, 0, sizeof(R));
        R.p[0] = h->Ub;
        R.p[1] = h->Wb;
        // The stored-digit Gram has a fixed cost of about 90 us (its per-chunk
        // chain); below k = 5 the FP32-pipe Gram over the few blocks is faster.
        // An autotuned handle takes the measured shape of iteration k instead.
        const lsba_tune_entry* tk = (h->mode == MODE_DF && h->tune_n == n && h->tune_s == s &&
                                     k < (int)h->tune.size() && h->tune[k].gram_kernel >= 0)
                                        ? &h->tune[k]
                                        : nullptr;
        if (h->use_tcs && gram_tcs_eligible(s, k, 2) && (tk ? tk->gram_kernel == 2 : k >= 5))
          do_gram_tcs(h, k, n, s, ctl);
        else do_gram(h, L, k, R, 2, n, s, ctl, 1, tk && tk->gram_kernel != 2 ? tk : nullptr);
        wait_side(h, k - 1);
        PROF(LSBA_K_SMALL, launch_small_step(st, w, k, 0));
        enqueue_side(h, k);
        BlockPtrs in = basis_list(h, n, s, k - 1);
        in.p[k - 1] = h->Ub;
        in.p[k] = h->Wb;
        double* Vk = h->basis + (size_t)(k - 1) * blk;
        if (h->use_tcs && k >= 2 && update_tcs_eligible(s, k + 1, true)) {
          prof_begin(h, LSBA_K_UPDATE);
          // V_k's digit planes come out of the same pass
          launch_update_tcs(st, h->dig, h->dexp, k - 1, (const float2*)h->Ub,
                            (const float2*)h->Wb, nullptr, n, (float2*)Vk, (float2*)h->Ub, w.coef1,
                            w.tri1, w.coef2, w.chain, skel == SK_LS ? w.tri2 : nullptr, h->cdf,
                            h->dig + (size_t)(k - 1) * digit_block_bytes(n, s),
                            h->dexp + (size_t)(k - 1) * digit_exp_count(n, s), ctl, k,
                            &h->d_ctl->error, h->num_sms,
                            tk && tk->update_kernel == 1 ? tk->update_ctas_per_sm : 0);
          prof_end(h);
        } else {
          do_update(h, in, k + 1, n, s, Vk, w.coef1, w.tri1, h->Ub, w.coef2, w.chain,
                    skel == SK_LS ? w.tri2 : nullptr, ctl, k,
                    tk && tk->update_kernel == 0 ? tk->update_ctas_per_sm : 0);
          if (h->use_tcs) split_basis(h, k - 1, n, s, ctl, k);
        }
      }
    }
  }
  wait_side(h, kmax);
}

// ||B - A X||_F / ||B||_F into ctl->relres_true (X, B in the solve's precision).
static void enqueue_true_residual(lsba_ctx* h, const lsba_csr* A, const double* Bw, const double* Xw,
                                  int64_t n, int s) {
  cudaStream_t st = h->stream;
  do_spmm(h, A, Xw, h->Wb, s, nullptr, 0);
  prof_begin(h, LSBA_K_UPDATE);
  if (h->mode == MODE_DF)
    launch_sub_df(st, n * s, (const float2*)Bw, (const float2*)h->Wb, (float2*)h->Ub);
  else
    launch_axpby(st, n, s, Bw, h->Wb, h->Ub);
  prof_end(h);
  BlockPtrs one;
  memset(&one, 0, sizeof(one));
  one.p[0] = h->Ub;
  do_gram(h, one, 1, one, 1, n, s, nullptr, 0);
  PROF(LSBA_K_SMALL, launch_true_relres(st, h->Gbuf, s, h->d_ctl));
}

extern "C" {

void lsba_default_options(lsba_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->modification = LSBA_GMRES;
  o->max_restarts = 50;
  o->adaptive_restart = 1;
  o->verify_true_residual = 1;
  o->record_history = 0;
  o->inject_flag_cycle = -1;
  o->inject_flag_relation = -1;
  o->profile = 0;
  o->precision = LSBA_PREC_AUTO;
  o->ir_max_outer = 10;
  o->ir_inner_tol = 1e-5;
  o->cuda_graphs = 1;
  o->tensor_cores = 1;
}

const char* lsba_status_string(int st) {
  switch (st) {
    case LSBA_OK: return "ok";
    case LSBA_NOT_CONVERGED: return "not converged";
    case LSBA_BREAKDOWN: return "breakdown: CholQR of B flagged";
    case LSBA_INVALID_ARG: return "invalid argument";
    case LSBA_OUT_OF_MEMORY: return "out of device memory";
    case LSBA_CUDA_ERROR: return "CUDA error";
    case LSBA_DEVICE_TIMEOUT: return "device timeout";
    default: return "unknown status";
  }
}

int lsba_create(lsba_handle* out, int device, void* cuda_stream, const lsba_options* opt) {
  if (!out) return LSBA_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  CK(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return LSBA_INVALID_ARG;
  CK(cudaSetDevice(device));
  lsba_ctx* h = new (std::nothrow) lsba_ctx();
  if (!h) return LSBA_OUT_OF_MEMORY;
  h->device = device;
  h->stream = (cudaStream_t)cuda_stream;
  if (!h->stream) {
    // The legacy default stream cannot be captured into a graph: run on a
    // blocking stream of the handle's own, which the legacy default stream
    // orders implicitly against its own work (same ordering for the caller).
    if (cudaStreamCreate(&h->stream) != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return LSBA_CUDA_ERROR;
    }
    h->own_stream = true;
  }
  if (opt) h->opt = *opt;
  else lsba_default_options(&h->opt);
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaMalloc(&h->d_ctl, sizeof(Ctl)) != cudaSuccess ||
      cudaMallocHost(&h->h_ctl, sizeof(Ctl)) != cudaSuccess ||
      cudaMalloc(&h->d_range, 4 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMallocHost(&h->h_range, 4 * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(h->d_ctl);
    cudaFree(h->d_range);
    cudaFreeHost(h->h_ctl);
    cudaFreeHost(h->h_range);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return LSBA_OUT_OF_MEMORY;
  }
  memset(h->h_ctl, 0, sizeof(Ctl));
  memset(&h->ws, 0, sizeof(h->ws));
  memset(&h->stats, 0, sizeof(h->stats));
  *out = h;
  return LSBA_OK;
}

int lsba_set_options(lsba_handle h, const lsba_options* opt) {
  if (!h || !opt) return LSBA_INVALID_ARG;
  const int old_restarts = h->opt.max_restarts;
  h->opt = *opt;
  if (opt->max_restarts > old_restarts) free_ws(h);  // history capacity depends on it
  return LSBA_OK;
}

int lsba_destroy(lsba_handle h) {
  if (!h) return LSBA_INVALID_ARG;
  cudaSetDevice(h->device);
  free_ws(h);
  cudaFree(h->d_ctl);
  cudaFreeHost(h->h_ctl);
  cudaFree(h->d_range);
  cudaFreeHost(h->h_range);
  ws_free(h, h->hA_rowptr);
  ws_free(h, h->hA_colidx);
  ws_free(h, h->hA_vals);
  ws_free(h, h->hB);
  ws_free(h, h->hX);
  ws_free(h, h->A_df);
  cudaStreamSynchronize(h->stream);
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  for (cudaEvent_t e : h->ev_main) cudaEventDestroy(e);
  for (cudaEvent_t e : h->ev_side) cudaEventDestroy(e);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
  return LSBA_OK;
}

static int skel_code(lsba_skeleton s) {
  switch (s) {
    case LSBA_BCGS: return SK_BCGS;
    case LSBA_BCGS_PIP: return SK_PIP;
    case LSBA_BCGSI_LS: return SK_LS;
    case LSBA_BMGS_ICWY: return SK_ICWY;
    case LSBA_BMGS_CWY: return SK_CWY;
    case LSBA_BMGS: return SK_BMGS;
    case LSBA_BCGS_PIO: return SK_PIO;
    case LSBA_BMGS_SVL: return SK_SVL;
    case LSBA_BMGS_LTS: return SK_LTS;
    default: return -1;
  }
}

// One restart cycle: control record to the device, the cycle's launches, the
// control record back, one host synchronisation.  With options.cuda_graphs the
// sequence is captured into a CUDA graph the second time its key is seen
// (stream capture in thread-local mode, so solves on other host threads are
// not disturbed) and replayed from then on; the copies of the pinned control
// record are part of the graph and read/write it when the graph runs.
static int run_cycle_body(lsba_handle h, const lsba_csr* A, const double* Rstart, int64_t n,
                          int s, int m_cur, int start_flags) {
  cudaStream_t st = h->stream;
  CycleGraph* g = nullptr;
  if (h->opt.cuda_graphs && !h->opt.profile) {
    CycleKey key;
    memset(&key, 0, sizeof(key));
    key.rowptr = A->d_rowptr;
    key.colidx = A->d_colidx;
    key.vals = A->d_vals;
    key.a_lowprec = h->mode == MODE_FP64 ? nullptr : h->A_df;
    key.rstart = Rstart;
    key.n = n;
    key.s = s;
    key.m_cur = m_cur;
    key.start_flags = start_flags;
    key.skel = h->ws.skel;
    key.modification = h->ws.modification;
    key.mode = h->mode;
    key.tensor_cores = h->opt.tensor_cores;
    key.global_ip = h->ws.global_ip;
    key.col_muscle = h->ws.col_muscle;
    key.pad = h->tune_gen;
    key.ws_gen = h->ws_gen;
    for (auto& e : h->graphs)
      if (e.key == key) g = &e;
    if (!g) {
      if (h->graphs.size() >= LSBA_MAX_CYCLE_GRAPHS) {
        size_t old = 0;
        for (size_t i = 1; i < h->graphs.size(); ++i)
          if (h->graphs[i].last_use < h->graphs[old].last_use) old = i;
        if (h->graphs[old].exec) cudaGraphExecDestroy(h->graphs[old].exec);
        h->graphs.erase(h->graphs.begin() + old);
      }
      h->graphs.push_back(CycleGraph{key, nullptr, ++h->graph_clock, false});
      g = nullptr;  // first sighting: issue directly
    } else {
      g->last_use = ++h->graph_clock;
      if (!g->exec && !g->failed) {
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          cudaMemcpyAsync(h->d_ctl, h->h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, st);
          enqueue_cycle(h, A, Rstart, n, s, m_cur, start_flags);
          cudaMemcpyAsync(h->h_ctl, h->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
          e = cudaStreamEndCapture(st, &graph);
        }
        cudaGraphExec_t exec = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
          cudaGetLastError();
          if (exec) cudaGraphExecDestroy(exec);
          g->failed = true;
        } else {
          g->exec = exec;
        }
      }
      if (g->failed) g = nullptr;
    }
  }
  if (g && g->exec) {
    CK(cudaGraphLaunch(g->exec, st));
    CK(cudaStreamSynchronize(st));
    return LSBA_OK;
  }
  int rc;
  if ((rc = push_ctl(h)) != LSBA_OK) return rc;
  enqueue_cycle(h, A, Rstart, n, s, m_cur, start_flags);
  CK(cudaGetLastError());
  return pull_ctl(h);
}

// Restart cycles of one (inner) solve of A X = B in the current working
// precision (h->mode), from X = 0.  Bw, Xw: B and X in that precision.
// Accumulates into h->stats; history of the first cycle when record_first.
static int run_cycles(lsba_handle h, const lsba_csr* A, const double* Bw, double* Xw, int64_t n,
                      int s, int m, double tol, bool verify, bool record_first, int* status_out) {
  SmallWs& w = h->ws;
  const int skel = w.skel;
  cudaStream_t st = h->stream;
  Ctl* c = h->h_ctl;
  lsba_stats& S = h->stats;
  const int vper = (skel == SK_LS) ? 4
                   : (skel == SK_PIP || skel == SK_PIO || skel == SK_SVL || skel == SK_LTS ||
                      lagged(skel))
                       ? 3
                       : 2;
  const int vcyc = lagged(skel) ? 1 : 0;
  int rc;
  CK(cudaMemsetAsync(Xw, 0, sizeof(double) * (size_t)n * s, st));
  c->tol = tol;
  c->update_step = -1;
  c->side_step = -1;
  int m_cur = m;
  const double* Rstart = Bw;
  int start_flags = 3;
  int status = LSBA_NOT_CONVERGED;
  int cycle = 0;
  while (true) {
    ++cycle;
    if (cycle > h->opt.max_restarts + 1) {
      status = LSBA_NOT_CONVERGED;
      --cycle;
      break;
    }
    c->cycle = cycle;
    c->record = (record_first && h->opt.record_history) ? 1 : 0;
    c->m_cur = m_cur;
    c->inject_relation = (cycle == h->opt.inject_flag_cycle) ? h->opt.inject_flag_relation : -1;
    c->muscle_syncs = 0;
    const int stall = (cycle == 1 && h->opt.inject_stall) ? 4 : 0;
    if ((rc = run_cycle_body(h, A, Rstart, n, s, m_cur, start_flags | stall)) != LSBA_OK) return rc;
    if (c->error) return LSBA_DEVICE_TIMEOUT;
    // the start block's muscle: CholQR one sync; the column muscle counts its
    // own syncs on the device (the start's and every step's)
    S.syncs += w.col_muscle ? c->muscle_syncs : 1;
    S.cycles += 1;
    if (c->start_flag) {
      status = (cycle == 1) ? LSBA_BREAKDOWN : LSBA_NOT_CONVERGED;
      break;
    }
    const int j = c->j;
    const int f = c->flagged ? 1 : 0;
    S.flags += f;
    h->h_cycle_m.push_back(j);
    h->h_cycle_flag.push_back(c->flagged);
    h->h_cycle_mcur.push_back(m_cur);
    S.steps += j;
    const int a_calls = lagged(skel) ? j + 1 + f : j + f;
    S.a_calls += a_calls;
    S.syncs += (skel == SK_SVL || skel == SK_LTS)
                   ? (w.col_muscle ? 2 * a_calls - f : 3 * a_calls - f)   // Y, (muscle), Z; a flagged step has no Z
               : (skel == SK_BCGS || skel == SK_PIO) ? 2 * a_calls
               : (skel == SK_BMGS) ? a_calls * (a_calls + 3) / 2   // k + 1 in step k
                                   : a_calls;
    S.v_apps += vper * j + (j > 0 ? vcyc : 0);
    if (!std::isnan(c->est)) S.relres_est = c->est;
    if (cycle == 1 && record_first && h->opt.record_history) {
      h->first_j = j;
      if (j > 0) {
        const int rows = (j + 1) * s, cols = j * s;
        h->h_first_H.resize((size_t)rows * cols);
        CK(cudaMemcpy2D(h->h_first_H.data(), sizeof(double) * rows, w.H, sizeof(double) * w.ldH,
                        sizeof(double) * rows, cols, cudaMemcpyDeviceToHost));
      }
      h->h_first_beta.resize((size_t)s * s);
      CK(cudaMemcpy(h->h_first_beta.data(), w.Bcyc, sizeof(double) * s * s, cudaMemcpyDeviceToHost));
    }
    if (c->flagged && h->opt.adaptive_restart) m_cur = c->flagged - 1;
    if (j == 0) {
      status = LSBA_NOT_CONVERGED;
      break;
    }
    if (w.modification == 0 && c->fom_singular) {
      status = LSBA_NOT_CONVERGED;
      break;
    }
    // Cycle end: X += V_j Xi C, U = V_{j+1} [M; -H], C <- c C.
    PROF(LSBA_K_SMALL, launch_small_end(st, w));
    if (h->use_ftc) {
      // on the FP64 tensor-core update; X's own term in FP64
      const unsigned char* Lp[LSBA_MAXB];
      const int* Le[LSBA_MAXB];
      for (int i = 0; i <= j; ++i) {
        Lp[i] = basis_planes(h, n, i);
        Le[i] = basis_exp(h, n, s, i);
      }
      do_update_ftc(h, Lp, Le, j + 1, Xw, n, Xw, nullptr, nullptr, h->Ub, h->fexp_U, h->fpl_U,
                    w.coef1, nullptr, w.coef2, nullptr, nullptr, h->d_ctl, LSBA_END_STEP);
    } else if (h->use_tcs && update_tcs_eligible(s, j + 1, true)) {
      // on the stored digit planes of V_1..V_{j+1}; X's own term in double-float
      prof_begin(h, LSBA_K_UPDATE);
      launch_update_tcs(st, h->dig, h->dexp, j + 1, nullptr, nullptr, (const float2*)Xw, n,
                        (float2*)Xw, (float2*)h->Ub, w.coef1, nullptr, w.coef2, nullptr, nullptr,
                        h->cdf, nullptr, nullptr, h->d_ctl, LSBA_END_STEP, &h->d_ctl->error,
                        h->num_sms);
      prof_end(h);
    } else {
      BlockPtrs in = basis_list(h, n, s, j + 1);
      in.p[j + 1] = Xw;
      do_update(h, in, j + 2, n, s, Xw, w.coef1, nullptr, h->Ub, w.coef2, nullptr, nullptr,
                h->d_ctl, LSBA_END_STEP);
    }
    CK(cudaGetLastError());
    if (c->flagged && !h->opt.adaptive_restart) {
      status = LSBA_NOT_CONVERGED;
      break;
    }
    if (c->converged) {
      if (verify) {
        enqueue_true_residual(h, A, Bw, Xw, n, s);
        if ((rc = pull_ctl(h)) != LSBA_OK) return rc;
        S.relres_true = c->relres_true;
        if (!(c->relres_true <= tol)) {
          Rstart = h->Ub;
          start_flags = 2;
          continue;
        }
      }
      status = LSBA_OK;
      break;
    }
    Rstart = h->Ub;
    start_flags = 0;
  }
  S.m_final = m_cur;
  *status_out = status;
  return LSBA_OK;
}

static int ensure_lowprec_A(lsba_handle h, const lsba_csr* A) {
  if ((size_t)A->nnz > h->A_df_cap) {
    ws_free(h, h->A_df);
    h->A_df = nullptr;
    h->A_df_cap = 0;
    if (ws_alloc(h, &h->A_df, sizeof(float2) * (A->nnz > 0 ? A->nnz : 1)) != cudaSuccess) {
      cudaGetLastError();
      return LSBA_OUT_OF_MEMORY;
    }
    h->A_df_cap = A->nnz;
  }
  return LSBA_OK;
}

// FP64 residual R = B - A X into Ub (double) and its norm ratio into
// ctl->relres_true (ratio to ctl->outer_normB; outer = 1 first stores ||B||).
static void enqueue_fp64_residual(lsba_ctx* h, const lsba_csr* A, const double* d_B,
                                  const double* d_X, int64_t n, int s, bool norm_of_B) {
  cudaStream_t st = h->stream;
  BlockPtrs one;
  memset(&one, 0, sizeof(one));
  const int mode = h->mode;
  h->mode = MODE_FP64;
  if (norm_of_B) {
    one.p[0] = d_B;
    do_gram(h, one, 1, one, 1, n, s, nullptr, 0);
    PROF(LSBA_K_SMALL, launch_outer_norm(st, h->Gbuf, s, h->d_ctl, 0));
  }
  do_spmm(h, A, d_X, h->Wb, s, nullptr, 0);
  PROF(LSBA_K_UPDATE, launch_axpby(st, n, s, d_B, h->Wb, h->Ub));
  one.p[0] = h->Ub;
  do_gram(h, one, 1, one, 1, n, s, nullptr, 0);
  PROF(LSBA_K_SMALL, launch_outer_norm(st, h->Gbuf, s, h->d_ctl, 1));
  h->mode = mode;
}

// Magnitude ranges of A's values and of B (one pass each, one host sync):
// amax, amin (smallest nonzero) of A and bmax of B; false if either holds a
// non-finite value.
static int input_ranges(lsba_ctx* h, const lsba_csr* A, const double* d_B, int64_t count_b,
                        double* amax, double* amin, double* bmax, bool* finite) {
  cudaStream_t st = h->stream;
  unsigned long long init[4] = {0ull, ~0ull, 0ull, ~0ull};
  memcpy(h->h_range, init, sizeof(init));
  CK(cudaMemcpyAsync(h->d_range, h->h_range, sizeof(init), cudaMemcpyHostToDevice, st));
  launch_absrange(st, A->nnz, A->d_vals, h->d_range, h->num_sms);
  launch_absrange(st, count_b, d_B, h->d_range + 2, h->num_sms);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(h->h_range, h->d_range, sizeof(init), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const unsigned long long inf_bits = 0x7FF0000000000000ull;
  *finite = h->h_range[0] < inf_bits && h->h_range[2] < inf_bits;
  double v[4];
  memcpy(v, h->h_range, sizeof(v));
  *amax = v[0];
  *amin = h->h_range[1] == ~0ull ? 0.0 : v[1];
  *bmax = v[2];
  return LSBA_OK;
}

// The power of two 2^p applied to an input whose largest magnitude is x: none
// (p = 0) while x is in [2^-32, 2^32], where every Gram of the solve stays far
// inside FP32's exponent range (for n up to 2^30 and s <= 32), else p with
// x 2^p in [1, 2).  p = 0 for x = 0 or non-finite x.
static int unit_scale_exp(double x) {
  if (!(x > 0.0) || !std::isfinite(x)) return 0;
  if (x >= std::ldexp(1.0, -32) && x <= std::ldexp(1.0, 32)) return 0;
  return -std::ilogb(x);
}

static int solve_impl(lsba_handle h, const lsba_csr* A, const double* d_B, double* d_X, int s, int m,
                      double tol, lsba_skeleton skel_in) {
  auto t0 = std::chrono::steady_clock::now();
  memset(&h->stats, 0, sizeof(h->stats));
  h->stats.relres_true = NAN;
  h->stats.relres_est = NAN;
  const int skel = skel_code(skel_in);
  if (!A || !d_B || !d_X || skel < 0 || s < 1 || s > LSBA_MAX_S || m < 1 ||
      (int64_t)(m + 1) * s > LSBA_MAX_MS || m + 3 > LSBA_MAXB || A->n < 1 || A->nnz < 0 ||
      A->nnz >= (int64_t)1 << 31 || !A->d_rowptr || (A->nnz > 0 && (!A->d_colidx || !A->d_vals)) ||
      !(tol >= 0.0) || h->opt.max_restarts < 0 ||
      (h->opt.inner_product != LSBA_IP_CLASSICAL && h->opt.inner_product != LSBA_IP_GLOBAL) ||
      (h->opt.muscle != LSBA_MUSCLE_CHOLQR &&
       (h->opt.muscle != LSBA_MUSCLE_COLUMN || (skel != SK_SVL && skel != SK_LTS) ||
        h->opt.inner_product != LSBA_IP_CLASSICAL)))
    return h->stats.status = LSBA_INVALID_ARG;
  const int64_t n = A->n;
  CK(cudaSetDevice(h->device));
  int rc = ensure_ws(h, n, s, m);
  if (rc != LSBA_OK) return h->stats.status = rc;
  SmallWs& w = h->ws;
  w.skel = skel;
  w.modification = h->opt.modification == LSBA_FOM ? 0 : 1;
  w.global_ip = h->opt.inner_product == LSBA_IP_GLOBAL ? 1 : 0;
  w.col_muscle = h->opt.muscle == LSBA_MUSCLE_COLUMN ? 1 : 0;
  cudaStream_t st = h->stream;
  const size_t blk = (size_t)n * s;
  // Working precision of the SpMM / Gram / update passes.
  const int prec = h->opt.precision;
  // The double-float kernels take every s (coefficient sets too large for
  // shared memory are read from global memory); the FP32 inner solver has
  // row kernels for s = 4, 8, 16 only and otherwise runs in double-float.
  const bool fits_f32 = (s == 4 || s == 8 || s == 16) && update_f32_smem(m + 3, s, true) <= 200 * 1024;
  const bool ir = prec == LSBA_PREC_FP32_IR && fits_f32;
  // Shapes the FP64 tensor-core passes take (the lagged skeletons, BCGS-PIP,
  // BCGS-PIO and BCGS; s = 8, m <= 22): under "auto" the lagged ones run
  // there, in FP64, rather than in double-float (they are faster on GB300 and
  // keep 53 bits); the others run in FP64 anyway.
  const bool ftc_skel = lagged(skel) || skel == SK_PIP || skel == SK_PIO || skel == SK_BCGS;
  const bool ftc_shape = s == 8 && h->opt.tensor_cores != 0 && ftc_skel &&
                         gram_f64tc_eligible(s, m + 1, 2, true) && update_f64tc_eligible(s, m + 2);
  if (ir) h->mode = MODE_F32;
  else if (prec == LSBA_PREC_DF || prec == LSBA_PREC_FP32_IR ||
           (prec == LSBA_PREC_AUTO && lagged(skel) && !ftc_shape))
    h->mode = MODE_DF;
  else h->mode = MODE_FP64;
  // Low-precision modes keep FP32's exponent range (2^-126 .. 2^128): A and B
  // whose largest magnitudes lie outside [2^-32, 2^32] are scaled by powers of
  // two (exact) to magnitudes near 1, and X is scaled back (the first cycle's
  // recorded Grams and Hessenberg are then those of the scaled problem).
  // Under "auto", double-float is taken only if
  // A's nonzero magnitudes then stay above 2^-90 (the low words of double-float
  // values keep their bits down to about 2^-102) and the inputs are finite;
  // otherwise the solve runs in FP64.
  int pA = 0, pB = 0;
  if (h->mode != MODE_FP64) {
    double amax = 0, amin = 0, bmax = 0;
    bool finite = true;
    if ((rc = input_ranges(h, A, d_B, (int64_t)blk, &amax, &amin, &bmax, &finite)) !=
        LSBA_OK)
      return h->stats.status = rc;
    pA = unit_scale_exp(amax);
    pB = unit_scale_exp(bmax);
    const bool spread_ok = amin == 0.0 || std::ldexp(amin, pA) >= std::ldexp(1.0, -90);
    if (prec == LSBA_PREC_AUTO && (!finite || !spread_ok)) {
      h->mode = MODE_FP64;
      pA = pB = 0;
    }
  }
  h->stats.precision = ir ? LSBA_PREC_FP32_IR : h->mode == MODE_DF ? LSBA_PREC_DF : LSBA_PREC_FP64;
  // Tensor-core Gram on stored digit planes: double-float lagged skeletons, s = 8.
  h->use_tcs = h->mode == MODE_DF && s == 8 && h->opt.tensor_cores != 0 && lagged(skel);
  if (h->use_tcs && ensure_digits(h) != LSBA_OK) h->use_tcs = false;
  // FP64 on the tensor cores: the skeletons above at s = 8, m <= 22.
  h->use_ftc = h->mode == MODE_FP64 && ftc_shape;
  if (h->use_ftc && ensure_f64tc(h) != LSBA_OK) h->use_ftc = false;
  h->stats.tensor_cores = (h->use_tcs || h->use_ftc) ? 1 : 0;

  Ctl* c = h->h_ctl;
  const int hist_cap = c->hist_cap, gram_cap = c->gram_hist_cap;
  memset(c, 0, sizeof(Ctl));
  c->hist_cap = hist_cap;
  c->gram_hist_cap = gram_cap;
  h->h_est.clear();
  h->h_est_cycle.clear();
  h->h_est_j.clear();
  h->h_cycle_m.clear();
  h->h_cycle_flag.clear();
  h->h_cycle_mcur.clear();
  h->h_first_H.clear();
  h->h_first_beta.clear();
  h->h_gram_data.clear();
  h->h_gram_rows.clear();
  h->h_gram_cols.clear();
  h->first_j = 0;
  lsba_stats& S = h->stats;
  int status = LSBA_NOT_CONVERGED;

  if (!ir) {
    const double* Bw = d_B;
    double* Xw = d_X;
    if (h->mode == MODE_DF) {
      if ((rc = ensure_lowprec_A(h, A)) != LSBA_OK) return S.status = rc;
      PROF(LSBA_K_UPDATE, launch_to_df(st, A->nnz, A->d_vals, h->A_df, std::ldexp(1.0, pA)));
      PROF(LSBA_K_UPDATE, launch_to_df(st, n * s, d_B, (float2*)h->Bdf, std::ldexp(1.0, pB)));
      Bw = h->Bdf;
      Xw = h->Xdf;
    }
    if ((rc = run_cycles(h, A, Bw, Xw, n, s, m, tol, h->opt.verify_true_residual != 0, true,
                         &status)) != LSBA_OK)
      return S.status = rc;
    // (2^pA A) X' = 2^pB B, so X = 2^(pA - pB) X'
    if (h->mode == MODE_DF)
      PROF(LSBA_K_UPDATE,
           launch_from_df(st, n * s, (const float2*)Xw, d_X, std::ldexp(1.0, pA - pB)));
    // True residual of the returned X (FP64).
    enqueue_fp64_residual(h, A, d_B, d_X, n, s, true);
    if ((rc = pull_ctl(h)) != LSBA_OK) return S.status = rc;
    S.relres_true = c->relres_true;
  } else {
    // FP64 iterative refinement around an FP32 inner BGMRES/BFOM:
    //   R = B - A X (FP64);  solve A D = R in FP32 to ir_inner_tol;  X += D (FP64).
    if ((rc = ensure_lowprec_A(h, A)) != LSBA_OK) return S.status = rc;
    PROF(LSBA_K_UPDATE, launch_to_f32(st, A->nnz, A->d_vals, (float*)h->A_df, std::ldexp(1.0, pA)));
    CK(cudaMemsetAsync(d_X, 0, sizeof(double) * blk, st));
    const double inner_tol = h->opt.ir_inner_tol > 0 ? h->opt.ir_inner_tol : 1e-5;
    const int max_outer = h->opt.ir_max_outer > 0 ? h->opt.ir_max_outer : 10;
    double prev = INFINITY;
    for (int it = 0; it <= max_outer; ++it) {
      enqueue_fp64_residual(h, A, d_B, d_X, n, s, it == 0);
      if ((rc = pull_ctl(h)) != LSBA_OK) return S.status = rc;
      S.relres_true = c->relres_true;
      if (c->relres_true <= tol) {
        status = LSBA_OK;
        break;
      }
      if (it == max_outer || !(c->relres_true < prev)) break;
      prev = c->relres_true;
      S.ir_outer += 1;
      // Inner FP32 solve of (2^pA A) D' = 2^pR R, R scaled as A is (by its
      // Frobenius norm) when outside [2^-32, 2^32] (R in Ub as FP64 -> FP32
      // into Bdf); then D = 2^(pA - pR) D'.
      const int pR = unit_scale_exp(c->relres_true * c->outer_normB);
      PROF(LSBA_K_UPDATE, launch_to_f32(st, n * s, h->Ub, (float*)h->Bdf, std::ldexp(1.0, pR)));
      int inner_status = 0;
      if ((rc = run_cycles(h, A, h->Bdf, h->Xdf, n, s, m, inner_tol, false, it == 0,
                           &inner_status)) != LSBA_OK)
        return S.status = rc;
      if (inner_status == LSBA_BREAKDOWN) break;
      PROF(LSBA_K_UPDATE,
           launch_add_f32(st, n * s, (const float*)h->Xdf, d_X, std::ldexp(1.0, pA - pR)));
    }
  }
  S.status = status;
  CK(cudaStreamSynchronize(st));
  if (h->opt.record_history) {
    const int ne = c->n_hist;
    h->h_est.resize(ne);
    h->h_est_cycle.resize(ne);
    h->h_est_j.resize(ne);
    if (ne > 0) {
      CK(cudaMemcpy(h->h_est.data(), w.hist_est, sizeof(double) * ne, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(h->h_est_cycle.data(), w.hist_cycle, sizeof(int) * ne, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(h->h_est_j.data(), w.hist_j, sizeof(int) * ne, cudaMemcpyDeviceToHost));
    }
    const int ng = c->n_gram_hist;
    std::vector<int> dims(2 * ng);
    if (ng > 0)
      CK(cudaMemcpy(dims.data(), w.gram_dims, sizeof(int) * 2 * ng, cudaMemcpyDeviceToHost));
    h->h_gram_rows.resize(ng);
    h->h_gram_cols.resize(ng);
    for (int i = 0; i < ng; ++i) {
      h->h_gram_rows[i] = dims[2 * i];
      h->h_gram_cols[i] = dims[2 * i + 1];
    }
    h->h_gram_data.resize(c->gram_hist_used);
    if (c->gram_hist_used > 0)
      CK(cudaMemcpy(h->h_gram_data.data(), w.gram_hist, sizeof(double) * c->gram_hist_used,
                    cudaMemcpyDeviceToHost));
  }
  auto t1 = std::chrono::steady_clock::now();
  S.solve_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  return status;
}

int lsba_solve(lsba_handle h, const lsba_csr* A, const double* d_B, double* d_X, int s, int m,
               double tol, lsba_skeleton skel) {
  if (!h) return LSBA_INVALID_ARG;
  return solve_impl(h, A, d_B, d_X, s, m, tol, skel);
}

int lsba_solve_host(lsba_handle h, int64_t n, int64_t nnz, const int32_t* h_rowptr,
                    const int32_t* h_colidx, const double* h_vals, const double* h_B, double* h_X,
                    int s, int m, double tol, lsba_skeleton skel) {
  if (!h || n < 1 || nnz < 0 || !h_rowptr || !h_B || !h_X || s < 1 || s > LSBA_MAX_S ||
      (nnz > 0 && (!h_colidx || !h_vals)))
    return LSBA_INVALID_ARG;
  CK(cudaSetDevice(h->device));
  if (n != h->host_n || nnz != h->host_nnz || s != h->host_s) {
    ws_free(h, h->hA_rowptr);
    ws_free(h, h->hA_colidx);
    ws_free(h, h->hA_vals);
    ws_free(h, h->hB);
    ws_free(h, h->hX);
    h->hA_rowptr = nullptr;
    h->hA_colidx = nullptr;
    h->hA_vals = nullptr;
    h->hB = h->hX = nullptr;
    h->host_n = h->host_nnz = 0;
    if (ws_alloc(h, &h->hA_rowptr, sizeof(int32_t) * (n + 1)) != cudaSuccess ||
        ws_alloc(h, &h->hA_colidx, sizeof(int32_t) * (nnz > 0 ? nnz : 1)) != cudaSuccess ||
        ws_alloc(h, &h->hA_vals, sizeof(double) * (nnz > 0 ? nnz : 1)) != cudaSuccess ||
        ws_alloc(h, &h->hB, sizeof(double) * n * s) != cudaSuccess ||
        ws_alloc(h, &h->hX, sizeof(double) * n * s) != cudaSuccess) {
      cudaGetLastError();
      return LSBA_OUT_OF_MEMORY;
    }
    h->host_n = n;
    h->host_nnz = nnz;
    h->host_s = s;
  }
  cudaStream_t st = h->stream;
  CK(cudaMemcpyAsync(h->hA_rowptr, h_rowptr, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, st));
  if (nnz > 0) {
    CK(cudaMemcpyAsync(h->hA_colidx, h_colidx, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(h->hA_vals, h_vals, sizeof(double) * nnz, cudaMemcpyHostToDevice, st));
  }
  CK(cudaMemcpyAsync(h->hB, h_B, sizeof(double) * n * s, cudaMemcpyHostToDevice, st));
  lsba_csr A;
  A.n = n;
  A.nnz = nnz;
  A.d_rowptr = h->hA_rowptr;
  A.d_colidx = h->hA_colidx;
  A.d_vals = h->hA_vals;
  int rc = solve_impl(h, &A, h->hB, h->hX, s, m, tol, skel);
  if (rc == LSBA_INVALID_ARG || rc == LSBA_CUDA_ERROR || rc == LSBA_OUT_OF_MEMORY) return rc;
  CK(cudaMemcpyAsync(h_X, h->hX, sizeof(double) * n * s, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return rc;
}

int lsba_release_workspace(lsba_handle h) {
  if (!h) return LSBA_INVALID_ARG;
  CK(cudaSetDevice(h->device));
  free_ws(h);
  ws_free(h, h->A_df);
  h->A_df = nullptr;
  h->A_df_cap = 0;
  ws_free(h, h->hA_rowptr);
  ws_free(h, h->hA_colidx);
  ws_free(h, h->hA_vals);
  ws_free(h, h->hB);
  ws_free(h, h->hX);
  h->hA_rowptr = h->hA_colidx = nullptr;
  h->hA_vals = h->hB = h->hX = nullptr;
  h->host_n = h->host_nnz = 0;
  h->host_s = 0;
  CK(cudaGetLastError());
  return LSBA_OK;
}

int64_t lsba_workspace_bytes(int64_t n, int64_t nnz, int s, int m) {
  if (n < 1 || s < 1 || s > LSBA_MAX_S || m < 1 || nnz < 0) return -1;
  // Every allocation of ensure_ws / ensure_lowprec_A at the largest settings:
  // basis (m+1 blocks), W, U, the low-precision B and X copies, the
  // low-precision matrix values, the small matrices with a full restart
  // history, the Gram partials of the largest plan, the converted update
  // coefficients and the integer history arrays.
  int num_sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      num_sms < 1) {
    cudaGetLastError();
    num_sms = 256;  // no device visible: a bound above any current part
  }
  const int64_t blk = n * s * (int64_t)sizeof(double);
  int64_t bytes = blk * (m + 5);
  bytes += (int64_t)sizeof(float2) * (nnz > 0 ? nnz : 1);
  const SmallLayout L = small_layout(s, m, LSBA_HIST_RESTARTS);
  bytes += (int64_t)(L.total * sizeof(double));
  size_t qmax = 0;
  const size_t partials = max_partials(n, s, m, num_sms, &qmax);
  bytes += (int64_t)((partials + qmax) * sizeof(double));
  bytes += (int64_t)(coef_df_count(m + 3, s, true) * sizeof(float2));
  bytes += (int64_t)((2 * L.hist_cap + 2 * (m + 4)) * sizeof(int));
  if (s == 8) {  // stored digit planes of the basis (double-float tensor-core Gram)
    bytes += (int64_t)((m + 1) * (digit_block_bytes(n, s) + sizeof(int) * digit_exp_count(n, s)));
    // exponents, digit planes and FP64 coefficients of the FP64 tensor-core passes
    bytes += (int64_t)(sizeof(int) * (size_t)(m + 4) * f64tc_exp_count(n, s) +
                       (size_t)(m + 4) * f64tc_plane_bytes(n) +
                       sizeof(double) * 2 * 8 * (size_t)(m + 3) * 8);
  }
  return bytes;
}

int lsba_get_profile(lsba_handle h, double* ms, int64_t* launches, int nclass) {
  if (!h || nclass < 0 || nclass > LSBA_K_NCLASS || (nclass > 0 && (!ms || !launches)))
    return LSBA_INVALID_ARG;
  for (int i = 0; i < nclass; ++i) {
    ms[i] = h->prof_ms[i];
    launches[i] = h->prof_n[i];
  }
  return LSBA_OK;
}

int lsba_reset_profile(lsba_handle h) {
  if (!h) return LSBA_INVALID_ARG;
  for (int i = 0; i < LSBA_K_NCLASS; ++i) {
    h->prof_ms[i] = 0.0;
    h->prof_n[i] = 0;
  }
  return LSBA_OK;
}

int lsba_get_stats(lsba_handle h, lsba_stats* out) {
  if (!h || !out) return LSBA_INVALID_ARG;
  *out = h->stats;
  return LSBA_OK;
}

int lsba_get_history(lsba_handle h, lsba_history* out) {
  if (!h || !out) return LSBA_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  out->n_est = (int32_t)h->h_est.size();
  out->est = h->h_est.data();
  out->est_cycle = h->h_est_cycle.data();
  out->est_j = h->h_est_j.data();
  out->n_cycles = (int32_t)h->h_cycle_m.size();
  out->cycle_m = h->h_cycle_m.data();
  out->cycle_flag = h->h_cycle_flag.data();
  out->cycle_mcur = h->h_cycle_mcur.data();
  out->first_j = h->first_j;
  out->first_H = h->h_first_H.data();
  out->first_beta = h->h_first_beta.data();
  out->n_grams = (int32_t)h->h_gram_rows.size();
  out->gram_rows = h->h_gram_rows.data();
  out->gram_cols = h->h_gram_cols.data();
  out->gram_data = h->h_gram_data.data();
  return LSBA_OK;
}

// ---------------------------------------------------------------- kernel-level entry points

int lsba_spmm(lsba_handle h, const lsba_csr* A, const double* d_V, double* d_W, int s) {
  if (!h || !A || !d_V || !d_W || s < 1 || s > LSBA_MAX_S || A->n < 1 || !A->d_rowptr ||
      (A->nnz > 0 && (!A->d_colidx || !A->d_vals)))
    return LSBA_INVALID_ARG;
  CK(cudaSetDevice(h->device));
  launch_spmm(h->stream, A->n, A->d_rowptr, A->d_colidx, A->d_vals, d_V, d_W, s, nullptr, 0);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  return LSBA_OK;
}

int lsba_gram(lsba_handle h, const double* d_L, int a, const double* d_R, int b, int64_t n, int s,
              double* d_G) {
  if (!h || !d_L || !d_R || !d_G || a < 1 || b < 1 || b > 2 || s < 1 || s > LSBA_MAX_S || n < 1 ||
      a + b > LSBA_MAXB || (int64_t)a * s > LSBA_MAX_MS)
    return LSBA_INVALID_ARG;
  CK(cudaSetDevice(h->device));
  GramPlan p = plan_gram(n, s, a, b, h->num_sms);
  const size_t need = (size_t)p.grid_x * p.q;
  if (need > h->partials_cap) {
    ws_free(h, h->partials);
    h->partials = nullptr;
    h->partials_cap = 0;
    if (ws_alloc(h, &h->partials, sizeof(double) * need) != cudaSuccess) {
      cudaGetLastError();
      return LSBA_OUT_OF_MEMORY;
    }
    h->partials_cap = need;
  }
  BlockPtrs L, R;
  memset(&L, 0, sizeof(L));
  memset(&R, 0, sizeof(R));
  for (int i = 0; i < a; ++i) L.p[i] = d_L + (size_t)i * n * s;
  for (int i = 0; i < b; ++i) R.p[i] = d_R + (size_t)i * n * s;
  launch_gram(h->stream, p, L, a, R, b, n, s, h->partials, d_G, nullptr, 0);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  return LSBA_OK;
}

// Measured kernel choices for the double-float lagged skeletons at s = 8: for
// every iteration k = 2..m+1, the stored-digit tensor-core Gram against the
// FP32-pipe Gram of [V_1..V_{k-1}, U]^T [U, W], and the tensor-core update with
// two against three CTAs per SM where three fit.  Each candidate runs once to
// warm up and three times under CUDA events on the handle's stream, on
// pseudo-random operands of the solve's shape (every digit busy) and their
// stored digit planes.
int lsba_autotune(lsba_handle h, int64_t n, int s, int m, int8_t* gram_choice,
                  int8_t* update_ctas, int cap) {
  if (!h || n < 1 || s < 1 || s > LSBA_MAX_S || m < 1 || (int64_t)(m + 1) * s > LSBA_MAX_MS ||
      m + 3 > LSBA_MAXB || cap < 0 || (cap > 0 && (!gram_choice || !update_ctas)))
    return LSBA_INVALID_ARG;
  CK(cudaSetDevice(h->device));
  int rc = ensure_ws(h, n, s, m);
  if (rc != LSBA_OK) return rc;
  // the stored-digit kernels (s = 8, tensor cores allowed) as the solver runs them
  const bool tcs = s == 8 && h->opt.tensor_cores != 0;
  if (tcs && (rc = ensure_digits(h)) != LSBA_OK) return rc;
  h->mode = MODE_DF;
  cudaStream_t st = h->stream;
  const size_t blk = (size_t)n * s;
  // Operands with every digit busy (not zeros): pseudo-random blocks and, for
  // the stored-digit kernels, their digit planes.
  launch_fill_df(st, (int64_t)(blk * (m + 1)), 0x5EED0001ull, (float2*)h->basis);
  launch_fill_df(st, (int64_t)blk, 0x5EED0002ull, (float2*)h->Ub);
  launch_fill_df(st, (int64_t)blk, 0x5EED0003ull, (float2*)h->Wb);
  Ctl* c = h->h_ctl;
  c->active = 1;
  c->update_step = -1;
  c->error = 0;
  if ((rc = push_ctl(h)) != LSBA_OK) return rc;
  if (tcs)
    for (int i = 0; i <= m; ++i) split_basis(h, i, n, s, h->d_ctl, -1);
  Ctl* ctl = h->d_ctl;
  const SmallWs& w = h->ws;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // microseconds a launch: one warm-up run, then three timed
  auto timed = [&](auto&& run) -> float {
    run();
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3; ++r) run();
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms * 1000.f / 3.f;
  };
  std::vector<lsba_tune_entry> tab(m + 2);
  for (auto& e : tab) {
    memset(&e, 0, sizeof(e));
    e.gram_kernel = -1;
  }
  for (int k = 2; k <= m + 1; ++k) {
    lsba_tune_entry& e = tab[k];
    e.k = k;
    BlockPtrs L = basis_list(h, n, s, k - 1);
    L.p[k - 1] = h->Ub;
    BlockPtrs R;
    memset(&R, 0, sizeof(R));
    R.p[0] = h->Ub;
    R.p[1] = h->Wb;
    // ---- Gram of iteration k: [V_1..V_{k-1}, U]^T [U, W]
    float best = 3.4e38f, dflt = 0.f;
    auto try_gram = [&](int kernel, int cps, int rows, float t) {
      if (t < best) {
        best = t;
        e.gram_kernel = kernel;
        e.gram_ctas_per_sm = cps;
        e.gram_rows = rows;
      }
    };
    // untuned rule: the stored-digit Gram from k = 5, else plan_gram_df's choice
    const bool def_tcs = tcs && gram_tcs_eligible(s, k, 2) && k >= 5;
    if (tcs && gram_tcs_eligible(s, k, 2)) {
      const float t = timed([&] { do_gram_tcs(h, k, n, s, ctl); });
      if (def_tcs) dflt = t;
      try_gram(2, 0, 0, t);
    }
    if (h->opt.tensor_cores != 0 && gram_tc_eligible(s, k, 2)) {
      lsba_tune_entry tk = e;
      tk.gram_kernel = 1;
      const float t = timed([&] { do_gram(h, L, k, R, 2, n, s, ctl, 1, &tk); });
      if (!def_tcs && plan_gram_df(n, s, k, 2, h->num_sms, h->opt.tensor_cores).tc) dflt = t;
      try_gram(1, 0, 0, t);
    }
    {
      const GramPlan d0 = plan_gram_df(n, s, k, 2, h->num_sms, 0);
      // candidates with the same launch shape (grid, chunk rows) are timed once
      int seen_grid[2 * LSBA_TUNE_MAX_CPS], seen_rc[2 * LSBA_TUNE_MAX_CPS], nseen = 0;
      float seen_t[2 * LSBA_TUNE_MAX_CPS];
      const bool def_fp = !def_tcs && !plan_gram_df(n, s, k, 2, h->num_sms, h->opt.tensor_cores).tc;
      for (int cps = 1; cps <= LSBA_TUNE_MAX_CPS; ++cps)
        for (int half = 0; half < 2; ++half) {
          const int rows = half ? (d0.rows_per_chunk + 1) / 2 : 0;
          const GramPlan pc = plan_gram_df(n, s, k, 2, h->num_sms, 0, cps, rows);
          // a CTA count the shared memory cannot hold resident is not a candidate,
          // except the rule's own shape
          const bool is_def = pc.grid_x == d0.grid_x && pc.rows_per_chunk == d0.rows_per_chunk;
          if (!is_def && cps > 1 && (size_t)cps * (pc.smem + 1024) > (size_t)228 * 1024) continue;
          int hit = -1;
          for (int i = 0; i < nseen; ++i)
            if (seen_grid[i] == pc.grid_x && seen_rc[i] == pc.rows_per_chunk) hit = i;
          float t;
          if (hit >= 0) {
            t = seen_t[hit];
          } else {
            lsba_tune_entry tk = e;
            tk.gram_kernel = 0;
            tk.gram_ctas_per_sm = cps;
            tk.gram_rows = rows;
            t = timed([&] { do_gram(h, L, k, R, 2, n, s, ctl, 1, &tk); });
            seen_grid[nseen] = pc.grid_x;
            seen_rc[nseen] = pc.rows_per_chunk;
            seen_t[nseen++] = t;
          }
          if (def_fp && is_def) dflt = t;
          try_gram(0, cps, rows, t);
        }
    }
    e.gram_us = best;
    e.gram_default_us = dflt;
    // ---- basis update of iteration k (two outputs, k + 1 inputs)
    double* Vk = h->basis + (size_t)(k - 1) * blk;
    if (tcs && update_tcs_eligible(s, k + 1, true)) {
      e.update_kernel = 1;
      auto upd = [&](int minb) {
        launch_update_tcs(st, h->dig, h->dexp, k - 1, (const float2*)h->Ub, (const float2*)h->Wb,
                          nullptr, n, (float2*)Vk, (float2*)h->Ub, w.coef1, nullptr, w.coef2,
                          nullptr, nullptr, h->cdf,
                          h->dig + (size_t)(k - 1) * digit_block_bytes(n, s),
                          h->dexp + (size_t)(k - 1) * digit_exp_count(n, s), ctl, -1,
                          &h->d_ctl->error, h->num_sms, minb);
      };
      const float t3 = 3 * (update_tcs_smem(k + 1) + 1024) <= 228 * 1024 ? timed([&] { upd(0); }) : 3.4e38f;
      const float t2 = timed([&] { upd(2); });
      e.update_ctas_per_sm = t2 < t3 ? 2 : 3;
      e.update_us = t2 < t3 ? t2 : t3;
      e.update_default_us = t3 < 3.4e38f ? t3 : t2;
    } else {
      e.update_kernel = 0;
      BlockPtrs in = basis_list(h, n, s, k - 1);
      in.p[k - 1] = h->Ub;
      in.p[k] = h->Wb;
      float bu = 3.4e38f;
      for (int cps : {1, 2, 4, 8}) {
        const float t = timed([&] {
          do_update(h, in, k + 1, n, s, Vk, w.coef1, nullptr, h->Ub, w.coef2, nullptr, nullptr, ctl, -1, cps);
        });
        if (cps == 4) e.update_default_us = t;
        if (t < bu) {
          bu = t;
          e.update_ctas_per_sm = cps;
        }
      }
      e.update_us = bu;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaGetLastError());
  if ((rc = pull_ctl(h)) != LSBA_OK) return rc;
  if (c->error) return LSBA_DEVICE_TIMEOUT;
  h->tune = tab;
  h->tune_n = n;
  h->tune_s = s;
  ++h->tune_gen;
  for (int k = 0; k < cap; ++k) {
    gram_choice[k] = k < (int)tab.size() ? (int8_t)tab[k].gram_kernel : -1;
    update_ctas[k] = k < (int)tab.size() && tab[k].gram_kernel >= 0 ? (int8_t)tab[k].update_ctas_per_sm : 0;
  }
  return LSBA_OK;
}

int lsba_autotune_table(lsba_handle h, lsba_tune_entry* out, int cap, int* count) {
  if (!h || cap < 0 || (cap > 0 && !out) || !count) return LSBA_INVALID_ARG;
  int nk = 0;
  for (const auto& e : h->tune)
    if (e.gram_kernel >= 0) {
      if (nk < cap) out[nk] = e;
      ++nk;
    }
  *count = nk;
  return LSBA_OK;
}

int lsba_gram_df(lsba_handle h, const double* d_L, int a, const double* d_R, int b, int64_t n,
                 int s, double* d_G, int tensor_cores) {
  if (!h || !d_L || !d_R || !d_G || a < 1 || b < 1 || b > 2 || s < 1 || s > LSBA_MAX_S || n < 1 ||
      a + b > LSBA_MAXB || (int64_t)a * s > LSBA_MAX_MS)
    return LSBA_INVALID_ARG;
  CK(cudaSetDevice(h->device));
  cudaStream_t st = h->stream;
  const bool stored = tensor_cores == 3;
  if (stored && !gram_tcs_eligible(s, a, b)) return LSBA_INVALID_ARG;
  GramPlan p = stored ? plan_gram_tcs(n, s, a, b, h->num_sms)
                      : plan_gram_df(n, s, a, b, h->num_sms, tensor_cores ? 2 : 0);
  const size_t need = (size_t)p.grid_x * p.q;
  if (need > h->partials_cap) {
    ws_free(h, h->partials);
    h->partials = nullptr;
    h->partials_cap = 0;
    if (ws_alloc(h, &h->partials, sizeof(double) * need) != cudaSuccess) {
      cudaGetLastError();
      return LSBA_OUT_OF_MEMORY;
    }
    h->partials_cap = need;
  }
  float2 *Ldf = nullptr, *Rdf = nullptr;
  const size_t la = (size_t)a * n * s, lb = (size_t)b * n * s;
  if (ws_alloc(h, &Ldf, sizeof(float2) * la) != cudaSuccess ||
      ws_alloc(h, &Rdf, sizeof(float2) * lb) != cudaSuccess) {
    cudaGetLastError();
    ws_free(h, Ldf);
    ws_free(h, Rdf);
    return LSBA_OUT_OF_MEMORY;
  }
  launch_to_df(st, (int64_t)la, d_L, Ldf);
  launch_to_df(st, (int64_t)lb, d_R, Rdf);
  BlockPtrs L, R;
  memset(&L, 0, sizeof(L));
  memset(&R, 0, sizeof(R));
  for (int i = 0; i < a; ++i) L.p[i] = (const double*)(Ldf + (size_t)i * n * s);
  for (int i = 0; i < b; ++i) R.p[i] = (const double*)(Rdf + (size_t)i * n * s);
  CK(cudaMemsetAsync(&h->d_ctl->error, 0, sizeof(int), st));
  unsigned char* dig = nullptr;
  int* dexp = nullptr;
  if (stored) {
    // Digit planes of L_1..L_{a-1}, as the solver keeps them for its basis;
    // the kernel splits R_1 (standing for L_a = U) and R_2 itself.
    const size_t db = digit_block_bytes(n, s), de = digit_exp_count(n, s);
    if (ws_alloc(h, &dig, db * (a - 1)) != cudaSuccess ||
        ws_alloc(h, &dexp, sizeof(int) * de * (a - 1)) != cudaSuccess) {
      cudaGetLastError();
      ws_free(h, dig);
      ws_free(h, dexp);
      ws_free(h, Ldf);
      ws_free(h, Rdf);
      return LSBA_OUT_OF_MEMORY;
    }
    for (int i = 0; i < a - 1; ++i)
      launch_split_digits(st, Ldf + (size_t)i * n * s, n, s, dig + i * db, dexp + i * de, h->d_ctl,
                          -1, h->num_sms);
  }
  prof_begin(h, LSBA_K_GRAM);
  if (stored)
    launch_gram_tcs(st, p, dig, dexp, n, s, a, Rdf, Rdf + (size_t)n * s, (float2*)h->partials, d_G,
                    nullptr, 0, &h->d_ctl->error);
  else
    launch_gram_df(st, p, L, a, R, b, n, s, (float2*)h->partials, d_G, nullptr, 0, &h->d_ctl->error);
  prof_end(h);
  CK(cudaGetLastError());
  int err = 0;
  CK(cudaMemcpyAsync(&h->h_ctl->error, &h->d_ctl->error, sizeof(int), cudaMemcpyDeviceToHost, st));
  ws_free(h, Ldf);
  ws_free(h, Rdf);
  ws_free(h, dig);
  ws_free(h, dexp);
  CK(cudaStreamSynchronize(st));
  prof_collect(h);
  err = h->h_ctl->error;
  return err ? LSBA_DEVICE_TIMEOUT : LSBA_OK;
}

int lsba_gram_fp64tc(lsba_handle h, const double* d_L, int a, const double* d_R, int b, int64_t n,
                     int s, double* d_G) {
  if (!h || !d_L || !d_R || !d_G || n < 1 || !gram_f64tc_eligible(s, a, b, false))
    return LSBA_INVALID_ARG;
  CK(cudaSetDevice(h->device));
  cudaStream_t st = h->stream;
  GramPlan p = plan_gram_f64tc(n, s, a, b, h->num_sms);
  const size_t need = (size_t)p.grid_x * p.q;
  if (need > h->partials_cap) {
    ws_free(h, h->partials);
    h->partials = nullptr;
    h->partials_cap = 0;
    if (ws_alloc(h, &h->partials, sizeof(double) * need) != cudaSuccess) {
      cudaGetLastError();
      return LSBA_OUT_OF_MEMORY;
    }
    h->partials_cap = need;
  }
  const size_t ec = f64tc_exp_count(n, s), pb = f64tc_plane_bytes(n);
  int* ex = nullptr;
  unsigned char* pl = nullptr;
  if (ws_alloc(h, &ex, sizeof(int) * ec * (a + b)) != cudaSuccess ||
      ws_alloc(h, &pl, pb * (a + b)) != cudaSuccess) {
    cudaGetLastError();
    ws_free(h, ex);
    ws_free(h, pl);
    return LSBA_OUT_OF_MEMORY;
  }
  const unsigned char* L[LSBA_MAXB];
  const int* Le[LSBA_MAXB];
  const unsigned char* R[2];
  const int* Re[2];
  for (int i = 0; i < a + b; ++i) {
    const double* blk = i < a ? d_L + (size_t)i * n * s : d_R + (size_t)(i - a) * n * s;
    launch_block_digits(st, blk, n, ex + (size_t)i * ec, pl + (size_t)i * pb, nullptr, 0);
    if (i < a) {
      L[i] = pl + (size_t)i * pb;
      Le[i] = ex + (size_t)i * ec;
    } else {
      R[i - a] = pl + (size_t)i * pb;
      Re[i - a] = ex + (size_t)i * ec;
    }
  }
  CK(cudaMemsetAsync(&h->d_ctl->error, 0, sizeof(int), st));
  prof_begin(h, LSBA_K_GRAM);
  launch_gram_f64tc(st, p, L, Le, a, R, Re, b, false, n, h->partials, d_G, nullptr, 0,
                    &h->d_ctl->error);
  prof_end(h);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(&h->h_ctl->error, &h->d_ctl->error, sizeof(int), cudaMemcpyDeviceToHost, st));
  ws_free(h, ex);
  ws_free(h, pl);
  CK(cudaStreamSynchronize(st));
  prof_collect(h);
  return h->h_ctl->error ? LSBA_DEVICE_TIMEOUT : LSBA_OK;
}

int lsba_combine_fp64tc(lsba_handle h, const double* d_in, int nin, int64_t n, int s,
                        const double* d_C1, const double* d_T, const double* d_C2, double* d_out1,
                        double* d_out2) {
  if (!h || !d_in || !d_C1 || !d_out1 || n < 1 || !update_f64tc_eligible(s, nin) ||
      (d_out2 && !d_C2))
    return LSBA_INVALID_ARG;
  CK(cudaSetDevice(h->device));
  cudaStream_t st = h->stream;
  const size_t ec = f64tc_exp_count(n, s), pb = f64tc_plane_bytes(n);
  int* ex = nullptr;
  double* cf = nullptr;
  unsigned char* pl = nullptr;
  if (ws_alloc(h, &ex, sizeof(int) * ec * nin) != cudaSuccess ||
      ws_alloc(h, &cf, sizeof(double) * 2 * 8 * (size_t)nin * 8) != cudaSuccess ||
      ws_alloc(h, &pl, pb * nin) != cudaSuccess) {
    cudaGetLastError();
    ws_free(h, ex);
    ws_free(h, cf);
    ws_free(h, pl);
    return LSBA_OUT_OF_MEMORY;
  }
  const unsigned char* in[LSBA_MAXB];
  const int* ein[LSBA_MAXB];
  for (int i = 0; i < nin; ++i) {
    in[i] = pl + (size_t)i * pb;
    ein[i] = ex + (size_t)i * ec;
    launch_block_digits(st, d_in + (size_t)i * n * s, n, ex + (size_t)i * ec, pl + (size_t)i * pb,
                        nullptr, 0);
  }
  CK(cudaMemsetAsync(&h->d_ctl->error, 0, sizeof(int), st));
  prof_begin(h, LSBA_K_UPDATE);
  launch_update_f64tc(st, in, ein, nin, nullptr, n, d_out1, nullptr, nullptr, d_out2, nullptr,
                      nullptr, d_C1, d_T, d_C2, nullptr, nullptr, cf, nullptr, -1, &h->d_ctl->error,
                      h->num_sms);
  prof_end(h);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(&h->h_ctl->error, &h->d_ctl->error, sizeof(int), cudaMemcpyDeviceToHost, st));
  ws_free(h, ex);
  ws_free(h, cf);
  ws_free(h, pl);
  CK(cudaStreamSynchronize(st));
  prof_collect(h);
  return h->h_ctl->error ? LSBA_DEVICE_TIMEOUT : LSBA_OK;
}

int lsba_combine(lsba_handle h, const double* d_in, int nin, int64_t n, int s, const double* d_C,
                 const double* d_T, double* d_out) {
  if (!h || !d_in || !d_C || !d_out || nin < 1 || nin > LSBA_MAXB || s < 1 || s > LSBA_MAX_S ||
      n < 1)
    return LSBA_INVALID_ARG;
  CK(cudaSetDevice(h->device));
  BlockPtrs in;
  memset(&in, 0, sizeof(in));
  for (int i = 0; i < nin; ++i) in.p[i] = d_in + (size_t)i * n * s;
  launch_update(h->stream, in, nin, n, s, d_out, d_C, d_T, nullptr, nullptr, nullptr, nullptr,
                nullptr, -1);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  return LSBA_OK;
}

}  // extern "C"
