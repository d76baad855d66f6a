// Internal declarations shared by the CUDA translation units of the solver.
// Not part of the public C ABI (include/lsba.h).
#pragma once
#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#define LSBA_MAXB 72          // blocks in one input list of a pass
#define LSBA_MAX_S 32
#define LSBA_MAX_MS 2048      // (m+1)*s limit
#define LSBA_SMALL_THREADS 512
#define LSBA_END_STEP (1 << 20)   // update_step value that enables the cycle-end pass

namespace lsba {

// Runs f() once per device for the calling thread's current device.  Kernel
// attributes (the dynamic shared-memory opt-in) belong to a device, and solver
// handles on several host threads may launch the first kernels concurrently:
// the bit is published only after f() has returned, and two threads that both
// run f() set the same attributes.
template <class F>
inline void once_per_device(std::atomic<unsigned long long>& done, F&& f) {
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return;
  f();
  done.fetch_or(bit, std::memory_order_release);
}

// Device-side control record of one solve.  Written by the small (single-CTA)
// kernels, read by every launch of the step so that a cycle that has ended
// turns the remaining launches of the enqueued cycle into no-ops.
struct Ctl {
  int active;          // 1 while the current cycle may complete more relations
  int j;               // relations completed in the current cycle
  int k;               // skeleton loop iterations done in the current cycle
  int flagged;         // relation whose Cholesky flagged (0: none)
  int converged;       // estimate <= tol at relation j
  int update_step;     // loop index whose basis update must run (-1: none)
  int start_flag;      // CholQR of the cycle's start block flagged
  int fom_singular;    // FOM small system singular at relation j
  int m_cur;           // maximum basis size of the current cycle
  int inject_relation; // force a flag when completing this relation (-1: none)
  int cycle;           // 1-based cycle number
  int record;          // record history
  int n_hist;          // estimates recorded so far
  int hist_cap;
  int n_gram_hist;     // Gram outputs recorded (first cycle)
  int gram_hist_used;  // doubles used in the Gram history buffer
  int gram_hist_cap;
  int muscle_syncs;    // syncs of the column muscle in the current cycle
  double est;          // last residual estimate
  double normB;        // ||B||_F
  double tol;
  double relres_true;
  int side_step;       // loop index whose side kernel must run (-1: none)
  int side_rel;        // relation the side kernel completes
  int side_J;          // side kernel also forms J (BCGSI+LS)
  int error;           // a bounded device wait gave up (LSBA_DEVICE_TIMEOUT)
  double outer_normB;  // ||B||_F of the outer (FP64) problem of iterative refinement
};

// Pointers of up to LSBA_MAXB blocks (each n x s, row-major, FP64).
struct BlockPtrs {
  const double* p[LSBA_MAXB];
};

// Device workspace of the small kernels (all device pointers).
// CTAs that share the s x s products of a BCGSI+LS step (k_ls_products).
#define LSBA_LS_PROD_CTAS 16

struct SmallWs {
  int s, m, skel, modification;
  int global_ip;       // 1: global block inner product (each s x s Gram block -> tr/s I)
  int col_muscle;      // 1: BMGS-SVL/LTS with the MGS-SVL/LTS column muscle
  double* mus;         // the column muscle's work area: R, T, coefficients, status, partials
  int ldH;             // (m+2)*s
  int ldT;             // (m+2)*s
  int ldR;             // (m+1)*s
  double* H;           // Hessenberg, ldH x (m+1)s, column-major
  double* T;           // ICWY/CWY auxiliary, ldT x ldT, column-major (strict upper part used)
  double* J;           // BCGSI+LS auxiliary, (m+1)s x s, column-major
  const double* G;     // reduced Gram output, row-major (rows x cols)
  double* coef1;       // update coefficients, [nin][s][s] row-major
  double* coef2;
  double* chain;       // s x s row-major
  double* tri1;        // s x s row-major upper (or unused)
  double* tri2;
  double* Rbar;        // QR of the block Hessenberg: R factor, ldR x ldR col-major
  double* refl;        // Householder vectors per block column: [(m+1)][2s x s] col-major
  double* tau;         // [(m+1)][s]
  double* Twy;         // compact WY factor per reflector set: [(m+1)][s x s] col-major
  double* g;           // transformed right-hand side E_1 Beta, (m+2)s x s col-major, ld (m+2)s
  double* Tfom;        // s x s col-major: last block of H_j's last column after j-1 reflector sets
  double* gfom;        // s x s: g block j before reflector set j
  double* cfom;        // s x s: FOM cospatial factor T_fom^{-1} gfom
  double* ufom;        // (m+1)s x s col-major: upper part of the last column after j-1 sets
  double* Cfac;        // s x s col-major: cumulative cospatial factor C
  double* Bcyc;        // s x s col-major: CholQR factor of the cycle's start block
  double* Xi;          // (m+1)s x s col-major
  double* Mvec;        // (m+1)s x s col-major
  double* work;        // scratch, >= 6*(m+2)s*s + 16*s*s doubles
  double* saveZP;      // BCGSI+LS: [Z; P] of the last iteration, (m+1)s x s
  double* saveY;       // BCGSI+LS: Y of the last iteration, (m+1)s x s
  double* saveR;       // BCGSI+LS: R = H_{k,k-1} of the last iteration, s x s
  double* prod;        // BCGSI+LS, s <= 16: per-CTA partial sums of Y^T Y and Y^T Z,
                       // [LSBA_LS_PROD_CTAS][2][s x s] (k_ls_products)
  double* hist_est;    // [hist_cap]
  int* hist_cycle;
  int* hist_j;
  double* gram_hist;   // [gram_hist_cap]
  int* gram_dims;      // [2 * (m+2)]
  Ctl* ctl;
};

// ---- launchers (stream-ordered, asynchronous) ----
// W = A V.  guard: skip when ctl->active == 0.
void launch_spmm(cudaStream_t st, int64_t n, const int32_t* rowptr, const int32_t* colidx,
                 const double* vals, const double* V, double* W, int s, const Ctl* ctl, int guard);
// R = B - W (elementwise), n x s.
void launch_axpby(cudaStream_t st, int64_t n, int s, const double* B, const double* W, double* R);

// Gram [L]^T [R] into per-CTA partials, then a fixed-order reduction into G.
struct GramPlan {
  int grid_x, grid_y, q, tile;
  size_t smem;
  int rows_per_chunk;
  int64_t rows_per_cta;
  int nl_max;     // bulk-copy Gram kernels: most left blocks one tile group reads
  int tc;         // double-float Gram on the tensor cores (k_gram_df_tc)
};

// Left blocks [first, first + count) that the output tiles tile_base ..
// tile_base + cnt - 1 of a bulk-copy Gram kernel read (tiles are 4 x 4, row
// tile it = T / ntj covers left columns 4 it .. 4 it + 3 of one block, s a
// multiple of 4).
__host__ __device__ inline void gram_tile_blocks(int tile_base, int cnt, int ntj, int s,
                                                 int* first, int* count) {
  const int it_lo = tile_base / ntj, it_hi = (tile_base + cnt - 1) / ntj;
  *first = (4 * it_lo) / s;
  *count = (4 * it_hi) / s - *first + 1;
}
GramPlan plan_gram(int64_t n, int s, int a, int b, int num_sms);
void launch_gram(cudaStream_t st, const GramPlan& p, const BlockPtrs& L, int a, const BlockPtrs& R,
                 int b, int64_t n, int s, double* partials, double* G, const Ctl* ctl, int guard);

// out_o = (sum_i in_i C_o[i] (+ out1 * chain for o = 2)) * tri_o^{-1}.
// Runs iff step < 0 or ctl->update_step == step.
void launch_update(cudaStream_t st, const BlockPtrs& in, int nin, int64_t n, int s,
                   double* out1, const double* coef1, const double* tri1,
                   double* out2, const double* coef2, const double* chain, const double* tri2,
                   const Ctl* ctl, int step);

// ---- double-float (FP64-accurate, FP32-pipe) variants; block vectors are float2 (hi, lo) ----
// in * scale -> double-float, and back (scale a power of two).
void launch_to_df(cudaStream_t st, int64_t count, const double* in, float2* out, double scale = 1.0);
void launch_from_df(cudaStream_t st, int64_t count, const float2* in, double* out,
                    double scale = 1.0);
// out[0] = bits of max |in|, out[1] = bits of the smallest nonzero |in| (out
// preset to {0, ~0}); a non-finite entry gives out[0] >= bits of +inf.
void launch_absrange(cudaStream_t st, int64_t count, const double* in, unsigned long long* out,
                     int num_sms);
void launch_sub_df(cudaStream_t st, int64_t count, const float2* B, const float2* W, float2* R);
void launch_spmm_df(cudaStream_t st, int64_t n, const int32_t* rowptr, const int32_t* colidx,
                    const float2* vals, const float2* V, float2* W, int s, const Ctl* ctl, int guard);
// tensor_cores: 0 FP32-pipe kernels only; 1 the tensor-core kernel where it
// measured faster (gram_tc_profitable); 2 wherever its shape allows.
// cps > 0: CTAs per SM of the FP32-pipe kernel (else its default, 2 or 3);
// rc_cap > 0: at most rc_cap rows a pipeline chunk (autotuned shapes).
#define LSBA_TUNE_MAX_CPS 4   // most CTAs per SM the autotuner gives the FP32-pipe Gram
GramPlan plan_gram_df(int64_t n, int s, int a, int b, int num_sms, int tensor_cores = 1, int cps = 0,
                      int rc_cap = 0);
// Tensor-core double-float Gram (kernels_tc.cu): shapes with s % 4 == 0,
// b s <= 16 and a s + b s <= 256.
bool gram_tc_eligible(int s, int a, int b);
bool gram_tc_profitable(int s, int a, int b);
void launch_gram_reduce_df(cudaStream_t st, const float2* partials, int nparts, int q, double* G,
                           const Ctl* ctl, int guard);
// Stored digit planes of basis blocks (kernels_tc.cu): bytes and exponent
// count of one n x s block (s % 8 == 0), the split kernel, and the Gram of
// [V_1..V_{a-1} (stored), U] x [U, W] (s = 8, b = 2, a s <= 168).
size_t digit_block_bytes(int64_t n, int s);
size_t digit_exp_count(int64_t n, int s);
// Pseudo-random double-float values (timing runs only).
void launch_fill_df(cudaStream_t st, int64_t count, uint64_t seed, float2* out);
void launch_split_digits(cudaStream_t st, const float2* V, int64_t n, int s, unsigned char* dig,
                         int* dexp, const Ctl* ctl, int step, int num_sms);
bool gram_tcs_eligible(int s, int a, int b);
// Coefficients of an update converted to double-float (k_coef_df layout).
void launch_coef_df(cudaStream_t st, int nin, int s, bool two, const double* coef1,
                    const double* coef2, const double* chain, const double* tri1,
                    const double* tri2, float2* cdf, const Ctl* ctl, int step);
// Tensor-core update (kernels_tcu.cu): inputs [V_1..V_a (stored digits), U, W]
// (U = W = nullptr: [V_1..V_a] only) plus an optional block X added in
// double-float (coefficients after the other inputs'), two outputs, s = 8,
// 8 nin <= 256 with nin the digit inputs.  dig_out / dexp_out (optional)
// receive out1's digit planes, as launch_split_digits would write them.
// Column muscle MGS-SVL / MGS-LTS (kernels_muscle.cu) on one n x s block in
// place (mode 0 FP64, 1 double-float, 2 FP32); R, T and the status in `area`.
#define MUS_PARTS 1024
size_t muscle_area_doubles(int s);
void launch_col_muscle(cudaStream_t st, void* X, int mode, int64_t n, int s, bool lts,
                       double* area, Ctl* ctl, int step, int num_sms);
bool update_tcs_eligible(int s, int nin, bool two);
void launch_update_tcs(cudaStream_t st, const unsigned char* dig, const int* dexp, int a,
                       const float2* U, const float2* W, const float2* X, int64_t n, float2* out1,
                       float2* out2, const double* coef1, const double* tri1, const double* coef2,
                       const double* chain, const double* tri2, float2* cdf, unsigned char* dig_out,
                       int* dexp_out, const Ctl* ctl, int step, int* err, int num_sms,
                       int minb = 0);   // CTAs per SM: 0 = 3 where they fit, else 2; 2 forces 2
size_t update_tcs_smem(int nin);
GramPlan plan_gram_tcs(int64_t n, int s, int a, int b, int num_sms);
void launch_gram_tcs(cudaStream_t st, const GramPlan& p, const unsigned char* dig,
                     const int* dexp, int64_t n, int s, int a, const float2* U, const float2* W,
                     float2* partials, double* G, const Ctl* ctl, int guard, int* err);
GramPlan plan_gram_tc(int64_t n, int s, int a, int b, int num_sms);
void launch_gram_tc(cudaStream_t st, const GramPlan& p, const BlockPtrs& L, int a,
                    const BlockPtrs& R, int b, int64_t n, int s, float2* partials,
                    const Ctl* ctl, int guard, int* err);
void launch_gram_df(cudaStream_t st, const GramPlan& p, const BlockPtrs& L, int a,
                    const BlockPtrs& R, int b, int64_t n, int s, float2* partials, double* G,
                    const Ctl* ctl, int guard, int* err);
__host__ __device__ size_t coef_df_count(int nin, int s, bool two);
size_t update_df_smem(int nin, int s, bool two);
void launch_update_df(cudaStream_t st, const BlockPtrs& in, int nin, int64_t n, int s, float2* out1,
                      const double* coef1, const double* tri1, float2* out2, const double* coef2,
                      const double* chain, const double* tri2, float2* cdf, const Ctl* ctl,
                      int step, int num_sms, int cps = 0);   // cps > 0: CTAs per SM (default 4)

// ---- FP32 variants (inner solver of FP64 iterative refinement); block vectors are float ----
void launch_to_f32(cudaStream_t st, int64_t count, const double* in, float* out, double scale = 1.0);
void launch_add_f32(cudaStream_t st, int64_t count, const float* d, double* x, double scale = 1.0);
void launch_spmm_f32(cudaStream_t st, int64_t n, const int32_t* rowptr, const int32_t* colidx,
                     const float* vals, const float* V, float* W, int s, const Ctl* ctl, int guard);
GramPlan plan_gram_f32(int64_t n, int s, int a, int b, int num_sms);
void launch_gram_f32(cudaStream_t st, const GramPlan& p, const BlockPtrs& L, int a,
                     const BlockPtrs& R, int b, int64_t n, int s, float* partials, double* G,
                     const Ctl* ctl, int guard, int* err);
__host__ __device__ size_t coef_f32_count(int nin, int s, bool two);
size_t update_f32_smem(int nin, int s, bool two);
void launch_update_f32(cudaStream_t st, const BlockPtrs& in, int nin, int64_t n, int s, float* out1,
                       const double* coef1, const double* tri1, float* out2, const double* coef2,
                       const double* chain, const double* tri2, float* cf, const Ctl* ctl, int step,
                       int num_sms);

// ---- FP64 on the tensor cores by exact digit products (kernels_f64tc.cu), s = 8 ----
// Per-(128-row tile, column) exponents E (max |x| < 2^E) of an n x s block:
// ex[tile * s + c]; f64tc_exp_count(n, s) ints per block.
size_t f64tc_exp_count(int64_t n, int s);
void launch_block_exp(cudaStream_t st, const double* V, int64_t n, int s, int* ex, const Ctl* ctl,
                      int guard);
// Exponents and digit planes (7 bytes a value, f64tc_plane_bytes(n) a block)
// of an n x 8 FP64 block, written by the pass that writes the block and read
// by the Gram and the update in place of its FP64 values.
size_t f64tc_plane_bytes(int64_t n);
void launch_block_digits(cudaStream_t st, const double* V, int64_t n, int* ex, unsigned char* planes,
                         const Ctl* ctl, int guard);
// W = A V (FP64, s = 8) with W's exponents and digit planes, in one pass.
void launch_spmm_digits(cudaStream_t st, int64_t n, const int32_t* rowptr, const int32_t* colidx,
                        const double* vals, const double* V, double* W, int* ex, unsigned char* planes,
                        const Ctl* ctl, int guard);
// Gram [L_1..L_a]^T [R_1..R_b] (blocks given by exponents and digit planes),
// reduced into G.  shared: R_1 is L_a (read once).
bool gram_f64tc_eligible(int s, int a, int b, bool shared);
GramPlan plan_gram_f64tc(int64_t n, int s, int a, int b, int num_sms);
void launch_gram_f64tc(cudaStream_t st, const GramPlan& p, const unsigned char* const* L,
                       const int* const* Le, int a, const unsigned char* const* R, const int* const* Re,
                       int b, bool shared, int64_t n, double* partials, double* G, const Ctl* ctl,
                       int guard, int* err);
// out1 = (sum_i in_i C1_i (+ X C1_X)) T1^{-1},
// out2 = (sum_i in_i C2_i (+ X C2_X) + out1 Chain) T2^{-1}  (out2 optional),
// with the inputs given by their exponents and digit planes, X (optional) in
// FP64, and the triangular factors and the chain folded into the
// coefficients first (into cf: 2 x 8 ncoef x 8 doubles, ncoef = nin (+1 with
// X)); the outputs' exponents and digit planes go to e_out / p_out (optional).
bool update_f64tc_eligible(int s, int nin);
size_t update_f64tc_smem(int nin);
void launch_update_f64tc(cudaStream_t st, const unsigned char* const* in, const int* const* ein,
                         int nin, const double* X, int64_t n, double* out1, int* e_out1,
                         unsigned char* p_out1, double* out2, int* e_out2, unsigned char* p_out2,
                         const double* coef1, const double* tri1, const double* coef2,
                         const double* chain, const double* tri2, double* cf, const Ctl* ctl,
                         int step, int* err, int num_sms);
// Fixed-order (CTA-order) sum of FP64 Gram partials [nparts][q] into G.
void launch_gram_reduce(cudaStream_t st, const double* partials, int nparts, int q, double* G,
                        const Ctl* ctl, int guard);

// Small single-CTA kernels (skeleton logic, Cholesky, least squares, estimate).
void launch_small_start(cudaStream_t st, const SmallWs& w, int flags);
void launch_true_relres(cudaStream_t st, const double* G, int s, Ctl* ctl);
// mode 0: ctl->outer_normB = sqrt(trace G); mode 1: ctl->relres_true = sqrt(trace G) / outer_normB.
void launch_outer_norm(cudaStream_t st, const double* G, int s, Ctl* ctl, int mode);
void launch_small_step(cudaStream_t st, const SmallWs& w, int k, int phase);
void launch_small_side(cudaStream_t st, const SmallWs& w, int k);
void launch_small_end(cudaStream_t st, const SmallWs& w);

}  // namespace lsba
