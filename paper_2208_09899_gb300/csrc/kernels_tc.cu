// Double-float block inner products G = L^T R on the tensor cores (tcgen05).
//
// The Gram step of every skeleton (the block inner product, Sec. 2 and
// Algorithms 2-7) is a contraction over the n rows: L = [L_1..L_a] and
// R = [R_1..R_b] are n x s blocks of double-float values (hi + lo FP32 pairs,
// 48 significand bits).  The bf16 tensor cores reach that accuracy by exact
// integer arithmetic on digits:
//
//   * Rows are processed in chunks of 32.  For each column c of the chunk
//     take e_c with max_k |hi| < 2^e_c, and write each value as six signed
//     digits, x = sum_t d_t 2^(e_c - 7 - 8t) + r with |r| <= 2^(e_c - 48):
//     digits of hi (|d| <= 128) plus digits of lo from the fourth on
//     (|lo| <= 2^(e_c - 25)), so |d_t| <= 128 for t < 3 and <= 256 after.
//     Every digit is an integer of at most 9 bits: exact in bf16.
//   * For each level l = t + u <= 5 the tensor core accumulates
//     S_l = sum_k sum_{t+u=l} dL_t dR_u over the 32 rows in FP32.  Every term
//     is an integer with |term| <= 2^15 and |S_l| <= 6 * 32 * 2^15 < 2^23, so
//     the accumulation is exact.  Levels above 5 (weights below 2^-48 of the
//     leading one) are not formed.
//   * The chunk's contribution sum_l S_l 2^(eL + eR - 14 - 8l) is added into
//     a double-float accumulator per output (error-free additions for levels
//     0-2, the small levels into the compensation term), as the FP32-pipe
//     kernel does with its products.
//
// Layout.  One CTA of 256 threads per row range; thread i owns column i of
// [L | R] (a s + b s <= 256) and loads its 32 values of a chunk straight from
// global memory (the next chunk's loads are in flight while the current one is
// split).  Digit planes live in shared memory in the no-swizzle K-major
// layout (core matrices of 8 columns x 8 rows, LBO = 128 B along the rows,
// SBO = 256 B along the columns), double-buffered so that splitting chunk c+1
// overlaps the MMAs of chunk c.  L columns form the MMA's M dimension (one or
// two tiles of 128; the second tile is the last 128 columns, overlapping the
// first); the six R digit planes are stacked along N (6 x 16 rows), so one
// MMA per L digit and 16-row slab covers every level it feeds.  Accumulators:
// 2 buffers x tiles x 6 levels x 16 tensor-memory columns.  Thread 0 issues
// the MMAs and commits them to an mbarrier; after each chunk the warps read their 32 tensor-memory lanes
// (warp w: tile w / 4, lanes 32 (w % 4) ...) and update the accumulators.  All
// waits are bounded; on a timeout the CTA records an error and returns after
// its MMAs have drained.
#include <cfloat>
#include <cuda_bf16.h>

#include "df.cuh"
#include "lsba_internal.cuh"
#include "tc.cuh"

namespace lsba {

#define GTC_THREADS 256
#define GTC_KC 32
#define GTC_NP 16

struct GramTcArgs {
  BlockPtrs L;
  BlockPtrs R;
  int s, as, bs;          // block width, a*s, b*s
  int ma;                 // rows of an L digit plane (>= 128, multiple of 8)
  int ntile, tile1;       // L tiles of 128 (1 or 2); first column of tile 1
  int64_t n, rows_per_cta;
  int q;                  // a*s*b*s
  uint32_t tcols;         // allocated tensor-memory columns
  uint32_t plane_bytes;   // one digit-plane buffer: 6 L planes + 6 R planes
  float2* partials;
  const Ctl* ctl;
  int guard;
  int* err;
};

__device__ __forceinline__ float gtc_round(float y) {  // nearest integer, |y| < 2^22
  return __fsub_rn(__fadd_rn(y, 12582912.f), 12582912.f);
}

// Digits of (hi, lo) in units of 2^(e - 7 - 8t); sc = 2^(7 - e).
__device__ __forceinline__ void gtc_digits(float2 x, float sc, float (&d)[6]) {
  float y = __fmul_rn(x.x, sc);
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const float q = gtc_round(y);
    d[t] = q;
    if (t < 5) y = __fmul_rn(__fsub_rn(y, q), 256.f);
  }
  float z = __fmul_rn(__fmul_rn(x.y, sc), 16777216.f);
#pragma unroll
  for (int t = 3; t < 6; ++t) {
    const float q = gtc_round(z);
    d[t] = __fadd_rn(d[t], q);
    if (t < 5) z = __fmul_rn(__fsub_rn(z, q), 256.f);
  }
}

__device__ __forceinline__ uint32_t gtc_pack(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// 2^k as a float, k in [-126, 127].
__device__ __forceinline__ float gtc_pow2(int k) { return __int_as_float((127 + k) << 23); }

// Column task of a thread: TPC = 4 / G threads share a column, each splits G
// groups of 8 rows of the 32-row chunk.
template <int G>
struct GtcCtx {
  const float2* src;      // column base: element (row) at src[row * s]
  bool has_col;
  int col, sub;           // column in [L | R]; sub-range of the chunk's rows
  uint32_t wofs;          // byte offset of the column's first 16-byte group in digit plane 0
  uint32_t wdig;          // bytes between digit planes of the column's operand
  uint32_t wslab;         // bytes between the two 16-row slabs of a plane
  int64_t r_begin, r_end;
};

template <int G>
__device__ __forceinline__ void gtc_load(const GramTcArgs& g, const GtcCtx<G>& cx, int c,
                                         float2 (&x)[8 * G]) {
  const int64_t r0 = cx.r_begin + (int64_t)c * GTC_KC + cx.sub * 8 * G;
#pragma unroll
  for (int k = 0; k < 8 * G; ++k) {
    const int64_t row = r0 + k;
    x[k] = (cx.has_col && row < cx.r_end) ? cx.src[row * g.s] : make_float2(0.f, 0.f);
  }
}

// Split the thread's rows of chunk c into the digit planes of buffer c & 1;
// the column's exponent (max over the 32 rows, combined over the TPC lanes)
// goes to exps.  Sets *bad on a non-finite value.
template <int G>
__device__ __forceinline__ void gtc_split(const GramTcArgs& g, const GtcCtx<G>& cx, int c,
                                          const float2 (&x)[8 * G], unsigned char* sm,
                                          int* exps, int* bad) {
  constexpr int TPC = 4 / G;
  const int buf = c & 1;
  float amax = 0.f;
  bool nonfinite = false;
#pragma unroll
  for (int k = 0; k < 8 * G; ++k) {
    const float v = fabsf(x[k].x);
    amax = fmaxf(amax, v);
    nonfinite |= !(v <= FLT_MAX);
  }
#pragma unroll
  for (int o = 1; o < TPC; o <<= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if (!cx.has_col) return;
  if (nonfinite) *bad = 1;
  int e = amax > 0.f ? ((__float_as_int(amax) >> 23) & 255) - 126 : 0;  // amax < 2^e
  e = max(e, -119);
  if (cx.sub == 0) exps[buf * GTC_THREADS + cx.col] = e;
  const float sc = gtc_pow2(7 - e);
  unsigned char* P = sm + (size_t)buf * g.plane_bytes;
#pragma unroll
  for (int i = 0; i < G; ++i) {
    const int grp = cx.sub * G + i;   // 8-row group of the chunk (0..3)
    float d[8][6];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) gtc_digits(x[8 * i + kk], sc, d[kk]);
    const uint32_t at = cx.wofs + (uint32_t)(grp >> 1) * cx.wslab + (uint32_t)(grp & 1) * 128;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      uint4 w;
      w.x = gtc_pack(d[0][t], d[1][t]);
      w.y = gtc_pack(d[2][t], d[3][t]);
      w.z = gtc_pack(d[4][t], d[5][t]);
      w.w = gtc_pack(d[6][t], d[7][t]);
      *reinterpret_cast<uint4*>(P + at + t * cx.wdig) = w;
    }
  }
}

// Thread 0: the MMAs of chunk c into accumulator buffer c & 1, committed to
// mmad[c & 1].  The R digit planes form one stack of 6 x 16 rows (digit u in
// rows 16 u ..), and the accumulators of one tile are the 6 level regions of
// 16 columns side by side.  So the MMA of L digit t against the first 6 - t
// digits of the stack (N = 16 (6 - t)), written at column region t, adds
// dL_t dR_u into level t + u for every u at once: 6 digits x 2 slabs = 12
// MMAs per tile.  The first (t = 0, slab 0) initialises all six levels.
__device__ __forceinline__ void gtc_issue(const GramTcArgs& g, int c, unsigned char* sm,
                                          uint32_t tmem, uint64_t* mmad) {
  const int buf = c & 1;
  const uint32_t pa = smem_addr(sm + (size_t)buf * g.plane_bytes);
  const uint32_t adig = (uint32_t)g.ma * 64, aslab = (uint32_t)g.ma * 32;
  const uint32_t pb = pa + 6 * adig, bslab = 6 * GTC_NP * 32;
  for (int T = 0; T < g.ntile; ++T) {
    const uint32_t rowoff = (uint32_t)(T == 0 ? 0 : g.tile1) * 32;
    const uint32_t dbase = tmem + (uint32_t)((buf * g.ntile + T) * 6 * GTC_NP);
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      const uint32_t idesc = tc_idesc_bf16_f32(128, GTC_NP * (6 - t));
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const uint64_t ad = tc_smem_desc(pa + t * adig + j * aslab + rowoff, 128, 256);
        const uint64_t bd = tc_smem_desc(pb + j * bslab, 128, 256);
        tc_mma_bf16(dbase + (uint32_t)(t * GTC_NP), ad, bd, idesc, (t | j) ? 1u : 0u);
      }
    }
  }
  tc_commit(&mmad[buf]);
}

// An epilogue warp: read the level sums of chunk c for its 32 tensor-memory
// lanes (L columns) and add them into the accumulators.
__device__ __forceinline__ void gtc_epilogue(const GramTcArgs& g, int c, uint32_t tmem, int T,
                                             int m, bool valid, const int* exps,
                                             dfacc (&acc)[GTC_NP]) {
  const int warp = threadIdx.x >> 5;
  const int buf = c & 1;
  const int eL = valid ? exps[buf * GTC_THREADS + m] : 0;
  const float sa = gtc_pow2(eL - 7);
  float w[GTC_NP];
#pragma unroll
  for (int i = 0; i < GTC_NP; ++i)
    w[i] = (valid && i < g.bs) ? __fmul_rn(sa, gtc_pow2(exps[buf * GTC_THREADS + g.as + i] - 7)) : 0.f;
  const uint32_t lanebase = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
#pragma unroll
  for (int l = 0; l < 6; ++l) {
    float v[16];
    tc_ld16(lanebase + (uint32_t)(((buf * g.ntile + T) * 6 + l) * GTC_NP), v);
#pragma unroll
    for (int i = 0; i < GTC_NP; ++i) {
      const float p = __fmul_rn(v[i], w[i]);
      w[i] = __fmul_rn(w[i], 0.00390625f);  // next level: weight / 2^8
      if (l < 3) {
        const float2 t = df_two_sum(acc[i].s, p);
        acc[i].s = t.x;
        acc[i].c = __fadd_rn(acc[i].c, t.y);
      } else {
        acc[i].c = __fadd_rn(acc[i].c, p);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < GTC_NP; ++i) df_renorm(acc[i]);
}

// Bounded wait that gives up for the whole warp once any lane has failed.
__device__ __forceinline__ void gtc_wait(uint64_t* bar, unsigned parity, bool& failed, int* err) {
  if (!failed && !mbar_wait_bounded(bar, parity)) {
    failed = true;
    if (err) atomicExch(err, 1);
  }
  failed = __any_sync(0xffffffffu, failed);
}

// Pipeline (no CTA-wide barrier inside the chunk loop).  Per chunk c, buffer
// b = c & 1 (digit planes, exponents, tensor-memory accumulators):
//   every warp: wait tfree[b] (the epilogue of chunk c - 2 has released b),
//     split its columns of chunk c, arrive full[b];
//   thread 0: wait full[b], issue the MMAs of chunk c, commit to mmad[b];
//   epilogue warps: wait full[b'] and mmad[b'] of chunk c - 1, read the level
//     sums, accumulate, arrive tfree[b'].
// Phase parity of every barrier of buffer b at chunk c: (c >> 1) & 1.
template <int G>
__global__ void __launch_bounds__(GTC_THREADS, 1) k_gram_df_tc(const __grid_constant__ GramTcArgs g) {
  if (g.guard && !*(volatile const int*)&g.ctl->active) return;
  extern __shared__ __align__(1024) unsigned char sm[];
  int* exps = reinterpret_cast<int*>(sm + 2 * (size_t)g.plane_bytes);   // [2][256]
  uint64_t* bars = reinterpret_cast<uint64_t*>(exps + 2 * GTC_THREADS);  // full[2], mmad[2], tfree[2]
  uint64_t* full = bars;
  uint64_t* mmad = bars + 2;
  uint64_t* tfree = bars + 4;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 6);
  int* bad = reinterpret_cast<int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nepi = g.ntile == 2 ? 8 : 4;   // epilogue warps

  // Zero both digit-plane buffers: padding columns (L beyond a s, R beyond
  // b s) stay zero for the whole kernel.
  for (uint32_t i = (uint32_t)tid * 16; i < 2 * g.plane_bytes; i += GTC_THREADS * 16)
    *reinterpret_cast<uint4*>(sm + i) = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    for (int b2 = 0; b2 < 2; ++b2) {
      mbar_init(&full[b2], GTC_THREADS / 32);
      mbar_init(&mmad[b2], 1);
      mbar_init(&tfree[b2], nepi);
    }
    *bad = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc_alloc(tslot, g.tcols);
  tc_fence_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  constexpr int TPC = 4 / G;
  GtcCtx<G> cx;
  cx.col = tid / TPC;
  cx.sub = tid % TPC;
  cx.has_col = cx.col < g.as + g.bs;
  cx.src = nullptr;
  if (cx.col < g.as) {
    cx.src = reinterpret_cast<const float2*>(g.L.p[cx.col / g.s]) + (cx.col % g.s);
    cx.wofs = (uint32_t)(cx.col >> 3) * 256 + (uint32_t)(cx.col & 7) * 16;
    cx.wdig = (uint32_t)g.ma * 64;
    cx.wslab = (uint32_t)g.ma * 32;
  } else {
    const int j = cx.has_col ? cx.col - g.as : 0;
    if (cx.has_col) cx.src = reinterpret_cast<const float2*>(g.R.p[j / g.s]) + (j % g.s);
    cx.wofs = 6u * (uint32_t)g.ma * 64 + (uint32_t)(j >> 3) * 256 + (uint32_t)(j & 7) * 16;
    cx.wdig = GTC_NP * 32;          // digit u occupies rows 16 u .. 16 u + 15 of the R stack
    cx.wslab = 6 * GTC_NP * 32;
  }
  cx.r_begin = (int64_t)blockIdx.x * g.rows_per_cta;
  cx.r_end = min(g.n, cx.r_begin + g.rows_per_cta);
  const int nch = cx.r_end > cx.r_begin ? (int)((cx.r_end - cx.r_begin + GTC_KC - 1) / GTC_KC) : 0;

  // Epilogue role: warp w covers tensor-memory lanes 32 (w % 4) .. of tile w / 4.
  const bool epi = warp < nepi;
  const int T = g.ntile == 2 ? (warp >> 2) : 0;
  const int m = (T == 0 ? 0 : g.tile1) + 32 * (warp & 3) + lane;
  const bool valid = epi && m < g.as && (T == 0 || m >= 128);
  const bool warp_has_out = __any_sync(0xffffffffu, valid);

  dfacc acc[GTC_NP];
#pragma unroll
  for (int i = 0; i < GTC_NP; ++i) acc[i] = dfacc{0.f, 0.f};

  bool failed = false;
  float2 xa[8 * G], xb[8 * G];
  if (nch > 0) gtc_load<G>(g, cx, 0, xa);
#define GTC_STEP(C, X)                                                              \
  {                                                                                 \
    const int b_ = (C) & 1;                                                         \
    if ((C) >= 2) gtc_wait(&tfree[b_], (unsigned)((((C) - 2) >> 1) & 1), failed, g.err); \
    if (!failed) gtc_split<G>(g, cx, (C), (X), sm, exps, bad);                      \
    tc_fence_smem();                                                                \
    __syncwarp();                                                                   \
    if (lane == 0) mbar_arrive(&full[b_]);                                          \
    if (tid == 0) {                                                                 \
      bool f0 = failed;                                                             \
      if (!f0 && !mbar_wait_bounded(&full[b_], (unsigned)(((C) >> 1) & 1))) {       \
        f0 = true;                                                                  \
        if (g.err) atomicExch(g.err, 1);                                            \
      }                                                                             \
      tc_fence_after();                                                             \
      if (!f0) gtc_issue(g, (C), sm, tmem, mmad);                                   \
      failed = f0;                                                                  \
    }                                                                               \
    failed = __any_sync(0xffffffffu, failed);                                       \
    if ((C) >= 1 && epi) {                                                          \
      const int pc = (C) - 1;                                                       \
      if (warp_has_out) {                                                           \
        gtc_wait(&full[pc & 1], (unsigned)((pc >> 1) & 1), failed, g.err);           \
        gtc_wait(&mmad[pc & 1], (unsigned)((pc >> 1) & 1), failed, g.err);           \
        tc_fence_after();                                                           \
        if (!failed) gtc_epilogue(g, pc, tmem, T, m, valid, exps, acc);             \
        tc_fence_before();                                                          \
      }                                                                             \
      __syncwarp();                                                                 \
      if (lane == 0) mbar_arrive(&tfree[pc & 1]);                                   \
    }                                                                               \
  }
  for (int c = 0; c < nch; c += 2) {
    if (c + 1 < nch) gtc_load<G>(g, cx, c + 1, xb);
    GTC_STEP(c, xa)
    if (c + 1 >= nch) break;
    if (c + 2 < nch) gtc_load<G>(g, cx, c + 2, xa);
    GTC_STEP(c + 1, xb)
  }
#undef GTC_STEP
  if (nch > 0 && epi && warp_has_out) {
    const int pc = nch - 1;
    gtc_wait(&full[pc & 1], (unsigned)((pc >> 1) & 1), failed, g.err);
    gtc_wait(&mmad[pc & 1], (unsigned)((pc >> 1) & 1), failed, g.err);
    tc_fence_after();
    if (!failed) gtc_epilogue(g, pc, tmem, T, m, valid, exps, acc);
  }
  tc_fence_before();
  const bool any_failed = __syncthreads_or(failed);
  tc_fence_after();
  if (any_failed) {
    if (tid == 0) {
      if (g.err) atomicExch(g.err, 1);
      // Let this CTA's outstanding MMAs finish before its tensor memory is freed.
      for (int b2 = 0; b2 < 2; ++b2) {
        mbar_wait_bounded(&mmad[b2], 0);
        mbar_wait_bounded(&mmad[b2], 1);
      }
    }
  } else if (valid) {
    const bool nan_out = *bad != 0;
    float2* out = g.partials + (int64_t)blockIdx.x * g.q + (int64_t)m * g.bs;
#pragma unroll
    for (int i = 0; i < GTC_NP; ++i)
      if (i < g.bs) out[i] = nan_out ? make_float2(__int_as_float(0x7fc00000), 0.f) : df_value(acc[i]);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tc_dealloc(tmem, g.tcols);
}

// ---------------------------------------------------------------- host side
bool gram_tc_eligible(int s, int a, int b) {
  const int as = a * s, bs = b * s;
  return (s % 4 == 0) && bs <= GTC_NP && as + bs <= GTC_THREADS && as >= 1;
}

// Where the digit kernel measured faster than the FP32-pipe kernel on GB300
// (n = 2^18, both kernels timed alone, s = 8, b = 2): a s >= 160 (one thread
// per column; 1.4-1.7x for a = 20..30).  Its cost per chunk depends little on
// the column count there, while the FP32-pipe kernel's grows with a b s^2.
bool gram_tc_profitable(int s, int a, int b) {
  return gram_tc_eligible(s, a, b) && b * s == GTC_NP && a * s >= 160;
}

static void gram_tc_shape(int s, int a, int b, int* ma, int* ntile, int* tile1, uint32_t* tcols,
                          uint32_t* plane_bytes) {
  const int as = a * s;
  const int ma8 = (as + 7) & ~7;
  *ma = ma8 > 128 ? ma8 : 128;
  *ntile = as > 128 ? 2 : 1;
  *tile1 = *ma - 128;
  const uint32_t need = 2u * (uint32_t)(*ntile) * 6u * GTC_NP;
  uint32_t c = 32;
  while (c < need) c <<= 1;
  *tcols = c;
  *plane_bytes = 6u * 64u * (uint32_t)(*ma + GTC_NP);
  (void)b;
}

size_t gram_tc_smem(int s, int a, int b) {
  int ma, nt, t1;
  uint32_t tc, pb;
  gram_tc_shape(s, a, b, &ma, &nt, &t1, &tc, &pb);
  return 2 * (size_t)pb + 2 * GTC_THREADS * sizeof(int) + 6 * sizeof(uint64_t) + 16;
}

GramPlan plan_gram_tc(int64_t n, int s, int a, int b, int num_sms) {
  GramPlan p{};
  p.q = a * s * b * s;
  p.tile = GTC_THREADS;
  p.grid_y = 1;
  p.rows_per_chunk = GTC_KC;
  p.nl_max = a;
  p.smem = gram_tc_smem(s, a, b);
  const int per_sm = p.smem <= 110 * 1024 ? 2 : 1;
  int64_t gx = (int64_t)per_sm * num_sms;
  const int64_t chunks = (n + GTC_KC - 1) / GTC_KC;
  if (gx > chunks) gx = chunks;
  if (gx < 1) gx = 1;
  int64_t rpc = (n + gx - 1) / gx;
  rpc = ((rpc + GTC_KC - 1) / GTC_KC) * GTC_KC;
  gx = (n + rpc - 1) / rpc;
  if (gx < 1) gx = 1;
  p.grid_x = (int)gx;
  p.rows_per_cta = rpc;
  return p;
}

void launch_gram_tc(cudaStream_t st, const GramPlan& p, const BlockPtrs& L, int a,
                    const BlockPtrs& R, int b, int64_t n, int s, float2* partials,
                    const Ctl* ctl, int guard, int* err) {
  static std::atomic<unsigned long long> attr_done{0};
  once_per_device(attr_done, [] {
    cudaFuncSetAttribute(k_gram_df_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  });
  GramTcArgs g;
  g.L = L;
  g.R = R;
  g.s = s;
  g.as = a * s;
  g.bs = b * s;
  gram_tc_shape(s, a, b, &g.ma, &g.ntile, &g.tile1, &g.tcols, &g.plane_bytes);
  g.n = n;
  g.rows_per_cta = p.rows_per_cta;
  g.q = p.q;
  g.partials = partials;
  g.ctl = ctl;
  g.guard = guard;
  g.err = err;
  // One thread per column (all 32 rows of a chunk) for every shape: the
  // variants with two or four threads per column were removed after an
  // unexplained launch failure in a build that ran one of them in solves.
  k_gram_df_tc<4><<<p.grid_x, GTC_THREADS, p.smem, st>>>(g);
}

// ============================================================================
// Stored digit planes: the basis split once, when it is written.
//
// Every Gram of BCGSI+LS reads the whole basis V_1..V_{k-1}; splitting it in
// every Gram costs ~45 FP32 instructions per value each time.  Instead each
// basis block is split once, right after the update that writes it, into the
// digits described above (per 32-row chunk and column), stored in HBM in the
// shared-memory operand layout of the Gram below, so that one bulk copy per
// block and chunk moves them.  The Gram then splits only U and W (the two
// blocks that are new at each step).
//
// Layout of one n x s block's digits (s % 8 == 0), per 32-row chunk c: s/8
// groups of 8 columns, group g at byte (c (s/8) + g) 3072; inside a group,
// digit t at t 512, rows 16 j.. of the chunk (slab j) at j 256, rows 8 kc..
// of the slab at kc 128, column (col % 8) at 16 (col % 8), row (row % 8) at
// 2 (row % 8).  As the Gram's A operand this is the no-swizzle K-major layout
// with LBO = 128 (rows) and SBO = 3072 (next 8 columns).  Exponents: int32
// [chunk][s], each the exponent of the column's maximum over the chunk's
// 128-row tile (chunks 4 t .. 4 t + 3).
// ============================================================================
#define DIG_GROUP 3072

size_t digit_block_bytes(int64_t n, int s) { return (size_t)((n + 31) / 32) * (s / 8) * DIG_GROUP; }
size_t digit_exp_count(int64_t n, int s) { return (size_t)((n + 31) / 32) * s; }

// One warp per (128-row tile, group of 8 columns); lane = row within each of
// the tile's four 32-row chunks.  A column's exponent is taken over the whole
// 128-row tile (so that the tensor-core update, whose MMA tile is 128 rows,
// sees one exponent per column) and stored for each of the four chunks.  The
// warp assembles each chunk's 3 KB in shared memory and stores it with
// 16-byte writes.  Runs iff step < 0 or ctl->update_step == step (the same
// condition as the update that wrote the block).
__global__ void __launch_bounds__(256) k_split_digits(const float2* __restrict__ V, int64_t n, int s,
                                                      unsigned char* __restrict__ dig,
                                                      int* __restrict__ dexp, const Ctl* ctl,
                                                      int step) {
  if (step >= 0 && *(volatile const int*)&ctl->update_step != step) return;
  __shared__ __align__(16) unsigned char st[8][DIG_GROUP];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int groups = s / 8;
  const int64_t nch = (n + 31) / 32, ntile = (n + 127) / 128, ntask = ntile * groups;
  unsigned char* my = st[warp];
  for (int64_t task = (int64_t)blockIdx.x * 8 + warp; task < ntask; task += (int64_t)gridDim.x * 8) {
    const int64_t tile = task / groups;
    const int g = (int)(task % groups);
    float2 x[4][8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t row = tile * 128 + q * 32 + lane;
#pragma unroll
      for (int i = 0; i < 8; ++i) x[q][i] = row < n ? V[row * s + g * 8 + i] : make_float2(0.f, 0.f);
    }
    int e[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float amax = fmaxf(fmaxf(fabsf(x[0][i].x), fabsf(x[1][i].x)), fmaxf(fabsf(x[2][i].x), fabsf(x[3][i].x)));
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
      e[i] = amax > 0.f ? ((__float_as_int(amax) >> 23) & 255) - 126 : 0;
      e[i] = max(e[i], -119);
    }
    const uint32_t rofs = (uint32_t)(lane >> 4) * 256 + (uint32_t)((lane >> 3) & 1) * 128 +
                          (uint32_t)(lane & 7) * 2;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t c = tile * 4 + q;   // 32-row chunk
      if (c >= nch) break;              // uniform across the warp
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (lane == i) dexp[c * s + g * 8 + i] = e[i];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        float d[6];
        gtc_digits(x[q][i], gtc_pow2(7 - e[i]), d);
#pragma unroll
        for (int t = 0; t < 6; ++t)
          *reinterpret_cast<__nv_bfloat16*>(my + t * 512 + rofs + i * 16) = __float2bfloat16_rn(d[t]);
      }
      __syncwarp();
      uint4* dst = reinterpret_cast<uint4*>(dig + (size_t)(c * groups + g) * DIG_GROUP);
      const uint4* src = reinterpret_cast<const uint4*>(my);
#pragma unroll
      for (int i = 0; i < DIG_GROUP / 16 / 32; ++i) dst[lane + 32 * i] = src[lane + 32 * i];
      __syncwarp();
    }
  }
}

void launch_split_digits(cudaStream_t st, const float2* V, int64_t n, int s, unsigned char* dig,
                         int* dexp, const Ctl* ctl, int step, int num_sms) {
  const int64_t tasks = ((n + 127) / 128) * (s / 8);
  int64_t grid = (tasks + 7) / 8;
  if (grid > 8LL * num_sms) grid = 8LL * num_sms;
  if (grid < 1) grid = 1;
  k_split_digits<<<(unsigned)grid, 256, 0, st>>>(V, n, s, dig, dexp, ctl, step);
}

// Gram with stored digits: L = [V_1..V_{a-1} (stored digits), U (split here)],
// R = [U, W] (split here), s = 8.  Three shared-memory buffers (bulk copies of
// chunk c + 2 in flight while chunk c is multiplied), two tensor-memory
// accumulator buffers.  Per chunk c (shared buffer c % 3, accumulators c % 2):
//   warps 0-7: wait tfree of chunk c - 2; warps 1-3 split U (L side) and U,
//     W (R side) of chunk c and arrive sfull; the epilogue warps add chunk
//     c - 1's level sums into the accumulators and arrive tfree;
//   warp 8 (one lane): wait tfree of chunk c - 2, sfull and tfull (the
//     copies) of chunk c, issue its MMAs (commit mmad); then wait tfree of
//     chunk c - 1 and copy chunk c + 2's stored digits and exponents into
//     the buffer chunk c - 1 used.
struct GramTcsArgs {
  const unsigned char* dig;  // stored digits of the basis: block i at dig + i * dig_stride
  const int* dexp;           // exponents: block i at dexp + i * dexp_stride
  size_t dig_stride, dexp_stride;
  const float2* U;
  const float2* W;
  int a, as, ma, ntile, tile1;
  int64_t n, rows_per_cta;
  int q;
  uint32_t tcols;
  uint32_t a_bytes;          // A region of one buffer: (ma / 8) groups x 3072
  uint32_t buf_bytes;        // A + B (12 x 512) + exponents (256 ints)
  float2* partials;
  const Ctl* ctl;
  int guard;
  int* err;
};

#define GTS_SPLIT_WARP0 1      // warps 1..3 split U and W (24 columns x 4 row groups)
#define GTS_THREADS (GTC_THREADS + 32)  // + warp 8: issues the bulk copies and the MMAs

__global__ void __launch_bounds__(GTS_THREADS, 1) k_gram_df_tcs(const __grid_constant__ GramTcsArgs g) {
  if (g.guard && !*(volatile const int*)&g.ctl->active) return;
  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + 3 * (size_t)g.buf_bytes);
  uint64_t* tfull = bars;        // [3] stored digits landed
  uint64_t* sfull = bars + 3;    // [3] split warps done
  uint64_t* mmad = bars + 6;     // [2]
  uint64_t* tfree = bars + 8;    // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 10);
  int* bad = reinterpret_cast<int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nepi = g.ntile == 2 ? 8 : 4;
  const int ast = g.a - 1;        // stored blocks
  constexpr int S = 8, NR = GTC_NP;

  for (uint32_t i = (uint32_t)tid * 16; i < 3 * g.buf_bytes; i += GTS_THREADS * 16)
    *reinterpret_cast<uint4*>(sm + i) = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    for (int b3 = 0; b3 < 3; ++b3) {
      mbar_init(&tfull[b3], 1);
      mbar_init(&sfull[b3], 3);
    }
    for (int b2 = 0; b2 < 2; ++b2) {
      mbar_init(&mmad[b2], 1);
      mbar_init(&tfree[b2], nepi);
    }
    *bad = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc_alloc(tslot, g.tcols);
  tc_fence_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;

  const int64_t r_begin = (int64_t)blockIdx.x * g.rows_per_cta;
  const int64_t r_end = min(g.n, r_begin + g.rows_per_cta);
  const int nch = r_end > r_begin ? (int)((r_end - r_begin + GTC_KC - 1) / GTC_KC) : 0;
  const int64_t chunk0 = r_begin / GTC_KC;   // rows_per_cta is a multiple of 32

  // Thread 0: bulk copies of chunk c's stored digits and exponents into buffer c % 3.
  auto copy_chunk = [&](int c) {
    unsigned char* B = sm + (size_t)(c % 3) * g.buf_bytes;
    int* ex = reinterpret_cast<int*>(B + g.a_bytes + 12 * 512);
    const int64_t gc = chunk0 + c;
    mbar_expect_tx(&tfull[c % 3], (unsigned)ast * (DIG_GROUP + S * 4));
    for (int i = 0; i < ast; ++i) {
      bulk_copy_g2s(B + (size_t)i * DIG_GROUP, g.dig + i * g.dig_stride + gc * DIG_GROUP, DIG_GROUP,
                    &tfull[c % 3]);
      bulk_copy_g2s(ex + i * S, g.dexp + i * g.dexp_stride + gc * S, S * 4, &tfull[c % 3]);
    }
  };

  // Split tasks of warps 1..3: 24 columns (U on the L side, then U and W on
  // the R side) x 4 groups of 8 rows.
  const int stask = tid - 32 * GTS_SPLIT_WARP0;
  const bool splitter = stask >= 0 && stask < 96;
  const int scol = splitter ? stask >> 2 : 0, ssub = stask & 3;
  const float2* ssrc = scol < S ? g.U + scol : (scol < 2 * S ? g.U + (scol - S) : g.W + (scol - 2 * S));

  const int T = g.ntile == 2 ? (warp >> 2) : 0;
  const int m = (T == 0 ? 0 : g.tile1) + 32 * (warp & 3) + lane;
  const bool epi = warp < nepi;
  const bool valid = epi && m < g.as && (T == 0 || m >= 128);
  const bool warp_has_out = __any_sync(0xffffffffu, valid);

  dfacc acc[NR];
#pragma unroll
  for (int i = 0; i < NR; ++i) acc[i] = dfacc{0.f, 0.f};
  bool failed = false;

  float2 xa[8], xb[8];
  auto load8 = [&](int c, float2 (&x)[8]) {
    const int64_t r0 = r_begin + (int64_t)c * GTC_KC + ssub * 8;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t row = r0 + k;
      x[k] = (splitter && row < r_end) ? ssrc[row * S] : make_float2(0.f, 0.f);
    }
  };
  auto split8 = [&](int c, const float2 (&x)[8]) {
    unsigned char* B = sm + (size_t)(c % 3) * g.buf_bytes;
    int* ex = reinterpret_cast<int*>(B + g.a_bytes + 12 * 512);
    float amax = 0.f;
    bool nonfinite = false;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float v = fabsf(x[k].x);
      amax = fmaxf(amax, v);
      nonfinite |= !(v <= FLT_MAX);
    }
    amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, 1));
    amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, 2));
    if (!splitter) return;
    if (nonfinite) *bad = 1;
    int e = amax > 0.f ? ((__float_as_int(amax) >> 23) & 255) - 126 : 0;
    e = max(e, -119);
    const float sc = gtc_pow2(7 - e);
    float d[8][6];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) gtc_digits(x[kk], sc, d[kk]);
    uint32_t at, dstride;
    if (scol < S) {            // U as the last L block
      const int col = g.as - S + scol;
      if (ssub == 0) ex[col] = e;
      at = (uint32_t)(col >> 3) * DIG_GROUP + (uint32_t)(col & 7) * 16;
      dstride = 512;
    } else {                   // R column j of [U, W]
      const int j = scol - S;
      if (ssub == 0) ex[g.as + j] = e;
      at = g.a_bytes + (uint32_t)(j >> 3) * 512 + (uint32_t)(j & 7) * 16;
      dstride = 2 * 512;       // digit u: rows 16 u .. of the R stack
    }
    at += (uint32_t)(ssub >> 1) * 256 + (uint32_t)(ssub & 1) * 128;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      uint4 w;
      w.x = gtc_pack(d[0][t], d[1][t]);
      w.y = gtc_pack(d[2][t], d[3][t]);
      w.z = gtc_pack(d[4][t], d[5][t]);
      w.w = gtc_pack(d[6][t], d[7][t]);
      *reinterpret_cast<uint4*>(B + at + t * dstride) = w;
    }
  };
  auto issue = [&](int c) {
    const uint32_t pa = smem_addr(sm + (size_t)(c % 3) * g.buf_bytes);
    const uint32_t pb = pa + g.a_bytes;
    for (int TT = 0; TT < g.ntile; ++TT) {
      const uint32_t aofs = (uint32_t)(TT == 0 ? 0 : g.tile1 / 8) * DIG_GROUP;
      const uint32_t dbase = tmem + (uint32_t)(((c & 1) * g.ntile + TT) * 6 * NR);
#pragma unroll
      for (int t = 0; t < 6; ++t) {
        const uint32_t idesc = tc_idesc_bf16_f32(128, NR * (6 - t));
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const uint64_t ad = tc_smem_desc(pa + aofs + t * 512 + j * 256, 128, DIG_GROUP);
          const uint64_t bd = tc_smem_desc(pb + j * 256, 128, 512);
          tc_mma_bf16(dbase + (uint32_t)(t * NR), ad, bd, idesc, (t | j) ? 1u : 0u);
        }
      }
    }
    tc_commit(&mmad[c & 1]);
  };
  auto epilogue = [&](int c) {
    const unsigned char* B = sm + (size_t)(c % 3) * g.buf_bytes;
    const int* ex = reinterpret_cast<const int*>(B + g.a_bytes + 12 * 512);
    const int eL = valid ? ex[m] : 0;
    const float sa = gtc_pow2(eL - 7);
    float w[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) w[i] = valid ? __fmul_rn(sa, gtc_pow2(ex[g.as + i] - 7)) : 0.f;
    const uint32_t lanebase = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
#pragma unroll
    for (int l = 0; l < 6; ++l) {
      float v[16];
      tc_ld16(lanebase + (uint32_t)((((c & 1) * g.ntile + T) * 6 + l) * NR), v);
#pragma unroll
      for (int i = 0; i < NR; ++i) {
        const float p = __fmul_rn(v[i], w[i]);
        w[i] = __fmul_rn(w[i], 0.00390625f);
        if (l < 3) {
          const float2 t = df_two_sum(acc[i].s, p);
          acc[i].s = t.x;
          acc[i].c = __fadd_rn(acc[i].c, t.y);
        } else {
          acc[i].c = __fadd_rn(acc[i].c, p);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < NR; ++i) df_renorm(acc[i]);
  };

  if (warp == GTC_THREADS / 32) {
    // Warp 8, one lane: the bulk copies two chunks ahead and the MMAs.
    if (lane == 0) {
      if (nch > 0) copy_chunk(0);
      if (nch > 1) copy_chunk(1);
      for (int c = 0; c < nch && !failed; ++c) {
        const unsigned par3 = (unsigned)((c / 3) & 1);
        // accumulators c & 1 free (chunk c - 2's epilogue done), operands in place
        if (c >= 2 && !mbar_wait_bounded(&tfree[c & 1], (unsigned)(((c - 2) >> 1) & 1))) failed = true;
        if (!failed && !mbar_wait_bounded(&sfull[c % 3], par3)) failed = true;
        if (!failed && !mbar_wait_bounded(&tfull[c % 3], par3)) failed = true;
        if (failed) break;
        tc_fence_after();
        issue(c);
        // buffer (c + 2) % 3 held chunk c - 1: refill it once that chunk's
        // epilogue (and so its MMAs) is done
        if (c + 2 < nch) {
          if (c >= 1 && !mbar_wait_bounded(&tfree[(c - 1) & 1], (unsigned)(((c - 1) >> 1) & 1))) {
            failed = true;
            break;
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          copy_chunk(c + 2);
        }
      }
      if (failed && g.err) atomicExch(g.err, 1);
    }
  } else if (epi) {
  // Warps 0-3 (and 4-7 with two tiles); the splitting warps 1-3 are among
  // them.  Warps with no role (4-7 with one tile) skip the loop: nothing
  // waits for them, so they must not wait on phases that run ahead.
  if (nch > 0) load8(0, xa);
  for (int c = 0; c < nch; ++c) {
    if (c + 1 < nch) load8(c + 1, xb);
    if (c >= 2) gtc_wait(&tfree[c & 1], (unsigned)(((c - 2) >> 1) & 1), failed, g.err);
    if (warp >= GTS_SPLIT_WARP0 && warp < GTS_SPLIT_WARP0 + 3) {
      if (!failed) split8(c, xa);
      tc_fence_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sfull[c % 3]);
    }
    if (c >= 1 && epi) {
      const int pc = c - 1;
      if (warp_has_out) {
        gtc_wait(&sfull[pc % 3], (unsigned)((pc / 3) & 1), failed, g.err);
        gtc_wait(&tfull[pc % 3], (unsigned)((pc / 3) & 1), failed, g.err);
        gtc_wait(&mmad[pc & 1], (unsigned)((pc >> 1) & 1), failed, g.err);
        tc_fence_after();
        if (!failed) epilogue(pc);
        tc_fence_before();
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&tfree[pc & 1]);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) xa[k] = xb[k];
  }
  if (nch > 0 && epi && warp_has_out) {
    const int pc = nch - 1;
    gtc_wait(&sfull[pc % 3], (unsigned)((pc / 3) & 1), failed, g.err);
    gtc_wait(&tfull[pc % 3], (unsigned)((pc / 3) & 1), failed, g.err);
    gtc_wait(&mmad[pc & 1], (unsigned)((pc >> 1) & 1), failed, g.err);
    tc_fence_after();
    if (!failed) epilogue(pc);
  }
  }
  tc_fence_before();
  const bool any_failed = __syncthreads_or(failed);
  tc_fence_after();
  if (any_failed) {
    if (tid == 0) {
      if (g.err) atomicExch(g.err, 1);
      for (int b2 = 0; b2 < 2; ++b2) {
        mbar_wait_bounded(&mmad[b2], 0);
        mbar_wait_bounded(&mmad[b2], 1);
      }
      for (int b3 = 0; b3 < 3; ++b3) {
        mbar_wait_bounded(&tfull[b3], 0);
        mbar_wait_bounded(&tfull[b3], 1);
      }
    }
  } else if (valid) {
    const bool nan_out = *bad != 0;
    float2* out = g.partials + (int64_t)blockIdx.x * g.q + (int64_t)m * NR;
#pragma unroll
    for (int i = 0; i < NR; ++i)
      out[i] = nan_out ? make_float2(__int_as_float(0x7fc00000), 0.f) : df_value(acc[i]);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tc_dealloc(tmem, g.tcols);
}

// Stored-digit Gram: s = 8, b = 2, 2 <= a and a s <= 168 (three buffers).
bool gram_tcs_eligible(int s, int a, int b) { return s == 8 && b == 2 && a >= 2 && a * s <= 168; }

GramPlan plan_gram_tcs(int64_t n, int s, int a, int b, int num_sms) {
  GramPlan p{};
  p.q = a * s * b * s;
  p.tile = GTC_THREADS;
  p.grid_y = 1;
  p.rows_per_chunk = GTC_KC;
  p.nl_max = a;
  p.tc = 2;
  const int as = a * s;
  const int ma8 = (as + 7) & ~7;
  const int ma = ma8 > 128 ? ma8 : 128;
  const size_t buf = (size_t)(ma / 8) * DIG_GROUP + 12 * 512 + GTC_THREADS * sizeof(int);
  p.smem = 3 * buf + 10 * sizeof(uint64_t) + 16;
  // one CTA per SM, one SM left for the small side kernel of the iteration
  int64_t gx = num_sms > 1 ? num_sms - 1 : 1;
  const int64_t chunks = (n + GTC_KC - 1) / GTC_KC;
  if (gx > chunks) gx = chunks;
  if (gx < 1) gx = 1;
  int64_t rpc = (n + gx - 1) / gx;
  rpc = ((rpc + GTC_KC - 1) / GTC_KC) * GTC_KC;
  gx = (n + rpc - 1) / rpc;
  if (gx < 1) gx = 1;
  p.grid_x = (int)gx;
  p.rows_per_cta = rpc;
  return p;
}

void launch_gram_tcs(cudaStream_t st, const GramPlan& p, const unsigned char* dig,
                     const int* dexp, int64_t n, int s, int a, const float2* U, const float2* W,
                     float2* partials, double* G, const Ctl* ctl, int guard, int* err) {
  static std::atomic<unsigned long long> attr_done{0};
  once_per_device(attr_done, [] {
    cudaFuncSetAttribute(k_gram_df_tcs, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  });
  GramTcsArgs g;
  g.dig = dig;
  g.dexp = dexp;
  g.dig_stride = digit_block_bytes(n, s);
  g.dexp_stride = digit_exp_count(n, s);
  g.U = U;
  g.W = W;
  g.a = a;
  g.as = a * s;
  const int ma8 = (g.as + 7) & ~7;
  g.ma = ma8 > 128 ? ma8 : 128;
  g.ntile = g.as > 128 ? 2 : 1;
  g.tile1 = g.ma - 128;
  const uint32_t need = 2u * (uint32_t)g.ntile * 6u * GTC_NP;
  uint32_t c = 32;
  while (c < need) c <<= 1;
  g.tcols = c;
  g.a_bytes = (uint32_t)(g.ma / 8) * DIG_GROUP;
  g.buf_bytes = g.a_bytes + 12 * 512 + GTC_THREADS * sizeof(int);
  g.n = n;
  g.rows_per_cta = p.rows_per_cta;
  g.q = p.q;
  g.partials = partials;
  g.ctl = ctl;
  g.guard = guard;
  g.err = err;
  k_gram_df_tcs<<<p.grid_x, GTS_THREADS, p.smem, st>>>(g);
  launch_gram_reduce_df(st, partials, p.grid_x, p.q, G, ctl, guard);
}

}  // namespace lsba
