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
    cudaFuncSetAttribute(k_gram_df_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    cudaFuncSetAttribute(k_gram_df_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
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
  // Threads per column: 4 (8 rows each) up to 64 columns, 2 up to 128, else 1.
  const int cols = g.as + g.bs;
  if (cols <= GTC_THREADS / 4) k_gram_df_tc<1><<<p.grid_x, GTC_THREADS, p.smem, st>>>(g);
  else if (cols <= GTC_THREADS / 2) k_gram_df_tc<2><<<p.grid_x, GTC_THREADS, p.smem, st>>>(g);
  else k_gram_df_tc<4><<<p.grid_x, GTC_THREADS, p.smem, st>>>(g);
}

}  // namespace lsba
