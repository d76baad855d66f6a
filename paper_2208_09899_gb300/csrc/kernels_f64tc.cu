// FP64 block inner products and basis updates on the tensor cores (tcgen05),
// by exact products of 8-bit digits of the FP64 values.
//
// The Gram step (the block inner product of Sec. 2 and Algorithms 2-7) and the
// basis update (Alg. 6 lines 17-18, Alg. 7 lines 16-17, the cycle end of
// Thm. 1) are contractions of FP64 blocks stored in HBM as FP64.  GB300 runs
// FP64 arithmetic at about 1 TFLOP/s, which leaves plain FP64 kernels 10-20x
// below the HBM roofline; the fp16 tensor cores can carry the same products
// exactly on integer digits (a splitting of each operand into small integers
// in the manner of Ozaki's error-free scheme for matrix products):
//
//   * Values are grouped by (128-row tile, column).  E is the group's exponent,
//     max |x| < 2^E (E >= -1021), written by the kernel that writes the block.
//     Each value becomes F = trunc(x 2^(54 - E)), |F| < 2^54 (53 bits relative
//     to the group maximum, the precision of FP64 at that maximum), and F is
//     written as seven signed 8-bit digits, F = sum_t d_t 2^(8(6 - t)),
//     t = 0 the most significant: the bytes of F + 0x0080808080808080 minus
//     128, so |d_0| <= 64 and |d_t| <= 128.  Every digit is exact in fp16.
//   * The fp16 tensor cores (kind::f16) sum digit products by level
//     l = t + u in FP32:
//     S_l = sum_k sum_{t+u=l} dL_t dR_u.  Per k every level is bounded by
//     98304 (level 6: 2 64 128 + 5 128^2; level 7: 6 128^2), so over a window
//     of at most 128 values of k every partial sum is an integer below 2^24
//     and the accumulation is exact in any order.  Levels 0..7 are formed;
//     the dropped levels weigh below 2^-57.7 of max|L| max|R| per k.
//   * A window's levels are combined in 64-bit integers,
//     T = ((sum_{l<=5} S_l 2^(8(5 - l))) << 3) + ((S_6 2^8 + S_7) >> 13),
//     |T| < 2^62.1, and added into an FP64 accumulator as T 2^(EL + ER - 55)
//     (one integer-to-FP64 conversion and one FMA per output and window).
//
// Layout of the digit operands in shared memory: the no-swizzle K-major
// canonical layout (tc.cuh): core matrices of 8 M (or N) rows x 8 K values
// (16 bytes a row), LBO = 128 B to the next 8 K values, SBO = 256 B to the
// next 8 rows.  The level of a product is fixed by where it accumulates: for
// digit t of the A operand the B operand is the stack of the other operand's
// digits u = 0, 1, ..., 7 (digit 7 all zeros), N = 16 (8 - t) rows of it, and
// the accumulator starts at tensor-memory column 16 t, so digit pair (t, u)
// lands in the 16 columns of level t + u.  The MMA of t = 0 covers all eight
// levels and starts each window (accumulate = 0).
#include <cstring>

#include <cuda_fp16.h>

#include "lsba_internal.cuh"
#include "tc.cuh"

namespace lsba {

#define FT_BIAS 0x0080808080808080ull
#define FT_EXP_MIN (-1021)

// Exponent of a group maximum given as the bits of |x| (sign cleared):
// max < 2^E, clamped below to -1021 (zero and subnormal groups).
__device__ __forceinline__ int ft_exp_of_bits(unsigned long long abits) {
  const int eb = (int)(abits >> 52);
  return max(eb - 1022, FT_EXP_MIN);
}

// F + BIAS with F = trunc(x 2^(54 - E)) for |x| < 2^E, E >= -1021.  A
// non-finite x sets nonfinite (its digits are then meaningless).
__device__ __forceinline__ unsigned long long ft_biased(double x, int E, bool& nonfinite) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int eb = (int)((bits >> 52) & 0x7FF);
  nonfinite |= eb == 0x7FF;
  const unsigned long long frac = bits & 0x000FFFFFFFFFFFFFull;
  // |x| = m 2^(max(eb, 1) - 1075), so F = (2 m) >> (E + 1022 - max(eb, 1))
  const unsigned long long m = eb ? (frac | 0x0010000000000000ull) : frac;
  const int r = max(E + 1022 - (eb ? eb : 1), 0);
  const unsigned long long F = r > 63 ? 0ull : ((m << 1) >> r);
  return (bits >> 63) ? FT_BIAS - F : FT_BIAS + F;
}

// Digit t (0 = most significant) of two values in biased form, as an fp16
// pair (element 0 in the low half), exact: the half word 0x6400 | b is
// 1024 + b, so one byte permutation, one mask-and-or and one packed
// subtraction of 1152 give (b0 - 128, b1 - 128).
__device__ __forceinline__ uint32_t ft_pair(unsigned long long g0, unsigned long long g1, int t) {
  const int byte = 6 - t;
  const uint32_t w0 = byte >= 4 ? (uint32_t)(g0 >> 32) : (uint32_t)g0;
  const uint32_t w1 = byte >= 4 ? (uint32_t)(g1 >> 32) : (uint32_t)g1;
  const uint32_t sel = (uint32_t)(byte & 3) | ((uint32_t)(4 + (byte & 3)) << 8);
  const uint32_t h = (__byte_perm(w0, w1, sel) & 0x00FF00FFu) | 0x64006400u;
  __half2 v = *reinterpret_cast<const __half2*>(&h);
  v = __hsub2(v, __halves2half2(__ushort_as_half((unsigned short)0x6480u),
                                __ushort_as_half((unsigned short)0x6480u)));
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Seven 16-byte core-matrix rows (one per digit) of eight values.
__device__ __forceinline__ void ft_digits8(const unsigned long long (&g)[8], uint4 (&d)[7]) {
#pragma unroll
  for (int t = 0; t < 7; ++t) {
    d[t].x = ft_pair(g[0], g[1], t);
    d[t].y = ft_pair(g[2], g[3], t);
    d[t].z = ft_pair(g[4], g[5], t);
    d[t].w = ft_pair(g[6], g[7], t);
  }
}

// acc + t 2^x (t an integer held in a double; exact scaling where 2^x is a
// normal number, else scalbn's rounding into the subnormal range).
__device__ __forceinline__ double ft_fma_pow2(double t, int x, double acc) {
  if (x >= -1022 && x <= 1023) return fma(t, __longlong_as_double((long long)(x + 1023) << 52), acc);
  return acc + scalbn(t, x);
}

// c 2^dx for dx <= 0 by the exponent field (integer arithmetic, exact) while
// the result stays normal; scalbn's rounding into the subnormal range below.
__device__ __forceinline__ double ft_scale_down(double c, int dx) {
  const long long b = __double_as_longlong(c);
  const int eb = (int)((b >> 52) & 0x7FF);
  if (eb == 0 || eb == 0x7FF) return eb == 0 && dx == 0 ? c : (eb == 0x7FF ? c : scalbn(c, dx));
  if (eb + dx >= 1) return __longlong_as_double(b + ((long long)dx << 52));
  return scalbn(c, dx);
}

// Level sums S_0..S_7 of 16 outputs, read level by level from tensor memory
// (16 consecutive columns per level), combined into T (see the file comment).
__device__ __forceinline__ void ft_levels16(uint32_t taddr, long long (&T)[16]) {
  int s6[16];
#pragma unroll
  for (int l = 0; l < 8; ++l) {
    float v[16];
    tc_ld16(taddr + (uint32_t)(16 * l), v);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int si = __float2int_rn(v[j]);
      if (l == 0) T[j] = si;
      else if (l <= 5) T[j] = (T[j] << 8) + si;
      else if (l == 6) s6[j] = si;
      else T[j] = (T[j] << 3) + (((long long)s6[j] * 256 + si) >> 13);
    }
  }
}

// The same for 8 outputs (8 consecutive columns per level).
__device__ __forceinline__ void ft_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                 "=r"(r[7])
               : "r"(taddr)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void ft_levels8(uint32_t taddr, long long (&T)[8]) {
  int s6[8];
#pragma unroll
  for (int l = 0; l < 8; ++l) {
    float v[8];
    ft_ld8(taddr + (uint32_t)(16 * l), v);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int si = __float2int_rn(v[j]);
      if (l == 0) T[j] = si;
      else if (l <= 5) T[j] = (T[j] << 8) + si;
      else if (l == 6) s6[j] = si;
      else T[j] = (T[j] << 3) + (((long long)s6[j] * 256 + si) >> 13);
    }
  }
}

// ---------------------------------------------------------------- exponents
// Per-(128-row tile, column) exponents of an n x s FP64 block (s <= 32): one
// CTA of 128 threads per tile, thread r owns row r of the tile.
__global__ void __launch_bounds__(128) k_block_exp(const double* __restrict__ V, int64_t n, int s,
                                                   int* __restrict__ ex, const Ctl* ctl, int guard) {
  if (guard && !*(volatile const int*)&ctl->active) return;
  __shared__ unsigned long long red[4][LSBA_MAX_S];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t tile = blockIdx.x, row = tile * 128 + tid;
  for (int c = 0; c < s; ++c) {
    unsigned long long b =
        row < n ? ((unsigned long long)__double_as_longlong(V[row * s + c]) & 0x7FFFFFFFFFFFFFFFull) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long y = __shfl_xor_sync(0xffffffffu, b, o);
      b = y > b ? y : b;
    }
    if (lane == 0) red[warp][c] = b;
  }
  __syncthreads();
  if (tid < s) {
    unsigned long long b = red[0][tid];
    for (int w = 1; w < 4; ++w) b = red[w][tid] > b ? red[w][tid] : b;
    ex[tile * s + tid] = ft_exp_of_bits(b);
  }
}

void launch_block_exp(cudaStream_t st, const double* V, int64_t n, int s, int* ex, const Ctl* ctl,
                      int guard) {
  const int64_t tiles = (n + 127) / 128;
  if (tiles > 0) k_block_exp<<<(unsigned)tiles, 128, 0, st>>>(V, n, s, ex, ctl, guard);
}

size_t f64tc_exp_count(int64_t n, int s) { return (size_t)((n + 127) / 128) * s; }

// ---------------------------------------------------------------- Gram
// G = L^T R with L = [L_1..L_a], R = [R_1..R_b] (s = 8), the partial sums of
// one CTA's row range (whole 128-row tiles) into partials[blockIdx.x][a s][b s].
// With `shared`, R_1 is L_a (the lagged skeletons' [V_1..V_{k-1}, U]^T [U, W])
// and is split once.
//
// Rows go in slabs of 16 (one MMA K step) and windows of 128 (one tile: the
// exponents' group and the exact accumulation window).  Roles (512 threads,
// 16 warps, so up to 128 registers a thread):
//   warps 0-9: split a slab's values from its stage into the digit operands
//     of slab buffer q % ndb (task = block slot x 8-row group);
//   warp 10: bulk copies (cp.async.bulk, the TMA engine) of every block's 16
//     rows of a slab (1 KB each, contiguous) into a ring of nst FP64 stages,
//     one block per lane, up to nst slabs ahead;
//   warp 11 (one lane): the MMAs of a slab once it is split;
//   warps 12-15: the epilogue of each 128-row window (tensor-memory lanes =
//     L columns; with two M tiles, tile 0 then tile 1), overlapping the
//     next window's splits and MMAs.
// Barriers (parity = use count & 1):
//   full[st]  bulk copies -> split warps        empty[st] split warps -> copies
//   dfull[b]  split warps -> MMA issue          dfree[b]  MMA commit -> split warps
//   wdone[w]  MMA commit at a window's end -> epilogue warps
//   tfree[w]  epilogue warps -> MMA issue (accumulator buffer w reusable)
#define GF_THREADS 512
#define GF_SPLIT_WARPS 10
#define GF_TMA_WARP 10
#define GF_MMA_WARP 11
#define GF_EPI_WARP0 12
#define GF_MAXSPLIT 24     // blocks split per slab: a + b - shared
#define GF_BSTRIDE 1088    // bytes per block in a stage: 16 rows x 64 B + 64 (bank offset)
#define GF_MAXST 6
#define GF_MAXDB 3         // digit slab buffers
#define GF_MAXTASK 5       // split tasks per warp and slab: 2 GF_MAXSPLIT / 10, rounded up

struct F64Blocks {
  const double* p[LSBA_MAXB];
  const int* e[LSBA_MAXB];   // per-(tile, column) exponents: e[i][tile * s + c]
};

struct GramF64Args {
  F64Blocks L, R;
  int a, b, as, bs, shared, nsplit;
  int ma, ntile, tile1;
  uint32_t dbuf_bytes, acc_bytes, stage_bytes, tcols;
  int nst, ndb;
  int64_t n;
  int tiles_per_cta;
  int q;
  double* partials;
  const Ctl* ctl;
  int guard;
  int* err;
};

__device__ __forceinline__ void gf_wait(uint64_t* bar, unsigned parity, bool& failed, int* err) {
  if (!failed && !mbar_wait_bounded(bar, parity)) {
    failed = true;
    if (err) atomicExch(err, 1);
  }
  failed = __any_sync(0xffffffffu, failed);
}

// Source block of split slot i (0 .. nsplit-1): L blocks, then the R blocks not shared.
__device__ __forceinline__ void gf_slot(const GramF64Args& g, int i, const double** p, const int** e,
                                        int* lblk, int* rblk) {
  if (i < g.a) {
    *p = g.L.p[i];
    *e = g.L.e[i];
    *lblk = i;
    *rblk = (g.shared && i == g.a - 1) ? 0 : -1;
  } else {
    const int r = i - g.a + (g.shared ? 1 : 0);
    *p = g.R.p[r];
    *e = g.R.e[r];
    *lblk = -1;
    *rblk = r;
  }
}

__global__ void __launch_bounds__(GF_THREADS, 1) k_gram_f64tc(const __grid_constant__ GramF64Args g) {
  if (g.guard && !*(volatile const int*)&g.ctl->active) return;
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* dbuf = sm;                                                   // [ndb] digit slabs
  double* accs = reinterpret_cast<double*>(sm + (size_t)g.ndb * g.dbuf_bytes);  // [16][ma]
  unsigned char* stage = sm + (size_t)g.ndb * g.dbuf_bytes + g.acc_bytes;     // [nst] FP64 stages
  uint64_t* bars = reinterpret_cast<uint64_t*>(stage + (size_t)g.nst * g.stage_bytes);
  uint64_t* full = bars;                    // [GF_MAXST]
  uint64_t* empty = bars + GF_MAXST;        // [GF_MAXST]
  uint64_t* dfull = bars + 2 * GF_MAXST;    // [GF_MAXDB]
  uint64_t* dfree = dfull + GF_MAXDB;       // [GF_MAXDB]
  uint64_t* wdone = dfree + GF_MAXDB;       // [2]
  uint64_t* tfree = wdone + 2;              // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tfree + 2);
  int* bad = reinterpret_cast<int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  for (uint32_t i = (uint32_t)tid * 16; i < (uint32_t)g.ndb * g.dbuf_bytes + g.acc_bytes; i += GF_THREADS * 16)
    *reinterpret_cast<uint4*>(sm + i) = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    for (int i = 0; i < g.nst; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], GF_SPLIT_WARPS);
    }
    for (int i = 0; i < g.ndb; ++i) {
      mbar_init(&dfull[i], GF_SPLIT_WARPS);
      mbar_init(&dfree[i], 1);
    }
    for (int b2 = 0; b2 < 2; ++b2) {
      mbar_init(&wdone[b2], 1);
      mbar_init(&tfree[b2], 4);
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

  const int64_t tile0 = (int64_t)blockIdx.x * g.tiles_per_cta;
  const int64_t r_begin = tile0 * 128;
  const int64_t r_end = min(g.n, r_begin + (int64_t)g.tiles_per_cta * 128);
  const int nslab = r_end > r_begin ? (int)((r_end - r_begin + 15) / 16) : 0;
  bool failed = false;

  if (warp == GF_TMA_WARP) {
    // ---- bulk copies of the slabs into the stage ring: lane i copies block
    // slot i (the copies of a slab are issued in parallel)
    for (int q = 0; q < nslab && !failed; ++q) {
      const int st = q % g.nst;
      bool f = false;
      if (lane == 0 && q >= g.nst && !mbar_wait_bounded(&empty[st], (unsigned)((q / g.nst - 1) & 1)))
        f = true;
      const int64_t r0 = r_begin + (int64_t)q * 16;
      const unsigned bytes = (unsigned)(min((int64_t)16, r_end - r0) * 64);
      if (lane == 0 && !f) mbar_expect_tx(&full[st], bytes * (unsigned)g.nsplit);
      failed = __any_sync(0xffffffffu, f);
      if (failed) break;
      unsigned char* dst = stage + (size_t)st * g.stage_bytes;
      for (int i = lane; i < g.nsplit; i += 32) {
        const double* p;
        const int* e;
        int lb, rb;
        gf_slot(g, i, &p, &e, &lb, &rb);
        bulk_copy_g2s(dst + (size_t)i * GF_BSTRIDE, p + r0 * 8, bytes, &full[st]);
      }
    }
    if (failed && lane == 0 && g.err) atomicExch(g.err, 1);
  } else if (warp == GF_MMA_WARP) {
    // ---- MMA issue
    if (lane == 0) {
      for (int q = 0; q < nslab && !failed; ++q) {
        const int w = q >> 3, wb = w & 1, b = q % g.ndb;
        if ((q & 7) == 0 && w >= 2 && !mbar_wait_bounded(&tfree[wb], (unsigned)(((w - 2) >> 1) & 1)))
          failed = true;
        if (!failed && !mbar_wait_bounded(&dfull[b], (unsigned)((q / g.ndb) & 1))) failed = true;
        if (failed) break;
        tc_fence_after();
        const uint32_t pa = smem_addr(dbuf + (size_t)b * g.dbuf_bytes);
        const uint32_t pb = pa + 224u * (uint32_t)g.ma;
        for (int T = 0; T < g.ntile; ++T) {
          const uint32_t aoff = T ? (uint32_t)(g.tile1 >> 3) * 256u : 0u;
          const uint32_t dcol = tmem + (uint32_t)((wb * g.ntile + T) * 128);
#pragma unroll
          for (int t = 0; t < 7; ++t) {
            const uint64_t ad = tc_smem_desc(pa + (uint32_t)t * 32u * g.ma + aoff, 128, 256);
            const uint64_t bd = tc_smem_desc(pb, 128, 256);
            const uint32_t accum = ((q & 7) || t) ? 1u : 0u;
            tc_mma_bf16(dcol + (uint32_t)(16 * t), ad, bd, tc_idesc_f16_f32(128, 16 * (8 - t)), accum);
          }
        }
        tc_commit(&dfree[b]);
        if ((q & 7) == 7 || q == nslab - 1) tc_commit(&wdone[wb]);
      }
      if (failed && g.err) atomicExch(g.err, 1);
    }
  } else if (warp >= GF_EPI_WARP0) {
    // ---- epilogue warps: lanes 32 (warp % 4) .. of each M tile = L columns
    for (int w = 0; w <= (nslab - 1) >> 3 && nslab > 0 && !failed; ++w) {
      const int wb = w & 1;
      gf_wait(&wdone[wb], (unsigned)((w >> 1) & 1), failed, g.err);
      tc_fence_after();
      if (!failed) {
        const int64_t tile = tile0 + w;
        for (int T = 0; T < g.ntile; ++T) {
          const int m = (T ? g.tile1 : 0) + 32 * (warp & 3) + lane;
          const bool valid = m < g.as && (T == 0 || m >= 128);
          const int EL = valid ? g.L.e[m >> 3][tile * 8 + (m & 7)] : 0;
          const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((wb * g.ntile + T) * 128);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            long long Tv[8];
            ft_levels8(ta + (uint32_t)(8 * h), Tv);
            if (valid && 8 * h < g.bs) {
              const int* er = g.R.e[h] + tile * 8;
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                double* a = accs + (size_t)(8 * h + j) * g.ma + m;
                *a = ft_fma_pow2((double)Tv[j], EL + er[j] - 55, *a);
              }
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tfree[wb]);
    }
    if (!failed) {
      for (int T = 0; T < g.ntile; ++T) {
        const int m = (T ? g.tile1 : 0) + 32 * (warp & 3) + lane;
        if (m < g.as && (T == 0 || m >= 128)) {
          double* out = g.partials + (int64_t)blockIdx.x * g.q + (int64_t)m * g.bs;
          const bool nan_out = *(volatile int*)bad != 0;
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (j < g.bs) out[j] = nan_out ? __longlong_as_double(0x7FF8000000000000ll) : accs[(size_t)j * g.ma + m];
        }
      }
    }
  } else {
    // ---- split warps.  Task = (block slot, 8-row group kg) of a slab:
    // lane = column (lane & 7) x row pair r2 = lane >> 3, the rows r2 and
    // r2 + 4 of the group, whose digits form fp16 pair r2 of the column's
    // 16-byte core-matrix row (the same order of the K values in both
    // operands, so the contraction is unchanged).
    const int col = lane & 7, r2 = lane >> 3;
    const int ntask = 2 * g.nsplit;
    // Exponents of the warp's tasks (task = warp + 10 i, the same every slab)
    // for the current window, and the next window's loaded one window ahead.
    int ecur[GF_MAXTASK], enext[GF_MAXTASK];
    auto load_exps = [&](int w, int (&ev)[GF_MAXTASK]) {
      const int64_t tile = tile0 + w;
#pragma unroll
      for (int i = 0; i < GF_MAXTASK; ++i) {
        const int task = warp + GF_SPLIT_WARPS * i;
        ev[i] = 0;
        if (task < ntask && tile * 128 < r_end) {
          const double* p;
          const int* e;
          int lb, rb;
          gf_slot(g, task >> 1, &p, &e, &lb, &rb);
          ev[i] = e[tile * 8 + col];
        }
      }
    };
    load_exps(0, ecur);
    load_exps(1, enext);
    for (int q = 0; q < nslab && !failed; ++q) {
      const int st = q % g.nst, b = q % g.ndb;
      const int64_t r0 = r_begin + (int64_t)q * 16;
      if ((q & 7) == 0 && q > 0) {
#pragma unroll
        for (int i = 0; i < GF_MAXTASK; ++i) ecur[i] = enext[i];
        load_exps((q >> 3) + 1, enext);
      }
      gf_wait(&full[st], (unsigned)((q / g.nst) & 1), failed, g.err);
      const unsigned char* S = stage + (size_t)st * g.stage_bytes;
      if (q >= g.ndb) gf_wait(&dfree[b], (unsigned)((q / g.ndb - 1) & 1), failed, g.err);
      unsigned char* D = dbuf + (size_t)b * g.dbuf_bytes;
      bool nf = false;
#pragma unroll
      for (int i = 0; i < GF_MAXTASK; ++i) {
        const int task = warp + GF_SPLIT_WARPS * i;
        if (task >= ntask || failed) break;
        const int sl = task >> 1, kg = task & 1;
        const int64_t row = r0 + kg * 8 + r2;
        const unsigned char* src = S + (size_t)sl * GF_BSTRIDE + (size_t)(kg * 8 + r2) * 64 + (size_t)col * 8;
        const double x0 = row < r_end ? *reinterpret_cast<const double*>(src) : 0.0;
        const double x1 = row + 4 < r_end ? *reinterpret_cast<const double*>(src + 256) : 0.0;
        const int E = ecur[i];
        const unsigned long long g0 = ft_biased(x0, E, nf), g1 = ft_biased(x1, E, nf);
        int lb, rb;
        if (sl < g.a) {
          lb = sl;
          rb = (g.shared && sl == g.a - 1) ? 0 : -1;
        } else {
          lb = -1;
          rb = sl - g.a + (g.shared ? 1 : 0);
        }
        const uint32_t dA = lb >= 0 ? (uint32_t)lb * 256u + (uint32_t)kg * 128u + (uint32_t)col * 16u +
                                          (uint32_t)r2 * 4u
                                    : ~0u;
        const uint32_t dB = rb >= 0 ? 224u * (uint32_t)g.ma + (uint32_t)rb * 256u + (uint32_t)kg * 128u +
                                          (uint32_t)col * 16u + (uint32_t)r2 * 4u
                                    : ~0u;
#pragma unroll
        for (int t = 0; t < 7; ++t) {
          const uint32_t d = ft_pair(g0, g1, t);
          if (dA != ~0u) *reinterpret_cast<uint32_t*>(D + dA + (uint32_t)t * 32u * g.ma) = d;
          // digit u = t of the R stack: N rows 16 u.. are 2 u core groups further
          if (dB != ~0u) *reinterpret_cast<uint32_t*>(D + dB + (uint32_t)t * 512u) = d;
        }
      }
      if (nf) *bad = 1;
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
      tc_fence_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&dfull[b]);
    }
  }
  tc_fence_before();
  const bool any_failed = __syncthreads_or(failed);
  tc_fence_after();
  if (any_failed && tid == 0) {
    if (g.err) atomicExch(g.err, 1);
    // let this CTA's MMAs and copies drain before its memory is released
    for (int i = 0; i < g.ndb; ++i) {
      mbar_wait_bounded(&dfree[i], 0);
      mbar_wait_bounded(&dfree[i], 1);
    }
    for (int i = 0; i < g.nst; ++i) {
      mbar_wait_bounded(&full[i], 0);
      mbar_wait_bounded(&full[i], 1);
    }
  }
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, g.tcols);
}

bool gram_f64tc_eligible(int s, int a, int b, bool shared) {
  return s == 8 && a >= 1 && b >= 1 && b <= 2 && a * s <= 256 &&
         a + b - (shared ? 1 : 0) <= GF_MAXSPLIT;
}

static void gram_f64tc_shape(int a, int* ma, int* ntile, int* tile1) {
  const int as = 8 * a;
  *ma = as > 128 ? ((as + 7) & ~7) : 128;
  *ntile = as > 128 ? 2 : 1;
  *tile1 = *ma - 128;
}

// Shared memory: ndb digit slabs, the accumulators, nst FP64 stages, barriers.
static size_t gram_f64tc_smem(int ma, int nsplit, int nst, int ndb) {
  return (size_t)ndb * ((size_t)224 * ma + 4096) + (size_t)16 * ma * 8 +
         (size_t)nst * nsplit * GF_BSTRIDE + (2 * GF_MAXST + 2 * GF_MAXDB + 4) * 8 + 16;
}
// Three digit slabs where at least three stages fit beside them, else two;
// then as many stages (<= 6) as fit.
static void gram_f64tc_buffers(int ma, int nsplit, int* nst, int* ndb) {
  *ndb = gram_f64tc_smem(ma, nsplit, 3, 3) <= 227 * 1024 ? 3 : 2;
  *nst = GF_MAXST;
  while (*nst > 2 && gram_f64tc_smem(ma, nsplit, *nst, *ndb) > 227 * 1024) --*nst;
}

GramPlan plan_gram_f64tc(int64_t n, int s, int a, int b, int num_sms) {
  GramPlan p{};
  p.q = a * s * b * s;
  p.tile = 128;
  p.grid_y = 1;
  p.rows_per_chunk = 16;
  p.nl_max = a;
  p.tc = 3;
  int ma, nt, t1;
  gram_f64tc_shape(a, &ma, &nt, &t1);
  const int nsplit = a + b;   // upper bound (shared splits one fewer)
  int nst, ndb;
  gram_f64tc_buffers(ma, nsplit, &nst, &ndb);
  p.smem = gram_f64tc_smem(ma, nsplit, nst, ndb);
  // one CTA per SM, one SM left for the small side kernel of the iteration
  const int64_t tiles = (n + 127) / 128;
  int64_t gx = num_sms > 1 ? num_sms - 1 : 1;
  if (gx > tiles) gx = tiles;
  if (gx < 1) gx = 1;
  const int64_t per = (tiles + gx - 1) / gx;
  gx = (tiles + per - 1) / per;
  p.grid_x = (int)(gx < 1 ? 1 : gx);
  p.rows_per_cta = per * 128;
  return p;
}

void launch_gram_f64tc(cudaStream_t st, const GramPlan& p, const double* const* L, const int* const* Le,
                       int a, const double* const* R, const int* const* Re, int b, bool shared,
                       int64_t n, double* partials, double* G, const Ctl* ctl, int guard, int* err) {
  static std::atomic<unsigned long long> attr_done{0};
  once_per_device(attr_done, [] {
    cudaFuncSetAttribute(k_gram_f64tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  });
  GramF64Args g;
  memset(&g, 0, sizeof(g));
  for (int i = 0; i < a; ++i) {
    g.L.p[i] = L[i];
    g.L.e[i] = Le[i];
  }
  for (int i = 0; i < b; ++i) {
    g.R.p[i] = R[i];
    g.R.e[i] = Re[i];
  }
  g.a = a;
  g.b = b;
  g.as = 8 * a;
  g.bs = 8 * b;
  g.shared = shared ? 1 : 0;
  g.nsplit = a + b - (shared ? 1 : 0);
  gram_f64tc_shape(a, &g.ma, &g.ntile, &g.tile1);
  g.dbuf_bytes = 224u * (uint32_t)g.ma + 4096u;
  g.acc_bytes = 16u * (uint32_t)g.ma * (uint32_t)sizeof(double);
  g.stage_bytes = (uint32_t)g.nsplit * GF_BSTRIDE;
  gram_f64tc_buffers(g.ma, g.nsplit, &g.nst, &g.ndb);
  g.tcols = g.ntile == 2 ? 512u : 256u;
  g.n = n;
  g.tiles_per_cta = (int)(p.rows_per_cta / 128);
  g.q = p.q;
  g.partials = partials;
  g.ctl = ctl;
  g.guard = guard;
  g.err = err;
  k_gram_f64tc<<<p.grid_x, GF_THREADS, gram_f64tc_smem(g.ma, g.nsplit, g.nst, g.ndb), st>>>(g);
  launch_gram_reduce(st, partials, p.grid_x, p.q, G, ctl, guard);
}


// ---------------------------------------------------------------- update
// out1 = sum_b in_b C1'_b (+ X C1'_X), out2 = sum_b in_b C2'_b (+ X C2'_X) for
// n x 8 FP64 blocks in_1..in_nin with per-tile exponents, coefficients folded
// beforehand (k_coef_fold64).  One CTA of 128 threads per 128-row tile at a
// time, thread r owning row r (the MMA's M = 128 rows, K = the 8 nin input
// columns, N = levels x 16 outputs):
//   * the tile's input exponents e_kk give E = max_kk e_kk; coefficient row kk
//     is scaled by 2^(e_kk - E) (exact) and split with one exponent f_n per
//     output column n, so sum_kk in[r][kk] C[kk][n] = 2^(E + f_n - 55) T[r][n];
//   * k-steps of 16 columns (two input blocks): each thread splits its row's
//     16 values into the digit planes of buffer ks & 1 (the 8 values of one
//     block are one 16-byte core-matrix row), thread 0 issues 7 MMAs against
//     the tile's coefficient digit stack; the accumulators are flushed into
//     FP64 every 8 k-steps (128 columns keep the level sums exact);
//   * X's own term is added in FP64 (X is much larger than its correction late
//     in a solve, so it does not go through the digits), the outputs are
//     stored, and the tile maxima of the output columns give their exponents.
#define UF_THREADS 128
#define UF_MAXIN 24
#define UF_FLUSH 8
#define UF_APLANE 4096
#define UF_ABUF (7 * UF_APLANE)

struct UpdF64Args {
  F64Blocks in;
  int nin, nks;
  const double* X;
  int64_t n;
  double* out1;
  double* out2;
  int* e_out1;
  int* e_out2;
  const double* cf;      // C1' [ncoef * 8][8] row-major, then C2' likewise
  int ncoef;
  const Ctl* ctl;
  int step;
  int* err;
};

template <int MINB>
__global__ void __launch_bounds__(UF_THREADS, MINB) k_update_f64tc(const __grid_constant__ UpdF64Args u) {
  if (u.step >= 0 && *(volatile const int*)&u.ctl->update_step != u.step) return;
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* Abuf = sm;                                   // [2][7][4096]
  unsigned char* Bst = sm + 2 * UF_ABUF;                      // [nks][4096]
  int* ex = reinterpret_cast<int*>(Bst + (size_t)u.nks * 4096);   // [8 UF_MAXIN]
  int* fexp = ex + 8 * UF_MAXIN;                              // [16]
  unsigned long long* red = reinterpret_cast<unsigned long long*>(fexp + 16);  // [4][16]
  int* misc = reinterpret_cast<int*>(red + 64);               // [0] bad coefficients
  uint64_t* mmad = reinterpret_cast<uint64_t*>(misc + 4);     // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mmad + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nin = u.nin, K = 8 * nin;
  const bool two = u.out2 != nullptr;
  const int64_t ntile = (u.n + 127) / 128;

  for (uint32_t i = (uint32_t)tid * 16; i < (uint32_t)u.nks * 4096u; i += UF_THREADS * 16)
    *reinterpret_cast<uint4*>(Bst + i) = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    mbar_init(&mmad[0], 1);
    mbar_init(&mmad[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc_alloc(tslot, 128);
  tc_fence_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t tlane = tmem + ((uint32_t)(32 * warp) << 16);
  bool failed = false;
  int gks = 0;   // k-steps issued by this CTA (mbarrier phases)

  auto load = [&](int64_t tile, int ks, double (&x)[16]) {
    const int64_t row = tile * 128 + tid;
#pragma unroll
    for (int kb = 0; kb < 2; ++kb) {
      const int blk = 2 * ks + kb;
      if (blk < nin && row < u.n) {
        const double2* p = reinterpret_cast<const double2*>(u.in.p[blk] + row * 8);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const double2 v = p[i];
          x[8 * kb + 2 * i] = v.x;
          x[8 * kb + 2 * i + 1] = v.y;
        }
      } else {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[8 * kb + i] = 0.0;
      }
    }
  };

  for (int64_t tile = blockIdx.x; tile < ntile && !failed; tile += gridDim.x) {
    const int64_t row = tile * 128 + tid;
    // ---- input exponents and their maximum
    for (int kk = tid; kk < K; kk += UF_THREADS) ex[kk] = u.in.e[kk >> 3][tile * 8 + (kk & 7)];
    if (tid < 16) fexp[tid] = -100000;
    if (tid == 0) misc[0] = 0;
    __syncthreads();
    int emax = FT_EXP_MIN;
    for (int kk = 0; kk < K; ++kk) emax = max(emax, ex[kk]);
    // ---- coefficient digits: unit = (output n, input block) -> 8 K values of one N row
    const int nunits = 16 * nin;
    for (int pass = 0; pass < 2; ++pass) {
      for (int un = tid; un < nunits; un += UF_THREADS) {
        const int n = un & 15, blk = un >> 4;
        if (n >= 8 && !two) continue;
        const double* cp = u.cf + (n < 8 ? 0 : (size_t)u.ncoef * 64) + (size_t)blk * 64 + (n & 7);
        double cs[8];
        bool nf = false;
        unsigned long long bmax = 0ull;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const double c = cp[q * 8];
          cs[q] = ft_scale_down(c, ex[blk * 8 + q] - emax);
          const unsigned long long b = (unsigned long long)__double_as_longlong(cs[q]) & 0x7FFFFFFFFFFFFFFFull;
          bmax = b > bmax ? b : bmax;
          nf |= !(fabs(c) <= 1.79769313486231570e308);
        }
        if (pass == 0) {
          atomicMax(&fexp[n], ft_exp_of_bits(bmax));
          if (nf) misc[0] = 1;
        } else {
          const int F = fexp[n];
          unsigned long long gv[8];
          bool nf2 = false;
#pragma unroll
          for (int q = 0; q < 8; ++q) gv[q] = ft_biased(cs[q], F, nf2);
          uint4 d[7];
          ft_digits8(gv, d);
          unsigned char* dst = Bst + (size_t)(blk >> 1) * 4096 + (size_t)(n >> 3) * 256 +
                               (size_t)(blk & 1) * 128 + (size_t)(n & 7) * 16;
#pragma unroll
          for (int t = 0; t < 7; ++t) *reinterpret_cast<uint4*>(dst + (size_t)t * 512) = d[t];
        }
      }
      __syncthreads();
    }
    // ---- k-steps
    double acc[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[j] = 0.0;
    bool rowbad = false;
    double xa[16], xb[16];
    load(tile, 0, xa);
    for (int ks = 0; ks < u.nks; ++ks) {
      const int b = gks & 1;
      if (ks + 1 < u.nks) load(tile, ks + 1, xb);
      if (gks >= 2 && !mbar_wait_bounded(&mmad[b], (unsigned)(((gks - 2) >> 1) & 1))) failed = true;
      unsigned char* A = Abuf + (size_t)b * UF_ABUF;
#pragma unroll
      for (int kb = 0; kb < 2; ++kb) {
        const int blk = 2 * ks + kb;
        unsigned char* dst = A + (size_t)(tid >> 3) * 256 + (size_t)kb * 128 + (size_t)(tid & 7) * 16;
        if (blk < nin) {
          unsigned long long gv[8];
#pragma unroll
          for (int c = 0; c < 8; ++c) gv[c] = ft_biased(xa[8 * kb + c], ex[blk * 8 + c], rowbad);
          uint4 d[7];
          ft_digits8(gv, d);
#pragma unroll
          for (int t = 0; t < 7; ++t) *reinterpret_cast<uint4*>(dst + (size_t)t * UF_APLANE) = d[t];
        } else {
#pragma unroll
          for (int t = 0; t < 7; ++t)
            *reinterpret_cast<uint4*>(dst + (size_t)t * UF_APLANE) = make_uint4(0u, 0u, 0u, 0u);
        }
      }
      tc_fence_smem();
      tc_fence_before();
      if (__syncthreads_or(failed)) {
        failed = true;
        break;
      }
      tc_fence_after();
      if (tid == 0) {
        const uint32_t pa = smem_addr(A), pb = smem_addr(Bst + (size_t)ks * 4096);
#pragma unroll
        for (int t = 0; t < 7; ++t) {
          const uint64_t ad = tc_smem_desc(pa + (uint32_t)t * UF_APLANE, 128, 256);
          const uint64_t bd = tc_smem_desc(pb, 128, 256);
          const uint32_t accum = ((ks % UF_FLUSH) || t) ? 1u : 0u;
          tc_mma_bf16(tmem + (uint32_t)(16 * t), ad, bd, tc_idesc_f16_f32(128, 16 * (8 - t)), accum);
        }
        tc_commit(&mmad[b]);
      }
      if ((ks % UF_FLUSH) == UF_FLUSH - 1 || ks + 1 == u.nks) {
        if (!mbar_wait_bounded(&mmad[b], (unsigned)((gks >> 1) & 1))) failed = true;
        tc_fence_after();
        if (!__syncthreads_or(failed)) {
          long long Tv[16];
          ft_levels16(tlane, Tv);
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[j] = ft_fma_pow2((double)Tv[j], emax + fexp[j] - 55, acc[j]);
        } else {
          failed = true;
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
      }
      ++gks;
      if (failed) break;
#pragma unroll
      for (int i = 0; i < 16; ++i) xa[i] = xb[i];
    }
    if (__syncthreads_or(failed)) {
      failed = true;
      break;
    }
    // ---- X's own term (FP64), outputs, output exponents
    if (u.X && row < u.n) {
      const double* xr = u.X + row * 8;   // read before out1 (which may be X) is written
      double xv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) xv[q] = xr[q];
      const double* c1 = u.cf + (size_t)nin * 64;
      const double* c2 = u.cf + (size_t)u.ncoef * 64 + (size_t)nin * 64;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        rowbad |= !(fabs(xv[q]) <= 1.79769313486231570e308);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          acc[c] = fma(xv[q], c1[q * 8 + c], acc[c]);
          if (two) acc[8 + c] = fma(xv[q], c2[q * 8 + c], acc[8 + c]);
        }
      }
    }
    if (rowbad || misc[0]) {
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j] = __longlong_as_double(0x7FF8000000000000ll);
    }
    if (row < u.n) {
      double2* d1 = reinterpret_cast<double2*>(u.out1 + row * 8);
#pragma unroll
      for (int i = 0; i < 4; ++i) d1[i] = make_double2(acc[2 * i], acc[2 * i + 1]);
      if (two) {
        double2* d2 = reinterpret_cast<double2*>(u.out2 + row * 8);
#pragma unroll
        for (int i = 0; i < 4; ++i) d2[i] = make_double2(acc[8 + 2 * i], acc[8 + 2 * i + 1]);
      }
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      unsigned long long b =
          row < u.n ? ((unsigned long long)__double_as_longlong(acc[j]) & 0x7FFFFFFFFFFFFFFFull) : 0ull;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, b, o);
        b = y > b ? y : b;
      }
      if (lane == 0) red[warp * 16 + j] = b;
    }
    __syncthreads();
    if (tid < 16) {
      unsigned long long b = red[tid];
      for (int w = 1; w < 4; ++w) b = red[w * 16 + tid] > b ? red[w * 16 + tid] : b;
      int* eo = tid < 8 ? u.e_out1 : u.e_out2;
      if (eo && (tid < 8 || two)) eo[tile * 8 + (tid & 7)] = ft_exp_of_bits(b);
    }
    __syncthreads();
  }
  if (failed) {
    if (tid == 0) {
      if (u.err) atomicExch(u.err, 1);
      for (int b2 = 0; b2 < 2; ++b2) {
        mbar_wait_bounded(&mmad[b2], 0);
        mbar_wait_bounded(&mmad[b2], 1);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tc_dealloc(tmem, 128);
}

size_t update_f64tc_smem(int nin) {
  const int nks = (nin + 1) / 2;
  return 2 * (size_t)UF_ABUF + (size_t)nks * 4096 + 8 * UF_MAXIN * 4 + 16 * 4 + 64 * 8 + 4 * 4 +
         2 * 8 + 16;
}

bool update_f64tc_eligible(int s, int nin) { return s == 8 && nin >= 1 && nin <= UF_MAXIN; }

// ---------------------------------------------------------------- coefficient fold
// C1' = C1 T1^{-1} and C2' = (C2 + C1' Chain) T2^{-1} for s = 8, row by row in
// FP64 (8 lanes per row, one column per lane; forward substitution with the
// reciprocal diagonal).  rows = 8 ncoef; C1, C2 are [rows][8] row-major; the
// result is C1' then C2' in `out`.  Runs iff step < 0 or ctl->update_step == step.
struct CoefFold64Args {
  const double* coef1;
  const double* coef2;
  const double* chain;
  const double* tri1;
  const double* tri2;
  int rows;
  double* out;
  const Ctl* ctl;
  int step;
};

__device__ __forceinline__ double fold64_trsm(double v, const double* T, const double* rinv, int c) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const double own = v * rinv[q];
    const double oq = __shfl_sync(0xffffffffu, own, q, 8);
    if (c == q) v = oq;
    else if (c > q) v = fma(-oq, T[q * 8 + c], v);
  }
  return v;
}

__global__ void __launch_bounds__(128) k_coef_fold64(const __grid_constant__ CoefFold64Args f) {
  if (f.step >= 0 && *(volatile const int*)&f.ctl->update_step != f.step) return;
  __shared__ double tm[3 * 64 + 16];   // T1, T2, Chain, 1 / diag(T1), 1 / diag(T2)
  const int tid = threadIdx.x;
  for (int e = tid; e < 208; e += 128) {
    double v = 0.0;
    if (e < 64) v = f.tri1 ? f.tri1[e] : 0.0;
    else if (e < 128) v = f.tri2 ? f.tri2[e - 64] : 0.0;
    else if (e < 192) v = f.chain ? f.chain[e - 128] : 0.0;
    else if (e < 200) v = f.tri1 ? 1.0 / f.tri1[(e - 192) * 9] : 0.0;
    else v = f.tri2 ? 1.0 / f.tri2[(e - 200) * 9] : 0.0;
    tm[e] = v;
  }
  __syncthreads();
  const int r = blockIdx.x * 16 + (tid >> 3), c = tid & 7;
  const bool live = r < f.rows;
  double o1 = live ? f.coef1[(size_t)r * 8 + c] : 0.0;
  if (f.tri1) o1 = fold64_trsm(o1, tm, tm + 192, c);
  double o2 = (live && f.coef2) ? f.coef2[(size_t)r * 8 + c] : 0.0;
  if (f.chain) {
#pragma unroll
    for (int q = 0; q < 8; ++q) o2 = fma(__shfl_sync(0xffffffffu, o1, q, 8), tm[128 + q * 8 + c], o2);
  }
  if (f.tri2) o2 = fold64_trsm(o2, tm + 64, tm + 200, c);
  if (live) {
    f.out[(size_t)r * 8 + c] = o1;
    f.out[(size_t)f.rows * 8 + (size_t)r * 8 + c] = o2;
  }
}

void launch_update_f64tc(cudaStream_t st, const double* const* in, const int* const* ein, int nin,
                         const double* X, int64_t n, double* out1, int* e_out1, double* out2,
                         int* e_out2, const double* coef1, const double* tri1, const double* coef2,
                         const double* chain, const double* tri2, double* cf, const Ctl* ctl,
                         int step, int* err, int num_sms) {
  const int ncoef = nin + (X ? 1 : 0);
  CoefFold64Args f;
  f.coef1 = coef1;
  f.coef2 = out2 ? coef2 : nullptr;
  f.chain = out2 ? chain : nullptr;
  f.tri1 = tri1;
  f.tri2 = out2 ? tri2 : nullptr;
  f.rows = 8 * ncoef;
  f.out = cf;
  f.ctl = ctl;
  f.step = step;
  k_coef_fold64<<<(f.rows + 15) / 16, 128, 0, st>>>(f);
  static std::atomic<unsigned long long> attr_done{0};
  once_per_device(attr_done, [] {
    cudaFuncSetAttribute(k_update_f64tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  });
  UpdF64Args u;
  memset(&u, 0, sizeof(u));
  for (int i = 0; i < nin; ++i) {
    u.in.p[i] = in[i];
    u.in.e[i] = ein[i];
  }
  u.nin = nin;
  u.nks = (nin + 1) / 2;
  u.X = X;
  u.n = n;
  u.out1 = out1;
  u.out2 = out2;
  u.e_out1 = e_out1;
  u.e_out2 = e_out2;
  u.cf = cf;
  u.ncoef = ncoef;
  u.ctl = ctl;
  u.step = step;
  u.err = err;
  // Two CTAs per SM, two short of filling the GPU: the SMs left with one CTA
  // have room for the iteration's small side kernel.
  const int64_t tiles = (n + 127) / 128;
  int64_t grid = 2LL * num_sms - 2;
  if (grid > tiles) grid = tiles;
  if (grid < 1) grid = 1;
  k_update_f64tc<2><<<(unsigned)grid, UF_THREADS, update_f64tc_smem(nin), st>>>(u);
}

}  // namespace lsba
