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

// Levels 0..7 of 8 outputs (8 columns a level at taddr + 16 l): all eight
// loads issued before one wait, then combined into T as in ft_levels16.
__device__ __forceinline__ void ft_levels8b(uint32_t taddr, long long (&T)[8]) {
  uint32_t r[8][8];
#pragma unroll
  for (int l = 0; l < 8; ++l)
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[l][0]), "=r"(r[l][1]), "=r"(r[l][2]), "=r"(r[l][3]), "=r"(r[l][4]),
                   "=r"(r[l][5]), "=r"(r[l][6]), "=r"(r[l][7])
                 : "r"(taddr + (uint32_t)(16 * l))
                 : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    long long t = 0;
    int s6 = 0;
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      const int si = __float2int_rn(__uint_as_float(r[l][j]));
      if (l == 0) t = si;
      else if (l <= 5) t = (t << 8) + si;
      else if (l == 6) s6 = si;
      else t = (t << 3) + (((long long)s6 * 256 + si) >> 13);
    }
    T[j] = t;
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

// ---------------------------------------------------------------- digit planes
// The stored digits of an n x 8 FP64 block: for tile tau (rows 128 tau ..),
// tile row r = 16 j + i (slab j of 16 rows, row i in it) and digit t (0 =
// most significant), the 8 bytes at
//   planes + tau * 7168 + j * 896 + t * 128 + i * 8 + c,  c = 0..7 (columns),
// are the biased digits d_t + 128 of F = trunc(x 2^(54 - E)) (x the value in
// row 128 tau + r, column c; E the tile column's exponent).  Rows past n hold
// digit 0 (byte 128).  7 KB a tile (7 bytes a value), a 16-row slab's 7
// digit rows contiguous (896 bytes): the update reads a tile's planes, the
// Gram a slab's, instead of the FP64 block, so the digits of a block are
// formed once, by the pass that writes it.  A tile column holding a non-finite value has E = 1025
// (the exponent of its maximum's bits), and its digits are meaningless.
#define FT_PLANE_TILE 7168
#define FT_PLANE_SLAB 896
#define FT_EXP_NONFINITE 1025

size_t f64tc_plane_bytes(int64_t n) { return (size_t)((n + 127) / 128) * FT_PLANE_TILE; }

// Byte p (0..7) of each of eight 64-bit words, packed in order (word c -> byte c).
__device__ __forceinline__ uint2 ft_gather_byte(const unsigned long long (&g)[8], int p) {
  const uint32_t b = (uint32_t)(p & 3), sel = b | ((4u + b) << 4);
  uint32_t w[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) w[c] = p >= 4 ? (uint32_t)(g[c] >> 32) : (uint32_t)g[c];
  const uint32_t p01 = __byte_perm(w[0], w[1], sel), p23 = __byte_perm(w[2], w[3], sel);
  const uint32_t p45 = __byte_perm(w[4], w[5], sel), p67 = __byte_perm(w[6], w[7], sel);
  return make_uint2(__byte_perm(p01, p23, 0x5410), __byte_perm(p45, p67, 0x5410));
}

// Eight biased digit bytes (d + 128) to eight fp16 digits d, exact: the half
// word 0x64 << 8 | b is 1024 + b, and 1024 + b - 1152 = d.
__device__ __forceinline__ uint4 ft_expand8(uint2 w) {
  const uint32_t k = 0x64646464u;
  uint32_t h[4] = {__byte_perm(w.x, k, 0x4140), __byte_perm(w.x, k, 0x4342),
                   __byte_perm(w.y, k, 0x4140), __byte_perm(w.y, k, 0x4342)};
  const __half2 off = __halves2half2(__ushort_as_half((unsigned short)0x6480u),
                                     __ushort_as_half((unsigned short)0x6480u));
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __half2 v = __hsub2(*reinterpret_cast<const __half2*>(&h[i]), off);
    h[i] = *reinterpret_cast<const uint32_t*>(&v);
  }
  return make_uint4(h[0], h[1], h[2], h[3]);
}

// Exponent of a tile column from the maximum of the high words of |x|.
__device__ __forceinline__ int ft_exp_of_hi(uint32_t hi) { return max((int)(hi >> 20) - 1022, FT_EXP_MIN); }

// The biased digit planes of 8 values (one row of a tile) with exponents e[c],
// stored at dst (the row's 8 bytes of digit plane 0; planes 128 bytes apart).
// Offset of tile row r's digit-0 bytes in a tile's plane set.
__device__ __forceinline__ size_t ft_row_off(int r) { return (size_t)(r >> 4) * FT_PLANE_SLAB + (size_t)(r & 15) * 8; }

__device__ __forceinline__ void ft_store_row_digits(const double (&x)[8], const int* e,
                                                    unsigned char* dst) {
  unsigned long long g[8];
  bool nf = false;
#pragma unroll
  for (int c = 0; c < 8; ++c) g[c] = ft_biased(x[c], e[c], nf);
#pragma unroll
  for (int t = 0; t < 7; ++t) *reinterpret_cast<uint2*>(dst + t * 128) = ft_gather_byte(g, 6 - t);
}

// Exponents and digit planes of an n x 8 FP64 block: one CTA of 128 threads
// per tile, thread r owns row r.
__global__ void __launch_bounds__(128) k_block_digits(const double* __restrict__ V, int64_t n,
                                                      int* __restrict__ ex,
                                                      unsigned char* __restrict__ planes,
                                                      const Ctl* ctl, int guard) {
  if (guard && !*(volatile const int*)&ctl->active) return;
  __shared__ uint32_t red[4][8];
  __shared__ int es[8];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t tile = blockIdx.x, row = tile * 128 + tid;
  double x[8];
  if (row < n) {
    const double2* p = reinterpret_cast<const double2*>(V + row * 8);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const double2 v = p[i];
      x[2 * i] = v.x;
      x[2 * i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = 0.0;
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const uint32_t hi = (uint32_t)((unsigned long long)__double_as_longlong(x[c]) >> 32) & 0x7FFFFFFFu;
    const uint32_t m = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) red[warp][c] = m;
  }
  __syncthreads();
  if (tid < 8) {
    const uint32_t m = max(max(red[0][tid], red[1][tid]), max(red[2][tid], red[3][tid]));
    const int e = ft_exp_of_hi(m);
    es[tid] = e;
    ex[tile * 8 + tid] = e;
  }
  __syncthreads();
  ft_store_row_digits(x, es, planes + (size_t)tile * FT_PLANE_TILE + ft_row_off(tid));
}

void launch_block_digits(cudaStream_t st, const double* V, int64_t n, int* ex, unsigned char* planes,
                         const Ctl* ctl, int guard) {
  const int64_t tiles = (n + 127) / 128;
  if (tiles > 0) k_block_digits<<<(unsigned)tiles, 128, 0, st>>>(V, n, ex, planes, ctl, guard);
}

// W = A V for s = 8 in FP64 (CSR, one thread per (row, column): the same
// summation as the plain SpMM), fused with W's tile exponents and digit
// planes: one CTA of 1024 threads per 128-row tile stages the tile's W in
// shared memory, reduces its column maxima and writes the digits, so W is not
// read back by a separate pass.
__global__ void __launch_bounds__(1024) k_spmm_digits(int64_t n, const int32_t* __restrict__ rowptr,
                                                      const int32_t* __restrict__ colidx,
                                                      const double* __restrict__ vals,
                                                      const double* __restrict__ V, double* __restrict__ W,
                                                      int* __restrict__ ex, unsigned char* __restrict__ planes,
                                                      const Ctl* ctl, int guard) {
  if (guard && !*(volatile const int*)&ctl->active) return;
  __shared__ double wt[128][9];   // the tile's W (padded rows)
  __shared__ uint32_t red[32][8];
  __shared__ int es[8];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r = tid >> 3, c = tid & 7;
  const int64_t tile = blockIdx.x, row = tile * 128 + r;
  double acc = 0.0;
  if (row < n) {
    const int p0 = rowptr[row], p1 = rowptr[row + 1];
    for (int p = p0; p < p1; ++p) acc = fma(vals[p], V[(int64_t)colidx[p] * 8 + c], acc);
    W[row * 8 + c] = acc;
  }
  wt[r][c] = acc;
  // column maxima (high words of |x|): lanes c, c + 8, c + 16, c + 24 share a column
  uint32_t hi = (uint32_t)((unsigned long long)__double_as_longlong(acc) >> 32) & 0x7FFFFFFFu;
  hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, 8));
  hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, 16));
  if (lane < 8) red[warp][lane] = hi;
  __syncthreads();
  if (tid < 8) {
    uint32_t m = 0;
    for (int w = 0; w < 32; ++w) m = max(m, red[w][tid]);
    const int e = ft_exp_of_hi(m);
    es[tid] = e;
    ex[tile * 8 + tid] = e;
  }
  __syncthreads();
  if (tid < 128) {
    double x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = wt[tid][q];
    ft_store_row_digits(x, es, planes + (size_t)tile * FT_PLANE_TILE + ft_row_off(tid));
  }
}

void launch_spmm_digits(cudaStream_t st, int64_t n, const int32_t* rowptr, const int32_t* colidx,
                        const double* vals, const double* V, double* W, int* ex, unsigned char* planes,
                        const Ctl* ctl, int guard) {
  const int64_t tiles = (n + 127) / 128;
  if (tiles > 0)
    k_spmm_digits<<<(unsigned)tiles, 1024, 0, st>>>(n, rowptr, colidx, vals, V, W, ex, planes, ctl, guard);
}

// ---------------------------------------------------------------- Gram
// G = L^T R with L = [L_1..L_a], R = [R_1..R_b] (s = 8) given by their
// exponents and digit planes, the partial sums of one CTA's rows (whole
// 128-row tiles) into partials[blockIdx.x][a s][b s].  With `shared`, R_1 is
// L_a (the lagged skeletons' [V_1..V_{k-1}, U]^T [U, W]), read once.
//
// Rows go in slabs of 16 (one MMA K step) and windows of 128 (one tile: the
// exponents' group and the exact accumulation window).  The A operand is
// L^T's digit plane t (M = L columns, K-major: the core-matrix row of column
// c holds its 8 rows of the group), the B operand the stack of R's digits
// u = 0..7 (N = 16 u + R column, slot 7 zero); the MMA of digit t writes from
// tensor-memory column 16 t, so pair (t, u) lands on level t + u.  Roles
// (512 threads, 16 warps, up to 128 registers a thread):
//   warps 0-9: expand a slab's digit bytes from its stage into the operands
//     of slab buffer q % ndb, warps 0-4 the even slabs and warps 5-9 the odd
//     ones (two slabs in flight).  Task = (digit t, 8-row group kg, block slot):
//     the 8 x 8 bytes of the group's rows and the block's columns are read
//     (64 contiguous bytes) and written column by column as fp16 (the byte
//     pair of rows 2i, 2i + 1 of a column is one fp16 pair, so the K order
//     is the row order in both operands);
//   warp 10: bulk copies (cp.async.bulk, the TMA engine) of every block's two
//     slabs of a stage (1792 contiguous bytes) into a ring of nst stages, one
//     block per lane;
//   warp 11 (one lane): the MMAs of a slab once it is expanded;
//   warps 12-15: the epilogue of each 128-row window (tensor-memory lanes =
//     L columns; with two M tiles, tile 0 then tile 1), overlapping the
//     next window's expansion and MMAs.
// Barriers (parity = use count & 1):
//   full[st]  bulk copies -> expansion warps     empty[st] expansion warps -> copies
//   dfull[b]  expansion warps -> MMA issue       dfree[b]  MMA commit -> expansion warps
//   wdone[w]  MMA commit at a window's end -> epilogue warps
//   tfree[w]  epilogue warps -> MMA issue (accumulator buffer w reusable)
// A tile column with a non-finite value (exponent 1025) makes G NaN.
#define GF_THREADS 512
#define GF_SPLIT_WARPS 10
#define GF_TMA_WARP 10
#define GF_MMA_WARP 11
#define GF_EPI_WARP0 12
#define GF_MAXSPLIT 24     // blocks read per slab: a + b - shared
#define GF_SSTRIDE 1808    // bytes per block in a stage: 2 slabs (1792) + 16 (bank offset)
#define GF_ASBO 272        // A operand: bytes from one 8-column group to the next (256 + 16)
#define GF_MAXST 6
#define GF_MAXDB 3         // digit slab buffers

struct F64Planes {
  const unsigned char* p[LSBA_MAXB];   // digit planes
  const int* e[LSBA_MAXB];             // per-(tile, column) exponents: e[i][tile * 8 + c]
};

struct GramF64Args {
  F64Planes L, R;
  int a, b, as, bs, shared, nsplit;
  int ma, ntile, tile1;
  uint32_t aplane_bytes, dbuf_bytes, acc_bytes, stage_bytes, tcols;
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

// Source block of slot i (0 .. nsplit-1): L blocks, then the R blocks not shared.
__device__ __forceinline__ void gf_slot(const GramF64Args& g, int i, const unsigned char** p, int* lblk,
                                        int* rblk) {
  if (i < g.a) {
    *p = g.L.p[i];
    *lblk = i;
    *rblk = (g.shared && i == g.a - 1) ? 0 : -1;
  } else {
    const int r = i - g.a + (g.shared ? 1 : 0);
    *p = g.R.p[r];
    *lblk = -1;
    *rblk = r;
  }
}

// fp16 digit pairs of column c (bytes c of rows 2i and 2i + 1, i = 0..3) of an
// 8 x 8 byte block held as rows w[0..7] (lo, hi words), as one 16-byte row.
__device__ __forceinline__ uint4 gf_column(const uint2 (&w)[8], int c) {
  const uint32_t b = (uint32_t)(c & 3), sel = b | ((4u + b) << 8);
  const __half2 off = __halves2half2(__ushort_as_half((unsigned short)0x6480u),
                                     __ushort_as_half((unsigned short)0x6480u));
  uint32_t h[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t x0 = c >= 4 ? w[2 * i].y : w[2 * i].x, x1 = c >= 4 ? w[2 * i + 1].y : w[2 * i + 1].x;
    const uint32_t v = (__byte_perm(x0, x1, sel) & 0x00FF00FFu) | 0x64006400u;
    const __half2 d = __hsub2(*reinterpret_cast<const __half2*>(&v), off);
    h[i] = *reinterpret_cast<const uint32_t*>(&d);
  }
  return make_uint4(h[0], h[1], h[2], h[3]);
}

__global__ void __launch_bounds__(GF_THREADS, 1) k_gram_f64tc(const __grid_constant__ GramF64Args g) {
  if (g.guard && !*(volatile const int*)&g.ctl->active) return;
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* dbuf = sm;                                                   // [ndb] digit slabs
  double* accs = reinterpret_cast<double*>(sm + (size_t)g.ndb * g.dbuf_bytes);  // [16][ma]
  unsigned char* stage = sm + (size_t)g.ndb * g.dbuf_bytes + g.acc_bytes;     // [nst] plane stages
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
      mbar_init(&dfull[i], GF_SPLIT_WARPS / 2);
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

  const int64_t ntile_all = (g.n + 127) / 128;
  const int64_t tile0 = (int64_t)blockIdx.x * g.tiles_per_cta;
  const int64_t tile_end = min(ntile_all, tile0 + (int64_t)g.tiles_per_cta);
  const int nslab = tile_end > tile0 ? (int)(tile_end - tile0) * 8 : 0;   // 16-row slabs
  const int nstg = nslab / 2;                                               // stages of two slabs
  bool failed = false;

  if (warp == GF_TMA_WARP) {
    // ---- bulk copies: stage qs holds slabs 2 qs, 2 qs + 1 of every block,
    // lane i copying block slot i
    for (int qs = 0; qs < nstg && !failed; ++qs) {
      const int st = qs % g.nst;
      bool f = false;
      if (lane == 0 && qs >= g.nst && !mbar_wait_bounded(&empty[st], (unsigned)((qs / g.nst - 1) & 1)))
        f = true;
      if (lane == 0 && !f) mbar_expect_tx(&full[st], 2u * FT_PLANE_SLAB * (unsigned)g.nsplit);
      failed = __any_sync(0xffffffffu, f);
      if (failed) break;
      const int64_t tile = tile0 + (qs >> 2);
      const size_t off = (size_t)tile * FT_PLANE_TILE + (size_t)(qs & 3) * 2 * FT_PLANE_SLAB;
      unsigned char* dst = stage + (size_t)st * g.stage_bytes;
      for (int i = lane; i < g.nsplit; i += 32) {
        const unsigned char* p;
        int lb, rb;
        gf_slot(g, i, &p, &lb, &rb);
        bulk_copy_g2s(dst + (size_t)i * GF_SSTRIDE, p + off, 2u * FT_PLANE_SLAB, &full[st]);
      }
    }
    if (failed && lane == 0 && g.err) atomicExch(g.err, 1);
  } else if (warp == GF_MMA_WARP) {
    // ---- MMA issue.  Descriptors are formed once: the start-address field
    // (address >> 4, 14 bits) of a base descriptor is advanced by adding
    // (byte offset >> 4), which cannot carry out of the field (shared memory
    // is below 256 KB).
    if (lane == 0) {
      const uint32_t pa0 = smem_addr(dbuf);
      const uint64_t adesc0 = tc_smem_desc(pa0, 128, GF_ASBO);
      const uint64_t bdesc0 = tc_smem_desc(pa0 + 7u * g.aplane_bytes, 128, 256);
      const uint64_t bstep = g.dbuf_bytes >> 4;   // one slab buffer further
      const uint64_t astep = g.aplane_bytes >> 4, a1 = (uint64_t)(((g.tile1 >> 3) * GF_ASBO) >> 4);
      int b = 0, bu = 0;   // slab buffer and its use count
      for (int q = 0; q < nslab && !failed; ++q) {
        const int w = q >> 3, wb = w & 1;
        if ((q & 7) == 0 && w >= 2 && !mbar_wait_bounded(&tfree[wb], (unsigned)(((w - 2) >> 1) & 1)))
          failed = true;
        if (!failed && !mbar_wait_bounded(&dfull[b], (unsigned)(bu & 1))) failed = true;
        if (failed) break;
        tc_fence_after();
        const uint64_t ab = adesc0 + (uint64_t)b * bstep, bd = bdesc0 + (uint64_t)b * bstep;
        const uint32_t first = (q & 7) ? 1u : 0u;
        for (int T = 0; T < g.ntile; ++T) {
          const uint64_t at = ab + (T ? a1 : 0ull);
          const uint32_t dcol = tmem + (uint32_t)((wb * g.ntile + T) * 128);
#pragma unroll
          for (int t = 0; t < 7; ++t)
            tc_mma_bf16(dcol + (uint32_t)(16 * t), at + (uint64_t)t * astep, bd, tc_idesc_f16_f32(128, 16 * (8 - t)),
                        t ? 1u : first);
        }
        tc_commit(&dfree[b]);
        if ((q & 7) == 7 || q == nslab - 1) tc_commit(&wdone[wb]);
        if (++b == g.ndb) {
          b = 0;
          ++bu;
        }
      }
      if (failed && g.err) atomicExch(g.err, 1);
    }
  } else if (warp >= GF_EPI_WARP0) {
    // ---- epilogue warps: lanes 32 (warp % 4) .. of each M tile = L columns.
    // The exponents of a window are loaded one window ahead.
    const int nwin = nslab > 0 ? ((nslab - 1) >> 3) + 1 : 0;
    int mcol[2];
    bool mvalid[2];
    for (int T = 0; T < 2; ++T) {
      mcol[T] = (T ? g.tile1 : 0) + 32 * (warp & 3) + lane;
      mvalid[T] = T < g.ntile && mcol[T] < g.as && (T == 0 || mcol[T] >= 128);
    }
    int ELn[2], ERn[16];
    auto load_exps = [&](int w) {
      const int64_t tile = tile0 + w;
#pragma unroll
      for (int T = 0; T < 2; ++T) ELn[T] = mvalid[T] ? g.L.e[mcol[T] >> 3][tile * 8 + (mcol[T] & 7)] : 0;
#pragma unroll
      for (int j = 0; j < 16; ++j) ERn[j] = j < g.bs ? g.R.e[j >> 3][tile * 8 + (j & 7)] : 0;
    };
    if (nwin > 0) load_exps(0);
    for (int w = 0; w < nwin && !failed; ++w) {
      const int wb = w & 1;
      int EL[2], ER[16];
#pragma unroll
      for (int T = 0; T < 2; ++T) EL[T] = ELn[T];
#pragma unroll
      for (int j = 0; j < 16; ++j) ER[j] = ERn[j];
      if (w + 1 < nwin) load_exps(w + 1);
      gf_wait(&wdone[wb], (unsigned)((w >> 1) & 1), failed, g.err);
      tc_fence_after();
      if (!failed) {
        for (int T = 0; T < g.ntile; ++T) {
          const int m = mcol[T];
          const bool valid = mvalid[T];
          if (valid && EL[T] >= FT_EXP_NONFINITE) *bad = 1;
          const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((wb * g.ntile + T) * 128);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            long long Tv[8];
            ft_levels8b(ta + (uint32_t)(8 * h), Tv);
            if (valid && 8 * h < g.bs) {
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int Ej = ER[8 * h + j];
                if (Ej >= FT_EXP_NONFINITE) *bad = 1;
                double* a = accs + (size_t)(8 * h + j) * g.ma + m;
                *a = ft_fma_pow2((double)Tv[j], EL[T] + Ej - 55, *a);
              }
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tfree[wb]);
    }
    // every epilogue warp's NaN marks before the outputs
    asm volatile("bar.sync 1, 128;" ::: "memory");
    if (!failed) {
      const bool nan_out = *(volatile int*)bad != 0;
      for (int T = 0; T < g.ntile; ++T) {
        const int m = (T ? g.tile1 : 0) + 32 * (warp & 3) + lane;
        if (m < g.as && (T == 0 || m >= 128)) {
          double* out = g.partials + (int64_t)blockIdx.x * g.q + (int64_t)m * g.bs;
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (j < g.bs) out[j] = nan_out ? __longlong_as_double(0x7FF8000000000000ll) : accs[(size_t)j * g.ma + m];
        }
      }
    }
  } else {
    // ---- expansion warps.  Task index k = (t * 2 + kg) * nsplit + slot, so
    // the lanes of a warp mostly share (t, kg) and take consecutive slots
    // (their shared-memory rows GF_SSTRIDE and GF_ASBO apart fall in
    // different banks).
    const int ntask = 14 * g.nsplit;
    const int grp = warp >= GF_SPLIT_WARPS / 2 ? 1 : 0, gtid = tid - grp * (GF_SPLIT_WARPS / 2) * 32;
    for (int q = grp; q < nslab && !failed; q += 2) {
      const int qs = q >> 1, st = qs % g.nst, b = q % g.ndb;
      gf_wait(&full[st], (unsigned)((qs / g.nst) & 1), failed, g.err);
      const unsigned char* S = stage + (size_t)st * g.stage_bytes + (size_t)(q & 1) * FT_PLANE_SLAB;
      if (q >= g.ndb) gf_wait(&dfree[b], (unsigned)((q / g.ndb - 1) & 1), failed, g.err);
      unsigned char* D = dbuf + (size_t)b * g.dbuf_bytes;
      if (!failed) {
        for (int k = gtid; k < ntask; k += (GF_SPLIT_WARPS / 2) * 32) {
          const int slot = k % g.nsplit, tk = k / g.nsplit, t = tk >> 1, kg = tk & 1;
          int lb, rb;
          if (slot < g.a) {
            lb = slot;
            rb = (g.shared && slot == g.a - 1) ? 0 : -1;
          } else {
            lb = -1;
            rb = slot - g.a + (g.shared ? 1 : 0);
          }
          const uint4* src = reinterpret_cast<const uint4*>(S + (size_t)slot * GF_SSTRIDE + (size_t)t * 128 +
                                                            (size_t)kg * 64);
          uint2 w[8];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const uint4 v = src[i];
            w[2 * i] = make_uint2(v.x, v.y);
            w[2 * i + 1] = make_uint2(v.z, v.w);
          }
          unsigned char* dA = lb >= 0 ? D + (size_t)t * g.aplane_bytes + (size_t)lb * GF_ASBO + (size_t)kg * 128
                                      : nullptr;
          // digit u = t of the R stack: N rows 16 u + 8 rb .. are 2 u + rb core groups further
          unsigned char* dB = rb >= 0 ? D + 7 * (size_t)g.aplane_bytes + (size_t)(2 * t + rb) * 256 + (size_t)kg * 128
                                      : nullptr;
          // digit plane t of the stored bytes is digit t (0 = most significant)
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const uint4 row = gf_column(w, c);
            if (dA) *reinterpret_cast<uint4*>(dA + c * 16) = row;
            if (dB) *reinterpret_cast<uint4*>(dB + c * 16) = row;
          }
        }
      }
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

static uint32_t gram_f64tc_aplane(int ma) { return (uint32_t)(ma / 8) * GF_ASBO; }

// Shared memory: ndb digit slabs, the accumulators, nst plane stages, barriers.
static size_t gram_f64tc_smem(int ma, int nsplit, int nst, int ndb) {
  return (size_t)ndb * (7 * (size_t)gram_f64tc_aplane(ma) + 4096) + (size_t)16 * ma * 8 +
         (size_t)nst * nsplit * GF_SSTRIDE + (2 * GF_MAXST + 2 * GF_MAXDB + 4) * 8 + 16;
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
  const int nsplit = a + b;   // upper bound (shared reads one fewer)
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

void launch_gram_f64tc(cudaStream_t st, const GramPlan& p, const unsigned char* const* L,
                       const int* const* Le, int a, const unsigned char* const* R, const int* const* Re,
                       int b, bool shared, int64_t n, double* partials, double* G, const Ctl* ctl,
                       int guard, int* err) {
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
  g.aplane_bytes = gram_f64tc_aplane(g.ma);
  g.dbuf_bytes = 7u * g.aplane_bytes + 4096u;
  g.acc_bytes = 16u * (uint32_t)g.ma * (uint32_t)sizeof(double);
  g.stage_bytes = (uint32_t)g.nsplit * GF_SSTRIDE;
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
// n x 8 blocks in_1..in_nin given by their exponents and digit planes, with
// the coefficients folded beforehand (k_coef_fold64); the outputs are written
// in FP64 together with their own exponents and digit planes.  For a 128-row
// tile (the MMA's M) with input exponents e_kk and E = max_kk e_kk,
// coefficient row kk is scaled by 2^(e_kk - E) and split with one exponent
// f_n per output column n, so sum_kk in[r][kk] C[kk][n] = 2^(E + f_n - 55)
// T[r][n]; K = 8 nin columns go in k-steps of 16 (two input blocks), and the
// level sums are flushed into FP64 every 8 k-steps (a window: 128 columns
// keep them exact).  X's own term is added in FP64 (late in a solve X is much
// larger than its correction, so it does not go through the digits).
//
// One persistent CTA an SM, 18 warps in four roles joined by mbarriers:
//   warps 0-7 (expansion), two groups of four taking alternate k-steps (two
//     k-steps in flight): per k-step, thread r of the group expands row r's 7
//     digit rows (8 bytes -> 8 fp16) of both blocks from the ring into the A
//     operand buffer g % 3, which lives in tensor memory (lane = row, 8
//     columns a digit plane: tcgen05.st, so the A digits never pass through
//     shared memory), and splits two coefficient values into the B stack in
//     shared memory (N = 8 digit slots x 16 outputs, slot 7 zero) from the
//     launch's significand table; at a tile's start all eight form E and the
//     f_n (parameter slot j % 8);
//   warp 16, lane 0: bulk copies (the TMA engine) of the plane sets (7 KB,
//     one block's tile) into a ring of UF_NST stages, across tiles;
//   warp 17, lane 0: the 7 MMAs of a k-step (digit t of A against slots
//     0..7-t, into accumulator column 16 t, so pair (t, u) lands on level
//     t + u) into accumulator buffer (window % 2);
//   warps 8-15 (epilogue; tensor-memory lanes = rows, warp 8 + 4 o + i for
//     lane quarter i and output half o): each window's levels into 8 FP64
//     accumulators a row, then X's term, the outputs, their exponents and
//     digit planes, while the next tile's k-steps run.
// Tensor memory: accumulators in columns [0, 256), A buffers of 56 columns
// from column 256.
// Barriers (parity = use count & 1): full/empty (ring), afull/afree (operand
// buffers), accfull/accfree (accumulators), pready/pfree (tile parameters).
// A wait that gives up sets the CTA's abort flag; from then on every wait
// returns at once and no copy or MMA is issued, so every role runs out its
// loops and the CTA ends after its copies and MMAs in flight have landed.
// A non-finite input (exponent 1025) or coefficient makes the tile's outputs
// NaN.
#define UF_THREADS 576
#define UF_EWARP0 8
#define UF_PWARP 16
#define UF_MWARP 17
#define UF_MAXIN 24
#define UF_FLUSH 8
#define UF_NST 12
#define UF_ND 3
#define UF_ACOL 256        // tensor-memory column of A buffer 0 (56 columns each)
#define UF_PSLOTS 8
#define UF_PSTRIDE 20
#define UF_OFF_B (UF_NST * FT_PLANE_TILE)
#define UF_OFF_CM (UF_OFF_B + UF_ND * 4096)
#define UF_OFF_CS (UF_OFF_CM + 8 * UF_MAXIN * 16 * 8)
#define UF_OFF_EX (UF_OFF_CS + 8 * UF_MAXIN * 16 * 2)
#define UF_OFF_PAR (UF_OFF_EX + 8 * UF_MAXIN * 4)
#define UF_OFF_RED (UF_OFF_PAR + UF_PSLOTS * UF_PSTRIDE * 4)
#define UF_OFF_BAR (UF_OFF_RED + 1024)
#define UF_SMEM (UF_OFF_BAR + 512)

struct UpdF64Args {
  const unsigned char* ip[UF_MAXIN];   // input digit planes
  const int* ie[UF_MAXIN];             // input exponents
  int nin, nks, nw;                    // inputs, k-steps and windows a tile
  const double* X;
  int64_t n;
  double* out1;
  double* out2;
  int* e_out1;
  int* e_out2;
  unsigned char* p_out1;
  unsigned char* p_out2;
  const double* cf;      // C1' [ncoef * 8][8] row-major, then C2' likewise
  int ncoef;
  const Ctl* ctl;
  int step;
  int* err;
};

__device__ __forceinline__ void uf_bar(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// A bounded wait that honours the CTA's abort flag (see above).
__device__ __forceinline__ bool uf_wait(uint64_t* bar, unsigned parity, volatile int* abortf, int* err) {
  if (*abortf) return false;
  if (mbar_wait_bounded(bar, parity)) return true;
  *abortf = 1;
  if (err) atomicExch(err, 1);
  return false;
}

// Tensor-memory stores of 4 columns (32-bit) for the warp's 32 lanes, and
// the MMA with the A operand in tensor memory (kind::f16, issued by one thread).
__device__ __forceinline__ void uf_st4(uint32_t taddr, uint4 v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(v.x),
               "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}
__device__ __forceinline__ void uf_mma_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__global__ void __launch_bounds__(UF_THREADS, 1) k_update_f64tc(const __grid_constant__ UpdF64Args u) {
  if (u.step >= 0 && *(volatile const int*)&u.ctl->update_step != u.step) return;
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* ring = sm;                                            // [UF_NST][7168] plane sets
  unsigned char* bst = sm + UF_OFF_B;                                  // [UF_ND][4096] fp16 B stacks
  unsigned long long* cm = reinterpret_cast<unsigned long long*>(sm + UF_OFF_CM);  // [8 nin][16]
  short* cs = reinterpret_cast<short*>(sm + UF_OFF_CS);                // [8 nin][16]
  int* exs = reinterpret_cast<int*>(sm + UF_OFF_EX);                   // [8 nin]
  int* par = reinterpret_cast<int*>(sm + UF_OFF_PAR);                  // [UF_PSLOTS][UF_PSTRIDE]
  int* redx = reinterpret_cast<int*>(sm + UF_OFF_RED);                 // [8][16] + [8]
  uint32_t* rede = reinterpret_cast<uint32_t*>(sm + UF_OFF_RED + 576); // [8 warps][8]
  int* eo = reinterpret_cast<int*>(sm + UF_OFF_RED + 832);             // [16]
  volatile int* abortf = reinterpret_cast<volatile int*>(sm + UF_OFF_RED + 960);
  int* badc = reinterpret_cast<int*>(sm + UF_OFF_RED + 964);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + UF_OFF_BAR);
  uint64_t* empty = full + UF_NST;
  uint64_t* afull = empty + UF_NST;
  uint64_t* afree = afull + UF_ND;
  uint64_t* accfull = afree + UF_ND;
  uint64_t* accfree = accfull + 2;
  uint64_t* pready = accfree + 2;
  uint64_t* pfree = pready + UF_PSLOTS;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + UF_OFF_BAR + 448);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nin = u.nin, K = 8 * nin, nks = u.nks, nw = u.nw;
  const bool two = u.out2 != nullptr;
  const int64_t ntile = (u.n + 127) / 128;
  const int64_t ntl = (int64_t)blockIdx.x < ntile ? (ntile - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t nq = ntl * nin;   // plane sets this CTA consumes, in (tile, block) order

  for (int i = tid * 16; i < UF_ND * 4096; i += UF_THREADS * 16)
    *reinterpret_cast<uint4*>(bst + i) = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    *abortf = 0;
    *badc = 0;
    for (int i = 0; i < UF_NST; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 4);
    }
    for (int i = 0; i < UF_ND; ++i) {
      mbar_init(&afull[i], 4);
      mbar_init(&afree[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accfull[i], 1);
      mbar_init(&accfree[i], 8);
    }
    for (int i = 0; i < UF_PSLOTS; ++i) {
      mbar_init(&pready[i], 1);
      mbar_init(&pfree[i], 8);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc_alloc(tslot, 512);
  tc_fence_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  // The coefficients' significand table (tile-independent): for (kk, n),
  // cm = 2 m | sign << 63 (m the 53-bit significand, 52 bits for subnormals)
  // and cs = 1022 - max(eb, 1), so that digit integer of C[kk][n] 2^(e_kk - E)
  // against group exponent F is (2 m) >> (F + E - e_kk + cs).
  for (int e = tid; e < 16 * K; e += UF_THREADS) {
    const int n = e & 15, kk = e >> 4;
    unsigned long long mv = 0ull;
    int sh = 1021;
    if (n < 8 || two) {
      const double c = u.cf[(n < 8 ? 0 : (size_t)u.ncoef * 64) + (size_t)kk * 8 + (n & 7)];
      const unsigned long long b = (unsigned long long)__double_as_longlong(c);
      const int eb = (int)((b >> 52) & 0x7FF);
      if (eb == 0x7FF) *badc = 1;
      const unsigned long long m = (b & 0x000FFFFFFFFFFFFFull) | (eb ? 0x0010000000000000ull : 0ull);
      mv = (m << 1) | (b & 0x8000000000000000ull);
      sh = 1022 - max(eb, 1);
    }
    cm[kk * 16 + n] = mv;
    cs[kk * 16 + n] = (short)sh;
  }
  __syncthreads();
  if (warp < UF_EWARP0) {
    // ================= expansion warps (256 threads)
    // group grp (warps 4 grp .. 4 grp + 3) takes the k-steps g = grp (mod 2);
    // thread gr of a group: row r = gr of both blocks (A) and coefficient
    // values gr, gr + 128 (B)
    const int grp = warp >> 2, gr = tid & 127, r = gr;
    int ne = (tid < K && ntl > 0) ? u.ie[tid >> 3][(int64_t)blockIdx.x * 8 + (tid & 7)] : 0;
    int64_t q = 0;
    int g = 0;
    for (int64_t j = 0; j < ntl; ++j) {
      const int64_t tile = blockIdx.x + j * gridDim.x;
      const int slot = (int)(j % UF_PSLOTS);
      int* pr = par + slot * UF_PSTRIDE;
      uf_bar(1, 256);   // the previous tile's reads of exs and redx are done
      if (tid == 0 && j >= UF_PSLOTS)
        uf_wait(&pfree[slot], (unsigned)(((j / UF_PSLOTS) - 1) & 1), abortf, u.err);
      if (tid < K) exs[tid] = ne;
      if (tid < K && j + 1 < ntl) ne = u.ie[tid >> 3][(tile + gridDim.x) * 8 + (tid & 7)];
      uf_bar(1, 256);
      {
        const int n = tid & 15;
        int mE = FT_EXP_MIN, mF = -100000;
        for (int kk = tid >> 4; kk < K; kk += 16) {
          const int e = exs[kk];
          mE = max(mE, e);
          mF = max(mF, 1022 - (int)cs[kk * 16 + n] + e);
        }
        mF = max(mF, __shfl_xor_sync(0xffffffffu, mF, 16));
        mE = __reduce_max_sync(0xffffffffu, mE);
        if (lane < 16) redx[warp * 16 + lane] = mF;
        if (lane == 0) redx[128 + warp] = mE;
      }
      uf_bar(1, 256);
      if (tid < 16) {
        int mF = redx[tid], mE = redx[128];
        for (int w = 1; w < 8; ++w) {
          mF = max(mF, redx[w * 16 + tid]);
          mE = max(mE, redx[128 + w]);
        }
        pr[2 + tid] = max(mF - mE - 1022, FT_EXP_MIN);
        if (tid == 0) {
          pr[0] = mE;
          pr[1] = mE >= FT_EXP_NONFINITE ? 1 : 0;
        }
      }
      uf_bar(1, 256);
      if (tid == 0) mbar_arrive(&pready[slot]);
      const int E = pr[0];
      int fnv[2];
#pragma unroll
      for (int i = 0; i < 2; ++i) fnv[i] = pr[2 + ((gr + 128 * i) >> 3 & 15)];
      for (int ks = 0; ks < nks; ++ks, ++g) {
        const int nb = (2 * ks + 1 < nin) ? 2 : 1;
        if ((g & 1) != grp) {   // the other group's k-step
          q += nb;
          continue;
        }
        const int d = g % UF_ND, v = g / UF_ND;
        bool ok = true;
        for (int hh = 0; hh < nb; ++hh) {
          const int64_t qq = q + hh;
          ok = uf_wait(&full[qq % UF_NST], (unsigned)((qq / UF_NST) & 1), abortf, u.err) && ok;
        }
        if (v >= 1) ok = uf_wait(&afree[d], (unsigned)((v - 1) & 1), abortf, u.err) && ok;
        ok = __all_sync(0xffffffffu, ok);   // the tensor-memory stores are warp-wide
        if (ok) {
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            // A: digit plane t of block hh -> columns UF_ACOL + 56 d + 8 t + 4 hh, lane r
            const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16) +
                                (uint32_t)(UF_ACOL + 56 * d + 4 * hh);
            if (hh < nb) {
              const unsigned char* S = ring + (size_t)((q + hh) % UF_NST) * FT_PLANE_TILE + ft_row_off(r);
              uint2 w[7];
#pragma unroll
              for (int t = 0; t < 7; ++t) w[t] = *reinterpret_cast<const uint2*>(S + t * 128);
#pragma unroll
              for (int t = 0; t < 7; ++t) uf_st4(ta + (uint32_t)(8 * t), ft_expand8(w[t]));
            } else {
#pragma unroll
              for (int t = 0; t < 7; ++t) uf_st4(ta + (uint32_t)(8 * t), make_uint4(0u, 0u, 0u, 0u));
            }
          }
          asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          // B: coefficient values v2 = gr + 128 i: (kk = 8 (2 ks + ckb) + cq, n = cn)
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            const int v2 = gr + 128 * i;
            const int cq = v2 & 7, cn = (v2 >> 3) & 15, ckb = v2 >> 7;
            const int blk = 2 * ks + ckb;
            unsigned long long gv = FT_BIAS;
            if (blk < nin) {
              const int kk = blk * 8 + cq;
              const unsigned long long mv = cm[kk * 16 + cn];
              const int rs = fnv[i] + E - exs[kk] + (int)cs[kk * 16 + cn];
              const unsigned long long F = rs > 63 ? 0ull : ((mv & 0x7FFFFFFFFFFFFFFFull) >> rs);
              gv = (mv >> 63) ? FT_BIAS - F : FT_BIAS + F;
            }
            unsigned short* Bd = reinterpret_cast<unsigned short*>(
                                     bst + (size_t)d * 4096 + (size_t)(cn >> 3) * 256 + (size_t)ckb * 128 +
                                     (size_t)(cn & 7) * 16) + cq;
#pragma unroll
            for (int t = 0; t < 7; ++t) {
              const int p = 6 - t;
              const uint32_t wd = p >= 4 ? (uint32_t)(gv >> 32) : (uint32_t)gv;
              const uint32_t hw = __byte_perm(wd, 0x64646464u, 0x40u | (uint32_t)(p & 3));
              const __half dg = __hsub(__ushort_as_half((unsigned short)(hw & 0xFFFFu)),
                                       __ushort_as_half((unsigned short)0x6480u));
              Bd[t * 256] = __half_as_ushort(dg);
            }
          }
        }
        tc_fence_smem();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&afull[d]);
          for (int hh = 0; hh < nb; ++hh) mbar_arrive(&empty[(q + hh) % UF_NST]);
        }
        q += nb;
      }
    }
  } else if (warp < UF_PWARP) {
    // ================= epilogue warps (256 threads): lane quarter i = warp & 3,
    // output half o (out1 / out2), row er of each tile
    const int ew = warp - UF_EWARP0, o = ew >> 2, qd = ew & 3, er = 32 * qd + lane;
    const uint32_t tl = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(8 * o);
    const bool olive = o == 0 || two;
    double* outp = o ? u.out2 : u.out1;
    int* eout = o ? u.e_out2 : u.e_out1;
    unsigned char* pout = o ? u.p_out2 : u.p_out1;
    const double* cx = u.cf + (o ? (size_t)u.ncoef * 64 : 0) + (size_t)nin * 64;   // X's coefficient rows
    int wi = 0;
    for (int64_t j = 0; j < ntl; ++j) {
      const int64_t tile = blockIdx.x + j * gridDim.x;
      const int slot = (int)(j % UF_PSLOTS);
      const int* pr = par + slot * UF_PSTRIDE;
      bool ok = uf_wait(&pready[slot], (unsigned)((j / UF_PSLOTS) & 1), abortf, u.err);
      double acc[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[c] = 0.0;
      const int E = pr[0];
      const bool tnan = pr[1] != 0;
      for (int wl = 0; wl < nw; ++wl, ++wi) {
        const int a = wi & 1, z = wi >> 1;
        const bool got = __all_sync(0xffffffffu, uf_wait(&accfull[a], (unsigned)(z & 1), abortf, u.err) && ok);
        if (got && olive) {
          tc_fence_after();
          long long T[8];
          ft_levels8b(tl + (uint32_t)(128 * a), T);
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[c] = ft_fma_pow2((double)T[c], E + pr[2 + 8 * o + c] - 55, acc[c]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&accfree[a]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&pfree[slot]);
      // X's own term (FP64), the outputs, their exponents and digit planes
      const int64_t row = tile * 128 + er;
      bool rowbad = false;
      if (u.X && row < u.n && olive) {
        const double* xr = u.X + row * 8;
        double xv[8];
#pragma unroll
        for (int qv = 0; qv < 8; ++qv) xv[qv] = xr[qv];
#pragma unroll
        for (int qv = 0; qv < 8; ++qv) {
          rowbad |= !(fabs(xv[qv]) <= 1.79769313486231570e308);
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[c] = fma(xv[qv], cx[qv * 8 + c], acc[c]);
        }
      }
      if (rowbad || tnan || *badc) {
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = __longlong_as_double(0x7FF8000000000000ll);
      }
      uf_bar(2, 256);   // every read of X (out1 may be X) before the stores
      if (olive && row < u.n) {
        double2* dp = reinterpret_cast<double2*>(outp + row * 8);
#pragma unroll
        for (int i = 0; i < 4; ++i) dp[i] = make_double2(acc[2 * i], acc[2 * i + 1]);
      }
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const uint32_t hi = (uint32_t)((unsigned long long)__double_as_longlong(acc[c]) >> 32) & 0x7FFFFFFFu;
        const uint32_t m = __reduce_max_sync(0xffffffffu, hi);
        if (lane == 0) rede[ew * 8 + c] = m;
      }
      uf_bar(2, 256);
      if (qd == 0 && lane < 8) {
        const uint32_t* rm = rede + o * 32 + lane;   // warps 4 o .. 4 o + 3
        const uint32_t m = max(max(rm[0], rm[8]), max(rm[16], rm[24]));
        const int e = ft_exp_of_hi(m);
        eo[8 * o + lane] = e;
        if (eout && olive) eout[tile * 8 + lane] = e;
      }
      uf_bar(2, 256);
      if (olive && pout)
        ft_store_row_digits(acc, eo + 8 * o, pout + (size_t)tile * FT_PLANE_TILE + ft_row_off(er));
    }
  } else if (warp == UF_PWARP) {
    // ================= bulk copies of the plane sets, in (tile, block) order
    if (lane == 0) {
      int64_t issued = 0, tl2 = blockIdx.x;
      int blk = 0, st = 0;
      unsigned ph = 0;   // parity of the stage's previous use
      for (int64_t qq = 0; qq < nq; ++qq) {
        if (qq >= UF_NST && !uf_wait(&empty[st], ph, abortf, u.err)) break;
        if (*abortf) break;
        mbar_expect_tx(&full[st], FT_PLANE_TILE);
        bulk_copy_g2s(ring + (size_t)st * FT_PLANE_TILE, u.ip[blk] + tl2 * FT_PLANE_TILE, FT_PLANE_TILE,
                      &full[st]);
        issued = qq + 1;
        if (++blk == nin) {
          blk = 0;
          tl2 += gridDim.x;
        }
        if (++st == UF_NST) {
          st = 0;
          if (qq >= UF_NST) ph ^= 1u;
        }
      }
      if (*abortf) {
        // the last copy issued into each stage lands before the CTA ends
        for (int64_t qq = issued > UF_NST ? issued - UF_NST : 0; qq < issued; ++qq)
          mbar_wait_bounded(&full[qq % UF_NST], (unsigned)((qq / UF_NST) & 1));
      }
    }
  } else {
    // ================= MMA issue (A from tensor memory, B from shared memory)
    if (lane == 0) {
      int g = 0, wi = 0, last = -1;
      for (int64_t j = 0; j < ntl; ++j) {
        for (int ks = 0; ks < nks; ++ks, ++g) {
          const int d = g % UF_ND, v = g / UF_ND;
          const int a = wi & 1, z = wi >> 1;
          bool ok = true;
          if ((ks % UF_FLUSH) == 0 && z >= 1) ok = uf_wait(&accfree[a], (unsigned)((z - 1) & 1), abortf, u.err);
          ok = uf_wait(&afull[d], (unsigned)(v & 1), abortf, u.err) && ok;
          const bool wend = (ks % UF_FLUSH) == UF_FLUSH - 1 || ks + 1 == nks;
          if (ok) {
            tc_fence_after();
            const uint64_t bd = tc_smem_desc(smem_addr(bst + (size_t)d * 4096), 128, 256);
#pragma unroll
            for (int t = 0; t < 7; ++t) {
              const uint32_t accum = ((ks % UF_FLUSH) || t) ? 1u : 0u;
              uf_mma_ta(tmem + (uint32_t)(128 * a + 16 * t), tmem + (uint32_t)(UF_ACOL + 56 * d + 8 * t), bd,
                        tc_idesc_f16_f32(128, 16 * (8 - t)), accum);
            }
            tc_commit(&afree[d]);
            if (wend) tc_commit(&accfull[a]);
            last = g;
          }
          if (wend) ++wi;
        }
      }
      // the last MMAs complete before the CTA ends
      if (*abortf && last >= 0) mbar_wait_bounded(&afree[last % UF_ND], (unsigned)((last / UF_ND) & 1));
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tc_dealloc(tmem, 512);
}

size_t update_f64tc_smem(int) { return UF_SMEM; }

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

void launch_update_f64tc(cudaStream_t st, const unsigned char* const* in, const int* const* ein,
                         int nin, const double* X, int64_t n, double* out1, int* e_out1,
                         unsigned char* p_out1, double* out2, int* e_out2, unsigned char* p_out2,
                         const double* coef1, const double* tri1, const double* coef2,
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
    cudaFuncSetAttribute(k_update_f64tc, cudaFuncAttributeMaxDynamicSharedMemorySize, UF_SMEM);
  });
  UpdF64Args u;
  memset(&u, 0, sizeof(u));
  for (int i = 0; i < nin; ++i) {
    u.ip[i] = in[i];
    u.ie[i] = ein[i];
  }
  u.nin = nin;
  u.nks = (nin + 1) / 2;
  u.nw = (u.nks + UF_FLUSH - 1) / UF_FLUSH;
  u.X = X;
  u.n = n;
  u.out1 = out1;
  u.out2 = out2;
  u.e_out1 = e_out1;
  u.e_out2 = e_out2;
  u.p_out1 = p_out1;
  u.p_out2 = p_out2;
  u.cf = cf;
  u.ncoef = ncoef;
  u.ctl = ctl;
  u.step = step;
  u.err = err;
  // One CTA an SM, one short of filling the GPU: the SM left free takes the
  // iteration's small side kernel.
  const int64_t tiles = (n + 127) / 128;
  int64_t grid = num_sms - 1;
  if (grid > tiles) grid = tiles;
  if (grid < 1) grid = 1;
  k_update_f64tc<<<(unsigned)grid, UF_THREADS, UF_SMEM, st>>>(u);
}

}  // namespace lsba
