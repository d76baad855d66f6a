// Double-float basis update on the tensor cores (tcgen05), s = 8.
//
// Iteration k >= 2 of a lagged skeleton (Alg. 6 and 7) writes two n x 8
// blocks in one pass over its inputs [V_1..V_{k-1}, U, W]:
//   out1 = V_k = (sum_b in_b C1_b) T1^{-1},
//   out2       = (sum_b in_b C2_b + out1 Chain) T2^{-1}   (T2 for BCGSI+LS only).
// The cycle end (Eq. (7) and Thm. 1) writes X and the next residual block from
// [V_1..V_{j+1}] and X in the same way, without the triangular factors; there
// X's own term X C1_X is added in double-float in the epilogue and only the
// basis terms go through the digits, so that the digit error is relative to
// the correction, not to X (a restarted solve adds one correction per cycle).
// The triangular factors and the chain term act on the columns only, so they
// are folded into the coefficients once per launch (k_coef_fold, FP64):
//   C1' = C1 T1^{-1},   C2' = (C2 + C1' Chain) T2^{-1},
// and out1 = sum_b in_b C1'_b, out2 = sum_b in_b C2'_b.  This is the same
// product taken in another order; the rounding of a term is still relative to
// its own size (the folded coefficients are rounded once to double-float).
// The contraction sum_b in_b [C1'_b | C2'_b] is a product of an n x K matrix
// (K = 8 nin) with a K x 16 one, done here exactly on digits as in the
// tensor-core Gram (kernels_tc.cu):
//   * rows are taken in tiles of 128 (the MMA's M); for column kk of the
//     inputs, e_kk is the exponent of its maximum over the tile (stored with
//     the basis digits; computed here for U and W), and each value is six
//     digits in units of 2^(e_kk - 7 - 8t);
//   * the coefficient rows are scaled by 2^(e_kk - e_max) (exact) and split
//     into six digits with one exponent f_n per output column n, so that
//     sum_kk A[r][kk] B[kk][n] = sum_{t,u} (sum_kk dA dB) 2^(e_max + f_n - 14 - 8(t+u));
//   * the level sums l = t + u <= 5 are exact in the FP32 tensor-memory
//     accumulators over 64 columns (every term an integer <= 2^15, a level
//     sum < 6 * 64 * 2^15 < 2^24), then added into a double-float accumulator
//     per row and output column.
// The A operand comes straight from the stored digit planes (MN-major: 8 rows
// of one column per 16 bytes, LBO = 12288 between 8-column blocks, SBO = 128
// between 8-row groups); U and W are split here.
#include <cfloat>
#include <cuda_bf16.h>

#include "df.cuh"
#include "lsba_internal.cuh"
#include "tc.cuh"

namespace lsba {

#define UT_THREADS 128           // one thread per row of the 128-row tile; two CTAs per SM
#define UT_SUB 2                 // blocks per sub-chunk: 16 columns, one K-step
#define UT_FLUSH 4               // sub-chunks per exact accumulation window (64 columns)
#define UT_BLK 12288             // one block's digits for a 128-row tile: 6 digits x 16 row groups x 128 B
#define UT_MAXK 256              // K = 8 nin <= 256
#define UT_DIG_GROUP 3072        // stored layout: one 32-row chunk of an 8-column group

struct UpdTcsArgs {
  const unsigned char* dig;      // stored digits: block i at dig + i * dig_stride
  const int* dexp;               // stored exponents: block i at dexp + i * dexp_stride
  size_t dig_stride, dexp_stride;
  int a;                         // stored input blocks V_1..V_a; inputs [V_1..V_a, U, W]
  int nsplit;                    // blocks split here: 2 (U, W) or 0
  int nin, kpad;                 // nin = a + nsplit; kpad = 8 nin rounded up to 32
  int ncoef;                     // coefficient blocks: nin, or nin + 1 with X
  const float2* U;
  const float2* W;
  const float2* X;               // optional addend block (coefficients after the nin blocks)
  int64_t n;
  float2* out1;
  float2* out2;
  const float2* cdf;             // folded coefficients: C1' (ncoef x 64), then C2'
  unsigned char* dig_out;        // optional: digit planes and exponents of out1, in the
  int* dexp_out;                 //   stored layout (kernels_tc.cu), written from registers
  const Ctl* ctl;
  int step;
  int* err;
};

__device__ __forceinline__ float ut_round(float y) {
  return __fsub_rn(__fadd_rn(y, 12582912.f), 12582912.f);
}
// Six digits of (hi, lo) in units of 2^(e - 7 - 8t); sc = 2^(7 - e).
__device__ __forceinline__ void ut_digits(float2 x, float sc, float (&d)[6]) {
  float y = __fmul_rn(x.x, sc);
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const float q = ut_round(y);
    d[t] = q;
    if (t < 5) y = __fmul_rn(__fsub_rn(y, q), 256.f);
  }
  float z = __fmul_rn(__fmul_rn(x.y, sc), 16777216.f);
#pragma unroll
  for (int t = 3; t < 6; ++t) {
    const float q = ut_round(z);
    d[t] = __fadd_rn(d[t], q);
    if (t < 5) z = __fmul_rn(__fsub_rn(z, q), 256.f);
  }
}
__device__ __forceinline__ float ut_pow2(int k) {  // 2^k, k clamped to the normal range
  k = max(-126, min(127, k));
  return __int_as_float((127 + k) << 23);
}
__device__ __forceinline__ int ut_exp_of(float amax) {  // e with amax < 2^e
  int e = amax > 0.f ? ((__float_as_int(amax) >> 23) & 255) - 126 : 0;
  return max(e, -119);
}
__device__ __forceinline__ uint32_t ut_pack(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
__device__ __forceinline__ void ut_cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void ut_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void ut_cp_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Warp-wide: 8 consecutive 32-bit tensor-memory columns of the warp's lanes.
__device__ __forceinline__ void ut_ld8(uint32_t taddr, float (&v)[8]) {
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

// MINB CTAs per SM: 3 where the shared memory of three fits (K <= 128), else 2.
template <int MINB>
__global__ void __launch_bounds__(UT_THREADS, MINB) k_update_df_tcs(const __grid_constant__ UpdTcsArgs u) {
  if (u.step >= 0 && *(volatile const int*)&u.ctl->update_step != u.step) return;
  extern __shared__ __align__(1024) unsigned char sm[];
  // Shared layout: A buffers [2][UT_SUB blocks][12 KB] | B digit stack | exponents | misc.
  unsigned char* Abuf = sm;
  unsigned char* Bst = sm + 2 * UT_SUB * UT_BLK;
  const uint32_t SB = (uint32_t)(u.kpad / 8) * 128;     // B: bytes per 8 stack rows
  int* ex = reinterpret_cast<int*>(Bst + 12 * SB);       // [UT_MAXK]
  float* red = reinterpret_cast<float*>(ex + UT_MAXK);   // [16][16]
  int* fexp = reinterpret_cast<int*>(red + 256);         // [16]
  uint64_t* mmad = reinterpret_cast<uint64_t*>(fexp + 32);  // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mmad + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nin = u.nin, K = 8 * nin, a = u.a;
  const int64_t nch = (u.n + 31) / 32, ntile = (u.n + 127) / 128;
  const float2* c1g = u.cdf;
  const float2* c2g = u.cdf + (size_t)u.ncoef * 64;

  // Zero the B stack once (padding columns stay zero).
  for (uint32_t i = (uint32_t)tid * 16; i < 12 * SB; i += UT_THREADS * 16)
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

  // U and W split tasks: column uc (0..7 U, 8..15 W), row groups ur0 and ur0 + 8.
  const int uc = tid & 15, ur0 = tid >> 4;
  const bool has_col = u.nsplit == 2;
  const float2* usrc = has_col ? (uc < 8 ? u.U + uc : u.W + (uc - 8)) : nullptr;
  bool failed = false;
  int gj = 0;  // sub-chunks issued so far (mbarrier phases)
  const int nsub = (nin + UT_SUB - 1) / UT_SUB;

  // Stored digit blocks go straight into an A buffer (MN-major per digit).
  auto load_stored = [&](int64_t tl, unsigned char* dst, int bi) {
    for (int p = tid; p < 768; p += UT_THREADS) {
      const int q = p / 192, rem = p % 192, t = rem >> 5, w = rem & 31;
      const int64_t c = tl * 4 + q;
      unsigned char* d = dst + t * 2048 + q * 512 + w * 16;
      if (c < nch)
        ut_cp16(d, u.dig + bi * u.dig_stride + (size_t)c * UT_DIG_GROUP + t * 512 + w * 16);
      else
        *reinterpret_cast<uint4*>(d) = make_uint4(0u, 0u, 0u, 0u);
    }
  };
  // A tile's first sub-chunk of stored blocks, its U and W rows and its stored
  // exponents are fetched while the previous tile is finished (overlap).
  float2 x[2][8];
  int exv[2] = {0, 0};
  auto prefetch = [&](int64_t tl) {
    for (int sl = 0; sl < UT_SUB && sl < a; ++sl) load_stored(tl, Abuf + sl * UT_BLK, sl);
    ut_cp_commit();
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int64_t row = tl * 128 + (ur0 + 8 * h) * 8 + k;
        x[h][k] = (has_col && row < u.n) ? usrc[row * 8] : make_float2(0.f, 0.f);
      }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int kk = tid + UT_THREADS * h;
      exv[h] = kk < 8 * a ? u.dexp[(kk >> 3) * u.dexp_stride + (tl * 4) * 8 + (kk & 7)] : 0;
    }
  };
  if (blockIdx.x < ntile) prefetch(blockIdx.x);

  for (int64_t tile = blockIdx.x; tile < ntile && !failed; tile += gridDim.x) {
    const int64_t r0 = tile * 128;
    // ---- exponents of the stored columns (the tile maximum, kept per chunk)
#pragma unroll
    for (int h = 0; h < 2; ++h)
      if (tid + UT_THREADS * h < 8 * a) ex[tid + UT_THREADS * h] = exv[h];
    // ---- U and W: exponent over the tile, digits kept in registers
    uint4 udig[2][6];
    if (has_col) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float am = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) am = fmaxf(am, fabsf(x[h][k].x));
        red[(ur0 + 8 * h) * 16 + uc] = am;
      }
      __syncthreads();
      float cm = 0.f;
#pragma unroll
      for (int i = 0; i < 16; ++i) cm = fmaxf(cm, red[i * 16 + uc]);
      const int ue = ut_exp_of(cm);
      if (ur0 == 0) ex[8 * a + uc] = ue;
      const float sc = ut_pow2(7 - ue);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float d[8][6];
#pragma unroll
        for (int k = 0; k < 8; ++k) ut_digits(x[h][k], sc, d[k]);
#pragma unroll
        for (int t = 0; t < 6; ++t) {
          udig[h][t].x = ut_pack(d[0][t], d[1][t]);
          udig[h][t].y = ut_pack(d[2][t], d[3][t]);
          udig[h][t].z = ut_pack(d[4][t], d[5][t]);
          udig[h][t].w = ut_pack(d[6][t], d[7][t]);
        }
      }
    }
    __syncthreads();  // ex complete; red free
    // ---- e_max over the columns, then the coefficient digits
    {
      int em = -1000;
      for (int kk = tid; kk < K; kk += UT_THREADS) em = max(em, ex[kk]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
      if (lane == 0) red[warp] = __int_as_float(em);
    }
    __syncthreads();
    int emax = -1000;
#pragma unroll
    for (int i = 0; i < UT_THREADS / 32; ++i) emax = max(emax, __float_as_int(red[i]));
    const int bn = tid & 15, bk0 = tid >> 4;   // coefficient task: output bn, rows bk0 + 8 i
    float bmx = 0.f;
    for (int kk = bk0; kk < K; kk += UT_THREADS / 16) {
      const int b = kk >> 3, q = kk & 7;
      const float2 v = bn < 8 ? c1g[b * 64 + q * 8 + bn] : c2g[b * 64 + q * 8 + (bn - 8)];
      const int dx = ex[kk] - emax;   // <= 0; below 2^-126 the column contributes nothing
      bmx = fmaxf(bmx, fabsf(__fmul_rn(v.x, dx < -126 ? 0.f : ut_pow2(dx))));
    }
    __syncthreads();  // everyone has read red (emax)
    red[bk0 * 16 + bn] = bmx;
    __syncthreads();
    float fm = 0.f;
#pragma unroll
    for (int i = 0; i < UT_THREADS / 16; ++i) fm = fmaxf(fm, red[i * 16 + bn]);
    const int fe = ut_exp_of(fm);
    if (bk0 == 0) fexp[bn] = fe;
    {
      const float sc = ut_pow2(7 - fe);
      for (int kk = bk0; kk < K; kk += UT_THREADS / 16) {
        const int b = kk >> 3, q = kk & 7;
        float2 v = bn < 8 ? c1g[b * 64 + q * 8 + bn] : c2g[b * 64 + q * 8 + (bn - 8)];
        const int dx = ex[kk] - emax;
        const float ps = dx < -126 ? 0.f : ut_pow2(dx);
        v = make_float2(__fmul_rn(v.x, ps), __fmul_rn(v.y, ps));
        float d[6];
        ut_digits(v, sc, d);
#pragma unroll
        for (int t = 0; t < 6; ++t) {
          const int r = 16 * t + bn;   // stack row: digit t of output bn
          *reinterpret_cast<__nv_bfloat16*>(Bst + (uint32_t)(r >> 3) * SB + (uint32_t)(kk >> 3) * 128 +
                                            (uint32_t)(r & 7) * 16 + (uint32_t)(kk & 7) * 2) =
              __float2bfloat16_rn(d[t]);
        }
      }
    }
    // ---- sub-chunks: digits of UT_SUB input blocks per buffer, MMAs, flushes
    auto load_sub = [&](int j) {
      unsigned char* A = Abuf + (size_t)(j & 1) * UT_SUB * UT_BLK;
      for (int sl = 0; sl < UT_SUB; ++sl) {
        const int bi = j * UT_SUB + sl;
        unsigned char* dst = A + sl * UT_BLK;
        if (bi < a) {
          if (j > 0) load_stored(tile, dst, bi);
        } else if (bi < nin) {
          // U (bi == a) or W (bi == a + 1): this thread's column, if it is that block's
          if ((uc < 8) == (bi == a)) {
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
              for (int t = 0; t < 6; ++t)
                *reinterpret_cast<uint4*>(dst + t * 2048 + (ur0 + 8 * h) * 128 + (uc & 7) * 16) = udig[h][t];
          }
        } else {
          for (int p = tid; p < UT_BLK / 16; p += UT_THREADS)
            *reinterpret_cast<uint4*>(dst + p * 16) = make_uint4(0u, 0u, 0u, 0u);
        }
      }
      ut_cp_commit();
    };
    dfacc acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = dfacc{0.f, 0.f};
    load_sub(0);
    for (int j = 0; j < nsub; ++j) {
      ut_cp_wait();
      tc_fence_smem();
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      const int gcur = gj + j;
      if (tid == 0) {
        const uint32_t pa = smem_addr(Abuf + (size_t)(j & 1) * UT_SUB * UT_BLK);
        const uint32_t pb = smem_addr(Bst);
#pragma unroll
        for (int t = 0; t < 6; ++t) {
          const uint32_t idesc = tc_idesc_bf16_f32(128, 16 * (6 - t)) | (1u << 15);  // A MN-major
#pragma unroll
          for (int ks = 0; ks < UT_SUB / 2; ++ks) {
            const uint64_t ad = tc_smem_desc(pa + ks * 2 * UT_BLK + t * 2048, UT_BLK, 128);
            const uint64_t bd = tc_smem_desc(pb + (uint32_t)(j * UT_SUB + 2 * ks) * 128, 128, SB);
            const uint32_t accum = ((j % UT_FLUSH) || t || ks) ? 1u : 0u;
            tc_mma_bf16(tmem + (uint32_t)(16 * t), ad, bd, idesc, accum);
          }
        }
        tc_commit(&mmad[gcur & 1]);
      }
      if (j + 1 < nsub) {
        // buffer (j + 1) & 1 held sub-chunk j - 1: wait for its MMAs
        if (j >= 1) {
          const int gp = gcur - 1;
          if (!mbar_wait_bounded(&mmad[gp & 1], (unsigned)((gp >> 1) & 1))) failed = true;
        }
        if (!failed) load_sub(j + 1);
      }
      if ((j % UT_FLUSH) == UT_FLUSH - 1 || j + 1 == nsub) {
        // flush: the level sums of this window into the accumulators
        if (!failed && !mbar_wait_bounded(&mmad[gcur & 1], (unsigned)((gcur >> 1) & 1))) failed = true;
        tc_fence_after();
        if (!__syncthreads_or(failed)) {
          const float s1 = ut_pow2(emax - 7);
          float w[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) w[i] = __fmul_rn(s1, ut_pow2(fexp[i] - 7));
          const uint32_t lb = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll
          for (int l = 0; l < 6; ++l) {
            float v[16];
            tc_ld16(lb + (uint32_t)(16 * l), v);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const float p = __fmul_rn(v[i], w[i]);
              w[i] = __fmul_rn(w[i], 0.00390625f);
              if (l < 3) {
                const float2 t2s = df_two_sum(acc[i].s, p);
                acc[i].s = t2s.x;
                acc[i].c = __fadd_rn(acc[i].c, t2s.y);
              } else {
                acc[i].c = __fadd_rn(acc[i].c, p);
              }
            }
          }
#pragma unroll
          for (int i = 0; i < 16; ++i) df_renorm(acc[i]);
        } else {
          failed = true;
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
      }
      if (failed) break;
    }
    gj += nsub;
    failed = __syncthreads_or(failed);
    if (failed) break;
    // Every MMA of this tile is done and both A buffers are free: start the
    // next tile's copies and loads before finishing this one.
    if (tile + gridDim.x < ntile) prefetch(tile + gridDim.x);
    // ---- row tid: out1 = acc[0..7], out2 = acc[8..15] (plus X's term)
    const int64_t row = r0 + tid;
    if (u.X && row < u.n) {
      // X's own term, in double-float (X may be out1: this thread reads the row first)
      const float4* xr = reinterpret_cast<const float4*>(u.X + row * 8);
      float2 xv[8];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float4 v = xr[i];
        xv[2 * i] = make_float2(v.x, v.y);
        xv[2 * i + 1] = make_float2(v.z, v.w);
      }
      const float2* cx1 = c1g + (size_t)nin * 64;
      const float2* cx2 = c2g + (size_t)nin * 64;
#pragma unroll
      for (int q = 0; q < 8; ++q)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          df_fma(acc[c], xv[q], cx1[q * 8 + c]);
          df_fma(acc[8 + c], xv[q], cx2[q * 8 + c]);
        }
    }
    float2 o1[8], o2[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      o1[c] = df_value(acc[c]);
      o2[c] = df_value(acc[8 + c]);
    }
    if (row < u.n) {
      float4* d1 = reinterpret_cast<float4*>(u.out1 + row * 8);
      float4* d2 = reinterpret_cast<float4*>(u.out2 + row * 8);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        d1[i] = make_float4(o1[2 * i].x, o1[2 * i].y, o1[2 * i + 1].x, o1[2 * i + 1].y);
        d2[i] = make_float4(o2[2 * i].x, o2[2 * i].y, o2[2 * i + 1].x, o2[2 * i + 1].y);
      }
    }
    if (u.dig_out) {
      // out1's digits for the later Grams and updates, exactly as the split
      // kernel would make them from the stored values (rows past n are zero):
      // per column the exponent of the tile maximum, then six digits per value
      // into the free A buffer, then 16-byte stores of the tile's four chunks.
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        float am = fabsf(o1[i].x);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) am = fmaxf(am, __shfl_xor_sync(0xffffffffu, am, o));
        if (lane == 0) red[warp * 8 + i] = am;
      }
      __syncthreads();
      unsigned char* stg = Abuf + UT_SUB * UT_BLK;
      const uint32_t rofs = (uint32_t)warp * UT_DIG_GROUP + (uint32_t)(lane >> 4) * 256 +
                            (uint32_t)((lane >> 3) & 1) * 128 + (uint32_t)(lane & 7) * 2;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float cm = fmaxf(fmaxf(red[i], red[8 + i]), fmaxf(red[16 + i], red[24 + i]));
        const int e = ut_exp_of(cm);
        float d[6];
        ut_digits(o1[i], ut_pow2(7 - e), d);
#pragma unroll
        for (int t = 0; t < 6; ++t)
          *reinterpret_cast<__nv_bfloat16*>(stg + rofs + t * 512 + i * 16) = __float2bfloat16_rn(d[t]);
      }
      const int nq = nch - tile * 4 < 4 ? (int)(nch - tile * 4) : 4;   // chunks inside n
      if (tid < 8 * nq) {
        const int i = tid & 7;
        const float cm = fmaxf(fmaxf(red[i], red[8 + i]), fmaxf(red[16 + i], red[24 + i]));
        u.dexp_out[(tile * 4 + (tid >> 3)) * 8 + i] = ut_exp_of(cm);
      }
      __syncthreads();
      uint4* dst = reinterpret_cast<uint4*>(u.dig_out + (size_t)tile * 4 * UT_DIG_GROUP);
      const uint4* src = reinterpret_cast<const uint4*>(stg);
      for (int p = tid; p < nq * (UT_DIG_GROUP / 16); p += UT_THREADS) dst[p] = src[p];
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
  ut_cp_wait();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tc_dealloc(tmem, 128);
}

bool update_tcs_eligible(int s, int nin, bool two) { return s == 8 && two && nin >= 1 && 8 * nin <= UT_MAXK; }

size_t update_tcs_smem(int nin) {
  const int kpad = ((8 * nin + 31) / 32) * 32;
  const size_t SB = (size_t)(kpad / 8) * 128;
  return 2 * UT_SUB * UT_BLK + 12 * SB + UT_MAXK * 4 + 256 * 4 + 32 * 4 + 2 * 8 + 16;
}

struct CoefFoldArgs {
  const double* coef1;           // K x 8 row-major (row q of block b at b * 8 + q)
  const double* coef2;
  const double* chain;           // 8 x 8, or nullptr
  const double* tri1;            // 8 x 8 upper triangular, or nullptr
  const double* tri2;
  int rows;                      // K = 8 ncoef
  float2* out;                   // C1' then C2', double-float
  const Ctl* ctl;
  int step;
};

#define FOLD_ROWS 16             // coefficient rows per 128-thread CTA, 8 lanes per row

// Right-multiply the row held by an 8-lane group by T^{-1} (T upper
// triangular, rinv its reciprocal diagonal): forward substitution in
// double-float, one column per lane.
__device__ __forceinline__ float2 fold_trsm(float2 v, const float2* T, const float2* rinv, int c) {
  dfacc t{v.x, v.y};
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float2 own = df_mul(df_value(t), rinv[q]);
    const float2 oq = make_float2(__shfl_sync(0xffffffffu, own.x, q, 8), __shfl_sync(0xffffffffu, own.y, q, 8));
    if (c == q) t = dfacc{oq.x, oq.y};
    else if (c > q) df_fms(t, oq, T[q * 8 + c]);
  }
  return df_value(t);
}

// C1' = C1 T1^{-1} and C2' = (C2 + C1' Chain) T2^{-1}, row by row.  FP64 is
// used only to convert the inputs (spread over all threads: the FP64 pipe is
// narrow); the substitutions run in double-float with one lane per column.
__global__ void __launch_bounds__(128) k_coef_fold(const __grid_constant__ CoefFoldArgs f) {
  if (f.step >= 0 && *(volatile const int*)&f.ctl->update_step != f.step) return;
  __shared__ float2 tm[3 * 64 + 16];               // T1, T2, Chain, 1 / diag(T1), 1 / diag(T2)
  __shared__ float2 cr[2][FOLD_ROWS * 8];          // this CTA's rows of C1 and C2
  const int tid = threadIdx.x;
  const int r0 = blockIdx.x * FOLD_ROWS;
  for (int e = tid; e < 3 * 64 + 16 + 2 * FOLD_ROWS * 8; e += 128) {
    float2 v = make_float2(0.f, 0.f);
    if (e < 64) {
      if (f.tri1) v = df_from_double(f.tri1[e]);
    } else if (e < 128) {
      if (f.tri2) v = df_from_double(f.tri2[e - 64]);
    } else if (e < 192) {
      if (f.chain) v = df_from_double(f.chain[e - 128]);
    } else if (e < 200) {
      if (f.tri1) v = df_from_double(1.0 / f.tri1[(e - 192) * 9]);
    } else if (e < 208) {
      if (f.tri2) v = df_from_double(1.0 / f.tri2[(e - 200) * 9]);
    } else {
      const int k = e - 208, m = k / (FOLD_ROWS * 8), o = k % (FOLD_ROWS * 8);
      const int r = r0 + o / 8;
      if (r < f.rows) v = df_from_double((m ? f.coef2 : f.coef1)[(size_t)r * 8 + (o & 7)]);
    }
    if (e < 208) tm[e] = v;
    else cr[(e - 208) / (FOLD_ROWS * 8)][(e - 208) % (FOLD_ROWS * 8)] = v;
  }
  __syncthreads();
  const int rl = tid >> 3, c = tid & 7, r = r0 + rl;
  float2 o1 = cr[0][rl * 8 + c];
  if (f.tri1) o1 = fold_trsm(o1, tm, tm + 192, c);
  dfacc a2{cr[1][rl * 8 + c].x, cr[1][rl * 8 + c].y};
  if (f.chain) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float2 oq = make_float2(__shfl_sync(0xffffffffu, o1.x, q, 8), __shfl_sync(0xffffffffu, o1.y, q, 8));
      df_fma(a2, oq, tm[128 + q * 8 + c]);
    }
  }
  float2 o2 = df_value(a2);
  if (f.tri2) o2 = fold_trsm(o2, tm + 64, tm + 200, c);
  if (r < f.rows) {
    f.out[(size_t)r * 8 + c] = o1;
    f.out[(size_t)f.rows * 8 + (size_t)r * 8 + c] = o2;
  }
}

void launch_update_tcs(cudaStream_t st, const unsigned char* dig, const int* dexp, int a,
                       const float2* U, const float2* W, const float2* X, int64_t n, float2* out1,
                       float2* out2, const double* coef1, const double* tri1, const double* coef2,
                       const double* chain, const double* tri2, float2* cdf, unsigned char* dig_out,
                       int* dexp_out, const Ctl* ctl, int step, int* err, int num_sms, int minb) {
  const int nsplit = U ? 2 : 0;
  const int nin = a + nsplit;
  const int ncoef = nin + (X ? 1 : 0);
  CoefFoldArgs f;
  f.coef1 = coef1;
  f.coef2 = coef2;
  f.chain = chain;
  f.tri1 = tri1;
  f.tri2 = tri2;
  f.rows = 8 * ncoef;
  f.out = cdf;
  f.ctl = ctl;
  f.step = step;
  k_coef_fold<<<(f.rows + FOLD_ROWS - 1) / FOLD_ROWS, 128, 0, st>>>(f);
  static std::atomic<unsigned long long> attr_done{0};
  once_per_device(attr_done, [] {
    cudaFuncSetAttribute(k_update_df_tcs<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k_update_df_tcs<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  });
  UpdTcsArgs u;
  u.dig = dig;
  u.dexp = dexp;
  u.dig_stride = digit_block_bytes(n, 8);
  u.dexp_stride = digit_exp_count(n, 8);
  u.a = a;
  u.nsplit = nsplit;
  u.nin = nin;
  u.ncoef = ncoef;
  u.kpad = ((8 * nin + 31) / 32) * 32;
  u.U = U;
  u.W = W;
  u.X = X;
  u.n = n;
  u.out1 = out1;
  u.out2 = out2;
  u.cdf = cdf;
  u.dig_out = dig_out;
  u.dexp_out = dexp_out;
  u.ctl = ctl;
  u.step = step;
  u.err = err;
  // Three CTAs per SM where their shared memory fits (228 KB per SM, 1 KB of it
  // reserved per CTA), else two CTAs per SM, two short of filling the GPU: the
  // SMs left with one CTA have room for the small side kernel of the same
  // iteration (512 threads x 64 registers), which then runs beside this pass.
  // With three per SM the side kernel runs after this pass, on the SMs the next
  // Gram leaves free.
  const int64_t tiles = (n + 127) / 128;
  const size_t smem = update_tcs_smem(nin);
  const bool three = 3 * (smem + 1024) <= 228 * 1024 && minb != 2;
  int64_t grid = three ? 3LL * num_sms : 2LL * num_sms - 2;
  if (grid > tiles) grid = tiles;
  if (grid < 1) grid = 1;
  if (three)
    k_update_df_tcs<3><<<(unsigned)grid, UT_THREADS, smem, st>>>(u);
  else
    k_update_df_tcs<2><<<(unsigned)grid, UT_THREADS, smem, st>>>(u);
}

}  // namespace lsba
