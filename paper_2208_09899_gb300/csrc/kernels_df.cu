// Double-float (FP64-accurate, FP32-pipe) versions of the bandwidth-shaped
// kernels of one block Arnoldi step.  GB300 executes FP64 at 1/72 of its FP32
// rate, which leaves the FP64 Gram and update kernels 10-20x below the HBM
// roofline; here every block vector is stored as hi + lo FP32 pairs (8 bytes
// per entry, the same footprint as FP64) and every product-sum runs as a
// compensated double-float accumulation (df.cuh) on the FP32 pipes.
//
//   k_spmm_df    W = A V                           (the paper's matvec, Sec. 2.1)
//   k_gram_df    [L_1..L_a]^T [R_1..R_b], one pass (the sync point of Alg. 3
//                line 4, Alg. 6 line 10, Alg. 7 line 10), register-tiled 4x4
//   k_update_df  out = (sum_i in_i C_i (+ out1 chain)) T^{-1}, two outputs in
//                one pass (Alg. 3 line 6, Alg. 6 lines 17-18, Alg. 7 lines 16-17)
// The Gram result and everything after it (the small kernels) are FP64.
#include "df.cuh"
#include "lsba_internal.cuh"
#include "tma.cuh"

namespace lsba {

static __device__ __forceinline__ int ctl_active_df(const Ctl* c) {
  return *(volatile const int*)&c->active;
}

static inline int next_pow2_df(int s) {
  int p = 1;
  while (p < s) p <<= 1;
  return p;
}

// ----------------------------------------------------------------- conversions
// scale is a power of two (exact unless a value leaves FP64's range).
__global__ void k_to_df(int64_t count, const double* __restrict__ in, float2* __restrict__ out,
                        double scale) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = df_from_double(in[i] * scale);
}
__global__ void k_from_df(int64_t count, const float2* __restrict__ in, double* __restrict__ out,
                          double scale) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = df_to_double(in[i]) * scale;
}
// Magnitude range of an FP64 array: out[0] = max |x|, out[1] = min |x| over the
// nonzero entries, as the bit patterns of the non-negative doubles (which order
// like unsigned integers; a NaN orders above +inf, so a non-finite input shows
// as out[0] >= the bits of +inf).  out must hold {0, ~0} before the launch.
__global__ void __launch_bounds__(256) k_absrange(int64_t count, const double* __restrict__ in,
                                                  unsigned long long* __restrict__ out) {
  unsigned long long mx = 0ull, mn = ~0ull;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(in[i]) & 0x7FFFFFFFFFFFFFFFull;
    mx = b > mx ? b : mx;
    if (b != 0ull) mn = b < mn ? b : mn;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, mx, o);
    const unsigned long long c = __shfl_xor_sync(0xffffffffu, mn, o);
    mx = a > mx ? a : mx;
    mn = c < mn ? c : mn;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out[0], mx);
    atomicMin(&out[1], mn);
  }
}
// R = B - W (double-float)
__global__ void k_sub_df(int64_t count, const float2* __restrict__ B, const float2* __restrict__ W,
                         float2* __restrict__ R) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) {
    dfacc a{B[i].x, B[i].y};
    const float2 w = W[i];
    df_add_to(a, make_float2(-w.x, -w.y));
    R[i] = df_value(a);
  }
}

// Pseudo-random double-float values for timing runs: entry i is u_i + v_i 2^-24
// with u_i, v_i uniform in [-1, 1) from a counter hash (SplitMix64's output
// function of seed + i), so every digit a kernel forms from them is busy.
__global__ void k_fill_df(int64_t count, uint64_t seed, float2* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + (uint64_t)i * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const float u = (float)(int32_t)(uint32_t)z * 0x1p-31f;
    const float v = (float)(int32_t)(uint32_t)(z >> 32) * 0x1p-31f;
    out[i] = make_float2(u, v * 0x1p-24f);
  }
}

void launch_fill_df(cudaStream_t st, int64_t count, uint64_t seed, float2* out) {
  if (count > 0) k_fill_df<<<1024, 256, 0, st>>>(count, seed, out);
}

void launch_to_df(cudaStream_t st, int64_t count, const double* in, float2* out, double scale) {
  if (count > 0) k_to_df<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(count, in, out, scale);
}
void launch_from_df(cudaStream_t st, int64_t count, const float2* in, double* out, double scale) {
  if (count > 0) k_from_df<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(count, in, out, scale);
}
void launch_absrange(cudaStream_t st, int64_t count, const double* in, unsigned long long* out,
                     int num_sms) {
  if (count <= 0) return;
  int64_t grid = (count + 255) / 256;
  if (grid > 4LL * num_sms) grid = 4LL * num_sms;
  k_absrange<<<(unsigned)grid, 256, 0, st>>>(count, in, out);
}
void launch_sub_df(cudaStream_t st, int64_t count, const float2* B, const float2* W, float2* R) {
  if (count > 0) k_sub_df<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(count, B, W, R);
}

// ----------------------------------------------------------------- SpMM
__global__ void __launch_bounds__(256) k_spmm_df(int64_t n, const int32_t* __restrict__ rowptr,
                                                 const int32_t* __restrict__ colidx,
                                                 const float2* __restrict__ vals,
                                                 const float2* __restrict__ V,
                                                 float2* __restrict__ W, int s, int S2,
                                                 const Ctl* ctl, int guard) {
  if (guard && !ctl_active_df(ctl)) return;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t row = idx / S2;
  const int c = (int)(idx % S2);
  if (row >= n || c >= s) return;
  const int p0 = rowptr[row], p1 = rowptr[row + 1];
  dfacc acc{0.f, 0.f};
  for (int p = p0; p < p1; ++p) df_fma(acc, vals[p], V[(int64_t)colidx[p] * s + c]);
  W[row * s + c] = df_value(acc);
}

// s = 8: one thread per row, all eight columns: the row's nonzeros and column
// indices are read once, each neighbour row of V arrives as four 16-byte
// loads, and a warp keeps 2 KB of V rows in flight per nonzero (the
// per-(row, column) kernel: 256 B).  Every output sums its products in the
// row's order, as the per-(row, column) kernel does.
__global__ void __launch_bounds__(256) k_spmm_df8(int64_t n, const int32_t* __restrict__ rowptr,
                                                  const int32_t* __restrict__ colidx,
                                                  const float2* __restrict__ vals,
                                                  const float2* __restrict__ V,
                                                  float2* __restrict__ W, const Ctl* ctl,
                                                  int guard) {
  if (guard && !ctl_active_df(ctl)) return;
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  const int p0 = rowptr[row], p1 = rowptr[row + 1];
  dfacc acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = dfacc{0.f, 0.f};
  for (int p = p0; p < p1; ++p) {
    const float2 a = vals[p];
    const float4* v = reinterpret_cast<const float4*>(V + (int64_t)colidx[p] * 8);
    float4 q[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) q[i] = v[i];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      df_fma(acc[2 * i], a, make_float2(q[i].x, q[i].y));
      df_fma(acc[2 * i + 1], a, make_float2(q[i].z, q[i].w));
    }
  }
  float4* w = reinterpret_cast<float4*>(W + row * 8);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 lo = df_value(acc[2 * i]), hi = df_value(acc[2 * i + 1]);
    w[i] = make_float4(lo.x, lo.y, hi.x, hi.y);
  }
}

void launch_spmm_df(cudaStream_t st, int64_t n, const int32_t* rowptr, const int32_t* colidx,
                    const float2* vals, const float2* V, float2* W, int s, const Ctl* ctl,
                    int guard) {
  if (s == 8) {
    if (n > 0)
      k_spmm_df8<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, rowptr, colidx, vals, V, W, ctl,
                                                              guard);
    return;
  }
  const int S2 = next_pow2_df(s);
  const int64_t threads = n * S2;
  if (threads == 0) return;
  k_spmm_df<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(n, rowptr, colidx, vals, V, W, s,
                                                                S2, ctl, guard);
}

// ----------------------------------------------------------------- Gram
// Shared-memory chunk layout: [block][row][sp] with sp = s rounded up to 4 (the
// padding columns are zero).  The output, in the padded index space
// (a sp) x (b sp), is cut into 4x4 thread tiles; a CTA owns up to 256 tiles
// (blockIdx.y) and a contiguous row range (blockIdx.x).  When it owns fewer
// than 256 tiles, groups of threads split the chunk's rows and are summed in
// shared memory at the end.  Per-CTA partials are double-float, reduced in
// CTA order by k_gram_reduce_df into FP64.
#define GDF_THREADS 256

struct GramDfArgs {
  BlockPtrs L;
  BlockPtrs R;
  int a, b, s, sp, rc;
  int64_t n, rows_per_cta;
  int q;          // a*s*b*s (unpadded outputs)
  int ntj;        // tiles along the padded column dimension (b*sp/4)
  int ntile;      // total tiles
  float2* partials;
  const Ctl* ctl;
  int guard;
};

__global__ void __launch_bounds__(GDF_THREADS) k_gram_df(const __grid_constant__ GramDfArgs g) {
  if (g.guard && !ctl_active_df(g.ctl)) return;
  extern __shared__ float2 smf[];
  const int s = g.s, sp = g.sp, rc = g.rc, a = g.a, b = g.b;
  const int nblk = a + b;
  const int tile_base = blockIdx.y * GDF_THREADS;
  const int cnt = min(GDF_THREADS, g.ntile - tile_base);
  const int groups = GDF_THREADS / cnt;
  const int grp = threadIdx.x / cnt;
  const int tl = threadIdx.x % cnt;
  const bool active = grp < groups;
  const int T = tile_base + tl;
  const int it = T / g.ntj, jt = T % g.ntj;
  // Element (blk, r, col) of the chunk lives at smf[(blk * rc + r) * sp + col].
  const int li = it * 4;                    // padded L index: block li/sp, column li%sp
  const int lofs = (li / sp) * rc * sp + (li % sp);
  const int rj = jt * 4;
  const int rofs = (a + rj / sp) * rc * sp + (rj % sp);

  dfacc acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[x][y] = dfacc{0.f, 0.f};

  const int64_t r_begin = (int64_t)blockIdx.x * g.rows_per_cta;
  const int64_t r_end = min(g.n, r_begin + g.rows_per_cta);
  // Zero the padding columns once (never overwritten by the chunk loads).
  if (sp != s) {
    for (int idx = threadIdx.x; idx < nblk * rc * (sp - s); idx += GDF_THREADS) {
      const int pc = idx % (sp - s), br = idx / (sp - s);
      smf[br * sp + s + pc] = make_float2(0.f, 0.f);
    }
  }
  for (int64_t r0 = r_begin; r0 < r_end; r0 += rc) {
    const int rows = (int)min((int64_t)rc, r_end - r0);
    const int per = rows * s;
    __syncthreads();
    if (sp == s) {
      // Each block's chunk is contiguous in global and in shared memory.
      const int per4 = per >> 1;  // float4 = two entries (s is a multiple of 4)
      for (int blk = 0; blk < nblk; ++blk) {
        const float4* src = (const float4*)((const float2*)(blk < a ? g.L.p[blk] : g.R.p[blk - a]) +
                                            r0 * s);
        float4* dst = (float4*)(smf + (size_t)blk * rc * sp);
        for (int i = threadIdx.x; i < per4; i += GDF_THREADS) dst[i] = src[i];
      }
    } else {
      for (int idx = threadIdx.x; idx < nblk * per; idx += GDF_THREADS) {
        const int blk = idx / per, off = idx - blk * per;
        const int r = off / s, c = off - r * s;
        const float2* src = (const float2*)(blk < a ? g.L.p[blk] : g.R.p[blk - a]);
        smf[(blk * rc + r) * sp + c] = src[r0 * s + off];
      }
    }
    __syncthreads();
    if (active) {
      for (int r = grp; r < rows; r += groups) {
        const float4* lp = (const float4*)(smf + lofs + r * sp);
        const float4* rp = (const float4*)(smf + rofs + r * sp);
        const float4 l01 = lp[0], l23 = lp[1], r01 = rp[0], r23 = rp[1];
        const float2 lv[4] = {make_float2(l01.x, l01.y), make_float2(l01.z, l01.w),
                              make_float2(l23.x, l23.y), make_float2(l23.z, l23.w)};
        const float2 rv[4] = {make_float2(r01.x, r01.y), make_float2(r01.z, r01.w),
                              make_float2(r23.x, r23.y), make_float2(r23.z, r23.w)};
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) df_fma(acc[x][y], lv[x], rv[y]);
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) df_renorm(acc[x][y]);
    }
  }
  // Sum the row groups (shared memory), then write this CTA's partials.
  if (groups > 1) {
    __syncthreads();
    float2* red = smf;  // [groups][cnt][16]
    if (active) {
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y)
          red[((size_t)grp * cnt + tl) * 16 + x * 4 + y] = make_float2(acc[x][y].s, acc[x][y].c);
    }
    __syncthreads();
    if (grp == 0) {
      for (int g2 = 1; g2 < groups; ++g2) {
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            const float2 v = red[((size_t)g2 * cnt + tl) * 16 + x * 4 + y];
            df_add_to(acc[x][y], make_float2(v.x, 0.f));
            df_add_to(acc[x][y], make_float2(v.y, 0.f));
          }
      }
    }
  }
  if (grp == 0) {
    const int bs = b * s;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int pi = li + x;               // padded row index
      const int i = (pi / sp) * s + (pi % sp);
      if (pi % sp >= s || pi >= a * sp) continue;
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int pj = rj + y;
        if (pj % sp >= s || pj >= b * sp) continue;
        const int j = (pj / sp) * s + (pj % sp);
        const float2 v = df_value(acc[x][y]);
        g.partials[(int64_t)blockIdx.x * g.q + (int64_t)i * bs + j] = v;
      }
    }
  }
}

// ---- Gram with asynchronous bulk copies (s a multiple of 4) ----------------
// The same computation as k_gram_df, but each chunk of rows is brought into
// shared memory by one-dimensional bulk copies (cp.async.bulk, the TMA engine)
// that complete on an mbarrier, two chunks in flight: the copy of chunk c+2
// overlaps the arithmetic on chunk c+1.  Every wait on an mbarrier is bounded;
// on a timeout the CTA records an error in *err, waits (bounded) for its own
// copies, and returns.
struct GramTmaArgs {
  BlockPtrs L;
  BlockPtrs R;
  int a, b, s, rc;
  int64_t n, rows_per_cta;
  int q, ntj, ntile;
  unsigned stage_elems;   // float2 per stage = (nl_max + b) * rc * s
  float2* partials;
  const Ctl* ctl;
  int guard;
  int* err;
};

__global__ void __launch_bounds__(GDF_THREADS) k_gram_df_tma(const __grid_constant__ GramTmaArgs g) {
  if (g.guard && !ctl_active_df(g.ctl)) return;
  extern __shared__ __align__(128) unsigned char smraw[];
  uint64_t* bars = (uint64_t*)smraw;
  float2* stage0 = (float2*)(smraw + 128);
  float2* stage1 = stage0 + g.stage_elems;
  const int s = g.s, rc = g.rc, b = g.b;
  const int tile_base = blockIdx.y * GDF_THREADS;
  const int cnt = min(GDF_THREADS, g.ntile - tile_base);
  const int groups = GDF_THREADS / cnt;
  const int grp = threadIdx.x / cnt;
  const int tl = threadIdx.x % cnt;
  const bool active = grp < groups;
  const int T = tile_base + tl;
  const int it = T / g.ntj, jt = T % g.ntj;
  const int li = it * 4, rj = jt * 4;
  // Only the left blocks this tile group reads are copied: [lb0, lb0 + nl).
  int lb0, nl;
  gram_tile_blocks(tile_base, cnt, g.ntj, s, &lb0, &nl);
  const int nblk = nl + b;
  const int lofs = (li / s - lb0) * rc * s + (li % s);
  const int rofs = (nl + rj / s) * rc * s + (rj % s);
  const int64_t r_begin = (int64_t)blockIdx.x * g.rows_per_cta;
  const int64_t r_end = min(g.n, r_begin + g.rows_per_cta);
  const int nchunks = r_end > r_begin ? (int)((r_end - r_begin + rc - 1) / rc) : 0;

  // bars[0..1]: stage full (copies landed); bars[2..3]: stage empty (every
  // warp has finished reading it).  Only the copy-issuing thread waits for a
  // stage to drain, so warps are not held in step by a CTA-wide barrier.
  uint64_t* empty = bars + 2;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&empty[0], GDF_THREADS / 32);
    mbar_init(&empty[1], GDF_THREADS / 32);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int c, int st) {
    const int64_t r0 = r_begin + (int64_t)c * rc;
    const int rows = (int)min((int64_t)rc, r_end - r0);
    const unsigned bytes = (unsigned)(rows * s * sizeof(float2));
    float2* dst = st ? stage1 : stage0;
    mbar_expect_tx(&bars[st], bytes * nblk);
    for (int blk = 0; blk < nblk; ++blk) {
      const float2* src = (const float2*)(blk < nl ? g.L.p[lb0 + blk] : g.R.p[blk - nl]) + r0 * s;
      bulk_copy_g2s(dst + (size_t)blk * rc * s, src, bytes, &bars[st]);
    }
  };
  if (threadIdx.x == 0) {
    if (nchunks > 0) issue(0, 0);
    if (nchunks > 1) issue(1, 1);
  }

  dfacc acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[x][y] = dfacc{0.f, 0.f};

  bool failed = false;
  for (int c = 0; c < nchunks; ++c) {
    const int st = c & 1;
    const unsigned parity = (unsigned)((c >> 1) & 1);
    if (!failed && !mbar_wait_bounded(&bars[st], parity)) failed = true;
    failed = __any_sync(0xffffffffu, failed);
    if (failed) break;
    const float2* buf = st ? stage1 : stage0;
    const int rows = (int)min((int64_t)rc, r_end - (r_begin + (int64_t)c * rc));
    if (active) {
      for (int r = grp; r < rows; r += groups) {
        const float4* lp = (const float4*)(buf + lofs + r * s);
        const float4* rp = (const float4*)(buf + rofs + r * s);
        const float4 l01 = lp[0], l23 = lp[1], r01 = rp[0], r23 = rp[1];
        const float2 lv[4] = {make_float2(l01.x, l01.y), make_float2(l01.z, l01.w),
                              make_float2(l23.x, l23.y), make_float2(l23.z, l23.w)};
        const float2 rv[4] = {make_float2(r01.x, r01.y), make_float2(r01.z, r01.w),
                              make_float2(r23.x, r23.y), make_float2(r23.z, r23.w)};
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) df_fma(acc[x][y], lv[x], rv[y]);
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) df_renorm(acc[x][y]);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);  // this warp is done reading the stage
    if (threadIdx.x == 0 && c + 2 < nchunks) {
      if (mbar_wait_bounded(&empty[st], parity)) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(c + 2, st);
      } else {
        failed = true;
      }
    }
  }
  if (__syncthreads_or(failed)) {
    if (threadIdx.x == 0) {
      if (g.err) atomicExch(g.err, 1);
      // Let this CTA's copies in flight land before the shared memory goes away.
      for (int c2 = 0; c2 < 2; ++c2) mbar_wait_bounded(&bars[c2], 0), mbar_wait_bounded(&bars[c2], 1);
    }
    __syncthreads();
    return;
  }
  if (groups > 1) {
    __syncthreads();
    float2* red = stage0;  // [groups][cnt][16], all copies have landed
    if (active) {
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y)
          red[((size_t)grp * cnt + tl) * 16 + x * 4 + y] = make_float2(acc[x][y].s, acc[x][y].c);
    }
    __syncthreads();
    if (grp == 0) {
      for (int g2 = 1; g2 < groups; ++g2) {
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            const float2 v = red[((size_t)g2 * cnt + tl) * 16 + x * 4 + y];
            df_add_to(acc[x][y], make_float2(v.x, 0.f));
            df_add_to(acc[x][y], make_float2(v.y, 0.f));
          }
      }
    }
  }
  if (grp == 0) {
    const int bs = b * s;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int i = li + x;
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int j = rj + y;
        g.partials[(int64_t)blockIdx.x * g.q + (int64_t)i * bs + j] = df_value(acc[x][y]);
      }
    }
  }
}

// 32 outputs per CTA; the 8 warps sum fixed eighths of the partials (warp y:
// partials [y P/8, (y+1) P/8) in order), then warp 0 adds the eight sums in
// order: a fixed summation order for a given plan.
__global__ void __launch_bounds__(256) k_gram_reduce_df(const float2* __restrict__ partials,
                                                        int nparts, int q, double* __restrict__ G,
                                                        const Ctl* ctl, int guard) {
  if (guard && !ctl_active_df(ctl)) return;
  __shared__ float2 part[8][32];
  const int ox = threadIdx.x & 31, gy = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + ox;
  dfacc acc{0.f, 0.f};
  if (e < q) {
    const int per = (nparts + 7) / 8;
    const int x0 = gy * per, x1 = min(nparts, x0 + per);
    // all loads of a chunk issued before the (ordered) sums
    for (int c0 = x0; c0 < x1; c0 += 24) {
      float2 v[24];
#pragma unroll
      for (int i = 0; i < 24; ++i) v[i] = c0 + i < x1 ? partials[(int64_t)(c0 + i) * q + e] : make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < 24; ++i)
        if (c0 + i < x1) df_add_to(acc, v[i]);
    }
  }
  part[gy][ox] = df_value(acc);
  __syncthreads();
  if (gy == 0 && e < q) {
    dfacc t{0.f, 0.f};
#pragma unroll
    for (int y = 0; y < 8; ++y) df_add_to(t, part[y][ox]);
    G[e] = dfacc_to_double(t);
  }
}

void launch_gram_reduce_df(cudaStream_t st, const float2* partials, int nparts, int q, double* G,
                           const Ctl* ctl, int guard) {
  k_gram_reduce_df<<<(q + 31) / 32, 256, 0, st>>>(partials, nparts, q, G, ctl, guard);
}

GramPlan plan_gram_df(int64_t n, int s, int a, int b, int num_sms, int tensor_cores, int cps,
                      int rc_cap) {
  if ((tensor_cores == 2 && gram_tc_eligible(s, a, b)) ||
      (tensor_cores == 1 && gram_tc_profitable(s, a, b))) {
    GramPlan t = plan_gram_tc(n, s, a, b, num_sms);
    t.tc = 1;
    return t;
  }
  GramPlan p{};
  p.tc = 0;
  const int sp = (s + 3) & ~3;
  p.q = a * s * b * s;
  const int ntile = (a * sp / 4) * (b * sp / 4);
  p.tile = GDF_THREADS;
  p.grid_y = (ntile + GDF_THREADS - 1) / GDF_THREADS;
  const size_t row_bytes = (size_t)(a + b) * sp * sizeof(float2);
  const size_t red_bytes = (size_t)GDF_THREADS * 16 * sizeof(float2);
  int rc;
  int ctas_per_sm;
  p.nl_max = a;
  if (sp == s) {
    // A tile group copies only the left blocks its tiles read.
    p.nl_max = 0;
    for (int y = 0; y < p.grid_y; ++y) {
      const int base = y * GDF_THREADS;
      const int cnt = ntile - base < GDF_THREADS ? ntile - base : GDF_THREADS;
      int first, count;
      gram_tile_blocks(base, cnt, b * s / 4, s, &first, &count);
      if (count > p.nl_max) p.nl_max = count;
    }
    const size_t row_bytes_g = (size_t)(p.nl_max + b) * s * sizeof(float2);
    // Two pipeline stages of <= 32 KB each: three CTAs per SM.
    rc = (int)((32 * 1024) / row_bytes_g);
    if (rc > 128) rc = 128;
    if (rc < 1) rc = 1;
    const size_t stages = 128 + 2 * row_bytes_g * rc;
    p.smem = stages > 128 + red_bytes ? stages : 128 + red_bytes;
    ctas_per_sm = 3;
  } else {
    rc = (int)((80 * 1024) / row_bytes);
    if (rc > 128) rc = 128;
    if (rc < 1) rc = 1;
    p.smem = row_bytes * rc > red_bytes ? row_bytes * rc : red_bytes;
    ctas_per_sm = 2;
  }
  // tuned shape: CTAs per SM and a cap on the rows of a pipeline chunk
  if (cps > 0) ctas_per_sm = cps;
  if (rc_cap > 0 && rc > rc_cap) {
    rc = rc_cap;
    if (sp == s) {
      const size_t stages = 128 + 2 * (size_t)(p.nl_max + b) * s * sizeof(float2) * rc;
      p.smem = stages > 128 + red_bytes ? stages : 128 + red_bytes;
    } else {
      p.smem = row_bytes * rc > red_bytes ? row_bytes * rc : red_bytes;
    }
  }
  p.rows_per_chunk = rc;
  int gx = (ctas_per_sm * num_sms + p.grid_y - 1) / p.grid_y;
  const int64_t max_gx = (n + rc - 1) / rc;
  if (gx > max_gx) gx = (int)max_gx;
  if (gx < 1) gx = 1;
  int64_t rpc = (n + gx - 1) / gx;
  rpc = ((rpc + rc - 1) / rc) * rc;
  if (rpc < rc) rpc = rc;
  gx = (int)((n + rpc - 1) / rpc);
  if (gx < 1) gx = 1;
  p.grid_x = gx;
  p.rows_per_cta = rpc;
  return p;
}

void launch_gram_df(cudaStream_t st, const GramPlan& p, const BlockPtrs& L, int a,
                    const BlockPtrs& R, int b, int64_t n, int s, float2* partials, double* G,
                    const Ctl* ctl, int guard, int* err) {
  static std::atomic<unsigned long long> attr_done{0};
  once_per_device(attr_done, [] {
    cudaFuncSetAttribute(k_gram_df, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_gram_df_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  if (p.tc) {
    launch_gram_tc(st, p, L, a, R, b, n, s, partials, ctl, guard, err);
    k_gram_reduce_df<<<(p.q + 31) / 32, 256, 0, st>>>(partials, p.grid_x, p.q, G, ctl, guard);
    return;
  }
  dim3 grid(p.grid_x, p.grid_y);
  const int sp = (s + 3) & ~3;
  if (sp == s) {
    GramTmaArgs g;
    g.L = L;
    g.R = R;
    g.a = a;
    g.b = b;
    g.s = s;
    g.rc = p.rows_per_chunk;
    g.n = n;
    g.rows_per_cta = p.rows_per_cta;
    g.q = p.q;
    g.ntj = b * s / 4;
    g.ntile = (a * s / 4) * g.ntj;
    g.stage_elems = (unsigned)((p.nl_max + b) * p.rows_per_chunk * s);
    g.partials = partials;
    g.ctl = ctl;
    g.guard = guard;
    g.err = err;
    k_gram_df_tma<<<grid, GDF_THREADS, p.smem, st>>>(g);
  } else {
    GramDfArgs g;
    g.L = L;
    g.R = R;
    g.a = a;
    g.b = b;
    g.s = s;
    g.sp = sp;
    g.rc = p.rows_per_chunk;
    g.n = n;
    g.rows_per_cta = p.rows_per_cta;
    g.q = p.q;
    g.ntj = b * g.sp / 4;
    g.ntile = (a * g.sp / 4) * g.ntj;
    g.partials = partials;
    g.ctl = ctl;
    g.guard = guard;
    k_gram_df<<<grid, GDF_THREADS, p.smem, st>>>(g);
  }
  k_gram_reduce_df<<<(p.q + 31) / 32, 256, 0, st>>>(partials, p.grid_x, p.q, G, ctl, guard);
}

// ----------------------------------------------------------------- Update
// The small kernels produce the update coefficients in FP64; k_coef_df
// converts them once per step with many CTAs (FP64->FP32 conversions run on
// the slow FP64 pipe), into the layout
//   [c1: nin*s*s][c2: nin*s*s if two][chain: s*s][t1: s*s][t2: s*s][r1: s][r2: s]
// (r = reciprocal diagonals of the triangular factors).  k_update_df runs a
// persistent grid; each CTA copies the converted coefficients to shared memory
// and walks row groups.  A row's s entries belong to a group of S2 lanes of one
// warp; input values are exchanged by shuffles.
__host__ __device__ size_t coef_df_count(int nin, int s, bool two) {
  const size_t ss = (size_t)s * s;
  return (size_t)nin * ss * (two ? 2 : 1) + 3 * ss + 2 * (size_t)s;
}

struct CoefDfArgs {
  const double* coef1;
  const double* coef2;
  const double* chain;
  const double* tri1;
  const double* tri2;
  int nin, s, two;
  float2* out;
  const Ctl* ctl;
  int step;
};

__global__ void k_coef_df(const __grid_constant__ CoefDfArgs a) {
  if (a.step >= 0 && *(volatile const int*)&a.ctl->update_step != a.step) return;
  const int s = a.s, ss = s * s;
  const int n1 = a.nin * ss, n2 = a.two ? n1 : 0;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  int o = e;
  if (o < n1) { a.out[e] = df_from_double(a.coef1[o]); return; }
  o -= n1;
  if (o < n2) { a.out[e] = df_from_double(a.coef2[o]); return; }
  o -= n2;
  if (o < ss) { a.out[e] = (a.two && a.chain) ? df_from_double(a.chain[o]) : make_float2(0.f, 0.f); return; }
  o -= ss;
  if (o < ss) { a.out[e] = a.tri1 ? df_from_double(a.tri1[o]) : make_float2(0.f, 0.f); return; }
  o -= ss;
  if (o < ss) { a.out[e] = (a.two && a.tri2) ? df_from_double(a.tri2[o]) : make_float2(0.f, 0.f); return; }
  o -= ss;
  if (o < s) { a.out[e] = a.tri1 ? df_from_double(1.0 / a.tri1[o * s + o]) : make_float2(0.f, 0.f); return; }
  o -= s;
  if (o < s) { a.out[e] = (a.two && a.tri2) ? df_from_double(1.0 / a.tri2[o * s + o]) : make_float2(0.f, 0.f); }
}

struct UpdDfArgs {
  BlockPtrs in;
  int nin, s, S2;
  int64_t n;
  float2* out1;
  float2* out2;
  const float2* cdf;
  int has_tri1, has_chain, has_tri2;
  int staged;          // coefficients copied to shared memory (else read from cdf)
  const Ctl* ctl;
  int step;
};

__device__ __forceinline__ float2 shfl_f2(float2 v, int src, int width) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src, width),
                     __shfl_sync(0xffffffffu, v.y, src, width));
}

// Right-multiply the row held by the lane group by T^{-1} (upper triangular):
// forward substitution over the columns in double-float.
__device__ __forceinline__ float2 row_trsm_df(dfacc t, const float2* T, const float2* rinv, int c,
                                              int s, int S2) {
  const float2 rc = c < s ? rinv[c] : make_float2(0.f, 0.f);
  for (int q = 0; q < s; ++q) {
    const float2 vq = shfl_f2(df_mul(df_value(t), rc), q, S2);
    if (c == q) {
      t.s = vq.x;
      t.c = vq.y;
    } else if (c > q && c < s) {
      df_fms(t, vq, T[q * s + c]);
    }
  }
  return df_value(t);
}

__global__ void __launch_bounds__(256) k_update_df(const __grid_constant__ UpdDfArgs u) {
  if (u.step >= 0 && *(volatile const int*)&u.ctl->update_step != u.step) return;
  extern __shared__ float2 cs[];
  const int s = u.s, S2 = u.S2, nin = u.nin;
  const int ss = s * s;
  const bool two = u.out2 != nullptr;
  // Coefficients that fit are staged in shared memory; larger sets (s = 32
  // with a long basis) are read from global memory, where every CTA reuses
  // the same few KB per input block through L1.
  const float2* c1 = u.cdf;
  if (u.staged) {
    const int total = (int)coef_df_count(nin, s, two);
    for (int e = threadIdx.x; e < total; e += blockDim.x) cs[e] = u.cdf[e];
    __syncthreads();
    c1 = cs;
  }
  const float2* c2 = c1 + (size_t)nin * ss;
  const float2* ch = c2 + (two ? (size_t)nin * ss : 0);
  const float2* t1 = ch + ss;
  const float2* t2 = t1 + ss;
  const float2* r1 = t2 + ss;
  const float2* r2 = r1 + s;
  const int c = threadIdx.x % S2;
  const int rows_per_cta = blockDim.x / S2;
  for (int64_t row0 = (int64_t)blockIdx.x * rows_per_cta; row0 < u.n;
       row0 += (int64_t)gridDim.x * rows_per_cta) {
    const int64_t row = row0 + threadIdx.x / S2;
    const bool live = (row < u.n) && (c < s);
    dfacc a1{0.f, 0.f}, a2{0.f, 0.f};
    for (int bk = 0; bk < nin; ++bk) {
      const float2 v = live ? ((const float2*)u.in.p[bk])[row * s + c] : make_float2(0.f, 0.f);
      const float2* k1 = c1 + (size_t)bk * ss;
      const float2* k2 = c2 + (size_t)bk * ss;
      for (int q = 0; q < s; ++q) {
        const float2 x = shfl_f2(v, q, S2);
        if (c < s) {
          df_fma(a1, x, k1[q * s + c]);
          if (two) df_fma(a2, x, k2[q * s + c]);
        }
      }
    }
    const float2 o1 = u.has_tri1 ? row_trsm_df(a1, t1, r1, c, s, S2) : df_value(a1);
    float2 o2 = make_float2(0.f, 0.f);
    if (two) {
      if (u.has_chain) {
        for (int q = 0; q < s; ++q) {
          const float2 x = shfl_f2(o1, q, S2);
          if (c < s) df_fma(a2, x, ch[q * s + c]);
        }
      }
      o2 = u.has_tri2 ? row_trsm_df(a2, t2, r2, c, s, S2) : df_value(a2);
    }
    __syncwarp();
    if (live) {
      u.out1[row * s + c] = o1;
      if (two) u.out2[row * s + c] = o2;
    }
  }
}

// One thread per row (s = 4, 8, 16): the row of every input block is loaded
// with 16-byte loads into registers, the coefficients (identical for all rows)
// are broadcast from shared memory, and both outputs accumulate in registers.
template <int S, bool TWO>
__global__ void __launch_bounds__(256) k_update_df_row(const __grid_constant__ UpdDfArgs u) {
  if (u.step >= 0 && *(volatile const int*)&u.ctl->update_step != u.step) return;
  extern __shared__ float2 cs[];
  const int nin = u.nin;
  constexpr int SS = S * S;
  const int total = (int)coef_df_count(nin, S, TWO);
  for (int e = threadIdx.x; e < total; e += blockDim.x) cs[e] = u.cdf[e];
  __syncthreads();
  const float2* c1 = cs;
  const float2* c2 = c1 + (size_t)nin * SS;
  const float2* ch = c2 + (TWO ? (size_t)nin * SS : 0);
  const float2* t1 = ch + SS;
  const float2* t2 = t1 + SS;
  const float2* r1 = t2 + SS;
  const float2* r2 = r1 + S;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < u.n;
       row += (int64_t)gridDim.x * blockDim.x) {
    dfacc a1[S], a2[S];
#pragma unroll
    for (int c = 0; c < S; ++c) {
      a1[c] = dfacc{0.f, 0.f};
      a2[c] = dfacc{0.f, 0.f};
    }
    for (int bk = 0; bk < nin; ++bk) {
      float2 v[S];
      const float4* src = (const float4*)((const float2*)u.in.p[bk] + row * S);
#pragma unroll
      for (int i = 0; i < S / 2; ++i) {
        const float4 t = src[i];
        v[2 * i] = make_float2(t.x, t.y);
        v[2 * i + 1] = make_float2(t.z, t.w);
      }
      const float2* k1 = c1 + (size_t)bk * SS;
      const float2* k2 = c2 + (size_t)bk * SS;
#pragma unroll
      for (int q = 0; q < S; ++q) {
#pragma unroll
        for (int c = 0; c < S; ++c) {
          df_fma(a1[c], v[q], k1[q * S + c]);
          if (TWO) df_fma(a2[c], v[q], k2[q * S + c]);
        }
      }
    }
    float2 o1[S];
    if (u.has_tri1) {
      // o1 = a1 T1^{-1}: forward substitution over the columns.
#pragma unroll
      for (int c = 0; c < S; ++c) {
#pragma unroll
        for (int q = 0; q < c; ++q) df_fms(a1[c], o1[q], t1[q * S + c]);
        o1[c] = df_mul(df_value(a1[c]), r1[c]);
      }
    } else {
#pragma unroll
      for (int c = 0; c < S; ++c) o1[c] = df_value(a1[c]);
    }
    float4* d1 = (float4*)(u.out1 + row * S);
#pragma unroll
    for (int i = 0; i < S / 2; ++i) d1[i] = make_float4(o1[2 * i].x, o1[2 * i].y, o1[2 * i + 1].x, o1[2 * i + 1].y);
    if (TWO) {
      if (u.has_chain) {
#pragma unroll
        for (int q = 0; q < S; ++q)
#pragma unroll
          for (int c = 0; c < S; ++c) df_fma(a2[c], o1[q], ch[q * S + c]);
      }
      float2 o2[S];
      if (u.has_tri2) {
#pragma unroll
        for (int c = 0; c < S; ++c) {
#pragma unroll
          for (int q = 0; q < c; ++q) df_fms(a2[c], o2[q], t2[q * S + c]);
          o2[c] = df_mul(df_value(a2[c]), r2[c]);
        }
      } else {
#pragma unroll
        for (int c = 0; c < S; ++c) o2[c] = df_value(a2[c]);
      }
      float4* d2 = (float4*)(u.out2 + row * S);
#pragma unroll
      for (int i = 0; i < S / 2; ++i) d2[i] = make_float4(o2[2 * i].x, o2[2 * i].y, o2[2 * i + 1].x, o2[2 * i + 1].y);
    }
  }
}

// s = 32: a pair of adjacent lanes per row, each owning 16 columns of both
// outputs (64 accumulator registers per lane).  Both lanes read the row's 32
// input values (one L1 transaction serves the pair); the coefficients come
// from global memory through L1 (every CTA reads the same 16 KB per input
// block).  The triangular solves run column by column: the lane that owns
// column q finishes it and hands it to its partner by a shuffle.
template <bool TWO>
__global__ void __launch_bounds__(256, 1) k_update_df_w32(const __grid_constant__ UpdDfArgs u) {
  if (u.step >= 0 && *(volatile const int*)&u.ctl->update_step != u.step) return;
  constexpr int S = 32, CG = 16, SS = S * S;
  const int nin = u.nin;
  const float2* c1 = u.cdf;
  const float2* c2 = c1 + (size_t)nin * SS;
  const float2* ch = c2 + (TWO ? (size_t)nin * SS : 0);
  const float2* t1 = ch + SS;
  const float2* t2 = t1 + SS;
  const float2* r1 = t2 + SS;
  const float2* r2 = r1 + S;
  const int half = threadIdx.x & 1;
  const int c0 = half * CG;
  const unsigned pair = 3u << (threadIdx.x & 30);
  const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 1;
  for (int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 1; row < u.n; row += stride) {
    dfacc a1[CG], a2[CG];
#pragma unroll
    for (int c = 0; c < CG; ++c) {
      a1[c] = dfacc{0.f, 0.f};
      a2[c] = dfacc{0.f, 0.f};
    }
    // Eight input values (a quarter row) per iteration; the next quarter is
    // loaded before the arithmetic on the current one.
    const int iters = nin * 4;
    float4 nxt[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) nxt[i] = ((const float4*)((const float2*)u.in.p[0] + row * S))[i];
#pragma unroll 1
    for (int itr = 0; itr < iters; ++itr) {
      const int bk = itr >> 2, qb = (itr & 3) * 8;
      float2 v[8];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        v[2 * i] = make_float2(nxt[i].x, nxt[i].y);
        v[2 * i + 1] = make_float2(nxt[i].z, nxt[i].w);
      }
      if (itr + 1 < iters) {
        const int bn = (itr + 1) >> 2, qn = ((itr + 1) & 3) * 8;
        const float4* src = (const float4*)((const float2*)u.in.p[bn] + row * S + qn);
#pragma unroll
        for (int i = 0; i < 4; ++i) nxt[i] = src[i];
      }
      const float2* k1 = c1 + (size_t)bk * SS + c0;
      const float2* k2 = c2 + (size_t)bk * SS + c0;
#pragma unroll
      for (int qq = 0; qq < 8; ++qq) {
        const float4* kr1 = (const float4*)(k1 + (qb + qq) * S);
        const float4* kr2 = (const float4*)(k2 + (qb + qq) * S);
#pragma unroll
        for (int c = 0; c < CG; c += 2) {
          const float4 k = __ldg(kr1 + c / 2);
          df_fma(a1[c], v[qq], make_float2(k.x, k.y));
          df_fma(a1[c + 1], v[qq], make_float2(k.z, k.w));
          if (TWO) {
            const float4 kk = __ldg(kr2 + c / 2);
            df_fma(a2[c], v[qq], make_float2(kk.x, kk.y));
            df_fma(a2[c + 1], v[qq], make_float2(kk.z, kk.w));
          }
        }
      }
    }
    // out1 = a1 T1^{-1}; the finished column values overwrite a1 (s = hi, c = lo).
    if (u.has_tri1) {
#pragma unroll
      for (int q = 0; q < S; ++q) {
        if (half == q / CG) {
          const float2 o = df_mul(df_value(a1[q % CG]), __ldg(r1 + q));
          a1[q % CG] = dfacc{o.x, o.y};
        }
        const float2 oq = make_float2(__shfl_sync(pair, a1[q % CG].s, q / CG, 2),
                                      __shfl_sync(pair, a1[q % CG].c, q / CG, 2));
#pragma unroll
        for (int c = 0; c < CG; ++c)
          if (c0 + c > q) df_fms(a1[c], oq, __ldg(t1 + q * S + c0 + c));
      }
    } else {
#pragma unroll
      for (int c = 0; c < CG; ++c) {
        const float2 o = df_value(a1[c]);
        a1[c] = dfacc{o.x, o.y};
      }
    }
    float4* d1 = (float4*)(u.out1 + row * S + c0);
#pragma unroll
    for (int i = 0; i < CG / 2; ++i)
      d1[i] = make_float4(a1[2 * i].s, a1[2 * i].c, a1[2 * i + 1].s, a1[2 * i + 1].c);
    if (TWO) {
      if (u.has_chain) {
#pragma unroll
        for (int q = 0; q < S; ++q) {
          const float2 oq = make_float2(__shfl_sync(pair, a1[q % CG].s, q / CG, 2),
                                        __shfl_sync(pair, a1[q % CG].c, q / CG, 2));
#pragma unroll
          for (int c = 0; c < CG; ++c) df_fma(a2[c], oq, __ldg(ch + q * S + c0 + c));
        }
      }
      if (u.has_tri2) {
#pragma unroll
        for (int q = 0; q < S; ++q) {
          if (half == q / CG) {
            const float2 o = df_mul(df_value(a2[q % CG]), __ldg(r2 + q));
            a2[q % CG] = dfacc{o.x, o.y};
          }
          const float2 oq = make_float2(__shfl_sync(pair, a2[q % CG].s, q / CG, 2),
                                        __shfl_sync(pair, a2[q % CG].c, q / CG, 2));
#pragma unroll
          for (int c = 0; c < CG; ++c)
            if (c0 + c > q) df_fms(a2[c], oq, __ldg(t2 + q * S + c0 + c));
        }
      } else {
#pragma unroll
        for (int c = 0; c < CG; ++c) {
          const float2 o = df_value(a2[c]);
          a2[c] = dfacc{o.x, o.y};
        }
      }
      float4* d2 = (float4*)(u.out2 + row * S + c0);
#pragma unroll
      for (int i = 0; i < CG / 2; ++i)
        d2[i] = make_float4(a2[2 * i].s, a2[2 * i].c, a2[2 * i + 1].s, a2[2 * i + 1].c);
    }
  }
}

size_t update_df_smem(int nin, int s, bool two) { return sizeof(float2) * coef_df_count(nin, s, two); }

// Largest coefficient set staged in shared memory by the update kernels.
static constexpr size_t UPDATE_DF_SMEM_MAX = 200 * 1024;

void launch_coef_df(cudaStream_t st, int nin, int s, bool two, const double* coef1,
                    const double* coef2, const double* chain, const double* tri1,
                    const double* tri2, float2* cdf, const Ctl* ctl, int step) {
  CoefDfArgs ca;
  ca.coef1 = coef1;
  ca.coef2 = coef2;
  ca.chain = chain;
  ca.tri1 = tri1;
  ca.tri2 = tri2;
  ca.nin = nin;
  ca.s = s;
  ca.two = two ? 1 : 0;
  ca.out = cdf;
  ca.ctl = ctl;
  ca.step = step;
  const int total = (int)coef_df_count(nin, s, two);
  k_coef_df<<<(total + 127) / 128, 128, 0, st>>>(ca);
}

void launch_update_df(cudaStream_t st, const BlockPtrs& in, int nin, int64_t n, int s, float2* out1,
                      const double* coef1, const double* tri1, float2* out2, const double* coef2,
                      const double* chain, const double* tri2, float2* cdf, const Ctl* ctl,
                      int step, int num_sms, int cps) {
  const bool two = out2 != nullptr;
  CoefDfArgs ca;
  ca.coef1 = coef1;
  ca.coef2 = coef2;
  ca.chain = chain;
  ca.tri1 = tri1;
  ca.tri2 = tri2;
  ca.nin = nin;
  ca.s = s;
  ca.two = two ? 1 : 0;
  ca.out = cdf;
  ca.ctl = ctl;
  ca.step = step;
  const int total = (int)coef_df_count(nin, s, two);
  k_coef_df<<<(total + 127) / 128, 128, 0, st>>>(ca);
  UpdDfArgs u;
  u.in = in;
  u.nin = nin;
  u.s = s;
  u.S2 = next_pow2_df(s);
  u.n = n;
  u.out1 = out1;
  u.out2 = out2;
  u.cdf = cdf;
  u.has_tri1 = tri1 != nullptr;
  u.has_chain = two && chain != nullptr;
  u.has_tri2 = two && tri2 != nullptr;
  u.ctl = ctl;
  u.step = step;
  const size_t smem_all = update_df_smem(nin, s, two);
  u.staged = smem_all <= UPDATE_DF_SMEM_MAX ? 1 : 0;
  const size_t smem = u.staged ? smem_all : 0;
  static std::atomic<unsigned long long> attr_done{0};
  once_per_device(attr_done, [] {
    cudaFuncSetAttribute(k_update_df, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_update_df_row<4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_update_df_row<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_update_df_row<8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_update_df_row<8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_update_df_row<16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_update_df_row<16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  if (u.staged && (s == 4 || s == 8 || s == 16)) {
    int64_t need = (n + 255) / 256;
    int64_t grid = (int64_t)(cps > 0 ? cps : 4) * num_sms;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
#define LAUNCH_ROW(SV)                                                        \
    if (two) k_update_df_row<SV, true><<<(unsigned)grid, 256, smem, st>>>(u); \
    else k_update_df_row<SV, false><<<(unsigned)grid, 256, smem, st>>>(u);
    if (s == 4) { LAUNCH_ROW(4) }
    else if (s == 8) { LAUNCH_ROW(8) }
    else { LAUNCH_ROW(16) }
#undef LAUNCH_ROW
    return;
  }
  if (s == 32) {
    const int64_t need = (n + 127) / 128;
    int64_t grid = (int64_t)(cps > 0 ? cps : 4) * num_sms;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    if (two) k_update_df_w32<true><<<(unsigned)grid, 256, 0, st>>>(u);
    else k_update_df_w32<false><<<(unsigned)grid, 256, 0, st>>>(u);
    return;
  }
  const int rows_per_cta = 256 / u.S2;
  const int64_t need = (n + rows_per_cta - 1) / rows_per_cta;
  int64_t grid = (int64_t)(cps > 0 ? cps : 4) * num_sms;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  k_update_df<<<(unsigned)grid, 256, smem, st>>>(u);
}

}  // namespace lsba
