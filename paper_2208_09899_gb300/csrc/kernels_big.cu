// Bandwidth-shaped kernels of one block Arnoldi step (all FP64):
//   SpMM        W = A V                                   (the paper's matvec, Sec. 2.1)
//   Gram        [L_1..L_a]^T [R_1..R_b]  in one pass        (the one sync point of Alg. 3
//                                                            line 4, Alg. 6 line 10, Alg. 7 line 10)
//   Update      out = (sum_i in_i C_i) T^{-1}, two outputs  (Alg. 3 line 6, Alg. 6 lines 17-18,
//               in one pass over the inputs                  Alg. 7 lines 16-17, cycle end Thm. 1)
// Block vectors are n x s row-major FP64.  A row's s values are handled by a
// group of S2 = next_pow2(s) lanes of one warp, so that a row is one coalesced
// segment and its values are exchanged with warp shuffles.
#include "lsba_internal.cuh"

namespace lsba {

static __device__ __forceinline__ int ctl_active(const Ctl* c) {
  return *(volatile const int*)&c->active;
}

static inline int next_pow2(int s) {
  int p = 1;
  while (p < s) p <<= 1;
  return p;
}

// ----------------------------------------------------------------- SpMM (CSR)
__global__ void __launch_bounds__(256) k_spmm(int64_t n, const int32_t* __restrict__ rowptr,
                                              const int32_t* __restrict__ colidx,
                                              const double* __restrict__ vals,
                                              const double* __restrict__ V, double* __restrict__ W,
                                              int s, int S2, const Ctl* ctl, int guard) {
  if (guard && !ctl_active(ctl)) return;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t row = idx / S2;
  const int c = (int)(idx % S2);
  if (row >= n || c >= s) return;
  const int p0 = rowptr[row], p1 = rowptr[row + 1];
  double acc = 0.0;
  for (int p = p0; p < p1; ++p) acc = fma(vals[p], V[(int64_t)colidx[p] * s + c], acc);
  W[row * s + c] = acc;
}

void launch_spmm(cudaStream_t st, int64_t n, const int32_t* rowptr, const int32_t* colidx,
                 const double* vals, const double* V, double* W, int s, const Ctl* ctl, int guard) {
  const int S2 = next_pow2(s);
  const int64_t threads = n * S2;
  const unsigned grid = (unsigned)((threads + 255) / 256);
  if (grid == 0) return;
  k_spmm<<<grid, 256, 0, st>>>(n, rowptr, colidx, vals, V, W, s, S2, ctl, guard);
}

__global__ void k_axpby(int64_t total, const double* __restrict__ B, const double* __restrict__ W,
                        double* __restrict__ R) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < total) R[i] = B[i] - W[i];
}

void launch_axpby(cudaStream_t st, int64_t n, int s, const double* B, const double* W, double* R) {
  const int64_t total = n * s;
  if (total == 0) return;
  k_axpby<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(total, B, W, R);
}

// ----------------------------------------------------------------- Gram
// Each CTA (x, y) owns a contiguous range of rows (x) and a tile of output
// entries (y).  Rows are staged chunk by chunk in shared memory for all a + b
// blocks; every thread accumulates up to GRAM_EPT output entries over the
// CTA's rows in row order, then writes its partial sums.  A second kernel adds
// the per-CTA partials in CTA order, so the result does not depend on timing.
#define GRAM_THREADS 256
#define GRAM_EPT 16

struct GramArgs {
  BlockPtrs L;
  BlockPtrs R;
  int a, b, s, rc;
  int64_t n, rows_per_cta;
  int q;
  double* partials;
  const Ctl* ctl;
  int guard;
};

__global__ void __launch_bounds__(GRAM_THREADS) k_gram(const __grid_constant__ GramArgs g) {
  if (g.guard && !ctl_active(g.ctl)) return;
  extern __shared__ double sm[];
  const int s = g.s, a = g.a, b = g.b, rc = g.rc;
  const int bs = b * s;
  const int nblk = a + b;
  const int64_t r_begin = (int64_t)blockIdx.x * g.rows_per_cta;
  const int64_t r_end = min(g.n, r_begin + g.rows_per_cta);
  const int tile0 = blockIdx.y * (GRAM_THREADS * GRAM_EPT);

  int loff[GRAM_EPT], roff[GRAM_EPT];
  double acc[GRAM_EPT];
#pragma unroll
  for (int t = 0; t < GRAM_EPT; ++t) {
    const int e = tile0 + threadIdx.x + t * GRAM_THREADS;
    acc[t] = 0.0;
    if (e < g.q) {
      const int i = e / bs, jj = e % bs;
      loff[t] = (i / s) * rc * s + (i % s);
      roff[t] = (a + jj / s) * rc * s + (jj % s);
    } else {
      loff[t] = -1;
      roff[t] = 0;
    }
  }

  for (int64_t r0 = r_begin; r0 < r_end; r0 += rc) {
    const int rows = (int)min((int64_t)rc, r_end - r0);
    const int per = rows * s;
    __syncthreads();
    for (int idx = threadIdx.x; idx < nblk * per; idx += GRAM_THREADS) {
      const int blk = idx / per, off = idx - blk * per;
      const double* src = blk < a ? g.L.p[blk] : g.R.p[blk - a];
      sm[blk * rc * s + off] = src[r0 * s + off];
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < GRAM_EPT; ++t) {
      if (loff[t] >= 0) {
        const double* lp = sm + loff[t];
        const double* rp = sm + roff[t];
        double v = acc[t];
        for (int r = 0; r < rows; ++r) v = fma(lp[r * s], rp[r * s], v);
        acc[t] = v;
      }
    }
  }
#pragma unroll
  for (int t = 0; t < GRAM_EPT; ++t) {
    const int e = tile0 + threadIdx.x + t * GRAM_THREADS;
    if (e < g.q) g.partials[(int64_t)blockIdx.x * g.q + e] = acc[t];
  }
}

// Sum of the per-CTA partials in a fixed order: a CTA of 8 warps handles 32
// consecutive outputs (lane = output); warp w sums the partials of CTAs
// [w P / 8, (w + 1) P / 8) in CTA order, four independent running sums per
// lane (partial x goes to sum x % 4, combined 0 + 1 + 2 + 3), and the eight
// warp sums are added in warp order.  The order depends only on the number of
// partials, so results are bitwise reproducible.
__global__ void __launch_bounds__(256) k_gram_reduce(const double* __restrict__ partials, int nparts,
                                                     int q, double* __restrict__ G, const Ctl* ctl,
                                                     int guard) {
  if (guard && !ctl_active(ctl)) return;
  __shared__ double part[8][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int e = blockIdx.x * 32 + lane;
  const int x0 = (int)((int64_t)warp * nparts / 8), x1 = (int)((int64_t)(warp + 1) * nparts / 8);
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  if (e < q) {
    // all loads of a chunk issued before the sums (one memory round trip a
    // chunk); the sums keep the order x0, x0 + 1, .. into a[(x - x0) % 4]
    for (int c0 = x0; c0 < x1; c0 += 24) {
      double v[24];
#pragma unroll
      for (int i = 0; i < 24; ++i) v[i] = c0 + i < x1 ? partials[(int64_t)(c0 + i) * q + e] : 0.0;
#pragma unroll
      for (int i = 0; i < 24; ++i)
        if (c0 + i < x1) a[i & 3] += v[i];   // (c0 - x0) is a multiple of 4
    }
  }
  part[warp][lane] = (a[0] + a[1]) + (a[2] + a[3]);
  __syncthreads();
  if (warp == 0 && e < q) {
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) v += part[w][lane];
    G[e] = v;
  }
}

GramPlan plan_gram(int64_t n, int s, int a, int b, int num_sms) {
  GramPlan p{};
  p.q = a * s * b * s;
  p.tile = GRAM_THREADS * GRAM_EPT;
  p.grid_y = (p.q + p.tile - 1) / p.tile;
  const size_t row_bytes = (size_t)(a + b) * s * sizeof(double);
  int rc = (int)((96 * 1024) / row_bytes);
  if (rc > 32) rc = 32;
  if (rc < 1) rc = 1;
  p.rows_per_chunk = rc;
  p.smem = row_bytes * rc;
  int gx = (2 * num_sms + p.grid_y - 1) / p.grid_y;
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

void launch_gram(cudaStream_t st, const GramPlan& p, const BlockPtrs& L, int a, const BlockPtrs& R,
                 int b, int64_t n, int s, double* partials, double* G, const Ctl* ctl, int guard) {
  GramArgs g;
  g.L = L;
  g.R = R;
  g.a = a;
  g.b = b;
  g.s = s;
  g.rc = p.rows_per_chunk;
  g.n = n;
  g.rows_per_cta = p.rows_per_cta;
  g.q = p.q;
  g.partials = partials;
  g.ctl = ctl;
  g.guard = guard;
  static std::atomic<unsigned long long> attr_done{0};
  once_per_device(attr_done, [] {
    cudaFuncSetAttribute(k_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  dim3 grid(p.grid_x, p.grid_y);
  k_gram<<<grid, GRAM_THREADS, p.smem, st>>>(g);
  launch_gram_reduce(st, partials, p.grid_x, p.q, G, ctl, guard);
}

void launch_gram_reduce(cudaStream_t st, const double* partials, int nparts, int q, double* G,
                        const Ctl* ctl, int guard) {
  if (q > 0) k_gram_reduce<<<(q + 31) / 32, 256, 0, st>>>(partials, nparts, q, G, ctl, guard);
}

// ----------------------------------------------------------------- Update
struct UpdArgs {
  BlockPtrs in;
  int nin, s, S2;
  int64_t n;
  double* out1;
  const double* coef1;
  const double* tri1;
  double* out2;
  const double* coef2;
  const double* chain;
  const double* tri2;
  const Ctl* ctl;
  int step;
};

// Right-multiply the row held by the lane group by T^{-1} (T upper triangular,
// row-major s x s): forward substitution over the columns, one column per step.
static __device__ __forceinline__ double row_trsm(double t, const double* __restrict__ T, int c, int s,
                                                  int S2) {
  const double rinv = (c < s) ? 1.0 / T[c * s + c] : 0.0;
  for (int q = 0; q < s; ++q) {
    const double vq = __shfl_sync(0xffffffffu, t * rinv, q, S2);
    if (c == q) t = vq;
    else if (c > q && c < s) t = fma(-vq, T[q * s + c], t);
  }
  return t;
}

__global__ void __launch_bounds__(256) k_update(const __grid_constant__ UpdArgs u) {
  if (u.step >= 0 && *(volatile const int*)&u.ctl->update_step != u.step) return;
  const int S2 = u.S2, s = u.s;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t row = idx / S2;
  const int c = (int)(idx % S2);
  const bool live = (row < u.n) && (c < s);
  const bool two = u.out2 != nullptr;
  double t1 = 0.0, t2 = 0.0;
  for (int bk = 0; bk < u.nin; ++bk) {
    const double v = live ? u.in.p[bk][row * s + c] : 0.0;
    const double* c1 = u.coef1 + (size_t)bk * s * s;
    const double* c2 = two ? u.coef2 + (size_t)bk * s * s : nullptr;
    for (int q = 0; q < s; ++q) {
      const double x = __shfl_sync(0xffffffffu, v, q, S2);
      if (c < s) {
        t1 = fma(x, c1[q * s + c], t1);
        if (two) t2 = fma(x, c2[q * s + c], t2);
      }
    }
  }
  if (u.tri1) t1 = row_trsm(t1, u.tri1, c, s, S2);
  if (two) {
    if (u.chain) {
      for (int q = 0; q < s; ++q) {
        const double x = __shfl_sync(0xffffffffu, t1, q, S2);
        if (c < s) t2 = fma(x, u.chain[q * s + c], t2);
      }
    }
    if (u.tri2) t2 = row_trsm(t2, u.tri2, c, s, S2);
  }
  __syncwarp();
  if (live) {
    u.out1[row * s + c] = t1;
    if (two) u.out2[row * s + c] = t2;
  }
}

void launch_update(cudaStream_t st, const BlockPtrs& in, int nin, int64_t n, int s, double* out1,
                   const double* coef1, const double* tri1, double* out2, const double* coef2,
                   const double* chain, const double* tri2, const Ctl* ctl, int step) {
  UpdArgs u;
  u.in = in;
  u.nin = nin;
  u.s = s;
  u.S2 = next_pow2(s);
  u.n = n;
  u.out1 = out1;
  u.coef1 = coef1;
  u.tri1 = tri1;
  u.out2 = out2;
  u.coef2 = coef2;
  u.chain = chain;
  u.tri2 = tri2;
  u.ctl = ctl;
  u.step = step;
  const int64_t threads = n * u.S2;
  const unsigned grid = (unsigned)((threads + 255) / 256);
  if (grid == 0) return;
  k_update<<<grid, 256, 0, st>>>(u);
}

}  // namespace lsba
