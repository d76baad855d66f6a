// FP32 kernels of the inner solver of FP64 iterative refinement (mixed
// precision).  Block vectors are FP32 (4 bytes per entry); the SpMM, the
// one-pass Gram and the basis update multiply and accumulate in FP32 on the
// FP32 pipes.  The per-CTA Gram partials are summed across CTAs in CTA order
// with compensated (TwoSum) FP32 arithmetic and converted to FP64; every small
// s x s / ks x s computation after the Gram (Cholesky,
// Hessenberg least squares, estimate) stays FP64, as do the outer residual
// B - A X and the solution update X += D.
//
//   k_spmm_f32      W = A V                       (Sec. 2.1 matvec)
//   k_gram_f32_tma  [L_1..L_a]^T [R_1..R_b]        (one pass; bulk-copy pipeline)
//   k_update_f32    out = (sum_i in_i C_i (+ out1 chain)) T^{-1}, two outputs
#include "lsba_internal.cuh"
#include "tma.cuh"

namespace lsba {

static __device__ __forceinline__ int ctl_on(const Ctl* c) { return *(volatile const int*)&c->active; }

// ----------------------------------------------------------------- conversions
// scale is a power of two: the inner solver works on a scaled copy whose
// largest entries are near 1, so FP32's exponent range is not left.
__global__ void k_to_f32(int64_t count, const double* __restrict__ in, float* __restrict__ out,
                         double scale) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = __double2float_rn(in[i] * scale);
}
// X += scale D (D in FP32): the FP64 solution update of iterative refinement.
__global__ void k_add_f32(int64_t count, const float* __restrict__ d, double* __restrict__ x,
                          double scale) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) x[i] += (double)d[i] * scale;
}
void launch_to_f32(cudaStream_t st, int64_t count, const double* in, float* out, double scale) {
  if (count > 0) k_to_f32<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(count, in, out, scale);
}
void launch_add_f32(cudaStream_t st, int64_t count, const float* d, double* x, double scale) {
  if (count > 0) k_add_f32<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(count, d, x, scale);
}

// ----------------------------------------------------------------- SpMM
__global__ void __launch_bounds__(256) k_spmm_f32(int64_t n, const int32_t* __restrict__ rowptr,
                                                  const int32_t* __restrict__ colidx,
                                                  const float* __restrict__ vals,
                                                  const float* __restrict__ V, float* __restrict__ W,
                                                  int s, int S2, const Ctl* ctl, int guard) {
  if (guard && !ctl_on(ctl)) return;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t row = idx / S2;
  const int c = (int)(idx % S2);
  if (row >= n || c >= s) return;
  const int p0 = rowptr[row], p1 = rowptr[row + 1];
  float acc = 0.f;
  for (int p = p0; p < p1; ++p) acc = fmaf(vals[p], V[(int64_t)colidx[p] * s + c], acc);
  W[row * s + c] = acc;
}

void launch_spmm_f32(cudaStream_t st, int64_t n, const int32_t* rowptr, const int32_t* colidx,
                     const float* vals, const float* V, float* W, int s, const Ctl* ctl, int guard) {
  int S2 = 1;
  while (S2 < s) S2 <<= 1;
  const int64_t threads = n * S2;
  if (threads == 0) return;
  k_spmm_f32<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(n, rowptr, colidx, vals, V, W, s,
                                                                 S2, ctl, guard);
}

// ----------------------------------------------------------------- Gram
// Same tiling as the double-float Gram: 4x4 output tiles per thread, up to 256
// tiles per CTA, row groups when a CTA has fewer tiles, two bulk-copy stages.
#define GF_THREADS 256

struct GramF32Args {
  BlockPtrs L;
  BlockPtrs R;
  int a, b, s, rc;
  int64_t n, rows_per_cta;
  int q, ntj, ntile;
  unsigned stage_elems;
  float* partials;
  const Ctl* ctl;
  int guard;
  int* err;
};

__global__ void __launch_bounds__(GF_THREADS) k_gram_f32_tma(const __grid_constant__ GramF32Args g) {
  if (g.guard && !ctl_on(g.ctl)) return;
  extern __shared__ __align__(128) unsigned char smraw[];
  uint64_t* bars = (uint64_t*)smraw;
  float* stage0 = (float*)(smraw + 128);
  float* stage1 = stage0 + g.stage_elems;
  const int s = g.s, rc = g.rc, a = g.a, b = g.b;
  const int nblk = a + b;
  const int tile_base = blockIdx.y * GF_THREADS;
  const int cnt = min(GF_THREADS, g.ntile - tile_base);
  const int groups = GF_THREADS / cnt;
  const int grp = threadIdx.x / cnt;
  const int tl = threadIdx.x % cnt;
  const bool active = grp < groups;
  const int T = tile_base + tl;
  const int it = T / g.ntj, jt = T % g.ntj;
  const int li = it * 4, rj = jt * 4;
  const int lofs = (li / s) * rc * s + (li % s);
  const int rofs = (a + rj / s) * rc * s + (rj % s);
  const int64_t r_begin = (int64_t)blockIdx.x * g.rows_per_cta;
  const int64_t r_end = min(g.n, r_begin + g.rows_per_cta);
  const int nchunks = r_end > r_begin ? (int)((r_end - r_begin + rc - 1) / rc) : 0;
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int c, int st) {
    const int64_t r0 = r_begin + (int64_t)c * rc;
    const int rows = (int)min((int64_t)rc, r_end - r0);
    const unsigned bytes = (unsigned)(rows * s * sizeof(float));
    float* dst = st ? stage1 : stage0;
    mbar_expect_tx(&bars[st], bytes * nblk);
    for (int blk = 0; blk < nblk; ++blk) {
      const float* src = (const float*)(blk < a ? g.L.p[blk] : g.R.p[blk - a]) + r0 * s;
      bulk_copy_g2s(dst + (size_t)blk * rc * s, src, bytes, &bars[st]);
    }
  };
  if (threadIdx.x == 0) {
    if (nchunks > 0) issue(0, 0);
    if (nchunks > 1) issue(1, 1);
  }
  float acc[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
  bool failed = false;
  for (int c = 0; c < nchunks; ++c) {
    const int st = c & 1;
    const bool ok = mbar_wait_bounded(&bars[st], (unsigned)((c >> 1) & 1));
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    const float* buf = st ? stage1 : stage0;
    const int rows = (int)min((int64_t)rc, r_end - (r_begin + (int64_t)c * rc));
    if (active) {
      for (int r = grp; r < rows; r += groups) {
        const float4 l = *(const float4*)(buf + lofs + r * s);
        const float4 rr = *(const float4*)(buf + rofs + r * s);
        const float lv[4] = {l.x, l.y, l.z, l.w};
        const float rv[4] = {rr.x, rr.y, rr.z, rr.w};
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(lv[x], rv[y], acc[x][y]);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && c + 2 < nchunks) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(c + 2, st);
    }
  }
  if (failed) {
    if (threadIdx.x == 0) {
      if (g.err) atomicExch(g.err, 1);
      for (int c2 = 0; c2 < 2; ++c2) mbar_wait_bounded(&bars[c2], 0), mbar_wait_bounded(&bars[c2], 1);
    }
    __syncthreads();
    return;
  }
  if (groups > 1) {
    __syncthreads();
    float* red = stage0;
    if (active) {
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) red[((size_t)grp * cnt + tl) * 16 + x * 4 + y] = acc[x][y];
    }
    __syncthreads();
    if (grp == 0) {
      for (int g2 = 1; g2 < groups; ++g2)
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] += red[((size_t)g2 * cnt + tl) * 16 + x * 4 + y];
    }
  }
  if (grp == 0) {
    const int bs = b * s;
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y)
        g.partials[(int64_t)blockIdx.x * g.q + (int64_t)(li + x) * bs + (rj + y)] = acc[x][y];
  }
}

__global__ void k_gram_reduce_f32(const float* __restrict__ partials, int nparts, int q,
                                  double* __restrict__ G, const Ctl* ctl, int guard) {
  if (guard && !ctl_on(ctl)) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= q) return;
  // Compensated (TwoSum) FP32 accumulation in CTA order; one FP64 conversion.
  float sum = 0.f, comp = 0.f;
  for (int x = 0; x < nparts; ++x) {
    const float p = partials[(int64_t)x * q + e];
    const float t = __fadd_rn(sum, p);
    const float bb = __fsub_rn(t, sum);
    comp = __fadd_rn(comp, __fadd_rn(__fsub_rn(sum, __fsub_rn(t, bb)), __fsub_rn(p, bb)));
    sum = t;
  }
  G[e] = (double)sum + (double)comp;
}

GramPlan plan_gram_f32(int64_t n, int s, int a, int b, int num_sms) {
  GramPlan p{};
  p.q = a * s * b * s;
  const int ntile = (a * s / 4) * (b * s / 4);
  p.tile = GF_THREADS;
  p.grid_y = (ntile + GF_THREADS - 1) / GF_THREADS;
  const size_t row_bytes = (size_t)(a + b) * s * sizeof(float);
  int rc = (int)((32 * 1024) / row_bytes);
  if (rc > 256) rc = 256;
  if (rc < 1) rc = 1;
  const size_t red_bytes = (size_t)GF_THREADS * 16 * sizeof(float);
  const size_t stages = 128 + 2 * row_bytes * rc;
  p.smem = stages > 128 + red_bytes ? stages : 128 + red_bytes;
  p.rows_per_chunk = rc;
  int gx = (3 * num_sms + p.grid_y - 1) / p.grid_y;
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

void launch_gram_f32(cudaStream_t st, const GramPlan& p, const BlockPtrs& L, int a,
                     const BlockPtrs& R, int b, int64_t n, int s, float* partials, double* G,
                     const Ctl* ctl, int guard, int* err) {
  static std::atomic<unsigned long long> attr_done{0};
  once_per_device(attr_done, [] {
    cudaFuncSetAttribute(k_gram_f32_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  GramF32Args g;
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
  g.stage_elems = (unsigned)((a + b) * p.rows_per_chunk * s);
  g.partials = partials;
  g.ctl = ctl;
  g.guard = guard;
  g.err = err;
  dim3 grid(p.grid_x, p.grid_y);
  k_gram_f32_tma<<<grid, GF_THREADS, p.smem, st>>>(g);
  k_gram_reduce_f32<<<(p.q + 255) / 256, 256, 0, st>>>(partials, p.grid_x, p.q, G, ctl, guard);
}

// ----------------------------------------------------------------- Update
// Coefficients are converted to FP32 once per step (k_coef_f32, many CTAs),
// then one thread per row (s = 4, 8, 16) forms both outputs in registers.
__host__ __device__ size_t coef_f32_count(int nin, int s, bool two) {
  const size_t ss = (size_t)s * s;
  return (size_t)nin * ss * (two ? 2 : 1) + 3 * ss + 2 * (size_t)s;
}

struct CoefF32Args {
  const double* coef1;
  const double* coef2;
  const double* chain;
  const double* tri1;
  const double* tri2;
  int nin, s, two;
  float* out;
  const Ctl* ctl;
  int step;
};

__global__ void k_coef_f32(const __grid_constant__ CoefF32Args a) {
  if (a.step >= 0 && *(volatile const int*)&a.ctl->update_step != a.step) return;
  const int s = a.s, ss = s * s;
  const int n1 = a.nin * ss, n2 = a.two ? n1 : 0;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  int o = e;
  float v = 0.f;
  if (o < n1) v = __double2float_rn(a.coef1[o]);
  else if ((o -= n1) < n2) v = __double2float_rn(a.coef2[o]);
  else if ((o -= n2) < ss) v = (a.two && a.chain) ? __double2float_rn(a.chain[o]) : 0.f;
  else if ((o -= ss) < ss) v = a.tri1 ? __double2float_rn(a.tri1[o]) : 0.f;
  else if ((o -= ss) < ss) v = (a.two && a.tri2) ? __double2float_rn(a.tri2[o]) : 0.f;
  else if ((o -= ss) < s) v = a.tri1 ? __double2float_rn(1.0 / a.tri1[o * s + o]) : 0.f;
  else if ((o -= s) < s) v = (a.two && a.tri2) ? __double2float_rn(1.0 / a.tri2[o * s + o]) : 0.f;
  else return;
  a.out[e] = v;
}

struct UpdF32Args {
  BlockPtrs in;
  int nin;
  int64_t n;
  float* out1;
  float* out2;
  const float* cf;
  int has_tri1, has_chain, has_tri2;
  const Ctl* ctl;
  int step;
};

template <int S, bool TWO>
__global__ void __launch_bounds__(256) k_update_f32(const __grid_constant__ UpdF32Args u) {
  if (u.step >= 0 && *(volatile const int*)&u.ctl->update_step != u.step) return;
  extern __shared__ float csf[];
  const int nin = u.nin;
  constexpr int SS = S * S;
  const int total = (int)coef_f32_count(nin, S, TWO);
  for (int e = threadIdx.x; e < total; e += blockDim.x) csf[e] = u.cf[e];
  __syncthreads();
  const float* c1 = csf;
  const float* c2 = c1 + (size_t)nin * SS;
  const float* ch = c2 + (TWO ? (size_t)nin * SS : 0);
  const float* t1 = ch + SS;
  const float* t2 = t1 + SS;
  const float* r1 = t2 + SS;
  const float* r2 = r1 + S;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < u.n;
       row += (int64_t)gridDim.x * blockDim.x) {
    float a1[S], a2[S];
#pragma unroll
    for (int c = 0; c < S; ++c) a1[c] = a2[c] = 0.f;
    for (int bk = 0; bk < nin; ++bk) {
      float v[S];
      const float4* src = (const float4*)((const float*)u.in.p[bk] + row * S);
#pragma unroll
      for (int i = 0; i < S / 4; ++i) {
        const float4 t = src[i];
        v[4 * i] = t.x;
        v[4 * i + 1] = t.y;
        v[4 * i + 2] = t.z;
        v[4 * i + 3] = t.w;
      }
      const float* k1 = c1 + (size_t)bk * SS;
      const float* k2 = c2 + (size_t)bk * SS;
#pragma unroll
      for (int q = 0; q < S; ++q)
#pragma unroll
        for (int c = 0; c < S; ++c) {
          a1[c] = fmaf(v[q], k1[q * S + c], a1[c]);
          if (TWO) a2[c] = fmaf(v[q], k2[q * S + c], a2[c]);
        }
    }
    if (u.has_tri1) {
#pragma unroll
      for (int c = 0; c < S; ++c) {
#pragma unroll
        for (int q = 0; q < c; ++q) a1[c] = fmaf(-a1[q], t1[q * S + c], a1[c]);
        a1[c] *= r1[c];
      }
    }
    float4* d1 = (float4*)(u.out1 + row * S);
#pragma unroll
    for (int i = 0; i < S / 4; ++i) d1[i] = make_float4(a1[4 * i], a1[4 * i + 1], a1[4 * i + 2], a1[4 * i + 3]);
    if (TWO) {
      if (u.has_chain) {
#pragma unroll
        for (int q = 0; q < S; ++q)
#pragma unroll
          for (int c = 0; c < S; ++c) a2[c] = fmaf(a1[q], ch[q * S + c], a2[c]);
      }
      if (u.has_tri2) {
#pragma unroll
        for (int c = 0; c < S; ++c) {
#pragma unroll
          for (int q = 0; q < c; ++q) a2[c] = fmaf(-a2[q], t2[q * S + c], a2[c]);
          a2[c] *= r2[c];
        }
      }
      float4* d2 = (float4*)(u.out2 + row * S);
#pragma unroll
      for (int i = 0; i < S / 4; ++i) d2[i] = make_float4(a2[4 * i], a2[4 * i + 1], a2[4 * i + 2], a2[4 * i + 3]);
    }
  }
}

size_t update_f32_smem(int nin, int s, bool two) { return sizeof(float) * coef_f32_count(nin, s, two); }

void launch_update_f32(cudaStream_t st, const BlockPtrs& in, int nin, int64_t n, int s, float* out1,
                       const double* coef1, const double* tri1, float* out2, const double* coef2,
                       const double* chain, const double* tri2, float* cf, const Ctl* ctl, int step,
                       int num_sms) {
  const bool two = out2 != nullptr;
  CoefF32Args ca;
  ca.coef1 = coef1;
  ca.coef2 = coef2;
  ca.chain = chain;
  ca.tri1 = tri1;
  ca.tri2 = tri2;
  ca.nin = nin;
  ca.s = s;
  ca.two = two ? 1 : 0;
  ca.out = cf;
  ca.ctl = ctl;
  ca.step = step;
  const int total = (int)coef_f32_count(nin, s, two);
  k_coef_f32<<<(total + 127) / 128, 128, 0, st>>>(ca);
  UpdF32Args u;
  u.in = in;
  u.nin = nin;
  u.n = n;
  u.out1 = out1;
  u.out2 = out2;
  u.cf = cf;
  u.has_tri1 = tri1 != nullptr;
  u.has_chain = two && chain != nullptr;
  u.has_tri2 = two && tri2 != nullptr;
  u.ctl = ctl;
  u.step = step;
  const size_t smem = update_f32_smem(nin, s, two);
  static std::atomic<unsigned long long> attr_done{0};
  once_per_device(attr_done, [] {
    cudaFuncSetAttribute(k_update_f32<4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_update_f32<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_update_f32<8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_update_f32<8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_update_f32<16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_update_f32<16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  int64_t need = (n + 255) / 256;
  int64_t grid = 4LL * num_sms;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
#define LAUNCH_F32(SV)                                                     \
  if (two) k_update_f32<SV, true><<<(unsigned)grid, 256, smem, st>>>(u); \
  else k_update_f32<SV, false><<<(unsigned)grid, 256, smem, st>>>(u);
  if (s == 4) { LAUNCH_F32(4) }
  else if (s == 8) { LAUNCH_F32(8) }
  else { LAUNCH_F32(16) }
#undef LAUNCH_F32
}

}  // namespace lsba
