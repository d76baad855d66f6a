// Column muscles MGS-SVL / MGS-LTS for BMGS-SVL / BMGS-LTS (Alg. 5 with block
// size 1 applied to the columns of one n x s block, in Gram-Schmidt form).
//
// Column j of X (in place; columns < j already hold Q):
//   j > 0: y = Q_{<j}^T x_j            (a reduction over the rows: one sync)
//          r = T^T y (SVL) or T^{-T} y (LTS), R_{<j,j} = r
//          x_j <- x_j - Q_{<j} r
//   d = x_j^T x_j                        (one sync); the NaN-flag of the
//          Cholesky reading for s = 1 fires iff d <= 0 or d is not finite
//   R_jj = sqrt(d), q_j = x_j / R_jj
//   j > 0: z = Q_{<j}^T q_j              (one sync); T_{<j,j} = -T z (SVL) or z
//          (LTS), T_jj = 1
// so a call costs 3s - 2 syncs.  Each sync is three launches: per-CTA partial
// dot products (`k_mus_dots`, fixed row ranges), a one-CTA step that sums
// them in CTA order and does the small algebra (`k_mus_step`), and a row pass
// (`k_mus_rows`).  The block may be FP64, double-float (float2) or FP32; the
// arithmetic is FP64.  The muscle is a comparator of the paper's classical
// BMGS-SVL/LTS configuration, not a bandwidth kernel.
//
// Work area (doubles): R (s x s, col-major) | T (s x s, col-major, unit upper)
// | coefficients (s) | status, column of the flag | partials [MUS_PARTS][s].
#include "df.cuh"
#include "lsba_internal.cuh"

namespace lsba {

#define MUS_THREADS 256

struct MusArgs {
  void* X;
  int mode;          // 0 FP64, 1 double-float (float2), 2 FP32
  int64_t n;
  int s, j, phase;   // phase 0: y and the update, 1: the norm, 2: z and T
  int lts;
  double* area;
  int parts;         // CTAs of the partial-sum launch
  Ctl* ctl;
  int step;          // run iff step < 0 or ctl->update_step == step
};

__device__ __forceinline__ double mus_ld(const MusArgs& a, int64_t i) {
  if (a.mode == 0) return static_cast<const double*>(a.X)[i];
  if (a.mode == 1) return df_to_double(static_cast<const float2*>(a.X)[i]);
  return (double)static_cast<const float*>(a.X)[i];
}
__device__ __forceinline__ void mus_st(const MusArgs& a, int64_t i, double v) {
  if (a.mode == 0) static_cast<double*>(a.X)[i] = v;
  else if (a.mode == 1) static_cast<float2*>(a.X)[i] = df_from_double(v);
  else static_cast<float*>(a.X)[i] = (float)v;
}

// starts_call: column 0's partial sums and step, which begin a call and so
// must not read the flag a previous call left.
__device__ __forceinline__ bool mus_on(const MusArgs& a, bool starts_call) {
  if (a.step >= 0 && *(volatile const int*)&a.ctl->update_step != a.step) return false;
  // a flag earlier in this call stops the rest of it
  if (!starts_call && a.area[2 * a.s * a.s + a.s] != 0.0) return false;
  return true;
}

// Per-CTA partial sums of X[:, q] . X[:, j] for q in [q0, q1): phase 0 and 2
// take q < j, phase 1 q = j.
__global__ void __launch_bounds__(MUS_THREADS) k_mus_dots(const __grid_constant__ MusArgs a) {
  if (!mus_on(a, a.j == 0 && a.phase == 1)) return;
  __shared__ double red[MUS_THREADS / 32];
  const int s = a.s, j = a.j;
  const int q0 = a.phase == 1 ? j : 0, q1 = a.phase == 1 ? j + 1 : j;
  const int64_t rows = (a.n + a.parts - 1) / a.parts;
  const int64_t r0 = (int64_t)blockIdx.x * rows;
  const int64_t r1 = r0 + rows < a.n ? r0 + rows : a.n;
  double* part = a.area + 2 * s * s + s + 8 + (size_t)blockIdx.x * s;
  for (int q = q0; q < q1; ++q) {
    double acc = 0.0;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += MUS_THREADS)
      acc = fma(mus_ld(a, r * s + q), mus_ld(a, r * s + j), acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < MUS_THREADS / 32; ++w) t += red[w];
      part[q] = t;
    }
    __syncthreads();
  }
}

// One thread: the partials summed in CTA order, then the small algebra.
__global__ void k_mus_step(const __grid_constant__ MusArgs a) {
  if (!mus_on(a, a.j == 0 && a.phase == 1) || threadIdx.x != 0) return;
  const int s = a.s, j = a.j;
  double* R = a.area;
  double* T = a.area + s * s;
  double* coef = a.area + 2 * s * s;
  double* status = coef + s;
  const double* part = status + 8;
  double v[LSBA_MAX_S];
  const int q0 = a.phase == 1 ? j : 0, q1 = a.phase == 1 ? j + 1 : j;
  for (int q = q0; q < q1; ++q) {
    double t = 0.0;
    for (int c = 0; c < a.parts; ++c) t += part[(size_t)c * s + q];
    v[q] = t;
  }
  a.ctl->muscle_syncs += 1;   // one sync of the muscle
  if (a.phase == 0) {
    // r = T^T y (SVL) or T^{-T} y (LTS), T unit upper triangular
    for (int i = 0; i < j; ++i) {
      double t = v[i];
      if (a.lts) {
        for (int q = 0; q < i; ++q) t = fma(-T[q + i * s], coef[q], t);
      } else {
        for (int q = 0; q < i; ++q) t = fma(T[q + i * s], v[q], t);
      }
      coef[i] = t;
      R[i + j * s] = t;
    }
  } else if (a.phase == 1) {
    if (j == 0) {
      for (int e = 0; e < s * s; ++e) {
        R[e] = 0.0;
        T[e] = (e % (s + 1) == 0) ? 1.0 : 0.0;
      }
      status[0] = 0.0;
    }
    const double d = v[j];
    if (!(d > 0.0) || !isfinite(d)) {
      status[0] = 1.0;
      status[1] = (double)j;
      return;
    }
    R[j + j * s] = sqrt(d);
    coef[0] = R[j + j * s];
  } else {
    // T_{<j,j} = z (LTS) or -T_{<j,<j} z (SVL)
    for (int i = 0; i < j; ++i) {
      double t = v[i];
      if (!a.lts)
        for (int q = i + 1; q < j; ++q) t = fma(T[i + q * s], v[q], t);
      T[i + j * s] = a.lts ? t : -t;
    }
  }
}

// Row pass: phase 0: x_j -= Q_{<j} r; phase 1: q_j = x_j / R_jj.
__global__ void __launch_bounds__(MUS_THREADS) k_mus_rows(const __grid_constant__ MusArgs a) {
  if (!mus_on(a, false)) return;
  const int s = a.s, j = a.j;
  const double* coef = a.area + 2 * s * s;
  for (int64_t r = (int64_t)blockIdx.x * MUS_THREADS + threadIdx.x; r < a.n;
       r += (int64_t)gridDim.x * MUS_THREADS) {
    if (a.phase == 0) {
      double t = mus_ld(a, r * s + j);
      for (int q = 0; q < j; ++q) t = fma(-mus_ld(a, r * s + q), coef[q], t);
      mus_st(a, r * s + j, t);
    } else {
      mus_st(a, r * s + j, mus_ld(a, r * s + j) / coef[0]);
    }
  }
}

size_t muscle_area_doubles(int s) { return (size_t)2 * s * s + s + 8 + (size_t)MUS_PARTS * s; }

void launch_col_muscle(cudaStream_t st, void* X, int mode, int64_t n, int s, bool lts,
                       double* area, Ctl* ctl, int step, int num_sms) {
  MusArgs a;
  a.X = X;
  a.mode = mode;
  a.n = n;
  a.s = s;
  a.lts = lts ? 1 : 0;
  a.area = area;
  int parts = 2 * num_sms;
  if (parts > MUS_PARTS) parts = MUS_PARTS;
  if ((int64_t)parts * 64 > n) parts = (int)((n + 63) / 64);
  if (parts < 1) parts = 1;
  a.parts = parts;
  a.ctl = ctl;
  a.step = step;
  int rgrid = 4 * num_sms;
  if ((int64_t)rgrid * MUS_THREADS > n) rgrid = (int)((n + MUS_THREADS - 1) / MUS_THREADS);
  if (rgrid < 1) rgrid = 1;
  for (int j = 0; j < s; ++j) {
    a.j = j;
    if (j > 0) {
      a.phase = 0;
      k_mus_dots<<<parts, MUS_THREADS, 0, st>>>(a);
      k_mus_step<<<1, 32, 0, st>>>(a);
      k_mus_rows<<<rgrid, MUS_THREADS, 0, st>>>(a);
    }
    a.phase = 1;
    k_mus_dots<<<parts, MUS_THREADS, 0, st>>>(a);
    k_mus_step<<<1, 32, 0, st>>>(a);
    k_mus_rows<<<rgrid, MUS_THREADS, 0, st>>>(a);
    if (j > 0) {
      a.phase = 2;
      k_mus_dots<<<parts, MUS_THREADS, 0, st>>>(a);
      k_mus_step<<<1, 32, 0, st>>>(a);
    }
  }
}

}  // namespace lsba
