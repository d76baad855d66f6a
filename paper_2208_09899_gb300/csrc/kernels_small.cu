// Small FP64 kernels of the block Arnoldi step: one CTA each, working on the
// s x s and (k s) x s matrices that follow one sync point.
//
//  k_small_start   CholQR of the cycle's start block (Sec. 2.3 muscle; Alg. 3/6/7 line 1)
//  k_small_step    one loop iteration of a skeleton after its Gram pass:
//                    BCGS (Sec. 3.1), BCGS-PIP (Alg. 3), BMGS-CWY/ICWY (Alg. 6),
//                    BCGSI+LS (Alg. 7); Cholesky NaN-flag and adaptive restart (Sec. 4);
//                    then, when an Arnoldi relation j completes, the residual
//                    estimate of Eq. (9) for BFOM / BGMRES (Eq. (7), Thm. 1).
//  k_small_end     end of a cycle: Xi_j, the cospatial factor, the BGMRES
//                    modification M, and the coefficients of X += V Xi C and
//                    U = V_{j+1} [M; -H_{j+1,j}] (Sec. 2.4.2).
//
// Least squares: the block Hessenberg matrix is reduced column by column with
// block Householder reflectors (one set of s reflectors per block column, each
// acting on 2s rows).  With Q_{1..j-1} the first j-1 sets:
//   BGMRES Xi = Rbar^{-1} g (the minimiser of ||E_1 Beta - Hbar Xi||_F, which the
//     harmonic modification of Eq. (7) reproduces), estimate ||g_{j+1} C||_F;
//   BFOM: with T = last s x s block of H_j's last column after Q_{1..j-1}^T,
//     c = T^{-1} g_j, estimate ||H_{j+1,j} c C||_F;
//   BGMRES modification M = H_j^{-T} E_j H_{j+1,j}^T H_{j+1,j} = Q_{1..j-1} [0; T^{-T} S].
// All three equal the paper's formulas in exact arithmetic; the CPU oracle
// evaluates the formulas literally.
#include <cmath>

#include "lsba_internal.cuh"
#include "tma.cuh"

namespace lsba {

#define NT LSBA_SMALL_THREADS
#define NWARPS (NT / 32)

enum { SK_BCGS = 0, SK_PIP = 1, SK_LS = 2, SK_ICWY = 3, SK_CWY = 4, SK_BMGS = 5, SK_PIO = 6,
       SK_SVL = 7, SK_LTS = 8 };

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// C(MxN, ldc) = alpha * op(A) op(B) + beta * C.  op(A) is M x K.
__device__ void cta_gemm(int M, int N, int K, double alpha, const double* A, int lda, bool ta,
                         const double* B, int ldb, bool tb, double beta, double* C, int ldc) {
  for (int e = threadIdx.x; e < M * N; e += NT) {
    const int i = e % M, j = e / M;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int q = 0;
    for (; q + 3 < K; q += 4) {
      a0 = fma(ta ? A[q + i * lda] : A[i + q * lda], tb ? B[j + q * ldb] : B[q + j * ldb], a0);
      a1 = fma(ta ? A[q + 1 + i * lda] : A[i + (q + 1) * lda],
               tb ? B[j + (q + 1) * ldb] : B[q + 1 + j * ldb], a1);
      a2 = fma(ta ? A[q + 2 + i * lda] : A[i + (q + 2) * lda],
               tb ? B[j + (q + 2) * ldb] : B[q + 2 + j * ldb], a2);
      a3 = fma(ta ? A[q + 3 + i * lda] : A[i + (q + 3) * lda],
               tb ? B[j + (q + 3) * ldb] : B[q + 3 + j * ldb], a3);
    }
    for (; q < K; ++q)
      a0 = fma(ta ? A[q + i * lda] : A[i + q * lda], tb ? B[j + q * ldb] : B[q + j * ldb], a0);
    const double v = (a0 + a1) + (a2 + a3);
    C[i + j * ldc] = alpha * v + (beta == 0.0 ? 0.0 : beta * C[i + j * ldc]);
  }
  __syncthreads();
}

// Dynamic shared-memory arena of every small kernel (doubles).
#define SMALL_ARENA_DOUBLES (12 * 1024)
extern __shared__ double small_arena[];

// The same product with op(A) and op(B) first staged in shared memory by one
// coalesced, parallel load (the small kernels' operands sit in L2; staging
// turns K dependent L2 round trips per thread into one).  Falls back to
// cta_gemm when the panels do not fit the arena.
__device__ void cta_gemm_s(int M, int N, int K, double alpha, const double* A, int lda, bool ta,
                           const double* B, int ldb, bool tb, double beta, double* C, int ldc) {
  if ((size_t)M * K + (size_t)K * N > SMALL_ARENA_DOUBLES || K == 0) {
    cta_gemm(M, N, K, alpha, A, lda, ta, B, ldb, tb, beta, C, ldc);
    return;
  }
  double* As = small_arena;          // M x K, col-major (ld M)
  double* Bs = small_arena + M * K;  // K x N, col-major (ld K)
  for (int e = threadIdx.x; e < M * K; e += NT) {
    int i, q;
    if (ta) { q = e % K; i = e / K; } else { i = e % M; q = e / M; }
    As[i + q * M] = ta ? A[q + i * lda] : A[i + q * lda];
  }
  for (int e = threadIdx.x; e < K * N; e += NT) {
    int q, j;
    if (tb) { j = e % N; q = e / N; } else { q = e % K; j = e / K; }
    Bs[q + j * K] = tb ? B[j + q * ldb] : B[q + j * ldb];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < M * N; e += NT) {
    const int i = e % M, j = e / M;
    const double* bj = Bs + j * K;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int q = 0;
    for (; q + 3 < K; q += 4) {
      a0 = fma(As[i + q * M], bj[q], a0);
      a1 = fma(As[i + (q + 1) * M], bj[q + 1], a1);
      a2 = fma(As[i + (q + 2) * M], bj[q + 2], a2);
      a3 = fma(As[i + (q + 3) * M], bj[q + 3], a3);
    }
    for (; q < K; ++q) a0 = fma(As[i + q * M], bj[q], a0);
    const double v = (a0 + a1) + (a2 + a3);
    C[i + j * ldc] = alpha * v + (beta == 0.0 ? 0.0 : beta * C[i + j * ldc]);
  }
  __syncthreads();
}

__device__ void cta_copy(double* dst, int ldd, const double* src, int lds, int rows, int cols,
                         double alpha = 1.0) {
  for (int e = threadIdx.x; e < rows * cols; e += NT) {
    const int i = e % rows, j = e / rows;
    dst[i + j * ldd] = alpha * src[i + j * lds];
  }
  __syncthreads();
}

// Upper Cholesky factor R (s x s, col-major, ld s, shared) of the symmetric
// matrix whose upper triangle is read from S (col-major, lds).  Returns 1 (the
// NaN-flag) if an upper entry is non-finite or a pivot is <= 0 or non-finite.
__device__ int cta_chol(const double* S, int lds, int s, double* R, int* sflag) {
  // Right-looking: pivot p reads the updated row p of the working matrix (in
  // R's lower-left free space is not used: the work copy lives in the strict
  // upper triangle of R itself and row p is finalised in place).  Each pivot
  // takes one reciprocal square root and two barriers: the row-p scaling and
  // the trailing update of rows > p use the unscaled row p, so they need no
  // barrier between them.
  __shared__ double wrk[LSBA_MAX_S * LSBA_MAX_S];
  if (threadIdx.x == 0) *sflag = 0;
  __syncthreads();
  for (int e = threadIdx.x; e < s * s; e += NT) {
    const int a = e % s, c = e / s;
    double v = 0.0;
    if (a <= c) {
      v = S[a + c * lds];
      if (!isfinite(v)) *sflag = 1;
    }
    wrk[a + c * s] = v;
    R[a + c * s] = 0.0;
  }
  __syncthreads();
  if (*sflag) return 1;
  // The pivot's reciprocal square root is formed once, by thread 0, and
  // shared: on GB300 an FP64 rsqrt costs ~430 cycles, and 512 threads forming
  // it redundantly queue ~1800 cycles on the SM's FP64 pipe.
  __shared__ double piv[2];
  for (int p = 0; p < s; ++p) {
    const double d = wrk[p + p * s];
    if (!(d > 0.0) || !isfinite(d)) return 1;   // uniform: every thread reads the same d
    if (threadIdx.x == 0) {
      const double r0 = rsqrt(d);
      piv[0] = r0;
      piv[1] = r0 * r0;
    }
    __syncthreads();
    const double ri = piv[0];
    const double id = piv[1];
    const int nt = s - p;                        // row p (c >= p) and rows a in (p, c]
    for (int e = threadIdx.x; e < nt * nt; e += NT) {
      const int a = p + e % nt, c = p + e / nt;
      if (a > c) continue;
      if (a == p) R[p + c * s] = (c == p) ? d * ri : wrk[p + c * s] * ri;
      else wrk[a + c * s] = fma(-wrk[p + a * s] * id, wrk[p + c * s], wrk[a + c * s]);
    }
    __syncthreads();
  }
  return 0;
}

// X (rows x s, ldx) <- X R^{-1}, R upper s x s col-major (ld s).
__device__ void cta_trsm_right(double* X, int ldx, int rows, const double* R, int s) {
  for (int q = 0; q < s; ++q) {
    const double rq = R[q + q * s];
    for (int r = threadIdx.x; r < rows; r += NT) X[r + q * ldx] = X[r + q * ldx] / rq;
    __syncthreads();
    const int nc = s - q - 1;
    for (int e = threadIdx.x; e < rows * nc; e += NT) {
      const int r = e % rows, c = q + 1 + e / rows;
      X[r + c * ldx] = fma(-X[r + q * ldx], R[q + c * s], X[r + c * ldx]);
    }
    __syncthreads();
  }
}

// Y (s x cols, ldy) <- R^{-T} Y, R upper s x s col-major (ld s): forward
// substitution with R^T, one row per step (two barriers per row).
__device__ void cta_trsm_left_T(const double* R, int s, double* Y, int ldy, int cols) {
  __shared__ double rowq[64];
  __shared__ double rdiag[LSBA_MAX_S];
  for (int q = threadIdx.x; q < s; q += NT) rdiag[q] = 1.0 / R[q + q * s];
  __syncthreads();
  for (int q = 0; q < s; ++q) {
    for (int c = threadIdx.x; c < cols; c += NT) {
      const double v = Y[q + c * ldy] * rdiag[q];
      Y[q + c * ldy] = v;
      rowq[c] = v;
    }
    __syncthreads();
    const int nr = s - q - 1;
    for (int e = threadIdx.x; e < nr * cols; e += NT) {
      const int r = q + 1 + e % nr, c = e / nr;
      Y[r + c * ldy] = fma(-R[q + r * s], rowq[c], Y[r + c * ldy]);
    }
    __syncthreads();
  }
}

// Inverse of an upper-triangular s x s R (col-major) into Ri (col-major).
__device__ void cta_tri_inverse(const double* R, int s, double* Ri) {
  for (int e = threadIdx.x; e < s * s; e += NT) Ri[e] = (e % s == e / s) ? 1.0 : 0.0;
  __syncthreads();
  // Ri <- I R^{-1}: rows of the identity times R^{-1}.
  cta_trsm_right(Ri, s, s, R, s);
}

// Y (kb*s x cols, ldy) <- T^{-T} Y for unit upper-triangular T (ldt) given by
// its strictly upper blocks: block forward substitution Y_i -= sum_{l<i} T_{l,i}^T Y_l.
// diag: T's diagonal blocks are unit upper triangular (the column muscle's T
// factors) rather than I_s, and their strict upper parts take part too.
__device__ void cta_unit_upper_T_solve(const double* T, int ldt, int kb, int s, double* Y, int ldy,
                                       int cols, bool diag = false) {
  for (int i = diag ? 0 : 1; i < kb; ++i) {
    // Y_i -= T(0:i s, i s:(i+1) s)^T Y(0:i s, :)
    for (int e = threadIdx.x; e < s * cols; e += NT) {
      const int a = e % s, c = e / s;
      double acc0 = 0.0, acc1 = 0.0;
      const double* tcol = T + (i * s + a) * ldt;
      int q = 0;
      for (; q + 1 < i * s; q += 2) {
        acc0 = fma(tcol[q], Y[q + c * ldy], acc0);
        acc1 = fma(tcol[q + 1], Y[q + 1 + c * ldy], acc1);
      }
      if (q < i * s) acc0 = fma(tcol[q], Y[q + c * ldy], acc0);
      Y[i * s + a + c * ldy] -= (acc0 + acc1);
    }
    __syncthreads();
    if (diag) {
      // Y_i <- T_ii^{-T} Y_i, forward substitution over the block's rows
      for (int a = 1; a < s; ++a) {
        for (int c = threadIdx.x; c < cols; c += NT) {
          double acc = 0.0;
          for (int b = 0; b < a; ++b) acc = fma(T[i * s + b + (i * s + a) * ldt], Y[i * s + b + c * ldy], acc);
          Y[i * s + a + c * ldy] -= acc;
        }
        __syncthreads();
      }
    }
  }
}

// Y <- T^T Y for unit upper-triangular T (the compact-WY branch of Alg. 6).
__device__ void cta_unit_upper_T_mult(const double* T, int ldt, int kb, int s, double* Y, int ldy,
                                      int cols, double* tmp, bool diag = false) {
  const int rows = kb * s;
  for (int e = threadIdx.x; e < rows * cols; e += NT) {
    const int r = e % rows, c = e / rows;
    const int qend = diag ? r : (r / s) * s;
    double acc = Y[r + c * ldy];
    const double* tcol = T + r * ldt;
    for (int q = 0; q < qend; ++q) acc = fma(tcol[q], Y[q + c * ldy], acc);
    tmp[r + c * rows] = acc;
  }
  __syncthreads();
  cta_copy(Y, ldy, tmp, rows, rows, cols);
}

// LU with partial pivoting: solve T x = B (s x s each, col-major ld s) into X.
// Returns 1 if a pivot is zero or the result is not finite.  One warp.
__device__ int warp_lu_solve(const double* Tin, const double* Bin, int s, double* X, double* sT,
                             int* spiv, int* sflag) {
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 32) {
    for (int e = lane; e < s * s; e += 32) {
      sT[e] = Tin[e];
      X[e] = Bin[e];
    }
    if (lane == 0) *sflag = 0;
    __syncwarp();
    for (int p = 0; p < s; ++p) {
      if (lane == 0) {
        int piv = p;
        double best = fabs(sT[p + p * s]);
        for (int i = p + 1; i < s; ++i) {
          const double v = fabs(sT[i + p * s]);
          if (v > best) {
            best = v;
            piv = i;
          }
        }
        *spiv = piv;
        if (!(best > 0.0)) *sflag = 1;
      }
      __syncwarp();
      const int piv = *spiv;
      if (piv != p && lane < s) {
        double t = sT[p + lane * s];
        sT[p + lane * s] = sT[piv + lane * s];
        sT[piv + lane * s] = t;
        t = X[p + lane * s];
        X[p + lane * s] = X[piv + lane * s];
        X[piv + lane * s] = t;
      }
      __syncwarp();
      if (*sflag) break;
      const double dinv = 1.0 / sT[p + p * s];
      // lane c updates column c of T (c > p) and of X.
      if (lane < s) {
        for (int i = p + 1; i < s; ++i) {
          const double l = sT[i + p * s] * dinv;
          if (lane > p) sT[i + lane * s] = fma(-l, sT[p + lane * s], sT[i + lane * s]);
          X[i + lane * s] = fma(-l, X[p + lane * s], X[i + lane * s]);
        }
      }
      __syncwarp();
    }
    if (!*sflag && lane < s) {
      for (int i = s - 1; i >= 0; --i) {
        double v = X[i + lane * s];
        for (int q = i + 1; q < s; ++q) v = fma(-sT[i + q * s], X[q + lane * s], v);
        v = v * (1.0 / sT[i + i * s]);
        if (!isfinite(v)) *sflag = 1;
        X[i + lane * s] = v;
      }
    }
    __syncwarp();
  }
  __syncthreads();
  return *sflag;
}

// Apply Q_i^T (transpose = 1) or Q_i (transpose = 0) of reflector set i to the
// 2s rows starting at row r0 of X (col-major, ldx, ncols columns).  One warp
// per column; a column's 2s <= 64 entries live two per lane.
__device__ void apply_set(const double* v, const double* tau, int s, double* X, int ldx, int r0,
                          int ncols, int transpose) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int h = 2 * s;
  for (int c = warp; c < ncols; c += NWARPS) {
    double* x = X + r0 + c * ldx;
    double x0 = lane < h ? x[lane] : 0.0;
    double x1 = lane + 32 < h ? x[lane + 32] : 0.0;
    for (int t = 0; t < s; ++t) {
      const int l = transpose ? t : s - 1 - t;
      const double tl = tau[l];
      if (tl == 0.0) continue;
      const double* vl = v + l * h;
      const double v0 = (lane >= l && lane < h) ? vl[lane] : 0.0;
      const double v1 = (lane + 32 >= l && lane + 32 < h) ? vl[lane + 32] : 0.0;
      const double d = warp_sum(fma(v0, x0, v1 * x1));
      x0 = fma(-tl * d, v0, x0);
      x1 = fma(-tl * d, v1, x1);
    }
    if (lane < h) x[lane] = x0;
    if (lane + 32 < h) x[lane + 32] = x1;
  }
  __syncthreads();
}

// Householder QR of the 2s x s block at rows r0.. of X (col-major, ldx):
// stores reflectors (unit leading entry, zeros above) in v (2s x s, ld 2s) and
// tau; the block is overwritten by [R; 0].
__device__ void house_qr(double* X, int ldx, int r0, int s, double* v, double* tau, double* sh) {
  const int h = 2 * s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int l = 0; l < s; ++l) {
    double* xl = X + r0 + l * ldx;
    if (warp == 0) {
      const double a0 = (lane >= l + 1 && lane < h) ? xl[lane] : 0.0;
      const double a1 = (lane + 32 >= l + 1 && lane + 32 < h) ? xl[lane + 32] : 0.0;
      const double xn2 = warp_sum(fma(a0, a0, a1 * a1));
      if (lane == 0) {
        // beta = -sign(alpha) ||x||, tau = (beta - alpha) / beta = 1 + |alpha| / ||x||,
        // v = x / (alpha - beta) below the leading 1: one rsqrt and one division.
        const double alpha = xl[l];
        double t = 0.0, beta = alpha, scale = 0.0;
        if (xn2 > 0.0) {
          const double n2 = fma(alpha, alpha, xn2);
          const double rn = rsqrt(n2);
          const double nrm = n2 * rn;
          beta = alpha >= 0.0 ? -nrm : nrm;
          t = fma(fabs(alpha), rn, 1.0);
          scale = 1.0 / (alpha - beta);
        }
        sh[0] = t;
        sh[1] = beta;
        sh[2] = scale;
        tau[l] = t;
      }
    }
    __syncthreads();
    const double t = sh[0], beta = sh[1], scale = sh[2];
    for (int r = threadIdx.x; r < h; r += NT) {
      double vr;
      if (r < l) vr = 0.0;
      else if (r == l) vr = 1.0;
      else vr = (t == 0.0) ? 0.0 : xl[r] * scale;
      v[r + l * h] = vr;
    }
    __syncthreads();
    if (threadIdx.x == 0) xl[l] = beta;
    for (int r = l + 1 + threadIdx.x; r < h; r += NT) xl[r] = 0.0;
    __syncthreads();
    // Apply H_l to the remaining columns l+1..s-1 (one warp per column).
    if (t != 0.0) {
      const double* vl = v + l * h;
      for (int c = l + 1 + warp; c < s; c += NWARPS) {
        double* x = X + r0 + c * ldx;
        const double v0 = (lane >= l && lane < h) ? vl[lane] : 0.0;
        const double v1 = (lane + 32 >= l && lane + 32 < h) ? vl[lane + 32] : 0.0;
        double x0 = lane < h ? x[lane] : 0.0;
        double x1 = lane + 32 < h ? x[lane + 32] : 0.0;
        const double d = warp_sum(fma(v0, x0, v1 * x1));
        x0 = fma(-t * d, v0, x0);
        x1 = fma(-t * d, v1, x1);
        if (lane < h) x[lane] = x0;
        if (lane + 32 < h) x[lane + 32] = x1;
      }
    }
    __syncthreads();
  }
}

// Compact WY form of reflector set i: H_0 H_1 ... H_{s-1} = I - V T V^T with T
// upper triangular (Schreiber and Van Loan's construction):
//   T(l,l) = tau_l,  T(0:l, l) = -tau_l T(0:l, 0:l) (V(:, 0:l)^T v_l).
// vtv: s x s scratch (global), T: s x s col-major.
__device__ void build_wy_T(const double* v, const double* tau, int s, double* T, double* vtv) {
  const int h = 2 * s;
  cta_gemm_s(s, s, h, 1.0, v, h, true, v, h, false, 0.0, vtv, s);
  for (int e = threadIdx.x; e < s * s; e += NT) T[e] = 0.0;
  __syncthreads();
  for (int l = 0; l < s; ++l) {
    const double tl = tau[l];
    for (int i = threadIdx.x; i < l; i += NT) {
      double acc = 0.0;
      for (int q = i; q < l; ++q) acc = fma(T[i + q * s], vtv[q + l * s], acc);
      T[i + l * s] = -tl * acc;
    }
    if (threadIdx.x == 0) T[l + l * s] = tl;
    __syncthreads();
  }
}

// X(r0:r0+2s, 0:ncols) <- Q^T X (transpose = 1) or Q X (transpose = 0) with
// Q = I - V T V^T: three small products, three barriers.  w1, w2: s x ncols scratch.
__device__ void apply_set_wy(const double* v, const double* T, int s, double* X, int ldx, int r0,
                             int ncols, int transpose, double* w1, double* w2) {
  const int h = 2 * s;
  cta_gemm_s(s, ncols, h, 1.0, v, h, true, X + r0, ldx, false, 0.0, w1, s);
  cta_gemm_s(s, ncols, s, 1.0, T, s, transpose != 0, w1, s, false, 0.0, w2, s);
  cta_gemm_s(h, ncols, s, -1.0, v, h, false, w2, s, false, 1.0, X + r0, ldx);
}

// ||X C||_F for s x s X (col-major, ldx) and C (col-major ld s).
__device__ double cta_norm_prod(const double* X, int ldx, const double* C, int s, double* red) {
  double part = 0.0;
  for (int e = threadIdx.x; e < s * s; e += NT) {
    const int i = e % s, j = e / s;
    double acc = 0.0;
    for (int q = 0; q < s; ++q) acc = fma(X[i + q * ldx], C[q + j * s], acc);
    part = fma(acc, acc, part);
  }
  part = warp_sum(part);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < NWARPS; ++w) t += red[w];
    red[NWARPS] = sqrt(t);
  }
  __syncthreads();
  const double r = red[NWARPS];
  __syncthreads();
  return r;
}

// Write coefficient block b of a [nin][s][s] row-major array from a col-major
// matrix M (s x s, ldm) times alpha; M == nullptr writes alpha * I.
__device__ void put_coef(double* coef, int b, int s, const double* M, int ldm, double alpha) {
  double* dst = coef + (size_t)b * s * s;
  for (int e = threadIdx.x; e < s * s; e += NT) {
    const int a = e / s, c = e % s;
    dst[a * s + c] = M ? alpha * M[a + c * ldm] : (a == c ? alpha : 0.0);
  }
}

__device__ void put_zero_coef(double* coef, int b, int s) {
  double* dst = coef + (size_t)b * s * s;
  for (int e = threadIdx.x; e < s * s; e += NT) dst[e] = 0.0;
}

// Row-major copy of an upper-triangular col-major s x s matrix (triangular solve operand).
__device__ void put_tri(double* tri, const double* R, int s) {
  for (int e = threadIdx.x; e < s * s; e += NT) {
    const int a = e / s, c = e % s;
    tri[a * s + c] = R[a + c * s];
  }
}

struct Shared {
  double R[LSBA_MAX_S * LSBA_MAX_S];
  double A[LSBA_MAX_S * LSBA_MAX_S];
  double B[LSBA_MAX_S * LSBA_MAX_S];
  double red[NWARPS + 4];
  int flag, flag2, piv;
};

__device__ void record_gram(const SmallWs& w, const double* G, int rows, int cols) {
  Ctl* ctl = w.ctl;
  if (!ctl->record || ctl->cycle != 1) return;
  const int used = ctl->gram_hist_used, idx = ctl->n_gram_hist;
  if (used + rows * cols > ctl->gram_hist_cap || idx >= 2 * (w.m + 2)) return;
  for (int e = threadIdx.x; e < rows * cols; e += NT) w.gram_hist[used + e] = G[e];
  __syncthreads();
  if (threadIdx.x == 0) {
    w.gram_dims[2 * idx] = rows;
    w.gram_dims[2 * idx + 1] = cols;
    ctl->gram_hist_used = used + rows * cols;
    ctl->n_gram_hist = idx + 1;
  }
  __syncthreads();
}

// Relation j of the current cycle is complete: H(1:j+1, j) is final.
// The dot product of cta_gemm_s's inner loop (four running sums over q, q+1,
// q+2, q+3, the rest into the first, combined (a0 + a1) + (a2 + a3)), on
// strided shared-memory operands.
__device__ __forceinline__ double dot4(const double* x, int sx, const double* y, int sy, int K) {
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int q = 0;
  for (; q + 3 < K; q += 4) {
    a0 = fma(x[q * sx], y[q * sy], a0);
    a1 = fma(x[(q + 1) * sx], y[(q + 1) * sy], a1);
    a2 = fma(x[(q + 2) * sx], y[(q + 2) * sy], a2);
    a3 = fma(x[(q + 3) * sx], y[(q + 3) * sy], a3);
  }
  for (; q < K; ++q) a0 = fma(x[q * sx], y[q * sy], a0);
  return (a0 + a1) + (a2 + a3);
}

// Q_1^T .. Q_{j-1}^T applied to col ((j+1)s x s, ld ldc, global), the
// reflector sets' V and T and col itself staged once in the shared-memory
// arena: the same products as apply_set_wy (transpose = 1) in the same order,
// without a global round trip per product.  Returns false (nothing done) if
// they do not fit the arena.
__device__ bool apply_sets_T_staged(const SmallWs& w, int j, double* col, int ldc) {
  const int s = w.s, h = 2 * s, ss = s * s, rows = (j + 1) * s;
  const size_t need = (size_t)(j - 1) * 3 * ss + (size_t)rows * s + 2 * (size_t)ss;
  if (j < 2 || need > SMALL_ARENA_DOUBLES) return false;
  double* Vs = small_arena;                          // [(j-1)][2s x s]
  double* Ts = Vs + (size_t)(j - 1) * 2 * ss;        // [(j-1)][s x s]
  double* cs = Ts + (size_t)(j - 1) * ss;            // rows x s, ld rows
  double* w1 = cs + (size_t)rows * s;                // s x s
  double* w2 = w1 + ss;                              // s x s
  for (int e = threadIdx.x; e < (j - 1) * 2 * ss; e += NT) Vs[e] = w.refl[e];
  for (int e = threadIdx.x; e < (j - 1) * ss; e += NT) Ts[e] = w.Twy[e];
  for (int e = threadIdx.x; e < rows * s; e += NT) cs[e] = col[(e % rows) + (size_t)(e / rows) * ldc];
  __syncthreads();
  for (int i = 1; i < j; ++i) {
    const double* V = Vs + (size_t)(i - 1) * 2 * ss;
    const double* T = Ts + (size_t)(i - 1) * ss;
    double* x = cs + (i - 1) * s;
    // w1 = V^T x  (s x s, K = 2s)
    for (int e = threadIdx.x; e < ss; e += NT) {
      const int l = e % s, c = e / s;
      w1[l + c * s] = dot4(V + l * h, 1, x + c * rows, 1, h);
    }
    __syncthreads();
    // w2 = T^T w1
    for (int e = threadIdx.x; e < ss; e += NT) {
      const int l = e % s, c = e / s;
      w2[l + c * s] = dot4(T + l * s, 1, w1 + c * s, 1, s);
    }
    __syncthreads();
    // x -= V w2  (2s x s)
    for (int e = threadIdx.x; e < h * s; e += NT) {
      const int r = e % h, c = e / h;
      const double v = dot4(V + r, h, w2 + c * s, 1, s);
      x[r + c * rows] = -1.0 * v + 1.0 * x[r + c * rows];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < rows * s; e += NT) col[(e % rows) + (size_t)(e / rows) * ldc] = cs[e];
  __syncthreads();
  return true;
}

__device__ void relation_complete(const SmallWs& w, int j, Shared& sh) {
  const int s = w.s, ldH = w.ldH, ldg = w.ldH, ldR = w.ldR;
  Ctl* ctl = w.ctl;
  double* col = w.work;                   // (j+1)s x s, ld = ldH
  const double* Hj = w.H + (size_t)(j - 1) * s * ldH;
  cta_copy(col, ldH, Hj, ldH, (j + 1) * s, s);
  double* w1 = w.work + (size_t)2 * w.ldH * s;   // s x s scratch (clear of col and of J's)
  double* w2 = w1 + (size_t)s * s;
  if (!apply_sets_T_staged(w, j, col, ldH))
    for (int i = 1; i < j; ++i)
      apply_set_wy(w.refl + (size_t)(i - 1) * 2 * s * s, w.Twy + (size_t)(i - 1) * s * s, s, col,
                   ldH, (i - 1) * s, s, 1, w1, w2);
  // BFOM pieces (before reflector set j).
  cta_copy(w.Tfom, s, col + (j - 1) * s, ldH, s, s);
  cta_copy(w.ufom, ldH, col, ldH, (j - 1) * s, s);
  cta_copy(w.gfom, s, w.g + (j - 1) * s, ldg, s, s);
  int sing = 0;
  if (w.modification == 0) sing = warp_lu_solve(w.Tfom, w.gfom, s, w.cfom, sh.A, &sh.piv, &sh.flag2);
  // Reflector set j and the R factor's block column j.
  house_qr(col, ldH, (j - 1) * s, s, w.refl + (size_t)(j - 1) * 2 * s * s, w.tau + (j - 1) * s, sh.red);
  build_wy_T(w.refl + (size_t)(j - 1) * 2 * s * s, w.tau + (j - 1) * s, s,
             w.Twy + (size_t)(j - 1) * s * s, w1);
  cta_copy(w.Rbar + (size_t)(j - 1) * s * ldR, ldR, col, ldH, j * s, s);
  apply_set_wy(w.refl + (size_t)(j - 1) * 2 * s * s, w.Twy + (size_t)(j - 1) * s * s, s, w.g, ldg,
               (j - 1) * s, s, 1, w1, w2);
  double est;
  if (w.modification == 1) {
    est = cta_norm_prod(w.g + j * s, ldg, w.Cfac, s, sh.red) / ctl->normB;
  } else if (!sing) {
    // ||H_{j+1,j} c C||_F
    cta_gemm_s(s, s, s, 1.0, w.H + j * s + (size_t)(j - 1) * s * ldH, ldH, false, w.cfom, s, false, 0.0,
             sh.B, s);
    est = cta_norm_prod(sh.B, s, w.Cfac, s, sh.red) / ctl->normB;
  } else {
    est = nan("");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl->j = j;
    ctl->fom_singular = sing;
    ctl->est = est;
    if (ctl->record && ctl->n_hist < ctl->hist_cap) {
      w.hist_est[ctl->n_hist] = est;
      w.hist_cycle[ctl->n_hist] = ctl->cycle;
      w.hist_j[ctl->n_hist] = j;
      ctl->n_hist += 1;
    }
    if (!sing && est <= ctl->tol) {
      ctl->converged = 1;
      ctl->active = 0;
    }
    if (j >= ctl->m_cur) ctl->active = 0;
  }
  __syncthreads();
}

__device__ void flag_exit(const SmallWs& w, int relation) {
  __syncthreads();
  if (threadIdx.x == 0) {
    w.ctl->flagged = relation;
    w.ctl->active = 0;
    w.ctl->update_step = -1;
  }
  __syncthreads();
}

__device__ __forceinline__ bool injected(const SmallWs& w, int relation) {
  return w.ctl->inject_relation == relation;
}

// ---------------------------------------------------------------- cycle start
// flags: bit 0 = first cycle (compute ||B||_F from the Gram), bit 1 = reset C = I.
// Global block inner product (Table 1): the Gram passes compute the classical
// products of the blocks; each s x s block of the reduced result (a x b blocks,
// row-major) becomes tr(block)/s I_s before anything reads it.  Every later
// small-matrix operation then stays in the span of I_s (chol(t I) = sqrt(t) I,
// products and solves of such blocks), which is the global method.
__device__ void project_global(const SmallWs& w, int a, int b) {
  double* G = const_cast<double*>(w.G);
  const int s = w.s, cols = b * s;
  for (int blk = threadIdx.x; blk < a * b; blk += NT) {
    double* g = G + (size_t)(blk / b) * s * cols + (size_t)(blk % b) * s;
    double t = 0.0;
    for (int i = 0; i < s; ++i) t += g[(size_t)i * cols + i];
    t /= s;
    for (int i = 0; i < s; ++i)
      for (int c = 0; c < s; ++c) g[(size_t)i * cols + c] = i == c ? t : 0.0;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(NT) k_small_start(SmallWs w, int flags) {
  const int first_cycle = flags & 1;
  __shared__ Shared sh;
  const int s = w.s;
  Ctl* ctl = w.ctl;
  if (flags & 4) {
    // Test hook: a bounded wait on an mbarrier that nothing arrives at (no
    // copies or MMAs in flight).  It gives up, the error is recorded, and the
    // cycle ends as after a flagged start (every later kernel skips its work).
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
      if (!mbar_wait_bounded(&bar, 0)) atomicExch(&ctl->error, 1);
      ctl->start_flag = 1;
      ctl->active = 0;
      ctl->j = 0;
      ctl->flagged = 0;
      ctl->converged = 0;
      ctl->update_step = -1;
    }
    return;
  }
  // G = R_start^T R_start (s x s row-major == col-major since symmetric in exact
  // arithmetic; the upper triangle read as G[a*s + c], a <= c).
  int flag;
  if (w.col_muscle) {
    // The column muscle has made V_1 from R_start in place: Beta = R, and its
    // T factor is T's first diagonal block; ||R_start||_F = ||R||_F.
    const double* mR = w.mus;
    const double* mT = w.mus + s * s;
    flag = w.mus[2 * s * s + s] != 0.0 ? 1 : 0;
    for (int e = threadIdx.x; e < s * s; e += NT) {
      const int a = e % s, c = e / s;
      sh.R[e] = flag ? 0.0 : mR[e];
      w.T[a + c * w.ldT] = a < c && !flag ? mT[e] : 0.0;
    }
    __syncthreads();
    if (first_cycle && threadIdx.x == 0) {
      double t = 0.0;
      for (int e = 0; e < s * s; ++e) t += mR[e] * mR[e];
      ctl->normB = sqrt(t);
    }
  } else {
    if (w.global_ip) project_global(w, 1, 1);
    flag = cta_chol(w.G, s, s, sh.R, &sh.flag);
    if (first_cycle) {
      if (threadIdx.x == 0) {
        double tr = 0.0;
        for (int a = 0; a < s; ++a) tr += w.G[a * s + a];
        ctl->normB = sqrt(tr);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl->start_flag = flag;
    ctl->active = flag ? 0 : 1;
    ctl->j = 0;
    ctl->k = 0;
    ctl->flagged = 0;
    ctl->converged = 0;
    ctl->fom_singular = 0;
    ctl->update_step = flag ? -1 : 0;
  }
  if (flag) return;
  cta_copy(w.Bcyc, s, sh.R, s, s, s);
  // g = E_1 Beta
  for (int e = threadIdx.x; e < w.ldH * s; e += NT) {
    const int r = e % w.ldH, c = e / w.ldH;
    w.g[e] = r < s ? sh.R[r + c * s] : 0.0;
  }
  if (flags & 2) {
    for (int e = threadIdx.x; e < s * s; e += NT) w.Cfac[e] = (e % s == e / s) ? 1.0 : 0.0;
  }
  put_coef(w.coef1, 0, s, nullptr, 0, 1.0);
  put_tri(w.tri1, sh.R, s);
}

// ---------------------------------------------------------------- one step
// The end of a PIP / PIO step once R = H_{k+1,k} is in sh.R: store H_{1:k+1,k}
// and the coefficients of V_{k+1} = (W - V_k Hc) R^{-1} (inputs [V_1..V_k, W]).
__device__ void pip_finish(const SmallWs& w, int k, Shared& sh);

__device__ void step_pip(const SmallWs& w, int k, Shared& sh) {
  const int s = w.s, ks = k * s;
  const double* G = w.G;  // ((k+1)s x s) row-major: element (i, c) at G[i*s + c]
  record_gram(w, G, (k + 1) * s, s);
  // S = Omega - Hc^T Hc ; Hc(i,c) = G[i*s+c] is, as a col-major matrix, Hc^T with ld s.
  cta_gemm_s(s, s, ks, -1.0, G, s, false, G, s, true, 0.0, sh.A, s);
  for (int e = threadIdx.x; e < s * s; e += NT) {
    const int a = e % s, c = e / s;
    sh.A[a + c * s] += G[(ks + a) * s + c];
  }
  __syncthreads();
  int flag = cta_chol(sh.A, s, s, sh.R, &sh.flag);
  if (flag || injected(w, k)) {
    flag_exit(w, k);
    return;
  }
  pip_finish(w, k, sh);
}

// BCGS-PIO (Alg. 4) with the CholQR muscle: the muscle's factor of
// [W 0; 0 Hc] is diag(R_W, R_H), R_W = chol(W^T W) (the Omega block of the
// fused Gram), R_H = chol(Hc^T Hc); then H_{k+1,k} = chol(R_W^T R_W - R_H^T R_H).
__device__ void step_pio(const SmallWs& w, int k, Shared& sh) {
  const int s = w.s, ks = k * s;
  const double* G = w.G;
  record_gram(w, G, ks, s);   // the inner product <V_k, W>; <W, W> is the muscle's
  cta_gemm_s(s, s, ks, 1.0, G, s, false, G, s, true, 0.0, sh.A, s);
  __syncthreads();
  const int flag_h = cta_chol(sh.A, s, s, sh.R, &sh.flag);
  for (int e = threadIdx.x; e < s * s; e += NT) {
    const int a = e % s, c = e / s;
    sh.B[e] = sh.R[e];
    sh.A[a + c * s] = G[(ks + a) * s + c];
  }
  __syncthreads();
  const int flag_w = cta_chol(sh.A, s, s, sh.R, &sh.flag);
  if (flag_w || flag_h || injected(w, k)) {
    flag_exit(w, k);
    return;
  }
  cta_gemm_s(s, s, s, 1.0, sh.R, s, true, sh.R, s, false, 0.0, sh.A, s);
  __syncthreads();
  cta_gemm_s(s, s, s, -1.0, sh.B, s, true, sh.B, s, false, 1.0, sh.A, s);
  __syncthreads();
  const int flag = cta_chol(sh.A, s, s, sh.R, &sh.flag);
  if (flag) {
    flag_exit(w, k);
    return;
  }
  pip_finish(w, k, sh);
}

__device__ void pip_finish(const SmallWs& w, int k, Shared& sh) {
  const int s = w.s, ks = k * s, ldH = w.ldH;
  const double* G = w.G;
  double* Hk = w.H + (size_t)(k - 1) * s * ldH;
  for (int e = threadIdx.x; e < ks * s; e += NT) {
    const int i = e % ks, c = e / ks;
    Hk[i + c * ldH] = G[i * s + c];
  }
  for (int e = threadIdx.x; e < s * s; e += NT) {
    const int a = e % s, c = e / s;
    Hk[ks + a + c * ldH] = sh.R[a + c * s];
  }
  // V_{k+1} = (W - V_k Hc) R^{-1}: inputs [V_1..V_k, W].
  for (int e = threadIdx.x; e < ks * s; e += NT) w.coef1[e] = -G[e];
  put_coef(w.coef1, k, s, nullptr, 0, 1.0);
  put_tri(w.tri1, sh.R, s);
  __syncthreads();
  if (threadIdx.x == 0) {
    w.ctl->update_step = k;
    w.ctl->side_step = k;
    w.ctl->side_rel = k;
    w.ctl->side_J = 0;
  }
}

__device__ void step_bcgs(const SmallWs& w, int k, int phase, Shared& sh) {
  const int s = w.s, ks = k * s, ldH = w.ldH;
  const double* G = w.G;
  double* Hk = w.H + (size_t)(k - 1) * s * ldH;
  if (phase == 0) {
    // Hc = V_k^T W (ks x s row-major); W' = W - V_k Hc in place.
    record_gram(w, G, ks, s);
    for (int e = threadIdx.x; e < ks * s; e += NT) {
      const int i = e % ks, c = e / ks;
      Hk[i + c * ldH] = G[i * s + c];
    }
    for (int e = threadIdx.x; e < ks * s; e += NT) w.coef1[e] = -G[e];
    put_coef(w.coef1, k, s, nullptr, 0, 1.0);
    __syncthreads();
    if (threadIdx.x == 0) w.ctl->update_step = k;
    return;
  }
  // phase 1: G = W'^T W' ; [V_{k+1}, H_{k+1,k}] = CholQR(W').
  int flag = cta_chol(G, s, s, sh.R, &sh.flag);
  if (flag || injected(w, k)) {
    flag_exit(w, k);
    return;
  }
  for (int e = threadIdx.x; e < s * s; e += NT) {
    const int a = e % s, c = e / s;
    Hk[ks + a + c * ldH] = sh.R[a + c * s];
  }
  put_coef(w.coef1, 0, s, nullptr, 0, 1.0);
  put_tri(w.tri1, sh.R, s);
  __syncthreads();
  if (threadIdx.x == 0) {
    w.ctl->update_step = k;
    w.ctl->side_step = k;
    w.ctl->side_rel = k;
    w.ctl->side_J = 0;
  }
}

// BMGS-Arnoldi (Alg. 2), iteration k.  Phase p < k: the Gram is V_{p+1}^T W;
// H_{p+1,k} = G and W <- W - V_{p+1} H_{p+1,k} in place (inputs [V_{p+1}, W]).
// Phase k: [V_{k+1}, H_{k+1,k}] = CholQR(W), as in BCGS.
__device__ void step_bmgs(const SmallWs& w, int k, int phase, Shared& sh) {
  if (phase >= k) {
    step_bcgs(w, k, 1, sh);
    return;
  }
  const int s = w.s, ldH = w.ldH;
  const double* G = w.G;
  double* Hk = w.H + (size_t)(k - 1) * s * ldH + (size_t)phase * s;
  if (phase == 0) record_gram(w, G, s, s);
  for (int e = threadIdx.x; e < s * s; e += NT) {
    const int i = e % s, c = e / s;
    Hk[i + c * ldH] = G[i * s + c];
  }
  for (int e = threadIdx.x; e < s * s; e += NT) w.coef1[e] = -G[e];
  put_coef(w.coef1, 1, s, nullptr, 0, 1.0);
  __syncthreads();
  if (threadIdx.x == 0) w.ctl->update_step = k;
}

// BMGS-SVL / BMGS-LTS-Arnoldi (Alg. 5), iteration k; T is unit block upper
// triangular (the muscle's T_{k+1,k+1} is I_s), its strict upper part in w.T.
// Phase 0: Y = <V_k, W> (ks x s); H_{1:k,k} = T^T Y (SVL) or T^{-T} Y (LTS);
//   W <- W - V_k H_{1:k,k} in place.
// Phase 1: [V_{k+1}, H_{k+1,k}] = CholQR(W), as in BCGS.
// Phase 2: Z = <V_k, V_{k+1}>; T_{1:k,k+1} = -T Z (SVL) or Z (LTS); the
//   relation is then complete for the side kernel.
__device__ void step_svl(const SmallWs& w, int k, int phase, bool lts, Shared& sh) {
  const int s = w.s, ks = k * s, ldH = w.ldH, ldT = w.ldT;
  const double* G = w.G;
  if (phase == 1 && !w.col_muscle) {
    step_bcgs(w, k, 1, sh);   // its side fields are reset by phase 2's entry
    return;
  }
  if (phase == 1) {
    // The column muscle has made W = V_{k+1} H_{k+1,k} in place (R and its
    // T factor in w.mus): H_{k+1,k} = R, T_{k+1,k+1} = T_m, then V_{k+1} = W.
    const double* mR = w.mus;
    const double* mT = w.mus + s * s;
    if (w.mus[2 * s * s + s] != 0.0 || injected(w, k)) {
      flag_exit(w, k);
      return;
    }
    double* Hk = w.H + (size_t)(k - 1) * s * ldH;
    double* Tkk = w.T + (size_t)ks * ldT + ks;
    for (int e = threadIdx.x; e < s * s; e += NT) {
      const int a = e % s, c = e / s;
      Hk[ks + a + c * ldH] = mR[a + c * s];
      Tkk[a + c * ldT] = a < c ? mT[a + c * s] : 0.0;   // strict upper part; the unit diagonal is implied
    }
    put_coef(w.coef1, 0, s, nullptr, 0, 1.0);
    __syncthreads();
    if (threadIdx.x == 0) w.ctl->update_step = k;
    return;
  }
  if (phase == 0) {
    record_gram(w, G, ks, s);
    double* ZP = w.work;             // ks x s, ld ks
    for (int e = threadIdx.x; e < ks * s; e += NT) {
      const int i = e % ks, c = e / ks;
      ZP[i + c * ks] = G[i * s + c];
    }
    __syncthreads();
    if (lts) cta_unit_upper_T_solve(w.T, ldT, k, s, ZP, ks, s, w.col_muscle != 0);
    else cta_unit_upper_T_mult(w.T, ldT, k, s, ZP, ks, s, w.work + ks * s, w.col_muscle != 0);
    double* Hk = w.H + (size_t)(k - 1) * s * ldH;
    for (int e = threadIdx.x; e < ks * s; e += NT) {
      const int i = e % ks, c = e / ks;
      Hk[i + c * ldH] = ZP[i + c * ks];
    }
    for (int b = 0; b < k; ++b) put_coef(w.coef1, b, s, ZP + b * s, ks, -1.0);
    put_coef(w.coef1, k, s, nullptr, 0, 1.0);
    __syncthreads();
    if (threadIdx.x == 0) w.ctl->update_step = k;
    return;
  }
  // T_{1:k,k+1} = -T_{1:k,1:k} Z T_{k+1,k+1} (SVL) or Z T_{k+1,k+1} (LTS); the
  // diagonal blocks of T are I_s except with the column muscle.
  double* Tk = w.T + (size_t)ks * ldT;            // block column k + 1, rows 1..k
  const double* Tm = Tk + ks;                      // T_{k+1,k+1}, strict upper part
  double* tmp = w.work;                            // ks x s, ld ks
  for (int e = threadIdx.x; e < ks * s; e += NT) {
    const int r = e % ks, c = e / ks;
    double acc = G[r * s + c];
    if (!lts) {
      for (int q = w.col_muscle ? r + 1 : (r / s + 1) * s; q < ks; ++q)
        acc = fma(w.T[r + q * ldT], G[q * s + c], acc);
      acc = -acc;
    }
    tmp[r + c * ks] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ks * s; e += NT) {
    const int i = e % ks, c = e / ks;
    double v = tmp[i + c * ks];
    if (w.col_muscle)
      for (int q = 0; q < c; ++q) v = fma(tmp[i + q * ks], Tm[q + c * ldT], v);
    Tk[i + c * ldT] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    w.ctl->side_step = k;
    w.ctl->side_rel = k;
    w.ctl->side_J = 0;
  }
}

// Lagged skeletons, iteration k = 1: H_{1,1} = <U, W> (= J), U <- W - V_1 H_{1,1}.
// Inputs [V_1, W]; out1 = U.
__device__ void step_lagged_first(const SmallWs& w, Shared& sh) {
  const int s = w.s, ldH = w.ldH;
  const double* G = w.G;
  record_gram(w, G, s, s);
  for (int e = threadIdx.x; e < s * s; e += NT) {
    const int a = e % s, c = e / s;
    w.H[a + c * ldH] = G[a * s + c];
    if (w.skel == SK_LS) w.J[a + c * ldH] = G[a * s + c];
  }
  for (int e = threadIdx.x; e < s * s; e += NT) w.coef1[e] = -G[e];
  put_coef(w.coef1, 1, s, nullptr, 0, 1.0);
  __syncthreads();
  if (threadIdx.x == 0) w.ctl->update_step = 1;
  __syncthreads();
}

// BMGS-CWY / BMGS-ICWY iteration k >= 2 (Alg. 6).  Inputs [V_1..V_{k-1}, U, W];
// out1 = V_k, out2 = U.
__device__ void step_cwy(const SmallWs& w, int k, bool inverse, Shared& sh) {
  const int s = w.s, ldH = w.ldH, ldT = w.ldT;
  const int k1s = (k - 1) * s, ks = k * s, cols = 2 * s;
  const double* G = w.G;  // (ks x 2s) row-major
  record_gram(w, G, ks, cols);
  // Omega = G[(k-1)s:, 0:s] (upper triangle read)
  for (int e = threadIdx.x; e < s * s; e += NT) {
    const int a = e % s, c = e / s;
    sh.A[a + c * s] = G[(k1s + a) * cols + c];
  }
  __syncthreads();
  int flag = cta_chol(sh.A, s, s, sh.R, &sh.flag);
  if (flag || injected(w, k - 1)) {
    flag_exit(w, k - 1);
    return;
  }
  double* ZP = w.work;                 // ks x s, ld ks
  double* YR = w.work + ks * s;        // (k-1)s x s
  double* tmp = w.work + 2 * ks * s;   // ks x s
  // P = R^{-T} Ptilde
  for (int e = threadIdx.x; e < s * s; e += NT) {
    const int a = e % s, c = e / s;
    ZP[k1s + a + c * ks] = G[(k1s + a) * cols + s + c];
  }
  for (int e = threadIdx.x; e < k1s * s; e += NT) {
    const int i = e % k1s, c = e / k1s;
    ZP[i + c * ks] = G[i * cols + s + c];
    YR[i + c * k1s] = G[i * cols + c];
  }
  __syncthreads();
  cta_trsm_left_T(sh.R, s, ZP + k1s, ks, s);
  // [Z; P] R^{-1} and Y R^{-1}
  cta_trsm_right(ZP, ks, ks, sh.R, s);
  cta_trsm_right(YR, k1s, k1s, sh.R, s);
  // T_{1:k-1,k}
  double* Tk = w.T + (size_t)k1s * ldT;  // column block k (0-based k-1)
  if (inverse) {
    cta_copy(Tk, ldT, YR, k1s, k1s, s);
  } else {
    // -T_{1:k-1,1:k-1} (Y R^{-1}); T unit upper.
    for (int e = threadIdx.x; e < k1s * s; e += NT) {
      const int r = e % k1s, c = e / k1s;
      double acc = YR[r + c * k1s];
      for (int q = (r / s + 1) * s; q < k1s; ++q) acc = fma(w.T[r + q * ldT], YR[q + c * k1s], acc);
      tmp[r + c * k1s] = -acc;
    }
    __syncthreads();
    cta_copy(Tk, ldT, tmp, k1s, k1s, s);
  }
  // H_{1:k,k} = T^{-T} ZP (ICWY) or T^T ZP (CWY)
  if (inverse) cta_unit_upper_T_solve(w.T, ldT, k, s, ZP, ks, s);
  else cta_unit_upper_T_mult(w.T, ldT, k, s, ZP, ks, s, tmp);
  double* Hk = w.H + (size_t)(k - 1) * s * ldH;
  double* Hkm1 = w.H + (size_t)(k - 2) * s * ldH;
  for (int e = threadIdx.x; e < ks * s; e += NT) {
    const int i = e % ks, c = e / ks;
    Hk[i + c * ldH] = ZP[i + c * ks];
  }
  for (int e = threadIdx.x; e < s * s; e += NT) {
    const int a = e % s, c = e / s;
    Hkm1[k1s + a + c * ldH] = sh.R[a + c * s];
  }
  // Coefficients: out1 = V_k = U R^{-1};
  // out2 = W R^{-1} - V_{1:k-1} Hc_{1:k-1} - V_k Hc_k.
  cta_tri_inverse(sh.R, s, sh.B);
  // (coefficient block b, row a, column c: all blocks in one pass)
  for (int e = threadIdx.x; e < (k - 1) * s * s; e += NT) {
    const int b = e / (s * s), a = (e / s) % s, c = e % s;
    w.coef1[e] = 0.0;
    w.coef2[e] = -ZP[b * s + a + c * ks];
  }
  put_coef(w.coef1, k - 1, s, nullptr, 0, 1.0);
  put_zero_coef(w.coef2, k - 1, s);
  put_zero_coef(w.coef1, k, s);
  put_coef(w.coef2, k, s, sh.B, s, 1.0);
  put_coef(w.chain, 0, s, ZP + k1s, ks, -1.0);
  put_tri(w.tri1, sh.R, s);
  __syncthreads();
  if (threadIdx.x == 0) {
    w.ctl->update_step = k;
    w.ctl->side_step = k;
    w.ctl->side_rel = k - 1;
    w.ctl->side_J = 0;
  }
}

// BCGSI+LS iteration k >= 2 (Alg. 7).  Inputs [V_1..V_{k-1}, U, W]; out1 = V_k, out2 = U.
// BCGSI+LS, s <= 16: the step's two s x s products Y^T Y and Y^T Z (Alg. 7
// lines 11 and 13; Y, Z the first (k-1)s rows of the reduced Gram [Y Z; Omega~
// P~]) split by row ranges over LSBA_LS_PROD_CTAS CTAs, one output a thread:
// on one SM the FP64 pipe (~1.7 FMA a clock) would take ~2 s^2 (k-1) s / 1.7
// cycles.  The small step adds the CTAs' partial sums in CTA order.
__global__ void __launch_bounds__(512) k_ls_products(SmallWs w, int k) {
  if (!*(volatile const int*)&w.ctl->active) return;
  const int s = w.s, ss = s * s, cols = 2 * s, K = (k - 1) * s;
  const int t = threadIdx.x;
  if (t >= 2 * ss) return;
  const int o = t % ss, which = t / ss, i = o % s, j = o / s;
  const int q0 = (int)((int64_t)blockIdx.x * K / LSBA_LS_PROD_CTAS);
  const int q1 = (int)((int64_t)(blockIdx.x + 1) * K / LSBA_LS_PROD_CTAS);
  const double* G = w.G;
  double a0 = 0.0, a1 = 0.0;
  int q = q0;
  for (; q + 1 < q1; q += 2) {
    a0 = fma(G[q * cols + i], G[q * cols + which * s + j], a0);
    a1 = fma(G[(q + 1) * cols + i], G[(q + 1) * cols + which * s + j], a1);
  }
  if (q < q1) a0 = fma(G[q * cols + i], G[q * cols + which * s + j], a0);
  w.prod[(size_t)blockIdx.x * 2 * ss + t] = a0 + a1;
}

__device__ void step_ls(const SmallWs& w, int k, Shared& sh) {
  const int s = w.s, ldH = w.ldH;
  const int k1s = (k - 1) * s, ks = k * s, cols = 2 * s;
  const double* G = w.G;
  record_gram(w, G, ks, cols);
  // Omega = Omega~ - Y^T Y.  Y(i,c) = G[i*cols + c] is Y^T col-major with ld cols.
  // sh.B = Y^T Z for P below.  For s <= 16 (classical inner product) both come
  // as k_ls_products' partial sums (output i + j s); under the global product
  // the Gram is projected in this kernel first, so they are formed here.
  if (s <= 16 && !w.global_ip) {
    for (int e = threadIdx.x; e < s * s; e += NT) {
      double v1 = 0.0, v2 = 0.0;
      for (int p = 0; p < LSBA_LS_PROD_CTAS; ++p) {
        v1 += w.prod[(size_t)p * 2 * s * s + e];
        v2 += w.prod[(size_t)p * 2 * s * s + s * s + e];
      }
      sh.A[e] = -v1;
      sh.B[e] = v2;
    }
    __syncthreads();
  } else {
    cta_gemm_s(s, s, k1s, -1.0, G, cols, false, G, cols, true, 0.0, sh.A, s);
    cta_gemm_s(s, s, k1s, 1.0, G, cols, false, G + s, cols, true, 0.0, sh.B, s);
  }
  for (int e = threadIdx.x; e < s * s; e += NT) {
    const int a = e % s, c = e / s;
    sh.A[a + c * s] += G[(k1s + a) * cols + c];
  }
  __syncthreads();
  int flag = cta_chol(sh.A, s, s, sh.R, &sh.flag);
  if (flag || injected(w, k - 1)) {
    flag_exit(w, k - 1);
    return;
  }
  double* Hkm1 = w.H + (size_t)(k - 2) * s * ldH;
  // H_{k,k-1} = R ; H_{1:k-1,k-1} = J + Y
  for (int e = threadIdx.x; e < s * s; e += NT) {
    const int a = e % s, c = e / s;
    Hkm1[k1s + a + c * ldH] = sh.R[a + c * s];
  }
  for (int e = threadIdx.x; e < k1s * s; e += NT) {
    const int i = e % k1s, c = e / k1s;
    Hkm1[i + c * ldH] = w.J[i + c * ldH] + G[i * cols + c];
  }
  // P = R^{-T} (P~ - Y^T Z), sh.B = Y^T Z (above)
  double* ZP = w.work;                // ks x s, ld ks
  for (int e = threadIdx.x; e < s * s; e += NT) {
    const int a = e % s, c = e / s;
    ZP[k1s + a + c * ks] = G[(k1s + a) * cols + s + c] - sh.B[a + c * s];
  }
  for (int e = threadIdx.x; e < k1s * s; e += NT) {
    const int i = e % k1s, c = e / k1s;
    ZP[i + c * ks] = G[i * cols + s + c];
  }
  __syncthreads();
  cta_trsm_left_T(sh.R, s, ZP + k1s, ks, s);
  // J = ([Z; P] - H_{1:k,1:k-1} Y) R^{-1} is needed only by the next iteration:
  // keep [Z; P], Y and R for the side kernel, which computes it off the
  // critical path.
  for (int e = threadIdx.x; e < ks * s; e += NT) w.saveZP[e] = ZP[e];
  for (int e = threadIdx.x; e < k1s * s; e += NT) {
    const int i = e % k1s, c = e / k1s;
    w.saveY[i + c * k1s] = G[i * cols + c];
  }
  for (int e = threadIdx.x; e < s * s; e += NT) w.saveR[e] = sh.R[e];
  // out1 = V_k = (U - V_{1:k-1} Y) R^{-1};  out2 = (W - V_{1:k-1} Z - V_k P) R^{-1}
  // (coefficient block b, row a, column c: all blocks in one pass)
  for (int e = threadIdx.x; e < (k - 1) * s * s; e += NT) {
    const int b = e / (s * s), a = (e / s) % s, c = e % s;
    w.coef1[e] = -G[(b * s + a) * cols + c];
    w.coef2[e] = -G[(b * s + a) * cols + s + c];
  }
  put_coef(w.coef1, k - 1, s, nullptr, 0, 1.0);
  put_zero_coef(w.coef2, k - 1, s);
  put_zero_coef(w.coef1, k, s);
  put_coef(w.coef2, k, s, nullptr, 0, 1.0);
  put_coef(w.chain, 0, s, ZP + k1s, ks, -1.0);
  put_tri(w.tri1, sh.R, s);
  put_tri(w.tri2, sh.R, s);
  __syncthreads();
  if (threadIdx.x == 0) {
    w.ctl->update_step = k;
    w.ctl->side_step = k;
    w.ctl->side_rel = k - 1;
    w.ctl->side_J = 1;
  }
}

__global__ void __launch_bounds__(NT) k_small_step(SmallWs w, int k, int phase) {
  __shared__ Shared sh;
  if (!*(volatile int*)&w.ctl->active) return;
  if (threadIdx.x == 0) {
    w.ctl->update_step = -1;
    w.ctl->side_step = -1;
    w.ctl->k = k;
  }
  __syncthreads();
  if (w.global_ip) {
    // block shape of this step's Gram
    int a = 1, b = 1;
    if (w.skel == SK_PIP || w.skel == SK_PIO) a = k + 1;
    else if (w.skel == SK_BCGS && phase == 0) a = k;
    else if ((w.skel == SK_SVL || w.skel == SK_LTS) && phase != 1) a = k;
    else if ((w.skel == SK_LS || w.skel == SK_ICWY || w.skel == SK_CWY) && k >= 2) a = k, b = 2;
    project_global(w, a, b);
  }
  switch (w.skel) {
    case SK_PIP: step_pip(w, k, sh); break;
    case SK_BCGS: step_bcgs(w, k, phase, sh); break;
    case SK_BMGS: step_bmgs(w, k, phase, sh); break;
    case SK_PIO: step_pio(w, k, sh); break;
    case SK_SVL: step_svl(w, k, phase, false, sh); break;
    case SK_LTS: step_svl(w, k, phase, true, sh); break;
    case SK_ICWY:
    case SK_CWY:
      if (k == 1) step_lagged_first(w, sh);
      else step_cwy(w, k, w.skel == SK_ICWY, sh);
      break;
    case SK_LS:
      if (k == 1) step_lagged_first(w, sh);
      else step_ls(w, k, sh);
      break;
  }
}

// ---------------------------------------------------------------- side kernel
// Work of loop iteration k that the next iteration's bandwidth kernels do not
// wait for, run on a second stream while they execute:
//   * BCGSI+LS: J = ([Z; P] - H_{1:k,1:k-1} Y) R^{-1} (Alg. 7 line 15), read only by
//     iteration k+1's small kernel.  H_{1:k,1:k-1} is block upper Hessenberg, so
//     row block i only meets column blocks >= i-1.
//   * the relation that iteration k completed: incremental least squares,
//     residual estimate (Eq. (9)), convergence and the basis-size limit.
__global__ void __launch_bounds__(NT) k_small_side(SmallWs w, int k) {
  __shared__ Shared sh;
  Ctl* ctl = w.ctl;
  if (*(volatile int*)&ctl->side_step != k) return;
  relation_complete(w, ctl->side_rel, sh);
}

// BCGSI+LS: J = ([Z; P] - H_{1:k,1:k-1} Y) R^{-1} (Alg. 7 line 15), needed only by
// the next iteration's small kernel.  Spread over many CTAs (the FP64 pipes of
// several SMs): one lane group of S2 lanes per row of J; H_{1:k,1:k-1} is block
// upper Hessenberg, so row block i only meets column blocks >= i-1; the row is
// then multiplied by R^{-1} by forward substitution across the lane group.
__global__ void __launch_bounds__(64) k_side_J(SmallWs w, int k, int S2) {
  Ctl* ctl = w.ctl;
  if (*(volatile int*)&ctl->side_step != k || !ctl->side_J) return;
  extern __shared__ double jsm[];
  const int s = w.s, ldH = w.ldH, ks = k * s, k1s = (k - 1) * s;
  const int rows = blockDim.x / S2;                 // rows of J in this CTA
  const int r0 = blockIdx.x * rows;
  double* Ys = jsm;                                 // k1s x s
  double* Hs = jsm + (size_t)k1s * s;               // rows x k1s
  for (int e = threadIdx.x; e < k1s * s; e += blockDim.x) Ys[e] = w.saveY[e];
  for (int e = threadIdx.x; e < rows * k1s; e += blockDim.x) {
    const int rr = e % rows, q = e / rows;
    Hs[rr + q * rows] = (r0 + rr < ks) ? w.H[(r0 + rr) + (size_t)q * ldH] : 0.0;
  }
  __syncthreads();
  const int rl = threadIdx.x / S2, c = threadIdx.x % S2;
  const int r = r0 + rl;
  const bool live = r < ks && c < s;
  double t = 0.0;
  if (live) {
    const int q0 = max(0, (r / s - 1) * s);
    const double* Yc = Ys + (size_t)c * k1s;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int q = q0;
    for (; q + 3 < k1s; q += 4) {
      a0 = fma(Hs[rl + q * rows], Yc[q], a0);
      a1 = fma(Hs[rl + (q + 1) * rows], Yc[q + 1], a1);
      a2 = fma(Hs[rl + (q + 2) * rows], Yc[q + 2], a2);
      a3 = fma(Hs[rl + (q + 3) * rows], Yc[q + 3], a3);
    }
    for (; q < k1s; ++q) a0 = fma(Hs[rl + q * rows], Yc[q], a0);
    t = w.saveZP[r + c * ks] - ((a0 + a1) + (a2 + a3));
  }
  const double rinv = (c < s) ? 1.0 / w.saveR[c + c * s] : 0.0;
  for (int q = 0; q < s; ++q) {
    const double vq = __shfl_sync(0xffffffffu, t * rinv, q, S2);
    if (c == q) t = vq;
    else if (c > q && c < s) t = fma(-vq, w.saveR[q + c * s], t);
  }
  if (live) w.J[r + c * ldH] = t;
}

// The same product without shared-memory staging, for Y too large to stage.
__global__ void __launch_bounds__(256) k_side_J_glob(SmallWs w, int k, int S2) {
  Ctl* ctl = w.ctl;
  if (*(volatile int*)&ctl->side_step != k || !ctl->side_J) return;
  const int s = w.s, ldH = w.ldH, ks = k * s, k1s = (k - 1) * s;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = idx / S2, c = idx % S2;
  const bool live = r < ks && c < s;
  double t = 0.0;
  if (live) {
    const int q0 = max(0, (r / s - 1) * s);
    double a0 = 0.0, a1 = 0.0;
    int q = q0;
    for (; q + 1 < k1s; q += 2) {
      a0 = fma(w.H[r + (size_t)q * ldH], w.saveY[q + (size_t)c * k1s], a0);
      a1 = fma(w.H[r + (size_t)(q + 1) * ldH], w.saveY[q + 1 + (size_t)c * k1s], a1);
    }
    if (q < k1s) a0 = fma(w.H[r + (size_t)q * ldH], w.saveY[q + (size_t)c * k1s], a0);
    t = w.saveZP[r + c * ks] - (a0 + a1);
  }
  const double rinv = (c < s) ? 1.0 / w.saveR[c + c * s] : 0.0;
  for (int q = 0; q < s; ++q) {
    const double vq = __shfl_sync(0xffffffffu, t * rinv, q, S2);
    if (c == q) t = vq;
    else if (c > q && c < s) t = fma(-vq, w.saveR[q + c * s], t);
  }
  if (live) w.J[r + c * ldH] = t;
}

// ---------------------------------------------------------------- cycle end
// Relation j = ctl->j.  Computes Xi_j, c = E_j^T Xi_j, M (BGMRES), and the
// coefficients of the pass over [V_1..V_{j+1}, X]:
//   out1 = X + V_{1:j} (Xi C),   out2 = U = V_{1:j+1} [M; -H_{j+1,j}];
// then C <- c C.
// The cycle end runs as three kernels:
//   k_small_end (one CTA): Xi's right-hand side (BGMRES: g; BFOM: the last
//     block c_fom and g_{1:j-1} - u c_fom) and, for BGMRES, Y_last =
//     T^{-T} S with S = H_{j+1,j}^T H_{j+1,j};
//   k_end_cols (one CTA per right-hand-side column): the block back
//     substitution with Rbar and, for BGMRES, M = Q_{1..j-1} [0; Y_last], both
//     column by column (the columns are independent; on one SM the FP64 pipe
//     made this the longest part of a cycle);
//   k_end_tail (one CTA): the coefficients of X += V Xi C and U = V [M; -H],
//     and C <- c C.
__device__ __forceinline__ bool end_skip(const SmallWs& w, const Ctl* ctl) {
  return ctl->j == 0 || (w.modification == 0 && ctl->fom_singular);
}

__global__ void __launch_bounds__(NT) k_small_end(SmallWs w) {
  __shared__ Shared sh;
  Ctl* ctl = w.ctl;
  const int j = ctl->j;
  const int s = w.s, ldH = w.ldH, ldg = w.ldH;
  if (end_skip(w, ctl)) {
    if (threadIdx.x == 0) ctl->update_step = -2;
    return;
  }
  const int js = j * s;
  double* Xi = w.Xi;     // js x s, ld ldH
  // Xi_j (last block)
  if (w.modification == 1) {
    cta_copy(Xi, ldH, w.g, ldg, js, s);
  } else {
    cta_copy(Xi + (j - 1) * s, ldH, w.cfom, s, s, s);
    cta_copy(Xi, ldH, w.g, ldg, (j - 1) * s, s);
    // g_{1:j-1} - u c
    cta_gemm_s((j - 1) * s, s, s, -1.0, w.ufom, ldH, false, w.cfom, s, false, 1.0, Xi, ldH);
  }
  // Inverses of Rbar's upper-triangular diagonal blocks (BGMRES: blocks 1..j;
  // BFOM: blocks 1..j-1), one thread per block column (back substitution for
  // R_ii z = e_c with the diagonal's reciprocals), for k_end_cols.
  const int top = (w.modification == 1) ? j : j - 1;
  const int ldR = w.ldR;
  double* Rinv = w.work + (size_t)4 * w.ldH * s;  // top blocks of s x s (clear of Ylast/XiC)
  for (int e = threadIdx.x; e < top * s; e += NT) {
    const int i = e / s, c = e % s;  // block i (0-based), column c
    const double* Rii = w.Rbar + (size_t)i * s + (size_t)i * s * ldR;
    double* Ri = Rinv + (size_t)i * s * s;
    for (int r = s - 1; r >= 0; --r) {
      double acc = (r == c) ? 1.0 : 0.0;
      if (r < c) {
        for (int p2 = r + 1; p2 <= c; ++p2) acc = fma(-Rii[r + (size_t)p2 * ldR], Ri[p2 + c * s], acc);
      }
      Ri[r + c * s] = (r <= c) ? acc / Rii[r + (size_t)r * ldR] : 0.0;
    }
  }
  __syncthreads();
  // M (BGMRES): Q_{1..j-1} [0; T^{-T} S], S = H_{j+1,j}^T H_{j+1,j}; here Y_last = T^{-T} S
  if (w.modification == 1) {
    const double* Hsub = w.H + js + (size_t)(j - 1) * s * ldH;
    cta_gemm_s(s, s, s, 1.0, Hsub, ldH, true, Hsub, ldH, false, 0.0, sh.B, s);
    // T^{-T} S: solve T^T Y = S  -> LU solve with T^T.
    for (int e = threadIdx.x; e < s * s; e += NT) {
      const int a = e % s, c = e / s;
      sh.R[a + c * s] = w.Tfom[c + a * s];
    }
    __syncthreads();
    double* Ylast = w.work;  // s x s
    warp_lu_solve(sh.R, sh.B, s, Ylast, w.work + s * s, &sh.piv, &sh.flag2);
  }
}

// Shared memory of k_end_cols.
static size_t end_cols_smem(int s, int m) {
  const size_t js = (size_t)(m + 1) * s;
  return sizeof(double) * (2 * js + 2 * (size_t)s);
}

__global__ void __launch_bounds__(256) k_end_cols(SmallWs w) {
  const Ctl* ctl = w.ctl;
  if (end_skip(w, ctl)) return;
  const int j = ctl->j;
  const int s = w.s, ldH = w.ldH, ldR = w.ldR, js = j * s, c = blockIdx.x, t = threadIdx.x;
  const int top = (w.modification == 1) ? j : j - 1;
  extern __shared__ double se[];
  double* x = se;                         // [js] column c of Xi
  double* mv = x + js;                    // [js] column c of M
  double* w1 = mv + js;                   // [s]
  double* w2 = w1 + s;                    // [s]
  const double* Ri = w.work + (size_t)4 * ldH * s;   // R_ii^{-1}, from k_small_end
  for (int r = t; r < js; r += 256) x[r] = w.Xi[r + (size_t)c * ldH];
  __syncthreads();
  // block back substitution, right-looking: x_i <- Ri_i x_i, then the rows
  // above drop R_{l,i} x_i
  for (int i = top; i >= 1; --i) {
    const int r0 = (i - 1) * s;
    if (t < s) {
      const double* Rb = Ri + (size_t)(i - 1) * s * s;
      double acc = 0.0;
      for (int q = 0; q < s; ++q) acc = fma(Rb[t + q * s], x[r0 + q], acc);
      w1[t] = acc;
    }
    __syncthreads();
    if (t < s) x[r0 + t] = w1[t];
    __syncthreads();
    for (int r = t; r < r0; r += 256) {
      double acc = x[r];
      for (int q = 0; q < s; ++q) acc = fma(-w.Rbar[r + (size_t)(r0 + q) * ldR], x[r0 + q], acc);
      x[r] = acc;
    }
    __syncthreads();
  }
  for (int r = t; r < js; r += 256) w.Xi[r + (size_t)c * ldH] = x[r];
  if (w.modification == 1) {
    // M = Q_{1..j-1} [0; Y_last]: reflector sets j-1 .. 1, Q_i = I - V T V^T on rows (i-1)s .. (i+1)s
    const double* Ylast = w.work;
    for (int r = t; r < js; r += 256)
      mv[r] = (r >= (j - 1) * s) ? Ylast[(r - (j - 1) * s) + c * s] : 0.0;
    __syncthreads();
    const int h = 2 * s;
    for (int i = j - 1; i >= 1; --i) {
      const double* V = w.refl + (size_t)(i - 1) * 2 * s * s;
      const double* T = w.Twy + (size_t)(i - 1) * s * s;
      const int r0 = (i - 1) * s;
      if (t < s) {
        double acc = 0.0;
        for (int q = 0; q < h; ++q) acc = fma(V[q + t * h], mv[r0 + q], acc);
        w1[t] = acc;
      }
      __syncthreads();
      if (t < s) {
        double acc = 0.0;
        for (int q = 0; q < s; ++q) acc = fma(T[t + q * s], w1[q], acc);
        w2[t] = acc;
      }
      __syncthreads();
      if (t < h) {
        double acc = 0.0;
        for (int l = 0; l < s; ++l) acc = fma(V[t + l * h], w2[l], acc);
        mv[r0 + t] -= acc;
      }
      __syncthreads();
    }
    for (int r = t; r < js; r += 256) w.Mvec[r + (size_t)c * ldH] = mv[r];
  }
}

__global__ void __launch_bounds__(NT) k_end_tail(SmallWs w) {
  __shared__ Shared sh;
  Ctl* ctl = w.ctl;
  if (end_skip(w, ctl)) return;
  const int j = ctl->j;
  const int s = w.s, ldH = w.ldH, js = j * s, ss = s * s;
  double* Xi = w.Xi;
  const double* Mv = w.Mvec;
  const double* Hsub = w.H + js + (size_t)(j - 1) * s * ldH;
  // c = Xi_j (s x s) -> sh.A
  cta_copy(sh.A, s, Xi + (j - 1) * s, ldH, s, s);
  // Coefficients.  Xi C -> coef1 blocks 0..j-1; coef1 block j = 0; block j+1 (X) = I.
  double* XiC = w.work + 2 * s * s;  // js x s, ld js
  cta_gemm_s(js, s, s, 1.0, Xi, ldH, false, w.Cfac, s, false, 0.0, XiC, js);
  // coefficient block b, row a, column cc: all blocks in one pass
  for (int e = threadIdx.x; e < j * ss; e += NT) {
    const int b = e / ss, a = (e / s) % s, cc = e % s;
    w.coef1[e] = XiC[b * s + a + cc * js];
    w.coef2[e] = (w.modification == 1) ? Mv[b * s + a + cc * ldH] : 0.0;
  }
  put_zero_coef(w.coef1, j, s);
  put_coef(w.coef2, j, s, Hsub, ldH, -1.0);
  put_coef(w.coef1, j + 1, s, nullptr, 0, 1.0);
  put_zero_coef(w.coef2, j + 1, s);
  // C <- c C
  cta_gemm_s(s, s, s, 1.0, sh.A, s, false, w.Cfac, s, false, 0.0, sh.B, s);
  cta_copy(w.Cfac, s, sh.B, s, s, s);
  if (threadIdx.x == 0) ctl->update_step = LSBA_END_STEP;
}

// ||R||_F / ||B||_F from the Gram R^T R (s x s) into ctl->relres_true.
__global__ void k_true_relres(const double* G, int s, Ctl* ctl) {
  if (threadIdx.x == 0) {
    double tr = 0.0;
    for (int a = 0; a < s; ++a) tr += G[a * s + a];
    ctl->relres_true = sqrt(tr) / ctl->normB;
  }
}

static void small_attrs() {
  static std::atomic<unsigned long long> attr_done{0};
  once_per_device(attr_done, [] {
    const int bytes = SMALL_ARENA_DOUBLES * sizeof(double);
    cudaFuncSetAttribute(k_small_start, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_small_step, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_small_side, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_small_end, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    cudaFuncSetAttribute(k_end_tail, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  });
}

void launch_small_start(cudaStream_t st, const SmallWs& w, int flags) {
  small_attrs();
  k_small_start<<<1, NT, SMALL_ARENA_DOUBLES * sizeof(double), st>>>(w, flags);
}
void launch_true_relres(cudaStream_t st, const double* G, int s, Ctl* ctl) {
  k_true_relres<<<1, 32, 0, st>>>(G, s, ctl);
}

__global__ void k_outer_norm(const double* G, int s, Ctl* ctl, int mode) {
  if (threadIdx.x == 0) {
    double tr = 0.0;
    for (int a = 0; a < s; ++a) tr += G[a * s + a];
    if (mode == 0) ctl->outer_normB = sqrt(tr);
    else ctl->relres_true = sqrt(tr) / ctl->outer_normB;
  }
}
void launch_outer_norm(cudaStream_t st, const double* G, int s, Ctl* ctl, int mode) {
  k_outer_norm<<<1, 32, 0, st>>>(G, s, ctl, mode);
}
void launch_small_step(cudaStream_t st, const SmallWs& w, int k, int phase) {
  if (w.skel == SK_LS && k >= 2 && w.s <= 16 && !w.global_ip)
    k_ls_products<<<LSBA_LS_PROD_CTAS, 2 * w.s * w.s, 0, st>>>(w, k);
  k_small_step<<<1, NT, SMALL_ARENA_DOUBLES * sizeof(double), st>>>(w, k, phase);
}
void launch_small_side(cudaStream_t st, const SmallWs& w, int k) {
  if (w.skel == SK_LS && k >= 2) {
    int S2 = 1;
    while (S2 < w.s) S2 <<= 1;
    const int rows = 64 / S2 > 0 ? 64 / S2 : 1;
    const int ctas = (k * w.s + rows - 1) / rows;
    const size_t smem = sizeof(double) * ((size_t)(k - 1) * w.s * w.s + (size_t)rows * (k - 1) * w.s);
    static std::atomic<unsigned long long> attr_done{0};
    once_per_device(attr_done, [] {
      cudaFuncSetAttribute(k_side_J, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
    if (smem <= 200 * 1024) {
      k_side_J<<<ctas, 64, smem, st>>>(w, k, S2);
    } else {
      const int threads = k * w.s * S2;
      k_side_J_glob<<<(threads + 255) / 256, 256, 0, st>>>(w, k, S2);
    }
  }
  k_small_side<<<1, NT, SMALL_ARENA_DOUBLES * sizeof(double), st>>>(w, k);
}
void launch_small_end(cudaStream_t st, const SmallWs& w) {
  small_attrs();
  k_small_end<<<1, NT, SMALL_ARENA_DOUBLES * sizeof(double), st>>>(w);
  k_end_cols<<<w.s, 256, end_cols_smem(w.s, w.m), st>>>(w);
  k_end_tail<<<1, NT, SMALL_ARENA_DOUBLES * sizeof(double), st>>>(w);
}

}  // namespace lsba
