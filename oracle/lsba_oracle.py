"""CPU oracle: plain, slow FP64 restarted BFOM/BGMRES with low-sync block Arnoldi.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may use it.  It shares no code with the CUDA path.

What it computes (K. Lund, "Adaptively restarted block Krylov subspace methods
with low-synchronization skeletons", arXiv 2208.09899):

* Problem A X = B, A n x n sparse, B n x s (Sec. 2, Eq. (1)); real FP64 only.
* Classical block inner product <X, Y> = X^T Y and scaling quotient
  N(X) = R of X = Q R (Sec. 2.2, Table 1); global block inner product
  <X, Y> = tr(X^T Y)/s I_s with N(X) = ||X||_F/sqrt(s) I_s (Table 1).
* Muscle CholQR: R = chol(X^T X), Q = X R^{-1} (Sec. 2.3; the muscle list of Sec. 5).
* Skeletons, each written from its algorithm in the paper's order:
  BMGS-Arnoldi (Alg. 2), BCGS (the condensed loop of Sec. 3.1),
  BCGS-PIP-Arnoldi (Alg. 3), BCGS-PIO-Arnoldi (Alg. 4, reading R12),
  BMGS-SVL / BMGS-LTS-Arnoldi (Alg. 5, both branches, reading R13),
  BMGS-CWY / BMGS-ICWY-Arnoldi (Alg. 6, both branches),
  BCGSI+LS-Arnoldi (Alg. 7).
* Modified BFOM  X_m = V_m (H_m + M)^{-1} E_1 B  (Eq. (7)); M = 0 gives BFOM,
  M = H_m^{-T} E_m H_{m+1,m}^T H_{m+1,m} E_m^T gives BGMRES (Sec. 2.4.1).
* Cospatial residual R_m = U_m (E_m^T Xi_m), U_m = V_{m+1} [M; -H_{m+1,m}]
  (Thm. 1, Eq. (8)) and the local residual norm estimate (Eq. (9)).
* Static restarting X <- X + D (Sec. 2.4.2), applied cycle after cycle.
* Adaptive restarting on a Cholesky NaN-flag (Sec. 4).

Readings taken where the paper is silent or garbled (each also listed in the
design notes of the repository):
  R1  chol's NaN-flag fires iff some pivot d_j = G_jj - sum_{i<j} R_ij^2 is <= 0
      or non-finite, or any entry of G's upper triangle is non-finite; only the
      upper triangle of G is read (MATLAB chol convention, Sec. 4).
  R2  Sec. 3.1's condensed BCGS update "W - W H" is read as W - V_k H_{1:k,k}.
  R3  Alg. 6's last two lines do not apply at k = 1 (H_{1,0} is undefined);
      for k >= 2 the product V_{k-1} H_{1:k,k} is read as V_k H_{1:k,k}, with
      the V_k just formed.
  R4  Alg. 7 sets H_{1,1} = J at k = 1 and overwrites the first block column
      with J + Y at k = 2; the final value is kept.
  R5  The lagged skeletons (Alg. 6, 7) run k = 1..m+1; iteration k completes
      Arnoldi relation j = k - 1.
  R6  The residual estimate is checked after every completed relation j; if
      H_j + M is singular the estimate at that j is skipped.
  R7  Restart bookkeeping across cycles: X += V_j Xi_j C, U = V_{j+1}[M; -H],
      C <- (E_j^T Xi_j) C, the next cycle starts from CholQR(U); the estimate is
      ||[M; -H] c C||_F / ||B||_F (Thm. 1 applied cycle after cycle, Sec. 2.4.2).
  R8  Adaptive restart (Sec. 4): a flag while completing relation j+1 ends the
      cycle with relation j and sets the maximum basis size to j for all later
      cycles; j = 0, or more than max_restarts restarts, ends the solve
      unconverged.  With adaptive restarting off, a flag ends the solve after
      the cycle's update.
  R9  Counting: an A-call or sync performed by a step that then flags is
      counted; the step itself is not.  V-application counts per cycle of j
      completed relations are defined to reproduce the appendix tables:
      BMGS 2j, BCGS 2j, PIP 3j, CWY/ICWY 3j+1, BCGSI+LS 4j+1.
  R10 (extension) verify_true_residual: when the estimate says converged but
      ||B - A X||_F / ||B||_F > tol, one more cycle starts from B - A X with C = I.
  R11 The paper's benchmark tables stop at a relative *error* tolerance
      ||X_k - X_*||_F / ||X_*||_F <= tol with X_* from a direct solve (Sec. 5,
      "reach a specified error tolerance"); ``X_star`` selects that stopping
      test instead of the residual estimate (used only to compare with the
      paper's tables).
  R12 Alg. 4 (BCGS-PIO) with the CholQR muscle: the muscle's R factor of
      [W 0; 0 H_{1:k,k}] is block diagonal, diag(chol(<W, W>), chol(H^T H))
      (the Cholesky factor of a block-diagonal Gram), so H_{k+1,k} =
      chol(R_W^T R_W - R_H^T R_H); a flag of either muscle factor is a flag
      of the step.  Two syncs per step (the inner product and the muscle's
      <W, W>); V-applications as for PIP (3 per step).  Under the global inner
      product the muscle acts on W with the global scaling quotient.
  R15 The column muscles MGS-SVL / MGS-LTS, which the paper names but does not
      list, are read as Alg. 5 with block size 1 over the columns of a block in
      Gram-Schmidt form (the column's own vector in place of A V_k): 3s - 2
      syncs per call (the appendix table's classical BMGS-SVL/LTS rows, 584
      syncs for 96 iterations in 2 cycles at s = 2, fit exactly this count),
      and their T factor (unit upper triangular) becomes T's diagonal block.
  R13 Alg. 5 (BMGS-SVL / BMGS-LTS) with a muscle whose T factor is I_s: CholQR
      (classical) or the global scaling quotient (global), whose blocks are
      orthonormal in the block inner product, so T_{k+1,k+1} = I_s and T stays
      unit block upper triangular.  The paper pairs the classical variants
      with the column muscles MGS-SVL / MGS-LTS (muscle "mgs", reading R15).
      Syncs: Y, the muscle and Z, three per step; V-applications 3 per step.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse

SKELETONS = ("bmgs", "bcgs", "bcgs_pip", "bcgs_pio", "bmgs_svl", "bmgs_lts", "bmgs_cwy",
             "bmgs_icwy", "bcgsi_ls")
LAGGED = ("bmgs_cwy", "bmgs_icwy", "bcgsi_ls")

OK, NOT_CONVERGED, BREAKDOWN = 0, 1, 2


# ---------------------------------------------------------------- primitives

def spmm(A, V: np.ndarray) -> np.ndarray:
    """W = A V for A in CSR form (the ``matvec`` of Sec. 2.1 on a block vector)."""
    M = scipy.sparse.csr_matrix((A.vals, A.colidx, A.rowptr), shape=(A.n, A.n))
    return np.asarray(M @ V)


def inner(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Classical block inner product <X, Y> = X^T Y (Table 1)."""
    return X.T @ Y


def global_inner(s: int):
    """The global block inner product of Table 1 for blocks of s columns:
    block (i, j) of <X, Y> is tr(X_i^T Y_j)/s I_s, X_i and Y_j the i-th and
    j-th s-column blocks of X and Y (a block vector list is concatenated)."""
    def ip(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
        a, b = X.shape[1] // s, Y.shape[1] // s
        G = np.zeros((a * s, b * s))
        for i in range(a):
            for j in range(b):
                t = np.sum(X[:, i * s:(i + 1) * s] * Y[:, j * s:(j + 1) * s]) / s
                G[i * s:(i + 1) * s, j * s:(j + 1) * s] = t * np.eye(s)
        return G
    return ip


def block_inner_product(name: str, s: int):
    """The block inner product named "classical" or "global" (Table 1)."""
    if name == "classical":
        return inner
    if name == "global":
        return global_inner(s)
    raise ValueError(name)


def chol_flag(G: np.ndarray, pivots: list | None = None):
    """Upper Cholesky factor R (G = R^T R) read from the upper triangle of G,
    with the NaN-flag of Sec. 4 (reading R1).  Returns (R, flag).  If
    ``pivots`` is a list, the pivots d_j computed are appended to it (the last
    one is the failing pivot of a flag)."""
    G = np.asarray(G, dtype=np.float64)
    s = G.shape[0]
    R = np.zeros((s, s))
    if not np.all(np.isfinite(np.triu(G))):
        if pivots is not None:
            pivots.append(float("nan"))
        return R, True
    for j in range(s):
        d = G[j, j] - np.dot(R[:j, j], R[:j, j])
        if pivots is not None:
            pivots.append(float(d))
        if not np.isfinite(d) or d <= 0.0:
            return R, True
        R[j, j] = np.sqrt(d)
        for c in range(j + 1, s):
            R[j, c] = (G[j, c] - np.dot(R[:j, j], R[:j, c])) / R[j, j]
    return R, False


def right_solve_upper(X: np.ndarray, R: np.ndarray) -> np.ndarray:
    """X R^{-1} for upper-triangular R, by forward substitution over the columns."""
    Q = np.array(X, dtype=np.float64, copy=True)
    s = R.shape[0]
    for c in range(s):
        Q[:, c] = (X[:, c] - Q[:, :c] @ R[:c, c]) / R[c, c]
    return Q


def left_solve_upper_T(R: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """R^{-T} Y for upper-triangular R (forward substitution with R^T)."""
    s = R.shape[0]
    Z = np.array(Y, dtype=np.float64, copy=True)
    for r in range(s):
        Z[r] = (Y[r] - R[:r, r] @ Z[:r]) / R[r, r]
    return Z


def cholqr(X: np.ndarray, ip=inner):
    """CholQR muscle: R = chol(<X, X>), Q = X R^{-1}.  Returns (Q, R, flag).
    Under the global inner product <X, X> = ||X||_F^2/s I_s, so R is the
    global scaling quotient ||X||_F/sqrt(s) I_s (Table 1)."""
    R, flag = chol_flag(ip(X, X))
    if flag:
        return None, R, True
    return right_solve_upper(X, R), R, False


def mgs_svl(X: np.ndarray, lts: bool = False):
    """Column muscle MGS-SVL (lts=False) or MGS-LTS (lts=True): Alg. 5 with
    block size 1 applied to the columns of X in Gram-Schmidt form (reading
    R15).  Column j: y = Q_{<j}^T x_j, r = T^T y (SVL) or T^{-T} y (LTS),
    w = x_j - Q_{<j} r, [q_j, r_jj] = normalisation of w (the NaN-flag of R1
    for s = 1), z = Q_{<j}^T q_j, T_{<j,j} = -T z (SVL) or z (LTS), T_jj = 1.
    Returns (Q, R, T, flag, syncs) with syncs = 3s - 2 for a full call (the
    syncs performed up to a flag otherwise)."""
    X = np.asarray(X, dtype=np.float64)
    n, s = X.shape
    Q = np.zeros((n, s))
    R = np.zeros((s, s))
    T = np.eye(s)
    syncs = 0
    for j in range(s):
        x = X[:, j]
        if j > 0:
            y = Q[:, :j].T @ x
            syncs += 1
            r = unit_upper_T_solve(T[:j, :j], y[:, None])[:, 0] if lts else T[:j, :j].T @ y
            R[:j, j] = r
            w = x - Q[:, :j] @ r
        else:
            w = x
        d = float(w @ w)
        syncs += 1
        if not np.isfinite(d) or d <= 0.0:
            return None, R, T, True, syncs
        R[j, j] = np.sqrt(d)
        Q[:, j] = w / R[j, j]
        if j > 0:
            z = Q[:, :j].T @ Q[:, j]
            syncs += 1
            T[:j, j] = z if lts else -(T[:j, :j] @ z)
    return Q, R, T, False, syncs


def unit_upper_T_solve(T: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """T^{-T} Y for unit upper-triangular T (forward substitution with T^T)."""
    Z = np.array(Y, dtype=np.float64, copy=True)
    for r in range(T.shape[0]):
        Z[r] = Y[r] - T[:r, r] @ Z[:r]
    return Z


# ---------------------------------------------------------------- skeletons

class _Arnoldi:
    """State of one block Arnoldi cycle.  ``advance()`` performs one loop
    iteration of the skeleton's algorithm and returns ("rel", j) when Arnoldi
    relation j is complete, ("flag", j) when chol flagged while completing
    relation j, or ("none", 0)."""

    def __init__(self, A, V1: np.ndarray, m: int, counts: dict, grams: list | None,
                 ip=inner):
        self.A, self.m = A, m
        self.ip = ip
        n, s = V1.shape
        self.n, self.s = n, s
        self.V = [V1]
        self.H = np.zeros(((m + 2) * s, (m + 1) * s))
        self.k = 0
        self.counts = counts
        self.grams = grams
        self.pivot_log = None   # BCGS-PIP: (k, smallest relative Cholesky pivot) per step

    def _blk(self, i, j):
        s = self.s
        return slice((i - 1) * s, i * s), slice((j - 1) * s, j * s)

    def Hb(self, i, j):
        r, c = self._blk(i, j)
        return self.H[r, c]

    def set_Hb(self, i, j, val):
        r, c = self._blk(i, j)
        self.H[r, c] = val

    def Hcol(self, i0, i1, j):
        """H_{i0:i1, j} (block rows i0..i1 inclusive)."""
        s = self.s
        return self.H[(i0 - 1) * s:i1 * s, (j - 1) * s:j * s]

    def set_Hcol(self, i0, i1, j, val):
        s = self.s
        self.H[(i0 - 1) * s:i1 * s, (j - 1) * s:j * s] = val

    def basis(self, k):
        return np.hstack(self.V[:k])

    def _matvec(self, X):
        self.counts["a_calls"] += 1
        return spmm(self.A, X)

    def _sync(self):
        self.counts["syncs"] += 1

    def _record(self, G):
        if self.grams is not None:
            self.grams.append(np.array(G))


class BMGS(_Arnoldi):
    """BMGS-Arnoldi, Alg. 2."""

    def advance(self, force_flag=False):
        self.k += 1
        k = self.k
        W = self._matvec(self.V[k - 1])
        for j in range(1, k + 1):
            Hjk = self.ip(self.V[j - 1], W)
            self._sync()
            if j == 1:
                self._record(Hjk)
            self.set_Hb(j, k, Hjk)
            W = W - self.V[j - 1] @ Hjk
        self._sync()
        Q, R, flag = cholqr(W, self.ip)
        if flag or force_flag:
            return ("flag", k)
        self.V.append(Q)
        self.set_Hb(k + 1, k, R)
        return ("rel", k)


class BCGS(_Arnoldi):
    """Block classical Gram-Schmidt Arnoldi, Sec. 3.1 (reading R2)."""

    def advance(self, force_flag=False):
        self.k += 1
        k = self.k
        W = self._matvec(self.V[k - 1])
        Vk = self.basis(k)
        Hc = self.ip(Vk, W)
        self._sync()
        self._record(Hc)
        self.set_Hcol(1, k, k, Hc)
        W = W - Vk @ Hc
        self._sync()
        Q, R, flag = cholqr(W, self.ip)
        if flag or force_flag:
            return ("flag", k)
        self.V.append(Q)
        self.set_Hb(k + 1, k, R)
        return ("rel", k)


class BCGS_PIP(_Arnoldi):
    """BCGS-PIP-Arnoldi, Alg. 3."""

    def advance(self, force_flag=False):
        self.k += 1
        k, s = self.k, self.s
        W = self._matvec(self.V[k - 1])
        Vk = self.basis(k)
        G = self.ip(np.hstack([Vk, W]), W)          # [H_{1:k,k}; Omega]
        self._sync()
        self._record(G)
        Hc, Om = G[:k * s], G[k * s:]
        piv = [] if self.pivot_log is not None else None
        R, flag = chol_flag(Om - Hc.T @ Hc, piv)
        if piv is not None:
            # smallest pivot relative to <W, W>'s diagonal: how far the
            # Pythagorean difference Omega - H^T H is from cancelling out
            self.pivot_log.append((k, min(p / Om[i, i] for i, p in enumerate(piv))))
        if flag or force_flag:
            return ("flag", k)
        self.set_Hcol(1, k, k, Hc)
        self.set_Hb(k + 1, k, R)
        self.V.append(right_solve_upper(W - Vk @ Hc, R))
        return ("rel", k)


class BCGS_PIO(_Arnoldi):
    """BCGS-PIO-Arnoldi, Alg. 4, with the CholQR muscle (reading R12)."""

    def advance(self, force_flag=False):
        self.k += 1
        k = self.k
        W = self._matvec(self.V[k - 1])
        Vk = self.basis(k)
        Hc = self.ip(Vk, W)
        self._sync()
        self._record(Hc)
        # The muscle on [W 0; 0 H_{1:k,k}]: its Gram is block diagonal, and so
        # is its Cholesky factor.
        RW, flag_w = chol_flag(self.ip(W, W))
        self._sync()
        RH, flag_h = chol_flag(Hc.T @ Hc)
        if flag_w or flag_h or force_flag:
            return ("flag", k)
        R, flag = chol_flag(RW.T @ RW - RH.T @ RH)
        if flag:
            return ("flag", k)
        self.set_Hcol(1, k, k, Hc)
        self.set_Hb(k + 1, k, R)
        self.V.append(right_solve_upper(W - Vk @ Hc, R))
        return ("rel", k)


class BMGS_SVL(_Arnoldi):
    """BMGS-SVL-Arnoldi, Alg. 5 (red branch), readings R13 and R15.  muscle =
    "cholqr" (T factor I_s) or "mgs" (MGS-SVL / MGS-LTS column muscle, whose
    T factor enters T's diagonal block); T11 is the start block's factor."""
    lts = False

    def __init__(self, *args, muscle: str = "cholqr", T11=None, **kw):
        super().__init__(*args, **kw)
        self.muscle = muscle
        self.T = np.eye((self.m + 2) * self.s)
        if T11 is not None:
            self.T[:self.s, :self.s] = T11

    def advance(self, force_flag=False):
        self.k += 1
        k, s = self.k, self.s
        W = self._matvec(self.V[k - 1])
        Vk = self.basis(k)
        Y = self.ip(Vk, W)
        self._sync()
        self._record(Y)
        Tk = self.T[:k * s, :k * s]
        Hc = unit_upper_T_solve(Tk, Y) if self.lts else Tk.T @ Y
        if self.muscle == "mgs":
            Q, R, Tm, flag, ns = mgs_svl(W - Vk @ Hc, self.lts)
            self.counts["syncs"] += ns
        else:
            self._sync()
            Q, R, flag = cholqr(W - Vk @ Hc, self.ip)
            Tm = np.eye(s)
        if flag or force_flag:
            return ("flag", k)
        self.V.append(Q)
        self.set_Hcol(1, k, k, Hc)
        self.set_Hb(k + 1, k, R)
        Z = self.ip(Vk, Q)
        self._sync()
        # T_{1:k,k+1} = -T Z T_{k+1,k+1} (SVL) or Z T_{k+1,k+1} (LTS)
        self.T[:k * s, k * s:(k + 1) * s] = (Z if self.lts else -Tk @ Z) @ Tm
        self.T[k * s:(k + 1) * s, k * s:(k + 1) * s] = Tm
        return ("rel", k)


class BMGS_LTS(BMGS_SVL):
    """BMGS-LTS-Arnoldi, Alg. 5 (blue branch), reading R13."""
    lts = True


class BMGS_CWY(_Arnoldi):
    """BMGS-CWY (red) / BMGS-ICWY (blue) Arnoldi, Alg. 6 (readings R3, R5)."""
    inverse = False

    def __init__(self, *a, **kw):
        super().__init__(*a, **kw)
        self.T = np.eye((self.m + 2) * self.s)
        self.U = self.V[0]

    def advance(self, force_flag=False):
        self.k += 1
        k, s = self.k, self.s
        W = self._matvec(self.U)
        if k == 1:
            H11 = self.ip(self.U, W)
            self._sync()
            self._record(H11)
            self.set_Hb(1, 1, H11)
            self.U = W - self.V[0] @ H11
            return ("none", 0)
        Vkm1 = self.basis(k - 1)
        G = self.ip(np.hstack([Vkm1, self.U]), np.hstack([self.U, W]))
        self._sync()
        self._record(G)
        Y, Z = G[:(k - 1) * s, :s], G[:(k - 1) * s, s:]
        Om, Pt = G[(k - 1) * s:, :s], G[(k - 1) * s:, s:]
        R, flag = chol_flag(Om)
        if flag or force_flag:
            return ("flag", k - 1)
        self.set_Hb(k, k - 1, R)
        P = left_solve_upper_T(R, Pt)
        YRi = right_solve_upper(Y, R)
        ZP = right_solve_upper(np.vstack([Z, P]), R)
        if self.inverse:
            self.T[:(k - 1) * s, (k - 1) * s:k * s] = YRi
            Hc = unit_upper_T_solve(self.T[:k * s, :k * s], ZP)
        else:
            self.T[:(k - 1) * s, (k - 1) * s:k * s] = -self.T[:(k - 1) * s, :(k - 1) * s] @ YRi
            Hc = self.T[:k * s, :k * s].T @ ZP
        self.set_Hcol(1, k, k, Hc)
        Vk = right_solve_upper(self.U, R)
        self.V.append(Vk)
        self.U = right_solve_upper(W, R) - self.basis(k) @ Hc
        return ("rel", k - 1)


class BMGS_ICWY(BMGS_CWY):
    inverse = True


class BCGSI_LS(_Arnoldi):
    """BCGSI+LS-Arnoldi, Alg. 7 (readings R4, R5)."""

    def __init__(self, *a, **kw):
        super().__init__(*a, **kw)
        self.U = self.V[0]
        self.J = None

    def advance(self, force_flag=False):
        self.k += 1
        k, s = self.k, self.s
        W = self._matvec(self.U)
        if k == 1:
            J = self.ip(self.U, W)
            self._sync()
            self._record(J)
            self.J = J
            self.set_Hb(1, 1, J)
            self.U = W - self.V[0] @ J
            return ("none", 0)
        Vkm1 = self.basis(k - 1)
        G = self.ip(np.hstack([Vkm1, self.U]), np.hstack([self.U, W]))
        self._sync()
        self._record(G)
        Y, Z = G[:(k - 1) * s, :s], G[:(k - 1) * s, s:]
        Omt, Pt = G[(k - 1) * s:, :s], G[(k - 1) * s:, s:]
        R, flag = chol_flag(Omt - Y.T @ Y)
        if flag or force_flag:
            return ("flag", k - 1)
        self.set_Hb(k, k - 1, R)
        self.set_Hcol(1, k - 1, k - 1, self.J + Y)
        P = left_solve_upper_T(R, Pt - Y.T @ Z)
        ZP = np.vstack([Z, P])
        Hk = self.H[:k * s, :(k - 1) * s]
        self.J = right_solve_upper(ZP - Hk @ Y, R)
        Vk = right_solve_upper(self.U - Vkm1 @ Y, R)
        self.V.append(Vk)
        self.U = right_solve_upper(W - self.basis(k) @ ZP, R)
        return ("rel", k - 1)


_CLASSES = {"bmgs": BMGS, "bcgs": BCGS, "bcgs_pip": BCGS_PIP, "bcgs_pio": BCGS_PIO,
            "bmgs_svl": BMGS_SVL, "bmgs_lts": BMGS_LTS,
            "bmgs_cwy": BMGS_CWY, "bmgs_icwy": BMGS_ICWY, "bcgsi_ls": BCGSI_LS}

_VAPPS = {"bmgs": (2, 0), "bcgs": (2, 0), "bcgs_pip": (3, 0), "bcgs_pio": (3, 0),
          "bmgs_svl": (3, 0), "bmgs_lts": (3, 0),
          "bmgs_cwy": (3, 1), "bmgs_icwy": (3, 1), "bcgsi_ls": (4, 1)}


def _start_block(R_start, skeleton, ip, muscle):
    """The cycle's start muscle: CholQR (or the global scaling quotient), or
    for BMGS-SVL/LTS with muscle "mgs" the column muscle (reading R15).
    Returns (V1, Beta, flag, syncs, extra constructor arguments)."""
    if skeleton in ("bmgs_svl", "bmgs_lts"):
        if muscle == "mgs":
            Q, R, T, flag, ns = mgs_svl(R_start, skeleton == "bmgs_lts")
            return Q, R, flag, ns, {"muscle": "mgs", "T11": T}
        if muscle != "cholqr":
            raise ValueError(muscle)
    elif muscle != "cholqr":
        raise ValueError("the column muscle belongs to BMGS-SVL / BMGS-LTS")
    V1, Beta, flag = cholqr(R_start, ip)
    return V1, Beta, flag, 1, {}


def arnoldi(A, B: np.ndarray, m: int, skeleton: str, inner_product: str = "classical",
            muscle: str = "cholqr"):
    """m steps of a block Arnoldi skeleton from B (no restarts, no flags expected).
    Returns (V_{m+1} as n x (m+1)s, H_{m+1,m}, Beta)."""
    counts = {"a_calls": 0, "syncs": 0}
    ip = block_inner_product(inner_product, B.shape[1])
    if muscle != "cholqr" and inner_product != "classical":
        raise ValueError("the global paradigm takes only the global muscle")
    V1, Beta, flag, _, extra = _start_block(B, skeleton, ip, muscle)
    if flag:
        raise FloatingPointError("CholQR of B flagged")
    ar = _CLASSES[skeleton](A, V1, m, counts, None, ip=ip, **extra)
    j = 0
    while j < m:
        kind, jj = ar.advance()
        if kind == "flag":
            raise FloatingPointError(f"chol flag at relation {jj}")
        if kind == "rel":
            j = jj
    s = B.shape[1]
    return ar.basis(m + 1), ar.H[:(m + 1) * s, :m * s].copy(), Beta


# ---------------------------------------------------------------- small solves

def cycle_coefficients(H: np.ndarray, j: int, s: int, Beta: np.ndarray, modification: str):
    """For relation j of a cycle: M vector, Xi_j and the cospatial factor.

    H_j = H[:js,:js], H_{j+1,j} = H[js:(j+1)s, (j-1)s:js].
    BFOM: M = 0.  BGMRES: M = H_j^{-T} E_j (H_{j+1,j}^T H_{j+1,j})  (Sec. 2.4.1).
    Xi_j = (H_j + M E_j^T)^{-1} E_1 Beta  (Eq. (7)); c = E_j^T Xi_j.
    Returns (Mvec, Xi, c) or None if the small system is singular (reading R6).
    """
    js = j * s
    Hj = H[:js, :js]
    Hsub = H[js:js + s, js - s:js]
    Ej = np.zeros((js, s))
    Ej[js - s:, :] = np.eye(s)
    E1B = np.zeros((js, s))
    E1B[:s, :] = Beta
    try:
        if modification == "gmres":
            Mvec = np.linalg.solve(Hj.T, Ej @ (Hsub.T @ Hsub))
        else:
            Mvec = np.zeros((js, s))
        Xi = np.linalg.solve(Hj + Mvec @ Ej.T, E1B)
    except np.linalg.LinAlgError:
        return None
    if not np.all(np.isfinite(Xi)):
        return None
    return Mvec, Xi, Xi[js - s:]


def residual_estimate(H, j, s, Mvec, c, C, normB):
    """||[M; -H_{j+1,j}] c C||_F / ||B||_F  (Eq. (9), reading R7)."""
    js = j * s
    Hsub = H[js:js + s, js - s:js]
    return np.linalg.norm(np.vstack([Mvec, -Hsub]) @ c @ C) / normB


# ---------------------------------------------------------------- driver

@dataclass
class Result:
    X: np.ndarray
    status: int
    cycles: int = 0
    steps: int = 0
    a_calls: int = 0
    syncs: int = 0
    v_apps: int = 0
    flags: int = 0
    cycle_m: list = field(default_factory=list)       # relations completed per cycle
    cycle_flag: list = field(default_factory=list)    # relation that flagged (0 = none)
    m_cur: list = field(default_factory=list)         # max basis size in force per cycle
    est_history: list = field(default_factory=list)   # (cycle, j, estimate)
    relres_est: float = float("nan")
    relres_true: float = float("nan")
    first_cycle: dict | None = None


def solve(A, B: np.ndarray, m: int, tol: float, skeleton: str = "bcgsi_ls",
          modification: str = "gmres", max_restarts: int = 50, adaptive: bool = True,
          verify_true_residual: bool = True, inject_flags=(), record_first_cycle: bool = False,
          true_residual_each_cycle: bool = False, X_star: np.ndarray | None = None,
          inner_product: str = "classical", muscle: str = "cholqr",
          pivot_trace: list | None = None) -> Result:
    """Restarted, adaptively restarted modified BFOM (BFOM or BGMRES) for A X = B
    with the given block Arnoldi skeleton; X_0 = 0.

    ``inject_flags`` is a set of (cycle, relation) pairs at which the chol flag
    is forced (test hook: a host-decided input, reading R8 applies).
    ``pivot_trace`` (a list, BCGS-PIP only) receives (cycle, relation, r) for
    every step, r the smallest Cholesky pivot of Omega - H^T H relative to
    Omega's diagonal: the margin by which the step's flag decision was taken,
    which decides whether another rounding order may decide differently.
    """
    if skeleton not in _CLASSES:
        raise ValueError(skeleton)
    B = np.asarray(B, dtype=np.float64)
    n, s = B.shape
    ip = block_inner_product(inner_product, s)
    if muscle != "cholqr" and inner_product != "classical":
        raise ValueError("the global paradigm takes only the global muscle")
    normB = np.linalg.norm(B)
    X = np.zeros((n, s))
    C = np.eye(s)
    m_cur = m
    R_start = B
    inject = set(tuple(x) for x in inject_flags)
    counts = {"a_calls": 0, "syncs": 0}
    res = Result(X=X, status=NOT_CONVERGED)
    vper, vcyc = _VAPPS[skeleton]
    cycle = 0
    while True:
        cycle += 1
        if cycle > max_restarts + 1:
            res.status = NOT_CONVERGED
            break
        V1, Beta, flag, ns, extra = _start_block(R_start, skeleton, ip, muscle)
        counts["syncs"] += ns
        if flag:
            res.status = BREAKDOWN if cycle == 1 else NOT_CONVERGED
            res.cycles = cycle
            break
        grams = [] if (record_first_cycle and cycle == 1) else None
        ar = _CLASSES[skeleton](A, V1, m_cur, counts, grams, ip=ip, **extra)
        if pivot_trace is not None:
            ar.pivot_log = []
        res.m_cur.append(m_cur)
        j, converged, flagged = 0, False, 0
        coeffs = None
        ests = []
        while j < m_cur:
            target = j + 1
            kind, jj = ar.advance(force_flag=(cycle, target) in inject and _lagged_ready(ar, skeleton))
            if kind == "none":
                continue
            if kind == "flag":
                flagged = jj
                res.flags += 1
                break
            j = jj
            cf = cycle_coefficients(ar.H, j, s, Beta, modification)
            if cf is None:
                ests.append(float("nan"))
                res.est_history.append((cycle, j, float("nan")))
                coeffs = None
                continue
            coeffs = cf
            est = residual_estimate(ar.H, j, s, cf[0], cf[2], C, normB)
            ests.append(est)
            res.est_history.append((cycle, j, est))
            res.relres_est = est
            if X_star is not None:
                Xj = X + ar.basis(j) @ (cf[1] @ C)
                if np.linalg.norm(Xj - X_star) <= tol * np.linalg.norm(X_star):
                    converged = True
                    break
            elif est <= tol:
                converged = True
                break
        res.cycles = cycle
        if pivot_trace is not None and ar.pivot_log is not None:
            pivot_trace.extend((cycle, k, r) for k, r in ar.pivot_log)
        res.cycle_m.append(j)
        res.cycle_flag.append(flagged)
        res.steps += j
        res.v_apps += vper * j + (vcyc if j > 0 else 0)
        if record_first_cycle and cycle == 1:
            res.first_cycle = {"H": ar.H[:(j + 1) * s, :j * s].copy(), "Beta": Beta.copy(),
                               "grams": grams, "V": ar.basis(j + 1) if j > 0 else V1,
                               "est": list(ests), "j": j}
        if flagged and adaptive:
            m_cur = flagged - 1
        if j == 0:
            res.status = NOT_CONVERGED
            break
        if coeffs is None:
            res.status = NOT_CONVERGED
            break
        Mvec, Xi, c = coeffs
        Vj = ar.basis(j)
        X = X + Vj @ (Xi @ C)
        Hsub = ar.H[j * s:(j + 1) * s, (j - 1) * s:j * s]
        U = ar.basis(j + 1) @ np.vstack([Mvec, -Hsub])
        C = c @ C
        if flagged and not adaptive:
            res.status = NOT_CONVERGED
            break
        if true_residual_each_cycle or (converged and verify_true_residual):
            Rt = B - spmm(A, X)
            res.relres_true = np.linalg.norm(Rt) / normB
        if converged:
            if verify_true_residual and res.relres_true > tol:
                R_start = Rt
                C = np.eye(s)
                continue
            res.status = OK
            break
        R_start = U
    res.X = X
    res.a_calls = counts["a_calls"]
    res.syncs = counts["syncs"]
    if np.isnan(res.relres_true):
        res.relres_true = np.linalg.norm(B - spmm(A, X)) / normB
    return res


def _lagged_ready(ar, skeleton):
    """A forced flag applies to the iteration that would complete the target
    relation: for lagged skeletons that is any iteration k >= 2."""
    if skeleton in LAGGED:
        return ar.k + 1 >= 2
    return True


# ---------------------------------------------------------------- diagnostics

def loss_of_orthogonality(Q: np.ndarray) -> float:
    """||I - <Q, Q>||_2  (Eq. (5))."""
    return np.linalg.norm(np.eye(Q.shape[1]) - Q.T @ Q, 2)


def arnoldi_residual(A, V: np.ndarray, H: np.ndarray, m: int, s: int) -> float:
    """||A V_m - V_{m+1} H_{m+1,m}||_F  (Eq. (6))."""
    return np.linalg.norm(spmm(A, V[:, :m * s]) - V[:, :(m + 1) * s] @ H[:(m + 1) * s, :m * s])
