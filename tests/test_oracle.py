"""Pins for the CPU oracle against facts fixed by the paper and by the mathematics
(not against the oracle itself).  CPU only."""
import json
import os

import numpy as np
import pytest

from oracle import lsba_oracle as O
from paper_2208_09899_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tridiag.json")


def _rand_csr(n, density, seed):
    rng = np.random.default_rng(seed)
    D = np.where(rng.random((n, n)) < density, rng.standard_normal((n, n)), 0.0)
    D += np.diag(np.full(n, 5.0))
    rows, cols = np.nonzero(D)
    return W._from_coo(n, rows, cols, D[rows, cols]), D


# ------------------------------------------------------------------ primitives

def test_spmm_matches_dense_product():
    A, D = _rand_csr(57, 0.1, 1)
    V = W.gaussian_block(57, 5, 2)
    assert np.allclose(O.spmm(A, V), D @ V, rtol=0, atol=1e-13)
    # An empty row and a ragged structure.
    A2 = W._from_coo(6, [0, 0, 2, 5], [1, 4, 2, 0], [1.0, 2.0, 3.0, 4.0])
    D2 = A2.to_dense()
    V2 = W.gaussian_block(6, 3, 3)
    assert np.allclose(O.spmm(A2, V2), D2 @ V2, atol=1e-15)
    assert np.all(O.spmm(A2, V2)[1] == 0.0)


def test_chol_flag_matches_textbook_and_reads_upper_triangle():
    rng = np.random.default_rng(0)
    for s in (1, 2, 5, 16, 32):
        X = rng.standard_normal((3 * s + 4, s))
        G = X.T @ X
        R, flag = O.chol_flag(G)
        assert not flag
        L = np.linalg.cholesky(G)
        assert np.allclose(R, L.T, rtol=1e-12, atol=1e-12 * np.abs(L).max())
        assert np.allclose(np.triu(R), R)
        # Garbage (even NaN) in the strict lower triangle is never read.
        Gl = G.copy()
        Gl[np.tril_indices(s, -1)] = np.nan
        R2, flag2 = O.chol_flag(Gl)
        assert not flag2 and np.array_equal(R, R2)


@pytest.mark.parametrize("case", ["indefinite", "singular", "nan", "inf", "negdiag"])
def test_chol_flag_fires(case):
    s = 4
    G = np.eye(s)
    if case == "indefinite":
        G = np.array([[1.0, 2.0], [2.0, 1.0]])
    elif case == "singular":
        v = np.arange(1.0, s + 1)
        G = np.outer(v, v)
    elif case == "nan":
        G[1, 3] = np.nan
    elif case == "inf":
        G[0, 0] = np.inf
    elif case == "negdiag":
        G[2, 2] = -1e-300
    _, flag = O.chol_flag(G)
    assert flag


def test_cholqr_is_a_qr_factorization():
    X = W.gaussian_block(200, 6, 4)
    Q, R, flag = O.cholqr(X)
    assert not flag
    assert np.linalg.norm(Q.T @ Q - np.eye(6)) < 1e-14
    assert np.linalg.norm(Q @ R - X) < 1e-13 * np.linalg.norm(X)
    Qh, Rh = np.linalg.qr(X)
    sg = np.sign(np.diag(Rh))
    assert np.allclose(R, sg[:, None] * Rh, rtol=1e-11, atol=1e-12)
    # A block with an exactly zero column has a zero pivot: the muscle flags.
    Xd = X.copy()
    Xd[:, 3] = 0.0
    assert O.cholqr(Xd)[2]


# ------------------------------------------------------------------ skeletons

def _problem(n=300, s=3, seed=0):
    return W.tridiag_const(n), W.gaussian_block(n, s, seed)


@pytest.mark.parametrize("sk", O.SKELETONS)
def test_arnoldi_relation_and_orthogonality(sk):
    """Eq. (6) holds, and the loss of orthogonality (Eq. (5)) obeys Table 2's
    bounds with kappa = kappa([B, A V_m]) measured independently on the dense
    matrix: O(eps) kappa for BMGS, O(eps) kappa^2 for PIP (when eps kappa^2 < 1);
    the CWY/ICWY/BCGSI+LS bounds are open, so the BMGS bound is used for them."""
    A, B = _problem()
    m, s = 12, 3
    V, H, Beta = O.arnoldi(A, B, m, sk)
    rel = O.arnoldi_residual(A, V, H, m, s) / (6.0 * np.linalg.norm(V[:, :m * s]))
    assert rel < 1e-13, rel
    eps = np.finfo(float).eps
    kappa = np.linalg.cond(np.hstack([B, A.to_dense() @ V[:, :m * s]]))
    loo = O.loss_of_orthogonality(V)
    if sk in ("bcgs_pip", "bcgs_pio", "bcgs"):
        if eps * kappa ** 2 < 1:
            assert loo <= 100 * eps * kappa ** 2
    else:
        assert loo <= 100 * eps * kappa, (loo, kappa)
    # Block upper Hessenberg; subdiagonal blocks upper triangular with positive diagonal.
    for j in range(1, m + 1):
        assert np.all(H[(j + 1) * s:, (j - 1) * s:j * s] == 0.0)
        Hs = H[j * s:(j + 1) * s, (j - 1) * s:j * s]
        assert np.allclose(np.tril(Hs, -1), 0.0) and np.all(np.diag(Hs) > 0)
    # V_1 Beta = B.
    assert np.linalg.norm(V[:, :s] @ Beta - B) < 1e-13 * np.linalg.norm(B)
    # Few steps, better-conditioned [B, A V]: orthogonal to O(eps) (O(eps) kappa^2
    # for the Pythagorean/classical skeletons).
    V4, _, _ = O.arnoldi(A, B, 3, sk)
    assert O.loss_of_orthogonality(V4) < (1e-10 if sk in ("bcgs_pip", "bcgs_pio", "bcgs") else 1e-13)


@pytest.mark.parametrize("sk", [k for k in O.SKELETONS if k != "bmgs"])
def test_skeletons_agree_with_bmgs(sk):
    """All BGS skeletons give the same QR in exact arithmetic (Remark 1).  The
    2D Laplacian keeps kappa([B, A V_m]) ~ 5e2, so rounding differences stay
    near eps * kappa."""
    A = W.laplacian_2d(20)
    B = W.gaussian_block(A.n, 3, 3)
    m = 10
    V0, H0, B0 = O.arnoldi(A, B, m, "bmgs")
    V1, H1, B1 = O.arnoldi(A, B, m, sk)
    assert np.linalg.norm(H1 - H0) <= 1e-12 * np.linalg.norm(H0)
    assert np.linalg.norm(V1 - V0) <= 1e-12 * np.linalg.norm(V0)
    assert np.array_equal(B0, B1)


@pytest.mark.parametrize("sk", O.SKELETONS)
def test_hessenberg_is_the_projection_and_basis_spans_krylov(sk):
    """H_m = V_m^T A V_m and span(V_m) contains B, AB, ..., A^{m-1}B (Eq. (4))."""
    n, s, m = 120, 2, 6
    A = W.laplacian_2d(12, 10)
    B = W.gaussian_block(n, s, 7)
    V, H, _ = O.arnoldi(A, B, m, sk)
    D = A.to_dense()
    Vm = V[:, :m * s]
    assert np.allclose(Vm.T @ D @ Vm, H[:m * s], atol=1e-12 * np.abs(D).max())
    K = B.copy()
    for i in range(m):
        assert np.linalg.norm(K - Vm @ (Vm.T @ K)) <= 1e-10 * np.linalg.norm(K)
        K = D @ K


def test_bgmres_is_block_least_squares_and_bfom_is_galerkin():
    """BGMRES as modified BFOM minimises ||E_1 Beta - Hbar Xi||_F (Sec. 2.4.1);
    BFOM's residual is orthogonal to V_m.  A is nonsymmetric so that H_m^T != H_m."""
    A = W.tridiag_const(225, -1.3, 4.0, -0.6)
    n, s, m = A.n, 4, 9
    B = W.gaussian_block(n, s, 11)
    V, H, Beta = O.arnoldi(A, B, m, "bcgsi_ls")
    rhs = np.zeros(((m + 1) * s, s))
    rhs[:s] = Beta
    _, Xi_g, _ = O.cycle_coefficients(H, m, s, Beta, "gmres")
    Xi_ls = np.linalg.lstsq(H, rhs, rcond=None)[0]
    assert np.linalg.norm(Xi_g - Xi_ls) <= 1e-10 * np.linalg.norm(Xi_ls)
    _, Xi_f, _ = O.cycle_coefficients(H, m, s, Beta, "fom")
    Xf = V[:, :m * s] @ Xi_f
    Rf = B - O.spmm(A, Xf)
    assert np.linalg.norm(V[:, :m * s].T @ Rf) <= 1e-11 * np.linalg.norm(B)


@pytest.mark.parametrize("mod", ["fom", "gmres"])
@pytest.mark.parametrize("sk", ["bcgs_pip", "bcgsi_ls", "bmgs_icwy", "bcgs"])
def test_estimate_equals_true_residual_every_cycle(sk, mod):
    """Eq. (9) (Thm. 1, exact arithmetic) across restarts: the estimate at each
    cycle end equals ||B - A X||_F / ||B||_F.  Pins the cospatial factor
    recurrence C <- c C and X += V Xi C."""
    A = W.laplacian_2d(20)
    B = W.gaussian_block(A.n, 3, 5)
    r = O.solve(A, B, 6, 1e-30, sk, modification=mod, max_restarts=4,
                verify_true_residual=False)
    # Re-run cycle by cycle with true residuals (deterministic: same arithmetic).
    ests = {}
    for (c, j, e) in r.est_history:
        ests[c] = e
    for cyc in range(1, r.cycles + 1):
        rr = O.solve(A, B, 6, 1e-30, sk, modification=mod, max_restarts=cyc - 1,
                     verify_true_residual=False, true_residual_each_cycle=True)
        assert abs(rr.relres_true - ests[cyc]) <= 1e-7 * ests[cyc], (cyc, rr.relres_true, ests[cyc])


def test_gmres_estimate_is_nonincreasing_within_a_cycle():
    A = W.laplacian_2d(24)
    B = W.gaussian_block(A.n, 4, 8)
    r = O.solve(A, B, 15, 1e-30, "bcgsi_ls", modification="gmres", max_restarts=2,
                verify_true_residual=False)
    by_cycle = {}
    for c, j, e in r.est_history:
        by_cycle.setdefault(c, []).append(e)
    for c, es in by_cycle.items():
        assert all(b <= a * (1 + 1e-10) for a, b in zip(es, es[1:])), es


def _textbook_gmres(D, b, m):
    """Single-vector GMRES(m) with modified Gram-Schmidt Arnoldi and Givens
    rotations (Saad, Iterative Methods for Sparse Linear Systems, Alg. 6.9),
    x0 = 0, no restart.  Returns x_m and the residual norms."""
    n = len(b)
    beta = np.linalg.norm(b)
    Vv = np.zeros((n, m + 1))
    Hh = np.zeros((m + 1, m))
    Vv[:, 0] = b / beta
    cs, sn = np.zeros(m), np.zeros(m)
    g = np.zeros(m + 1)
    g[0] = beta
    res = []
    for j in range(m):
        w = D @ Vv[:, j]
        for i in range(j + 1):
            Hh[i, j] = w @ Vv[:, i]
            w = w - Hh[i, j] * Vv[:, i]
        Hh[j + 1, j] = np.linalg.norm(w)
        Vv[:, j + 1] = w / Hh[j + 1, j]
        for i in range(j):
            t = cs[i] * Hh[i, j] + sn[i] * Hh[i + 1, j]
            Hh[i + 1, j] = -sn[i] * Hh[i, j] + cs[i] * Hh[i + 1, j]
            Hh[i, j] = t
        rr = np.hypot(Hh[j, j], Hh[j + 1, j])
        cs[j], sn[j] = Hh[j, j] / rr, Hh[j + 1, j] / rr
        Hh[j, j], Hh[j + 1, j] = rr, 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        res.append(abs(g[j + 1]))
    y = np.zeros(m)
    for i in range(m - 1, -1, -1):
        y[i] = (g[i] - Hh[i, i + 1:m] @ y[i + 1:]) / Hh[i, i]
    return Vv[:, :m] @ y, np.array(res)


@pytest.mark.parametrize("sk", ["bmgs", "bcgs_pip", "bcgsi_ls", "bmgs_icwy"])
def test_s1_bgmres_is_textbook_gmres(sk):
    A, D = _rand_csr(80, 0.08, 21)
    b = W.gaussian_block(80, 1, 22)
    m = 12
    x_ref, res_ref = _textbook_gmres(D, b[:, 0], m)
    r = O.solve(A, b, m, 1e-30, sk, modification="gmres", max_restarts=0,
                verify_true_residual=False)
    assert r.cycle_m == [m]
    assert np.linalg.norm(r.X[:, 0] - x_ref) <= 1e-10 * np.linalg.norm(x_ref)
    est = np.array([e for (c, j, e) in r.est_history])
    assert np.allclose(est, res_ref / np.linalg.norm(b), rtol=1e-8)


@pytest.mark.parametrize("mod", ["fom", "gmres"])
@pytest.mark.parametrize("sk", O.SKELETONS)
def test_solution_matches_direct_solve(sk, mod):
    """Final X against a dense direct solve (Sec. 5 uses backslash likewise)."""
    A = W.laplacian_2d(12)
    n, s = A.n, 3
    B = W.gaussian_block(n, s, 30)
    r = O.solve(A, B, 10, 1e-10, sk, modification=mod, max_restarts=100)
    assert r.status == O.OK
    D = A.to_dense()
    Xs = np.linalg.solve(D, B)
    assert r.relres_true <= 1e-10
    kappa = np.linalg.cond(D)
    assert np.linalg.norm(r.X - Xs) <= 2 * kappa * 1e-10 * np.linalg.norm(Xs)


@pytest.mark.parametrize("sk", O.SKELETONS)
def test_counter_identities(sk):
    """Sync / A-call / V-application counts per cycle of j relations (Table 2 and
    the appendix tables): BMGS 1+j(j+1)/2+j syncs; PIP 1+j; lagged 1+(j+1);
    BCGS 1+2j.  A-calls j (j+1 lagged)."""
    A = W.laplacian_2d(16)
    B = W.gaussian_block(A.n, 2, 9)
    r = O.solve(A, B, 7, 1e-9, sk, modification="gmres", max_restarts=200,
                verify_true_residual=False)
    assert r.status == O.OK and r.flags == 0
    js = r.cycle_m
    lag = sk in O.LAGGED
    syn = {"bmgs": lambda j: 1 + j * (j + 1) // 2 + j, "bcgs": lambda j: 1 + 2 * j,
           "bcgs_pip": lambda j: 1 + j, "bcgs_pio": lambda j: 1 + 2 * j,
           "bmgs_svl": lambda j: 1 + 3 * j, "bmgs_lts": lambda j: 1 + 3 * j}.get(sk, lambda j: 1 + j + 1)
    assert r.syncs == sum(syn(j) for j in js)
    assert r.a_calls == sum(j + (1 if lag else 0) for j in js)
    assert r.steps == sum(js)


def test_paper_tridiag_table():
    """Appendix table for tridiag (n=1000, s=2, m=70, FOM, tol 1e-10).  The
    paper's tables stop on the relative error (reading R11).  Stable skeletons:
    2 cycles and 94 +- 2 iterations, with the table's own count identities."""
    g = json.load(open(GOLDEN))
    A, B = W.paper_tridiag(1000)
    Xs = np.linalg.solve(A.to_dense(), B)
    for sk in ("bmgs", "bmgs_cwy", "bmgs_icwy", "bcgsi_ls"):
        row = g["classical_rows"][sk]
        r = O.solve(A, B, 70, 1e-10, sk, modification="fom", max_restarts=100,
                    verify_true_residual=False, X_star=Xs)
        assert r.status == O.OK
        assert r.cycles == row["cycles"]
        assert abs(r.steps - row["iters"]) <= 2
        # The table's identities, evaluated on our run.
        assert row["A"] - row["iters"] == r.a_calls - r.steps
        if sk == "bmgs":
            assert r.syncs == sum(1 + j * (j + 1) // 2 + j for j in r.cycle_m)
            assert row["sync"] == sum(1 + j * (j + 1) // 2 + j for j in (70, 24))
        else:
            assert r.syncs == r.steps + 2 * r.cycles
            assert row["sync"] == row["iters"] + 2 * row["cycles"]
        vper = {"bmgs": 2, "bmgs_cwy": 3, "bmgs_icwy": 3, "bcgsi_ls": 4}[sk]
        vcyc = 0 if sk == "bmgs" else 1
        assert row["V"] == vper * row["iters"] + vcyc * row["cycles"]
        assert r.v_apps == vper * r.steps + vcyc * r.cycles


def test_paper_multithread_example_pip_flag_step():
    """Sec. 4: tridiag n=100, no restarts, m=50: single-threaded BCGS-PIP reaches
    35 iterations before chol raises the NaN-flag."""
    g = json.load(open(GOLDEN))["multithread_example"]
    A, B = W.paper_tridiag(g["n"])
    r = O.solve(A, B, g["m"], 0.0, "bcgs_pip", modification="fom", max_restarts=0,
                adaptive=False, verify_true_residual=False)
    assert r.cycle_m == [g["bcgs_pip_relations_before_flag"]]
    assert r.cycle_flag == [g["bcgs_pip_relations_before_flag"] + 1]
    assert r.status == O.NOT_CONVERGED


@pytest.mark.parametrize("sk", ["bcgs_pip", "bcgsi_ls", "bmgs_icwy", "bcgs"])
def test_adaptive_restart_shrinks_m(sk):
    """Sec. 4: on a flag, the cycle ends at the last safe relation and the
    maximum basis size drops to it for all later cycles."""
    A = W.laplacian_2d(16)
    B = W.gaussian_block(A.n, 2, 12)
    r = O.solve(A, B, 8, 1e-9, sk, modification="gmres", max_restarts=200,
                inject_flags=[(1, 5)])
    assert r.cycle_flag[0] == 5 and r.cycle_m[0] == 4
    assert r.m_cur[0] == 8 and all(mc == 4 for mc in r.m_cur[1:])
    assert r.status == O.OK
    # A flag on the very first relation cannot be resolved (Sec. 5.4).
    r0 = O.solve(A, B, 8, 1e-9, sk, modification="gmres", inject_flags=[(1, 1)])
    assert r0.status == O.NOT_CONVERGED and r0.cycle_m == [0]


def test_rank_deficient_rhs_breaks_down():
    A = W.laplacian_2d(8)
    B = W.gaussian_block(A.n, 3, 1)
    B[:, 2] = 0.0
    r = O.solve(A, B, 5, 1e-8, "bcgsi_ls")
    assert r.status == O.BREAKDOWN


def test_cwy_and_icwy_agree():
    A = W.laplacian_2d(14)
    B = W.gaussian_block(A.n, 4, 2)
    _, H0, _ = O.arnoldi(A, B, 9, "bmgs_cwy")
    _, H1, _ = O.arnoldi(A, B, 9, "bmgs_icwy")
    assert np.linalg.norm(H0 - H1) <= 1e-12 * np.linalg.norm(H0)


def test_low_sync_corrections_on_the_paper_tridiag():
    """On the paper's tridiag with n=100 (Sec. 4: kappa([B, A V_k]) exceeds 1e8
    near step 15), BCGSI+LS keeps O(eps) orthogonality and an Arnoldi relation
    at the rounding level of ||H||; BMGS-ICWY's loss of orthogonality stays far
    below BCGS-PIP's, which flags at step 36 (pinned separately)."""
    A, B = W.paper_tridiag(100)
    V, H, _ = O.arnoldi(A, B, 30, "bcgsi_ls")
    assert O.loss_of_orthogonality(V) < 1e-13
    assert O.arnoldi_residual(A, V, H, 30, 2) <= 3.5e-16 * np.linalg.norm(H)
    V, H, _ = O.arnoldi(A, B, 20, "bmgs_icwy")
    assert O.loss_of_orthogonality(V) < 1e-4


# ------------------------------------------------------------------ global inner product

def _kron_identity(A, s):
    """I_s (x) A in CSR: the operator of the vectorized block system."""
    rows, cols, vals = [], [], []
    D = A.to_dense()
    r, c = np.nonzero(D)
    for b in range(s):
        rows.append(r + b * A.n)
        cols.append(c + b * A.n)
        vals.append(D[r, c])
    return W._from_coo(A.n * s, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def test_global_inner_product_definition():
    """Table 1: block (i, j) of <X, Y> is tr(X_i^T Y_j)/s I_s; for s = 1 it is
    the classical product; the global scaling quotient is ||X||_F/sqrt(s) I_s."""
    rng = np.random.default_rng(7)
    s = 3
    X, Y = rng.standard_normal((40, 2 * s)), rng.standard_normal((40, 3 * s))
    G = O.global_inner(s)(X, Y)
    for i in range(2):
        for j in range(3):
            t = np.trace(X[:, i * s:(i + 1) * s].T @ Y[:, j * s:(j + 1) * s]) / s
            assert np.allclose(G[i * s:(i + 1) * s, j * s:(j + 1) * s], t * np.eye(s), atol=1e-13)
    x, y = rng.standard_normal((40, 4)), rng.standard_normal((40, 4))
    assert np.allclose(O.global_inner(1)(x, y), x.T @ y, atol=1e-13)
    Q, R, flag = O.cholqr(X[:, :s], O.global_inner(s))
    assert not flag
    assert np.allclose(R, np.linalg.norm(X[:, :s]) / np.sqrt(s) * np.eye(s), rtol=1e-14)
    assert np.isclose(np.linalg.norm(Q), np.sqrt(s), rtol=1e-14)


@pytest.mark.parametrize("sk", O.SKELETONS)
def test_global_method_is_the_vectorized_single_vector_method(sk):
    """Under the global inner product a block method on (A, B) is the s = 1
    method on (I_s (x) A, vec B) (the global product is the Euclidean product of
    the vectorized blocks, divided by s): same restart log and steps, the same X,
    and H = h (x) I_s with h the single-vector Hessenberg matrix."""
    A = W.laplacian_2d(12, 11)
    s = 3
    B = W.gaussian_block(A.n, s, 5)
    K = _kron_identity(A, s)
    b = B.T.reshape(-1, 1).copy()
    g = O.solve(A, B, 6, 1e-10, sk, inner_product="global", max_restarts=400)
    c = O.solve(K, b, 6, 1e-10, sk, max_restarts=400)
    assert g.status == c.status == O.OK
    assert g.cycle_m == c.cycle_m and g.steps == c.steps
    Xc = c.X.reshape(s, A.n).T
    assert np.linalg.norm(g.X - Xc) <= 1e-12 * np.linalg.norm(Xc)
    V, H, Beta = O.arnoldi(A, B, 5, sk, inner_product="global")
    v, h, beta = O.arnoldi(K, b, 5, sk)
    assert np.allclose(H, np.kron(h, np.eye(s)), rtol=0, atol=1e-12 * np.abs(h).max())
    assert np.allclose(Beta, beta[0, 0] / np.sqrt(s) * np.eye(s), rtol=1e-14)
    # global block orthonormality: tr(V_i^T V_j)/s = delta_ij
    Gv = O.global_inner(s)(V, V)
    assert np.allclose(Gv, np.eye(6 * s), atol=1e-12)


@pytest.mark.parametrize("sk", ["bmgs", "bmgs_svl", "bmgs_lts", "bmgs_cwy", "bmgs_icwy", "bcgsi_ls",
                                "bcgs_pip"])
def test_paper_tridiag_table_global_rows(sk):
    """Appendix table for tridiag, global rows (gl-skeleton o gl-fom): the
    global inner product with the global muscle reproduces the printed cycle,
    iteration, A-call, V-application and sync counts exactly."""
    g = json.load(open(GOLDEN))
    row = g["global_rows"][sk]
    A, B = W.paper_tridiag(1000)
    Xs = np.linalg.solve(A.to_dense(), B)
    r = O.solve(A, B, 70, 1e-10, sk, modification="fom", max_restarts=100,
                verify_true_residual=False, X_star=Xs, inner_product="global")
    assert r.status == O.OK
    assert (r.cycles, r.steps, r.a_calls, r.v_apps, r.syncs) == \
        (row["cycles"], row["iters"], row["A"], row["V"], row["sync"])


@pytest.mark.parametrize("sk", ["bmgs_svl", "bmgs_lts"])
def test_svl_lts_classical_rows_and_stability(sk):
    """Alg. 5 with the CholQR muscle (reading R13).  The appendix table's
    classical rows use the column muscles MGS-SVL / MGS-LTS; the skeleton still
    takes 2 cycles and 96 +- 2 iterations with the table's identities
    (A-calls = iterations, V = 3 x iterations).  Table 1: loss of
    orthogonality O(eps) kappa, like BMGS, on the paper's tridiag (n = 100),
    where BCGS has already lost orthogonality completely."""
    g = json.load(open(GOLDEN))
    row = g["classical_rows"][sk]
    A, B = W.paper_tridiag(1000)
    Xs = np.linalg.solve(A.to_dense(), B)
    r = O.solve(A, B, 70, 1e-10, sk, modification="fom", max_restarts=100,
                verify_true_residual=False, X_star=Xs)
    assert r.status == O.OK and r.cycles == row["cycles"]
    assert abs(r.steps - row["iters"]) <= 2
    assert row["A"] == row["iters"] and r.a_calls == r.steps
    assert row["V"] == 3 * row["iters"] and r.v_apps == 3 * r.steps
    Ap, Bp = W.paper_tridiag(100)
    V, H, _ = O.arnoldi(Ap, Bp, 20, sk)
    kappa = np.linalg.cond(np.hstack([Bp, Ap.to_dense() @ V[:, :40]]))
    assert O.loss_of_orthogonality(V) <= 100 * np.finfo(float).eps * kappa
    Vb, _, _ = O.arnoldi(Ap, Bp, 20, "bcgs")
    assert O.loss_of_orthogonality(Vb) > 0.1


def test_column_muscles_mgs_svl_lts():
    """Reading R15: MGS-SVL / MGS-LTS give X = Q R with R the (sign-normalised)
    R of Householder QR, 3s - 2 syncs, a unit upper-triangular T, and a loss of
    orthogonality O(eps) kappa(X) like MGS: at kappa = 1e8 and 1e10, where
    CholQR raises the NaN-flag (eps kappa^2 > 1) and classical Gram-Schmidt has
    lost orthogonality completely."""
    rng = np.random.default_rng(3)
    n, s = 200, 8
    U, _ = np.linalg.qr(rng.standard_normal((n, s)))
    Vr, _ = np.linalg.qr(rng.standard_normal((s, s)))
    eps = np.finfo(float).eps
    X0 = rng.standard_normal((n, s))
    Rh = np.linalg.qr(X0)[1]
    Rh = np.diag(np.sign(np.diag(Rh))) @ Rh
    for lts in (False, True):
        Q, R, T, flag, ns = O.mgs_svl(X0, lts)
        assert not flag and ns == 3 * s - 2
        assert np.allclose(R, Rh, rtol=0, atol=1e-12 * np.abs(Rh).max())
        assert np.allclose(np.tril(T, -1), 0.0) and np.all(np.diag(T) == 1.0)
        for kappa in (1e8, 1e10):
            X = U @ np.diag(np.logspace(0, -np.log10(kappa), s)) @ Vr.T
            Q, R, T, flag, ns = O.mgs_svl(X, lts)
            assert not flag
            assert np.linalg.norm(np.eye(s) - Q.T @ Q) <= 100 * eps * kappa
            assert np.linalg.norm(Q @ R - X) <= 1e-14 * np.linalg.norm(X)
            assert O.cholqr(X)[2]


@pytest.mark.parametrize("sk", ["bmgs_svl", "bmgs_lts"])
def test_paper_tridiag_table_classical_svl_lts_with_column_muscles(sk):
    """Appendix table, cl-BMGS-SVL o MGS-SVL and cl-BMGS-LTS o MGS-LTS rows
    (2 cycles, 96 iterations, 584 syncs at s = 2): the same cycles, iterations
    within 2, and the sync identity 6 per iteration + 4 per cycle (Y, the
    3s - 2 = 4 syncs of the column muscle and Z per step; the muscle per cycle
    start), which the printed row satisfies exactly."""
    g = json.load(open(GOLDEN))
    row = g["classical_rows"][sk]
    A, B = W.paper_tridiag(1000)
    Xs = np.linalg.solve(A.to_dense(), B)
    r = O.solve(A, B, 70, 1e-10, sk, modification="fom", max_restarts=100,
                verify_true_residual=False, X_star=Xs, muscle="mgs")
    assert r.status == O.OK and r.cycles == row["cycles"]
    assert abs(r.steps - row["iters"]) <= 2
    assert r.syncs == 6 * r.steps + 4 * r.cycles
    assert row["sync"] == 6 * row["iters"] + 4 * row["cycles"]
    assert r.v_apps == 3 * r.steps and row["V"] == 3 * row["iters"]
