"""Mutation check of the oracle's pins: plant a plausible mistake in a copy of
the oracle (on the CPU) and confirm that at least one pin catches it."""
import importlib.util
import os
import sys
import types

import numpy as np
import pytest

from paper_2208_09899_gb300 import workloads as W

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "lsba_oracle.py")

MUTATIONS = {
    # sign of the Pythagorean correction in PIP (Alg. 3)
    "pip_sign": ("R, flag = chol_flag(Om - Hc.T @ Hc, piv)", "R, flag = chol_flag(Om + Hc.T @ Hc, piv)"),
    # dropped Y^T Z term in BCGSI+LS (Alg. 7)
    "ls_drop_term": ("P = left_solve_upper_T(R, Pt - Y.T @ Z)", "P = left_solve_upper_T(R, Pt)"),
    # ICWY uses T instead of T^{-T} (Alg. 6, blue)
    "icwy_no_solve": ("Hc = unit_upper_T_solve(self.T[:k * s, :k * s], ZP)", "Hc = ZP"),
    # ICWY: V_{k-1} instead of V_k in the U update (reading R3) -- omit the new V_k
    "icwy_vkm1": ("self.U = right_solve_upper(W, R) - self.basis(k) @ Hc",
                  "self.U = right_solve_upper(W, R) - self.basis(k - 1) @ Hc[:(k - 1) * s]"),
    # cospatial factor multiplied on the wrong side (Sec. 2.4.2)
    "C_order": ("C = c @ C", "C = C @ c"),
    # BGMRES modification without the transpose of H_m (Sec. 2.4.1)
    "gmres_no_T": ("Mvec = np.linalg.solve(Hj.T, Ej @ (Hsub.T @ Hsub))",
                   "Mvec = np.linalg.solve(Hj, Ej @ (Hsub.T @ Hsub))"),
    # estimate without the cospatial factor C (Eq. (9))
    "est_no_C": ("return np.linalg.norm(np.vstack([Mvec, -Hsub]) @ c @ C) / normB",
                 "return np.linalg.norm(np.vstack([Mvec, -Hsub]) @ c) / normB"),
    # BCGSI+LS keeps H_{1:k-1,k-1} = J without the +Y correction (reading R4)
    "ls_no_Y": ("self.set_Hcol(1, k - 1, k - 1, self.J + Y)", "self.set_Hcol(1, k - 1, k - 1, self.J)"),
    # chol reads the lower triangle (R1)
    "chol_lower": ("R[j, c] = (G[j, c] - np.dot(R[:j, j], R[:j, c])) / R[j, j]",
                   "R[j, c] = (G[c, j] * 1.0000001 - np.dot(R[:j, j], R[:j, c])) / R[j, j]"),
    # adaptive restart keeps the flagged relation (Sec. 4)
    "restart_off_by_one": ("m_cur = flagged - 1", "m_cur = flagged"),
    # sign of the Pythagorean correction in PIO (Alg. 4)
    "pio_sign": ("R, flag = chol_flag(RW.T @ RW - RH.T @ RH)", "R, flag = chol_flag(RW.T @ RW + RH.T @ RH)"),
    # PIO's muscle factor of H taken from H H^T's wrong side
    "pio_HHt": ("RH, flag_h = chol_flag(Hc.T @ Hc)", "RH, flag_h = chol_flag(Hc[-Hc.shape[1]:] @ Hc[-Hc.shape[1]:].T)"),
    # SVL's T column without its sign (Alg. 5, red)
    "svl_sign": ("self.T[:k * s, k * s:(k + 1) * s] = (Z if self.lts else -Tk @ Z) @ Tm",
                 "self.T[:k * s, k * s:(k + 1) * s] = (Z if self.lts else Tk @ Z) @ Tm"),
    # LTS multiplies by T^T instead of solving with it (Alg. 5, blue)
    "lts_mult": ("Hc = unit_upper_T_solve(Tk, Y) if self.lts else Tk.T @ Y", "Hc = Tk.T @ Y"),
    # MGS-SVL's T column without its sign (column muscle, reading R15)
    "mgs_svl_sign": ("T[:j, j] = z if lts else -(T[:j, :j] @ z)", "T[:j, j] = z if lts else (T[:j, :j] @ z)"),
    # MGS-LTS multiplies by T^T instead of solving with it
    "mgs_lts_mult": ("r = unit_upper_T_solve(T[:j, :j], y[:, None])[:, 0] if lts else T[:j, :j].T @ y",
                     "r = T[:j, :j].T @ y"),
    # global inner product without the 1/s of Table 1
    "global_no_scale": ("t = np.sum(X[:, i * s:(i + 1) * s] * Y[:, j * s:(j + 1) * s]) / s",
                        "t = np.sum(X[:, i * s:(i + 1) * s] * Y[:, j * s:(j + 1) * s])"),
    # global inner product summing every entry product of the two blocks (not the trace)
    "global_all_pairs": ("t = np.sum(X[:, i * s:(i + 1) * s] * Y[:, j * s:(j + 1) * s]) / s",
                         "t = np.sum(X[:, i * s:(i + 1) * s].T @ Y[:, j * s:(j + 1) * s]) / s"),
}


def _load_mutant(name):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    mod = types.ModuleType(f"lsba_oracle_mutant_{name}")
    sys.modules[mod.__name__] = mod
    exec(compile(src.replace(old, new), SRC, "exec"), mod.__dict__)
    return mod


def _pins_pass(O):
    """A compact subset of the pins in test_oracle.py; True if all hold."""
    try:
        # Low-sync corrections (Y-terms) vanish in exact arithmetic: only the
        # loss of orthogonality on a fast-converging problem shows them (Table 2).
        At = W.tridiag_const(300)
        Bt = W.gaussian_block(300, 3, 0)
        for sk in ("bmgs", "bmgs_cwy", "bmgs_icwy", "bcgsi_ls"):
            V, H, _ = O.arnoldi(At, Bt, 12, sk)
            kappa = np.linalg.cond(np.hstack([Bt, At.to_dense() @ V[:, :36]]))
            if O.loss_of_orthogonality(V) > 100 * np.finfo(float).eps * kappa:
                return False
        # The paper's tridiag (n=100), where kappa([B, A V]) grows past 1e8 within
        # ~15 steps (Sec. 4): ICWY's T-solve and BCGSI+LS's Y-corrections decide
        # the loss of orthogonality and the Arnoldi relation there.
        Ap, Bp = W.paper_tridiag(100)
        V, H, _ = O.arnoldi(Ap, Bp, 20, "bmgs_icwy")
        if O.loss_of_orthogonality(V) > 1e-4:
            return False
        for sk in ("bmgs_svl", "bmgs_lts"):
            V, H, _ = O.arnoldi(Ap, Bp, 20, sk)
            kappa = np.linalg.cond(np.hstack([Bp, Ap.to_dense() @ V[:, :40]]))
            if O.loss_of_orthogonality(V) > 100 * np.finfo(float).eps * kappa:
                return False
        V, H, _ = O.arnoldi(Ap, Bp, 30, "bcgsi_ls")
        if O.loss_of_orthogonality(V) > 1e-12:
            return False
        if O.arnoldi_residual(Ap, V, H, 30, 2) > 3.5e-16 * np.linalg.norm(H):
            return False
        # A nonsymmetric matrix, so that H_m^T differs from H_m.
        A = W.tridiag_const(196, -1.3, 4.0, -0.6)
        B = W.gaussian_block(A.n, 3, 2)
        for sk in O.SKELETONS:
            V, H, Beta = O.arnoldi(A, B, 8, sk)
            if O.arnoldi_residual(A, V, H, 8, 3) > 1e-12 * np.linalg.norm(V):
                return False
            if O.loss_of_orthogonality(V) > (1e-6 if sk in ("bcgs_pip", "bcgs_pio") else 1e-10):
                return False
            rhs = np.zeros((27, 3))
            rhs[:3] = Beta
            Xi = O.cycle_coefficients(H, 8, 3, Beta, "gmres")[1]
            if np.linalg.norm(Xi - np.linalg.lstsq(H, rhs, rcond=None)[0]) > 1e-9 * np.linalg.norm(Xi):
                return False
        for mod in ("fom", "gmres"):
            for cyc in (1, 2, 3):
                r = O.solve(A, B, 5, 1e-30, "bcgsi_ls", modification=mod, max_restarts=cyc - 1,
                            verify_true_residual=False, true_residual_each_cycle=True)
                if abs(r.relres_true - r.est_history[-1][2]) > 1e-7 * r.relres_true:
                    return False
        G = np.array([[4.0, 2.0], [2.0, 3.0]])
        if not np.allclose(O.chol_flag(G)[0], np.linalg.cholesky(G).T):
            return False
        r = O.solve(A, B, 8, 1e-9, "bcgs_pip", inject_flags=[(1, 5)])
        if r.cycle_m[0] != 4 or any(mc != 4 for mc in r.m_cur[1:]):
            return False
        # Column muscles: loss of orthogonality O(eps) kappa at kappa = 1e10.
        rng = np.random.default_rng(3)
        Uq, _ = np.linalg.qr(rng.standard_normal((200, 8)))
        Vq, _ = np.linalg.qr(rng.standard_normal((8, 8)))
        Xm = Uq @ np.diag(np.logspace(0, -10, 8)) @ Vq.T
        for lts in (False, True):
            Qm, Rm, Tm, fm, _ = O.mgs_svl(Xm, lts)
            if fm or np.linalg.norm(np.eye(8) - Qm.T @ Qm) > 100 * np.finfo(float).eps * 1e10:
                return False
        # Global inner product: the block method is the single-vector method on
        # (I_s (x) A, vec B) (Table 1).
        Ag = W.laplacian_2d(9, 8)
        Bg = W.gaussian_block(Ag.n, 2, 5)
        D = Ag.to_dense()
        r_, c_ = np.nonzero(D)
        K = W._from_coo(2 * Ag.n, np.concatenate([r_, r_ + Ag.n]), np.concatenate([c_, c_ + Ag.n]),
                        np.concatenate([D[r_, c_], D[r_, c_]]))
        g = O.solve(Ag, Bg, 5, 1e-10, "bcgsi_ls", inner_product="global", max_restarts=300)
        c = O.solve(K, Bg.T.reshape(-1, 1).copy(), 5, 1e-10, "bcgsi_ls", max_restarts=300)
        if g.steps != c.steps or np.linalg.norm(g.X - c.X.reshape(2, Ag.n).T) > 1e-12 * np.linalg.norm(g.X):
            return False
        return True
    except Exception:
        return False


def test_unmutated_oracle_passes_the_compact_pins():
    spec = importlib.util.spec_from_file_location("lsba_oracle_clean", SRC)
    mod = importlib.util.module_from_spec(spec)
    sys.modules["lsba_oracle_clean"] = mod
    spec.loader.exec_module(mod)
    assert _pins_pass(mod)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    assert not _pins_pass(_load_mutant(name))
