"""FP64 on the tensor cores (exact digit products): the Gram and update
kernels against the oracle's FP64 products, and solves at s = 8 in FP64
(lagged skeletons, BCGS-PIP, BCGS-PIO, BCGS), which run on them, against the
oracle.

Bound of the kernels (per output entry): every value is represented to
2^-53 of its (128-row tile, column) maximum, so a product term L_ri R_rj is
in error by at most 2^-53 (ML |R_rj| + |L_ri| MR) + 2^-55 ML MR (ML, MR the
tile maxima of the two columns, the last term for the dropped digit levels),
and the FP64 accumulation over tiles and CTAs adds at most ~2^-53 per
addition; the reference product itself is FP64 (error <= n 2^-53 |L|^T |R|,
far less in practice).  The tests assert the error is below 4 times the sum
of these terms."""
import numpy as np
import pytest

from oracle import lsba_oracle as O
from paper_2208_09899_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U53 = 2.0 ** -53


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_09899_gb300 import build, lsba
    build.build()
    lsba.load()
    return torch, lsba


def _tile_max(X):
    n = X.shape[0]
    t = (n + 127) // 128
    pad = np.zeros((t * 128, X.shape[1]))
    pad[:n] = np.abs(X)
    return np.repeat(pad.reshape(t, 128, -1).max(axis=1), 128, axis=0)[:n]


def _bound(Lh, Rh):
    ML, MR = _tile_max(Lh), _tile_max(Rh)
    aL, aR = np.abs(Lh), np.abs(Rh)
    n = Lh.shape[0]
    terms = ML.T @ aR + aL.T @ MR + 0.25 * (ML.T @ MR)
    return 4 * (U53 * terms + (n // 128 + 64) * U53 * (aL.T @ aR))


def _blocks(rng, k, n, s=8):
    return rng.standard_normal((k, n, s)) * np.exp(rng.uniform(-4, 4, size=(k, 1, s)))


@pytest.mark.parametrize("a,b,n", [(1, 1, 1), (1, 1, 1000), (2, 2, 1000), (3, 1, 70001),
                                   (16, 2, 4099), (17, 2, 262147), (21, 2, 70001), (23, 1, 31),
                                   (22, 2, 5003), (8, 2, 128), (5, 2, 129)])
def test_gram_fp64tc_matches_oracle(env, a, b, n):
    torch, lsba = env
    rng = np.random.default_rng(a * 31 + b + n)
    L = _blocks(rng, a, n)
    R = _blocks(rng, b, n)
    sv = lsba.Solver(0)
    dL, dR = torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()
    dG = torch.empty((a * 8, b * 8), dtype=torch.float64, device="cuda")
    sv.gram_fp64tc(dL, dR, dG)
    G = dG.cpu().numpy()
    Lh, Rh = np.hstack(list(L)), np.hstack(list(R))
    ref = O.inner(Lh, Rh)
    err = np.abs(G - ref)
    bound = _bound(Lh, Rh)
    print(f"GRAMF64 a={a} b={b} n={n} max err/bound {np.max(err / bound):.2e} "
          f"err/(|L|^T|R|) {np.max(err / O.inner(np.abs(Lh), np.abs(Rh))):.2e}")
    assert np.all(err <= bound)
    sv.gram_fp64tc(dL, dR, dG)
    assert np.array_equal(G, dG.cpu().numpy())


def test_gram_fp64tc_special_values(env):
    """Zero columns, a value 2^1000 and one of 2^-1060 (subnormal) in the same
    blocks, and a NaN that must reach the output."""
    torch, lsba = env
    rng = np.random.default_rng(7)
    n = 1000
    L = rng.standard_normal((3, n, 8))
    R = rng.standard_normal((2, n, 8))
    L[0, :, 3] = 0.0
    L[1, 17, 2] = 2.0 ** 500
    R[0, 17, 5] = 2.0 ** 490
    L[2, 400, 1] = 2.0 ** -1060
    sv = lsba.Solver(0)
    dG = torch.empty((24, 16), dtype=torch.float64, device="cuda")
    sv.gram_fp64tc(torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda(), dG)
    G = dG.cpu().numpy()
    Lh, Rh = np.hstack(list(L)), np.hstack(list(R))
    ref = O.inner(Lh, Rh)
    assert np.all(np.isfinite(G))
    assert np.all(np.abs(G - ref) <= _bound(Lh, Rh))
    L[1, 5, 0] = np.nan
    sv.gram_fp64tc(torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda(), dG)
    assert np.all(np.isnan(dG.cpu().numpy()))


@pytest.mark.parametrize("nin,n,tri,two", [(1, 1000, True, False), (2, 70001, False, True),
                                           (3, 4099, True, True), (16, 262147, True, True),
                                           (17, 40003, False, True), (22, 9999, True, True),
                                           (24, 31, True, True), (7, 128, False, False)])
def test_combine_fp64tc_matches_oracle(env, nin, n, tri, two):
    torch, lsba = env
    rng = np.random.default_rng(nin * 7 + n)
    IN = _blocks(rng, nin, n)
    C1 = rng.standard_normal((nin * 8, 8)) * np.exp(rng.uniform(-3, 3, size=(nin * 8, 1)))
    C2 = rng.standard_normal((nin * 8, 8))
    T = np.triu(rng.standard_normal((8, 8))) + 4 * np.eye(8)
    sv = lsba.Solver(0)
    dIN = torch.from_numpy(IN).cuda()
    d1 = torch.empty((n, 8), dtype=torch.float64, device="cuda")
    d2 = torch.empty((n, 8), dtype=torch.float64, device="cuda") if two else None
    sv.combine_fp64tc(dIN, torch.from_numpy(C1).cuda(), torch.from_numpy(T).cuda() if tri else None,
                      d1, torch.from_numpy(C2).cuda() if two else None, d2)
    INh = np.hstack(list(IN))
    # the kernel folds T into the coefficients first: C1' = C1 T^-1 (FP64)
    C1f = O.right_solve_upper(C1, T) if tri else C1
    ML = _tile_max(INh)
    aI = np.abs(INh)
    K = INh.shape[1]
    for got, Cf in ((d1, C1f),) + (((d2, C2),) if two else ()):
        g = got.cpu().numpy()
        ref = INh @ Cf
        aC = np.abs(Cf)
        # the coefficients are scaled by the inputs' tile exponents and split
        # per output column: their error per term is bounded by the largest
        # scaled term max_k ML[r, k] |C[k, j]| of the row's tile
        mterm = np.stack([np.max(ML * aC[:, j][None, :], axis=1) for j in range(8)], axis=1)
        bound = 4 * U53 * (ML @ aC + 2.5 * K * mterm) + 64 * U53 * (aI @ aC)
        err = np.abs(g - ref)
        print(f"COMBF64 nin={nin} n={n} max err/bound {np.max(err / bound):.2e} "
              f"err/(|in||C|) {np.max(err / (aI @ aC)):.2e}")
        assert np.all(err <= bound)


_SK8 = ["bcgsi_ls", "bmgs_icwy", "bmgs_cwy", "bcgs_pip", "bcgs_pio", "bcgs"]


def _cmp(lsba, A, B, m, tol, sk, mod, **kw):
    from tests.test_gpu_parity import _compare_solve
    X, st, hist, ref = _compare_solve(lsba, A, B, m, tol, sk, mod, precision="fp64", **kw)
    assert st["precision"] == lsba.PRECISIONS["fp64"] and st["tensor_cores"] == 1
    return X, st, hist, ref


@pytest.mark.parametrize("mod", ["gmres", "fom"])
@pytest.mark.parametrize("sk", _SK8)
def test_fp64_tensor_core_solves(env, sk, mod):
    """The lagged skeletons, BCGS-PIP, BCGS-PIO and BCGS at s = 8 in FP64 run
    their Gram and update passes on the digit kernels: the oracle's restart
    log, counters, first-cycle Grams and Hessenberg within 1e-11, estimates,
    and X within 1e-8."""
    torch, lsba = env
    A = W.laplacian_2d(40, 37)
    B = W.gaussian_block(A.n, 8, 3)
    _cmp(lsba, A, B, 8, 1e-10, sk, mod, max_restarts=200)


@pytest.mark.parametrize("sk", _SK8)
def test_fp64_tensor_core_injected_flag_and_global(env, sk):
    torch, lsba = env
    A = W.laplacian_2d(30)
    B = W.gaussian_block(A.n, 8, 4)
    X, st, hist, ref = _cmp(lsba, A, B, 8, 1e-9, sk, "gmres", max_restarts=300,
                            inject_flag_cycle=1, inject_flag_relation=5)
    assert hist["cycle_m"][0] == 4
    _cmp(lsba, A, B, 8, 1e-9, sk, "gmres", max_restarts=300, inner_product="global")


def test_fp64_tensor_cores_off_uses_fp64_kernels(env):
    """tensor_cores = 0 keeps the native FP64 kernels; both paths match the
    oracle and each other to the solve tolerances."""
    torch, lsba = env
    A = W.laplacian_2d(33, 29)
    B = W.gaussian_block(A.n, 8, 6)
    X1, st1, _, _ = _cmp(lsba, A, B, 10, 1e-10, "bcgsi_ls", "gmres", max_restarts=300)
    from tests.test_gpu_parity import _compare_solve
    X0, st0, _, _ = _compare_solve(lsba, A, B, 10, 1e-10, "bcgsi_ls", "gmres", max_restarts=300,
                                   precision="fp64", tensor_cores=0)
    assert st0["tensor_cores"] == 0
    assert np.linalg.norm(X1 - X0) <= 1e-8 * np.linalg.norm(X0)
