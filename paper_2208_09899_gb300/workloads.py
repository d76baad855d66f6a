"""Seeded synthetic inputs for the block Krylov solver: sparse matrices in CSR
form and block right-hand sides.

This module only builds inputs.  It holds none of the solver's arithmetic, so
that the CPU oracle and the CUDA path can both be fed from it without sharing
any part of the method.

Every generator returns plain numpy arrays:
  rowptr int32 [n+1], colidx int32 [nnz] (sorted within each row, 0-based),
  vals float64 [nnz];  block right-hand sides are float64 (n, s) C-contiguous
  (row-major, a row's s values contiguous).

Workloads (shapes follow the paper's test problems, Sec. 5, Table 5):
  * ``tridiag_const``    A = tridiag(lo, d, up), e.g. tridiag(-1, 4, -1).
  * ``paper_tridiag``    the paper's ``tridiag`` case (Sec. 5.1): off-diagonals
                          1, diagonal -1, -2, ..., -n; B = [1/sqrt(n) * ones, (1..n)].
  * ``laplacian_2d``     5-point Dirichlet Laplacian (stencil 4, -1 x 4),
                          lexicographic ordering (the ``lapl_2d`` shape, Sec. 5.7).
  * ``laplacian_3d``     7-point Dirichlet Laplacian + shift * I.
  * ``rgg_laplacian``    graph Laplacian of a random geometric graph in [0,1)^2
                          with log-uniform edge weights plus a small diagonal
                          shift: an ill-conditioned SPD matrix.
  * ``gaussian_block``   i.i.d. N(0,1) block vector from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    """A square sparse matrix in compressed sparse row form (0-based)."""
    n: int
    rowptr: np.ndarray   # int32 [n+1]
    colidx: np.ndarray   # int32 [nnz]
    vals: np.ndarray     # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        """Dense copy (small n only), by scattering each stored entry."""
        D = np.zeros((self.n, self.n))
        for i in range(self.n):
            for p in range(self.rowptr[i], self.rowptr[i + 1]):
                D[i, self.colidx[p]] += self.vals[p]
        return D


def _from_coo(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> CSR:
    """Sort COO triplets by (row, col) and compress; duplicates are summed."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    key = rows * n + cols
    order = np.argsort(key, kind="stable")
    key, vals = key[order], vals[order]
    uniq, start = np.unique(key, return_index=True)
    summed = np.add.reduceat(vals, start) if len(vals) else vals
    r = (uniq // n).astype(np.int64)
    c = (uniq % n).astype(np.int32)
    counts = np.bincount(r, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2 ** 31:
        raise ValueError("nnz >= 2^31 is not supported by the int32 CSR layout")
    return CSR(n, rowptr.astype(np.int32), c, np.ascontiguousarray(summed))


def tridiag_const(n: int, lo: float = -1.0, d: float = 4.0, up: float = -1.0) -> CSR:
    """tridiag(lo, d, up) of order n."""
    i = np.arange(n)
    rows = np.concatenate([i, i[1:], i[:-1]])
    cols = np.concatenate([i, i[:-1], i[1:]])
    vals = np.concatenate([np.full(n, d), np.full(n - 1, lo), np.full(n - 1, up)])
    return _from_coo(n, rows, cols, vals)


def paper_tridiag(n: int):
    """The paper's ``tridiag`` problem (Sec. 5.1): A has 1 on both off-diagonals
    and -1, -2, ..., -n on the diagonal; B = [ones/sqrt(n), (1, 2, ..., n)^T]."""
    i = np.arange(n)
    rows = np.concatenate([i, i[1:], i[:-1]])
    cols = np.concatenate([i, i[:-1], i[1:]])
    vals = np.concatenate([-(i + 1.0), np.ones(n - 1), np.ones(n - 1)])
    A = _from_coo(n, rows, cols, vals)
    B = np.empty((n, 2))
    B[:, 0] = 1.0 / np.sqrt(n)
    B[:, 1] = i + 1.0
    return A, B


def laplacian_2d(nx: int, ny: int | None = None) -> CSR:
    """5-point Dirichlet Laplacian on an nx x ny grid, lexicographic ordering
    (index = y * nx + x), stencil 4 on the diagonal and -1 for each neighbour."""
    ny = nx if ny is None else ny
    n = nx * ny
    idx = np.arange(n).reshape(ny, nx)
    rows = [idx.ravel()]
    cols = [idx.ravel()]
    vals = [np.full(n, 4.0)]
    for a, b in ((idx[:, 1:], idx[:, :-1]), (idx[:, :-1], idx[:, 1:]),
                 (idx[1:, :], idx[:-1, :]), (idx[:-1, :], idx[1:, :])):
        rows.append(a.ravel())
        cols.append(b.ravel())
        vals.append(np.full(a.size, -1.0))
    return _from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def laplacian_3d(N: int, shift: float = 0.0) -> CSR:
    """7-point Dirichlet Laplacian on an N^3 grid (stencil 6, -1 x 6) + shift*I,
    lexicographic ordering i = (z*N + y)*N + x.  Built row by row in column
    order (offsets -N^2, -N, -1, 0, +1, +N, +N^2), no sort needed."""
    n = N ** 3
    i = np.arange(n, dtype=np.int64)
    x, y, z = i % N, (i // N) % N, i // (N * N)
    offs = (-N * N, -N, -1, 0, 1, N, N * N)
    ok = (z > 0, y > 0, x > 0, np.ones(n, bool), x < N - 1, y < N - 1, z < N - 1)
    cols = np.stack([i + o for o in offs], axis=1)
    mask = np.stack(ok, axis=1)
    vals = np.where(np.arange(7) == 3, 6.0 + shift, -1.0)
    vals = np.broadcast_to(vals, (n, 7))
    rowptr = np.zeros(n + 1, dtype=np.int32)
    np.cumsum(mask.sum(axis=1), out=rowptr[1:])
    return CSR(n, rowptr, cols[mask].astype(np.int32), np.ascontiguousarray(vals[mask]))


def rgg_laplacian(n: int, seed: int = 0, avg_degree: float = 6.0,
                  wmin: float = 1e-3, wmax: float = 1e3, rel_shift: float = 1e-6) -> CSR:
    """Laplacian of a random geometric graph plus a small diagonal shift.

    Points are uniform in [0,1)^2; i and j are joined when |p_i - p_j| < r with
    r = sqrt(avg_degree / (pi n)) (expected degree avg_degree, ignoring the
    boundary).  Edge weights are 10^U(log10 wmin, log10 wmax).  The matrix is
    L = D - W + rel_shift * max(diag(D)) * I, symmetric positive definite and
    ill-conditioned.  Neighbours are found with a k-d tree
    (scipy.spatial.cKDTree.query_pairs); pairs are sorted so the result is
    independent of the tree's traversal order.
    """
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 2))
    r = np.sqrt(avg_degree / (np.pi * n))
    pairs = cKDTree(pts).query_pairs(r, output_type="ndarray")
    pairs = pairs[np.lexsort((pairs[:, 1], pairs[:, 0]))]
    I = pairs[:, 0].astype(np.int64)
    J = pairs[:, 1].astype(np.int64)
    w = 10.0 ** rng.uniform(np.log10(wmin), np.log10(wmax), size=len(I))
    deg = np.bincount(I, weights=w, minlength=n) + np.bincount(J, weights=w, minlength=n)
    shift = rel_shift * deg.max()
    rows = np.concatenate([I, J, np.arange(n)])
    cols = np.concatenate([J, I, np.arange(n)])
    vals = np.concatenate([-w, -w, deg + shift])
    return _from_coo(n, rows, cols, vals)


def gaussian_block(n: int, s: int, seed: int = 0) -> np.ndarray:
    """i.i.d. N(0,1) n x s block, row-major, from numpy's PCG64 with ``seed``."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.standard_normal((n, s)))


# Named workloads with the paper-shaped sizes used by the tests and the bench.
def workload(name: str, seed: int = 0):
    """Return (A, B) for a named workload.

    tridiag2000_s4     A = tridiag(-1,4,-1), n=2000, B 2000x4 N(0,1)
    lapl512_s8         2D Laplacian 512x512 (n=262144), B n x 8 N(0,1)
    rgg1M_s16          random geometric graph Laplacian, n=2^20, B n x 16
    lapl2048_s16       2D Laplacian 2048x2048 (n=4194304), B n x 16
    """
    if name == "tridiag2000_s4":
        return tridiag_const(2000), gaussian_block(2000, 4, seed)
    if name == "lapl512_s8":
        return laplacian_2d(512), gaussian_block(512 * 512, 8, seed)
    if name == "rgg1M_s16":
        n = 1 << 20
        return rgg_laplacian(n, seed), gaussian_block(n, 16, seed + 1000)
    if name == "lapl2048_s16":
        return laplacian_2d(2048), gaussian_block(2048 * 2048, 16, seed)
    raise KeyError(name)
