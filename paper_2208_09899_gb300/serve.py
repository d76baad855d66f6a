"""Continuous-batching solve server for block linear systems A X = B.

Requests (a CSR matrix, a block right-hand side, a basis size m, a tolerance and
a skeleton) arrive over time.  A request is admitted when a worker slot is free
and the device memory its solve needs (lib `lsba_workspace_bytes`: the Krylov
basis, its Hessenberg and small matrices, the matrix and block copies) fits
under the server's HBM cap next to the requests already running.  Admission is
first-in first-out with backfill: when the oldest waiting request does not fit,
a younger one that fits may start, unless the oldest has waited longer than
`max_backfill_wait` seconds.

Each slot owns one solver handle and one CUDA stream, so admitted solves run
concurrently on the GPU; the library allocates and releases its workspace in
stream order (no device-wide synchronisation), keeps each basis and its
Hessenberg matrix on the device across all restart cycles of its solve, and
returns the workspace to the device pool when the solve ends.  Every kernel is
deterministic (fixed-order reductions), so a request's result does not depend
on what else is running.

The solver call is pluggable (``solve_fn_factory``) so that the scheduling can be
exercised without a GPU.
"""
from __future__ import annotations

import collections
import threading
import time
from dataclasses import dataclass

import numpy as np


@dataclass
class Request:
    rid: int
    A: object                 # workloads.CSR
    B: np.ndarray             # (n, s) float64
    m: int
    tol: float
    skeleton: str = "bcgsi_ls"
    modification: str = "gmres"
    precision: str = "auto"
    max_restarts: int = 500
    arrival: float = 0.0      # seconds after the server's start

    @property
    def n(self):
        return self.A.n

    @property
    def s(self):
        return self.B.shape[1]


@dataclass
class Result:
    rid: int
    X: np.ndarray | None
    stats: dict
    arrival: float
    start: float
    end: float
    slot: int
    need_bytes: int

    @property
    def latency(self):
        return self.end - self.arrival

    @property
    def wait(self):
        return self.start - self.arrival


def request_bytes(req: Request) -> int:
    """Device memory of one request: the library's workspace bound plus the
    device copies of A, B and X the slot makes."""
    from . import lsba
    ws = lsba.workspace_bytes(req.n, req.A.nnz, req.s, req.m)
    copies = req.A.nnz * 12 + (req.n + 1) * 4 + 2 * req.n * req.s * 8
    return int(ws + copies)


class _GpuSlot:
    """One worker slot: a solver handle on its own CUDA stream."""

    def __init__(self, device: int):
        import torch

        from . import lsba
        self.torch = torch
        self.lsba = lsba
        self.device = device
        self.stream = torch.cuda.Stream(device=device)
        self.solver = lsba.Solver(device, stream=self.stream)

    def __call__(self, req: Request):
        torch, lsba = self.torch, self.lsba
        dev = f"cuda:{self.device}"
        with torch.cuda.stream(self.stream):
            dA = lsba.DeviceCSR.from_host(req.A, dev)
            dB = torch.from_numpy(np.ascontiguousarray(req.B)).to(dev)
            dX = torch.empty_like(dB)
            self.solver.set_options(modification=req.modification, max_restarts=req.max_restarts,
                                    precision=req.precision)
            self.solver.solve(dA, dB, dX, req.m, req.tol, req.skeleton)
            X = dX.cpu().numpy()
            st = self.solver.stats()
            self.solver.release_workspace()
            self.stream.synchronize()
        return X, st

    def close(self):
        self.solver.close()


class SolveServer:
    """Admission-controlled concurrent solver (see the module docstring).

    slots:            concurrent solves (worker threads, one stream each)
    hbm_cap_bytes:    admission cap on the summed memory of running requests
    solve_fn_factory: slot index -> callable(Request) -> (X, stats); default: a
                      GPU slot on ``device``
    need_fn:          Request -> bytes (default: request_bytes)
    """

    def __init__(self, slots: int = 8, hbm_cap_bytes: float = 150e9, device: int = 0,
                 solve_fn_factory=None, need_fn=None, max_backfill_wait: float = 5.0):
        self.slots = slots
        self.cap = float(hbm_cap_bytes)
        self.max_backfill_wait = max_backfill_wait
        self.need_fn = need_fn or request_bytes
        self._factory = solve_fn_factory or (lambda i: _GpuSlot(device))
        self._lock = threading.Condition()
        self._pending: collections.deque = collections.deque()
        self._in_use = 0.0
        self._peak = 0.0
        self._running = 0
        self._closed = False
        self._results: list[Result] = []
        self._t0 = None
        self._workers = []
        self._slot_fns = [self._factory(i) for i in range(slots)]

    # -- admission ---------------------------------------------------------
    def _pick(self, now):
        """Index of the pending request to start now, or None (lock held).

        A request starts when its memory fits next to the running ones; one
        larger than the whole cap starts only on an idle server (it then
        reports its own allocation error, if any).  Younger requests are
        considered only while the oldest has waited at most max_backfill_wait."""
        for i, (req, need) in enumerate(self._pending):
            if req.arrival > now:
                break
            if self._in_use + need <= self.cap or (need > self.cap and self._running == 0):
                return i
            if i == 0 and now - req.arrival > self.max_backfill_wait:
                return None
        return None

    def _worker(self, slot: int):
        fn = self._slot_fns[slot]
        while True:
            with self._lock:
                while True:
                    if self._closed and not self._pending:
                        return
                    i = self._pick(time.perf_counter() - self._t0)
                    if i is not None:
                        req, need = self._pending[i]
                        del self._pending[i]
                        self._in_use += need
                        self._peak = max(self._peak, self._in_use)
                        self._running += 1
                        break
                    self._lock.wait(0.002)
            start = time.perf_counter() - self._t0
            try:
                X, st = fn(req)
            except Exception as exc:  # a failed solve is reported, not fatal
                X, st = None, {"error": repr(exc)}
            end = time.perf_counter() - self._t0
            with self._lock:
                self._in_use -= need
                self._running -= 1
                self._results.append(Result(req.rid, X, st, req.arrival, start, end, slot, need))
                self._lock.notify_all()

    # -- public ------------------------------------------------------------
    def run(self, requests, keep_x: bool = True):
        """Serve ``requests`` (their ``arrival`` times are honoured, in seconds
        from now) and return the results in request-id order."""
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        self._results = []
        self._closed = False
        self._t0 = time.perf_counter()
        with self._lock:
            for r in reqs:
                self._pending.append((r, self.need_fn(r)))
        self._workers = [threading.Thread(target=self._worker, args=(i,), daemon=True)
                         for i in range(self.slots)]
        for t in self._workers:
            t.start()
        with self._lock:
            self._closed = True
            self._lock.notify_all()
        for t in self._workers:
            t.join()
        out = sorted(self._results, key=lambda r: r.rid)
        if not keep_x:
            for r in out:
                r.X = None
        return out

    @property
    def peak_bytes(self):
        return self._peak

    def close(self):
        for fn in self._slot_fns:
            if hasattr(fn, "close"):
                fn.close()


def summarize(results, t_first=None):
    """p50/p99 latency, mean wait, solves/s of a served batch."""
    lat = np.array([r.latency for r in results])
    t0 = min(r.arrival for r in results) if t_first is None else t_first
    t1 = max(r.end for r in results)
    ok = sum(1 for r in results if r.stats.get("status", -1) == 0)
    errors = sorted({r.stats["error"] for r in results if "error" in r.stats})
    return {"requests": len(results), "converged": ok, "errors": errors,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_wait_s": float(np.mean([r.wait for r in results])),
            "solves_per_s": len(results) / max(t1 - t0, 1e-9), "makespan_s": t1 - t0}


def poisson_arrivals(count: int, rate: float, seed: int = 0):
    """Arrival times (s) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def serving_requests(count: int, seed: int = 0, side_range=(22, 100), s_choices=(1, 4, 8, 16, 32),
                     m_range=(8, 32), tol: float = 1e-8, precision: str = "auto",
                     max_restarts: int = 500):
    """Seeded request mix: 3D 7-point Laplacian + delta I with delta ~ U[0, 0.1],
    grid side N ~ U{side_range} (n = N^3), s ~ U{s_choices}, m ~ U{m_range},
    B ~ N(0, 1).  The Laplacian of each side is built once; a request copies its
    values and adds its own delta on the diagonal."""
    from . import workloads as W
    rng = np.random.default_rng(seed)
    base, diag = {}, {}
    reqs = []
    for i in range(count):
        N = int(rng.integers(side_range[0], side_range[1] + 1))
        delta = float(rng.uniform(0.0, 0.1))
        s = int(rng.choice(s_choices))
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        if N not in base:
            L = W.laplacian_3d(N)
            rows = np.repeat(np.arange(L.n), np.diff(L.rowptr))
            base[N], diag[N] = L, np.flatnonzero(rows == L.colidx)
        L = base[N]
        vals = L.vals.copy()
        vals[diag[N]] += delta
        A = W.CSR(L.n, L.rowptr, L.colidx, vals)
        B = W.gaussian_block(A.n, s, seed * 100003 + i)
        reqs.append(Request(i, A, B, m, tol, precision=precision, max_restarts=max_restarts))
    return reqs
