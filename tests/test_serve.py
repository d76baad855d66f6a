"""Continuous-batching server: admission and scheduling on the CPU with a fake
solver; on the GPU, each served result equals the same request solved alone."""
import threading
import time
from types import SimpleNamespace

import numpy as np
import pytest

from paper_2208_09899_gb300 import serve


class Tracker:
    """Fake solver slots that sleep and record what ran concurrently."""

    def __init__(self, need_fn, fail_ids=()):
        self.lock = threading.Lock()
        self.need_fn = need_fn
        self.running = {}
        self.max_bytes = 0.0
        self.max_running = 0
        self.log = []          # (event, rid, running ids)
        self.fail_ids = set(fail_ids)

    def factory(self, slot):
        def run(req):
            with self.lock:
                self.running[req.rid] = self.need_fn(req)
                self.max_bytes = max(self.max_bytes, sum(self.running.values()))
                self.max_running = max(self.max_running, len(self.running))
                self.log.append(("start", req.rid, tuple(sorted(self.running))))
            time.sleep(req.m * 1e-3)
            with self.lock:
                del self.running[req.rid]
            if req.rid in self.fail_ids:
                raise RuntimeError("fake failure")
            return np.full((req.n, req.s), float(req.rid)), {"status": 0}
        return run


def fake(rid, n, s=1, m=5, arrival=0.0):
    A = SimpleNamespace(n=n, nnz=3 * n)
    return serve.Request(rid, A, np.zeros((n, s)), m, 1e-8, arrival=arrival)


def need(req):
    return float(req.n)


def test_cap_and_slots_respected():
    rng = np.random.default_rng(0)
    reqs = [fake(i, int(rng.integers(10, 60)), m=int(rng.integers(2, 8))) for i in range(40)]
    tr = Tracker(need)
    srv = serve.SolveServer(slots=4, hbm_cap_bytes=100, solve_fn_factory=tr.factory, need_fn=need)
    out = srv.run(reqs)
    assert [r.rid for r in out] == list(range(40))
    assert tr.max_bytes <= 100 and srv.peak_bytes <= 100
    assert tr.max_running <= 4
    assert tr.max_running >= 2          # it does run requests concurrently
    for r in out:
        assert r.X[0, 0] == r.rid and r.start >= r.arrival and r.end >= r.start


def test_backfill_and_strict_fifo():
    # rid 0 (60) runs; rid 1 (60) does not fit next to it; rid 2 (30) does.
    reqs = [fake(0, 60, m=40), fake(1, 60, m=5), fake(2, 30, m=5)]
    tr = Tracker(need)
    srv = serve.SolveServer(slots=3, hbm_cap_bytes=100, solve_fn_factory=tr.factory, need_fn=need,
                            max_backfill_wait=10.0)
    out = srv.run(reqs)
    assert out[2].start < out[1].start          # backfilled past the blocked head
    assert out[1].start >= out[0].end - 1e-3    # the head waited for memory
    # With no backfill allowed, requests start in arrival order.
    tr = Tracker(need)
    srv = serve.SolveServer(slots=3, hbm_cap_bytes=100, solve_fn_factory=tr.factory, need_fn=need,
                            max_backfill_wait=0.0)
    out = srv.run(reqs)
    starts = [r.start for r in out]
    assert starts[1] <= starts[2] + 1e-4


def test_oversized_runs_alone_and_failure_reported():
    reqs = [fake(0, 50, m=10), fake(1, 500, m=5), fake(2, 50, m=10), fake(3, 20, m=3)]
    tr = Tracker(need, fail_ids={3})
    srv = serve.SolveServer(slots=4, hbm_cap_bytes=100, solve_fn_factory=tr.factory, need_fn=need,
                            max_backfill_wait=0.0)
    out = srv.run(reqs)
    starts = {rid: running for ev, rid, running in tr.log if ev == "start"}
    assert starts[1] == (1,)                    # the request above the cap ran alone
    assert out[3].X is None and "fake failure" in out[3].stats["error"]
    assert all(out[i].stats.get("status") == 0 for i in range(3))
    sm = serve.summarize(out)
    assert sm["converged"] == 3 and len(sm["errors"]) == 1 and "fake failure" in sm["errors"][0]


def test_arrivals_honoured_and_summary():
    arr = serve.poisson_arrivals(12, rate=400.0, seed=1)
    assert np.all(np.diff(arr) > 0)
    reqs = [fake(i, 10, m=2, arrival=float(a)) for i, a in enumerate(arr)]
    tr = Tracker(need)
    srv = serve.SolveServer(slots=2, hbm_cap_bytes=100, solve_fn_factory=tr.factory, need_fn=need)
    out = srv.run(reqs, keep_x=False)
    assert all(r.start >= r.arrival - 1e-6 for r in out)
    assert all(r.X is None for r in out)
    sm = serve.summarize(out)
    assert sm["requests"] == 12 and sm["converged"] == 12 and sm["errors"] == []
    assert 0 <= sm["p50_s"] <= sm["p99_s"] and sm["solves_per_s"] > 0


def test_request_mix_shapes():
    reqs = serve.serving_requests(8, seed=3, side_range=(6, 9))
    for r in reqs:
        N = round(r.n ** (1 / 3))
        assert N ** 3 == r.n and 6 <= N <= 9
        assert r.s in (1, 4, 8, 16, 32) and 8 <= r.m <= 32
        d = np.repeat(np.arange(r.n), np.diff(r.A.rowptr)) == r.A.colidx
        delta = r.A.vals[d] - 6.0
        assert np.all((delta >= 0) & (delta <= 0.1)) and np.ptp(delta) < 1e-12
        assert np.all(r.A.vals[~d] == -1.0)


def test_workspace_bound_covers_basis():
    pytest.importorskip("ctypes")
    from paper_2208_09899_gb300 import lsba
    try:
        lsba.load()
    except (RuntimeError, OSError) as exc:
        pytest.skip(f"library not built: {exc}")
    n, s, m = 100000, 8, 20
    b = lsba.workspace_bytes(n, 7 * n, s, m)
    assert b >= 8 * n * s * (m + 1)            # the basis itself
    assert b < 8 * n * s * (m + 1) * 2 + 7 * n * 8 + (1 << 28)
    assert lsba.workspace_bytes(n, 7 * n, 64, m) == -1


@pytest.mark.gpu
def test_served_results_equal_solo():
    import torch
    from paper_2208_09899_gb300 import lsba
    reqs = serve.serving_requests(10, seed=11, side_range=(10, 22), m_range=(6, 14),
                                  s_choices=(1, 4, 8, 16, 32), tol=1e-8)
    for i, r in enumerate(reqs):
        r.precision = ("auto", "fp32_ir", "df", "fp64")[i % 4]
        r.skeleton = ("bcgsi_ls", "bcgs_pip", "bmgs_icwy")[i % 3]
    solo = []
    sv = lsba.Solver(0)
    for r in reqs:
        dA = lsba.DeviceCSR.from_host(r.A, "cuda:0")
        dB = torch.from_numpy(r.B).cuda()
        dX = torch.empty_like(dB)
        sv.set_options(modification=r.modification, max_restarts=r.max_restarts,
                       precision=r.precision)
        sv.solve(dA, dB, dX, r.m, r.tol, r.skeleton)
        torch.cuda.synchronize()
        solo.append((dX.cpu().numpy(), sv.stats()))
    sv.close()
    srv = serve.SolveServer(slots=5, hbm_cap_bytes=40e9, device=0)
    try:
        out = srv.run(reqs)
    finally:
        srv.close()
    for r, res, (X, st) in zip(reqs, out, solo):
        assert "error" not in res.stats, res.stats
        assert res.stats["cycles"] == st["cycles"] and res.stats["status"] == st["status"]
        assert np.array_equal(res.X, X), f"request {r.rid} differs in the mix"
        assert st["status"] == 0
        R = r.B - _spmm(r.A, X)
        assert np.linalg.norm(R) <= 10 * r.tol * np.linalg.norm(r.B)


def _spmm(A, X):
    import scipy.sparse as sp
    return sp.csr_matrix((A.vals, A.colidx, A.rowptr), shape=(A.n, A.n)) @ X


def _lapl3d_kappa(A):
    """kappa of the 3D 7-point Laplacian + delta I of a served request."""
    N = round(A.n ** (1 / 3))
    d = np.repeat(np.arange(A.n), np.diff(A.rowptr)) == A.colidx
    delta = float(A.vals[d][0] - 6.0)
    c = np.cos(np.pi / (N + 1))
    return (delta + 6 * (1 + c)) / (delta + 6 * (1 - c))


@pytest.mark.gpu
def test_served_results_match_oracle():
    """Every served request against the CPU oracle on the same (A, B, m, tol,
    skeleton, modification, restarts): FP64, double-float and auto requests
    have the oracle's status, cycles, relations, A-calls and syncs and X within
    1e-8; FP32-inner requests reach tol and their error against the oracle is
    within kappa(A) (relres_gpu + relres_oracle) (iterative refinement reaches
    the same solution to the conditioning of the problem)."""
    from oracle import lsba_oracle as O
    reqs = serve.serving_requests(8, seed=17, side_range=(10, 18), m_range=(6, 12),
                                  s_choices=(1, 4, 8, 16), tol=1e-8)
    precisions = ("auto", "fp64", "df", "fp32_ir")
    skeletons = ("bcgsi_ls", "bcgs_pip", "bmgs_icwy", "bcgsi_ls")
    for i, r in enumerate(reqs):
        r.precision = precisions[i % 4]
        r.skeleton = skeletons[i % 4]
    # one request on the FP64 tensor-core passes (lagged skeleton, s = 8)
    reqs[1].skeleton, reqs[1].precision = "bcgsi_ls", "fp64"
    reqs[1].B = np.ascontiguousarray(
        np.random.default_rng(5).standard_normal((reqs[1].A.n, 8)))
    srv = serve.SolveServer(slots=4, hbm_cap_bytes=40e9, device=0)
    try:
        out = srv.run(reqs)
    finally:
        srv.close()
    for r, res in zip(reqs, out):
        assert "error" not in res.stats, res.stats
        ref = O.solve(r.A, r.B, r.m, r.tol, r.skeleton, modification=r.modification,
                      max_restarts=r.max_restarts)
        st = res.stats
        err = np.linalg.norm(res.X - ref.X) / np.linalg.norm(ref.X)
        print(f"SERVED rid={r.rid} n={r.n} s={r.s} m={r.m} {r.skeleton} {r.precision}: "
              f"cycles {st['cycles']}/{ref.cycles} relres {st['relres_true']:.2e} error {err:.2e}")
        assert st["status"] == ref.status == 0
        assert st["relres_true"] <= r.tol and ref.relres_true <= r.tol
        if r.precision == "fp32_ir":
            assert err <= _lapl3d_kappa(r.A) * (st["relres_true"] + ref.relres_true)
        else:
            assert (st["cycles"], st["steps"], st["a_calls"], st["syncs"]) == \
                (ref.cycles, ref.steps, ref.a_calls, ref.syncs)
            assert err <= 1e-8
