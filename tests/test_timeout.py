"""Bounded device waits: a wait that runs out ends the solve with
LSBA_DEVICE_TIMEOUT, read on the host, and leaves the handle and the CUDA
context usable.

The failure is made without a fault: the `inject_stall` test hook makes the
first cycle's start kernel wait on an mbarrier that nothing arrives at (no
copies or MMAs in flight), through the same bounded-wait routine the
tensor-core and bulk-copy kernels use.  The wait gives up after one second."""
import time

import numpy as np
import pytest

from oracle import lsba_oracle as O
from paper_2208_09899_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_09899_gb300 import build, lsba
    build.build()
    lsba.load()
    return torch, lsba


@pytest.mark.parametrize("skeleton,precision", [("bcgsi_ls", "auto"), ("bcgs_pip", "fp64")])
def test_stalled_wait_reports_timeout_and_handle_recovers(env, skeleton, precision):
    torch, lsba = env
    A = W.laplacian_3d(12)
    n = A.n
    B = W.gaussian_block(n, 8, seed=5)
    m, tol = 10, 1e-9
    dA = lsba.DeviceCSR.from_host(A, "cuda:0")
    dB = torch.from_numpy(B).to("cuda:0")
    dX = torch.zeros_like(dB)
    sv = lsba.Solver(0, precision=precision, inject_stall=1, max_restarts=40)
    try:
        t0 = time.perf_counter()
        with pytest.raises(lsba.LSBAError, match="device timeout"):
            sv.solve(dA, dB, dX, m, tol, skeleton)
        dt = time.perf_counter() - t0
        print(f"stalled solve ({skeleton}, {precision}) returned the timeout after {dt:.2f} s")
        assert dt < 30.0
        # the context and the handle still work: the same solve without the hook
        sv.set_options(inject_stall=0)
        st = sv.solve(dA, dB, dX, m, tol, skeleton)
        torch.cuda.synchronize()
        stats = sv.stats()
    finally:
        sv.close()
    assert st == lsba.LSBA_OK and stats["status"] == lsba.LSBA_OK
    ref = O.solve(A, B, m, tol, skeleton, max_restarts=40)
    X = dX.cpu().numpy()
    assert np.linalg.norm(X - ref.X) <= 1e-7 * np.linalg.norm(ref.X)
    assert stats["relres_true"] <= tol
