"""lsba_gram_noalloc: the block inner product for callers that cannot allocate
device memory (serving loops that may not pay for an allocation, hosts that
keep the device's memory footprint fixed).  It must give the same G as
lsba_gram and as a NumPy FP64 product, on consecutive calls that reuse its
fixed scratch array, and refuse sizes beyond that array."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2208_09899_gb300 import build, lsba
    build.build()
    return torch, lsba, lsba.load()


def _noalloc(lib, torch, L, R, G):
    a, n, s = L.shape
    b = R.shape[0]
    stream = torch.cuda.current_stream().cuda_stream
    return lib.lsba_gram_noalloc(C.c_void_p(L.data_ptr()), a, C.c_void_p(R.data_ptr()), b, n, s,
                                 C.c_void_p(G.data_ptr()), C.c_void_p(stream))


@pytest.mark.parametrize("calls", [[(8, 21, 2, 70001), (4, 3, 1, 1000)],
                                   [(16, 17, 2, 40003), (16, 17, 2, 40003)]])
def test_noalloc_matches_gram_on_consecutive_calls(env, calls):
    torch, lsba, lib = env
    sv = lsba.Solver(0)
    for i, (s, a, b, n) in enumerate(calls):
        rng = np.random.default_rng(100 + i)
        L = torch.from_numpy(rng.standard_normal((a, n, s))).cuda()
        R = torch.from_numpy(rng.standard_normal((b, n, s))).cuda()
        G_ref = torch.empty((a * s, b * s), dtype=torch.float64, device="cuda")
        sv.gram(L, R, G_ref)
        G = torch.full((a * s, b * s), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc(lib, torch, L, R, G) == 0
        torch.cuda.synchronize()
        g, gr = G.cpu().numpy(), G_ref.cpu().numpy()
        assert np.linalg.norm(g - gr) <= 1e-13 * np.linalg.norm(gr)
        # independent of the kernels both entry points share: the FP64 product
        # of the stacked blocks, computed on the host
        Lh = np.hstack(list(L.cpu().numpy()))
        Rh = np.hstack(list(R.cpu().numpy()))
        gn = Lh.T @ Rh
        assert np.linalg.norm(g - gn) <= 1e-13 * np.linalg.norm(gn)


def test_noalloc_rejects_oversized_output(env):
    torch, lsba, lib = env
    s, a, b, n = 32, 64, 2, 64   # (a s)(b s) = 2048 * 64 = 2^17 > 2^16
    L = torch.zeros((a, n, s), dtype=torch.float64, device="cuda")
    R = torch.zeros((b, n, s), dtype=torch.float64, device="cuda")
    G = torch.zeros((a * s, b * s), dtype=torch.float64, device="cuda")
    assert _noalloc(lib, torch, L, R, G) == lsba.LSBA_INVALID_ARG
