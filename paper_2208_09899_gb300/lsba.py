"""Thin ctypes binding of liblsba.so (the C ABI in include/lsba.h).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  Device arrays are torch CUDA tensors (FP64, C-contiguous); host
arrays are numpy arrays.  If the library is missing or cannot be loaded, every
entry point raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "liblsba.so")

LSBA_OK, LSBA_NOT_CONVERGED, LSBA_BREAKDOWN, LSBA_INVALID_ARG = 0, 1, 2, 3
LSBA_OUT_OF_MEMORY, LSBA_CUDA_ERROR, LSBA_DEVICE_TIMEOUT = 4, 5, 6
SKELETONS = {"bcgs": 0, "bcgs_pip": 1, "bcgsi_ls": 2, "bmgs_icwy": 3, "bmgs_cwy": 4, "bmgs": 5,
             "bcgs_pio": 6, "bmgs_svl": 7, "bmgs_lts": 8}
MODIFICATIONS = {"fom": 0, "gmres": 1}
PRECISIONS = {"fp64": 0, "df": 1, "auto": 2, "fp32_ir": 3}
INNER_PRODUCTS = {"classical": 0, "global": 1}
MUSCLES = {"cholqr": 0, "mgs": 1}

EXPORTED = ("lsba_default_options", "lsba_create", "lsba_set_options", "lsba_solve",
            "lsba_solve_host", "lsba_get_stats", "lsba_get_history", "lsba_status_string",
            "lsba_autotune", "lsba_autotune_table",
            "lsba_destroy", "lsba_spmm", "lsba_gram", "lsba_combine", "lsba_get_profile",
            "lsba_reset_profile", "lsba_gram_noalloc", "lsba_release_workspace",
            "lsba_workspace_bytes", "lsba_gram_df", "lsba_gram_fp64tc", "lsba_combine_fp64tc")
KERNEL_CLASSES = ("spmm", "gram", "update", "small")


class Options(C.Structure):
    _fields_ = [("modification", C.c_int32), ("max_restarts", C.c_int32),
                ("adaptive_restart", C.c_int32), ("verify_true_residual", C.c_int32),
                ("record_history", C.c_int32), ("inject_flag_cycle", C.c_int32),
                ("inject_flag_relation", C.c_int32), ("profile", C.c_int32),
                ("precision", C.c_int32), ("ir_max_outer", C.c_int32),
                ("ir_inner_tol", C.c_double), ("cuda_graphs", C.c_int32),
                ("tensor_cores", C.c_int32), ("inner_product", C.c_int32),
                ("muscle", C.c_int32), ("inject_stall", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("cycles", C.c_int32), ("steps", C.c_int32),
                ("a_calls", C.c_int32), ("syncs", C.c_int32), ("v_apps", C.c_int32),
                ("flags", C.c_int32), ("m_final", C.c_int32), ("relres_est", C.c_double),
                ("relres_true", C.c_double), ("solve_ms", C.c_double),
                ("precision", C.c_int32), ("ir_outer", C.c_int32), ("tensor_cores", C.c_int32)]


class History(C.Structure):
    _fields_ = [("n_est", C.c_int32), ("est", C.POINTER(C.c_double)),
                ("est_cycle", C.POINTER(C.c_int32)), ("est_j", C.POINTER(C.c_int32)),
                ("n_cycles", C.c_int32), ("cycle_m", C.POINTER(C.c_int32)),
                ("cycle_flag", C.POINTER(C.c_int32)), ("cycle_mcur", C.POINTER(C.c_int32)),
                ("first_j", C.c_int32), ("first_H", C.POINTER(C.c_double)),
                ("first_beta", C.POINTER(C.c_double)), ("n_grams", C.c_int32),
                ("gram_rows", C.POINTER(C.c_int32)), ("gram_cols", C.POINTER(C.c_int32)),
                ("gram_data", C.POINTER(C.c_double))]


class TuneEntry(C.Structure):
    _fields_ = [("k", C.c_int32), ("gram_kernel", C.c_int32), ("gram_ctas_per_sm", C.c_int32),
                ("gram_rows", C.c_int32), ("update_kernel", C.c_int32),
                ("update_ctas_per_sm", C.c_int32), ("gram_us", C.c_float), ("update_us", C.c_float),
                ("gram_default_us", C.c_float), ("update_default_us", C.c_float)]


class CSRDesc(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("d_rowptr", C.c_void_p),
                ("d_colidx", C.c_void_p), ("d_vals", C.c_void_p)]


_lib = None


def load(path: str = LIB_PATH):
    """Load liblsba.so (raises if it is missing: build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"liblsba.so not built ({path}); run paper_2208_09899_gb300.build.build()")
    lib = C.CDLL(path)
    vp, i32, i64, f64 = C.c_void_p, C.c_int, C.c_int64, C.c_double
    lib.lsba_default_options.argtypes = [C.POINTER(Options)]
    lib.lsba_default_options.restype = None
    lib.lsba_create.argtypes = [C.POINTER(vp), i32, vp, C.POINTER(Options)]
    lib.lsba_set_options.argtypes = [vp, C.POINTER(Options)]
    lib.lsba_solve.argtypes = [vp, C.POINTER(CSRDesc), vp, vp, i32, i32, f64, i32]
    lib.lsba_solve_host.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp, i32, i32, f64, i32]
    lib.lsba_autotune.argtypes = [vp, i64, i32, i32, vp, vp, i32]
    lib.lsba_autotune_table.argtypes = [vp, C.POINTER(TuneEntry), i32, C.POINTER(C.c_int)]
    lib.lsba_get_stats.argtypes = [vp, C.POINTER(Stats)]
    lib.lsba_get_history.argtypes = [vp, C.POINTER(History)]
    lib.lsba_status_string.argtypes = [i32]
    lib.lsba_status_string.restype = C.c_char_p
    lib.lsba_destroy.argtypes = [vp]
    lib.lsba_spmm.argtypes = [vp, C.POINTER(CSRDesc), vp, vp, i32]
    lib.lsba_gram.argtypes = [vp, vp, i32, vp, i32, i64, i32, vp]
    lib.lsba_combine.argtypes = [vp, vp, i32, i64, i32, vp, vp, vp]
    lib.lsba_get_profile.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64), i32]
    lib.lsba_reset_profile.argtypes = [vp]
    lib.lsba_gram_noalloc.argtypes = [vp, i32, vp, i32, i64, i32, vp, vp]
    lib.lsba_release_workspace.argtypes = [vp]
    lib.lsba_workspace_bytes.argtypes = [i64, i64, i32, i32]
    lib.lsba_gram_df.argtypes = [vp, vp, i32, vp, i32, i64, i32, vp, i32]
    lib.lsba_gram_fp64tc.argtypes = [vp, vp, i32, vp, i32, i64, i32, vp]
    lib.lsba_combine_fp64tc.argtypes = [vp, vp, i32, i64, i32, vp, vp, vp, vp, vp]
    for name in EXPORTED:
        if name not in ("lsba_default_options", "lsba_status_string"):
            getattr(lib, name).restype = C.c_int
    lib.lsba_workspace_bytes.restype = C.c_int64
    _lib = lib
    return lib


def workspace_bytes(n: int, nnz: int, s: int, m: int) -> int:
    """Upper bound of the device memory one solve allocates (admission control)."""
    return int(load().lsba_workspace_bytes(n, nnz, s, m))


def status_string(code: int) -> str:
    return load().lsba_status_string(code).decode()


class LSBAError(RuntimeError):
    pass


def _check(code: int, allowed=(LSBA_OK,)):
    if code not in allowed:
        raise LSBAError(f"lsba error {code}: {status_string(code)}")
    return code


def _ptr(t) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


@dataclass
class DeviceCSR:
    """A CSR matrix resident on the GPU (torch tensors kept alive here)."""
    n: int
    nnz: int
    rowptr: object
    colidx: object
    vals: object

    @classmethod
    def from_host(cls, A, device="cuda"):
        import torch
        return cls(A.n, A.nnz,
                   torch.from_numpy(np.ascontiguousarray(A.rowptr, dtype=np.int32)).to(device),
                   torch.from_numpy(np.ascontiguousarray(A.colidx, dtype=np.int32)).to(device),
                   torch.from_numpy(np.ascontiguousarray(A.vals, dtype=np.float64)).to(device))

    def desc(self) -> CSRDesc:
        import torch
        d = CSRDesc()
        d.n, d.nnz = self.n, self.nnz
        d.d_rowptr = self.rowptr.data_ptr()
        d.d_colidx = self.colidx.data_ptr() if self.nnz else None
        d.d_vals = self.vals.data_ptr() if self.nnz else None
        return d


def _host_ptr(a) -> int:
    """Address of a contiguous host array (numpy array or CPU torch tensor)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be contiguous")
        return a.ctypes.data
    if a.device.type != "cpu" or not a.is_contiguous():
        raise ValueError("host tensors must be contiguous CPU tensors")
    return a.data_ptr()


class PinnedCSR:
    """A host CSR matrix copied into page-locked memory (the H2D copies of
    lsba_solve_host then run as DMA at the link's bandwidth)."""

    def __init__(self, A):
        import torch
        self.n, self.nnz = int(A.n), int(A.nnz)
        self.rowptr = torch.from_numpy(np.ascontiguousarray(A.rowptr, dtype=np.int32)).pin_memory()
        self.colidx = torch.from_numpy(np.ascontiguousarray(A.colidx, dtype=np.int32)).pin_memory()
        self.vals = torch.from_numpy(np.ascontiguousarray(A.vals, dtype=np.float64)).pin_memory()


class Solver:
    """A solver handle bound to one device and the current torch stream."""

    def __init__(self, device: int = 0, stream=None, **opts):
        import torch
        lib = load()
        self.lib = lib
        self.opt = Options()
        lib.lsba_default_options(C.byref(self.opt))
        self._apply(opts)
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = C.c_void_p()
        _check(lib.lsba_create(C.byref(h), device, C.c_void_p(stream.cuda_stream), C.byref(self.opt)))
        self.h = h

    def _apply(self, opts):
        for k, v in opts.items():
            if k == "modification" and isinstance(v, str):
                v = MODIFICATIONS[v]
            if k == "precision" and isinstance(v, str):
                v = PRECISIONS[v]
            if k == "inner_product" and isinstance(v, str):
                v = INNER_PRODUCTS[v]
            if k == "muscle" and isinstance(v, str):
                v = MUSCLES[v]
            if isinstance(v, bool):
                v = int(v)
            setattr(self.opt, k, v)

    def set_options(self, **opts):
        self._apply(opts)
        _check(self.lib.lsba_set_options(self.h, C.byref(self.opt)))

    def close(self):
        if getattr(self, "h", None):
            self.lib.lsba_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, A: DeviceCSR, B, X, m: int, tol: float, skeleton: str = "bcgsi_ls") -> int:
        n, s = B.shape
        self._last_s = s
        d = A.desc()
        return _check(self.lib.lsba_solve(self.h, C.byref(d), C.c_void_p(_ptr(B)), C.c_void_p(_ptr(X)),
                                          s, m, tol, SKELETONS[skeleton]),
                      (LSBA_OK, LSBA_NOT_CONVERGED, LSBA_BREAKDOWN))

    def solve_host(self, A, B, m: int, tol: float, skeleton: str = "bcgsi_ls", X=None):
        """Host buffers in, host X out (copies inside the call).

        A is a host CSR (numpy arrays, or a `PinnedCSR`); B (n x s) and the
        optional output X are numpy arrays or CPU torch tensors (pinned memory
        makes the copies asynchronous DMA).  Returns (X, status)."""
        if isinstance(A, PinnedCSR):
            rp, ci, va = A.rowptr, A.colidx, A.vals
        else:
            rp = np.ascontiguousarray(A.rowptr, dtype=np.int32)
            ci = np.ascontiguousarray(A.colidx, dtype=np.int32)
            va = np.ascontiguousarray(A.vals, dtype=np.float64)
        if isinstance(B, np.ndarray):
            B = np.ascontiguousarray(B, dtype=np.float64)
            if X is None:
                X = np.empty_like(B)
        else:
            import torch
            if B.dtype != torch.float64 or B.device.type != "cpu" or not B.is_contiguous():
                raise ValueError("B must be a contiguous float64 CPU tensor")
            if X is None:
                X = torch.empty_like(B)
        if tuple(X.shape) != tuple(B.shape):
            raise ValueError("X must have the shape of B")
        self._last_s = B.shape[1]
        st = self.lib.lsba_solve_host(self.h, A.n, A.nnz, _host_ptr(rp), _host_ptr(ci),
                                      _host_ptr(va), _host_ptr(B), _host_ptr(X), B.shape[1], m,
                                      tol, SKELETONS[skeleton])
        _check(st, (LSBA_OK, LSBA_NOT_CONVERGED, LSBA_BREAKDOWN))
        return X, st

    def autotune(self, n: int, s: int, m: int) -> dict:
        """Time the candidate shapes of the double-float lagged skeletons'
        Gram and update for every iteration of an m-step cycle on n rows, block
        size s; later solves with the same n and s run the fastest.  Returns
        {k: (Gram kernel, update CTAs per SM)} (kernel 0 FP32 pipe, 1
        split-digit tensor cores, 2 stored-digit tensor cores)."""
        g = (C.c_int8 * (m + 2))()
        u = (C.c_int8 * (m + 2))()
        _check(self.lib.lsba_autotune(self.h, n, s, m, g, u, m + 2))
        return {k: (g[k], u[k]) for k in range(2, m + 2) if g[k] >= 0}

    def tune_table(self) -> list:
        """The last autotune's shapes and times, one dict per iteration k."""
        cnt = C.c_int(0)
        _check(self.lib.lsba_autotune_table(self.h, None, 0, C.byref(cnt)))
        arr = (TuneEntry * max(cnt.value, 1))()
        _check(self.lib.lsba_autotune_table(self.h, arr, cnt.value, C.byref(cnt)))
        return [{f: getattr(arr[i], f) for f, _ in TuneEntry._fields_} for i in range(cnt.value)]

    def stats(self) -> dict:
        s = Stats()
        _check(self.lib.lsba_get_stats(self.h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def profile(self) -> dict:
        ms = (C.c_double * 4)()
        cnt = (C.c_int64 * 4)()
        _check(self.lib.lsba_get_profile(self.h, ms, cnt, 4))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_CLASSES)}

    def release_workspace(self):
        _check(self.lib.lsba_release_workspace(self.h))

    def reset_profile(self):
        _check(self.lib.lsba_reset_profile(self.h))

    def history(self) -> dict:
        hs = History()
        _check(self.lib.lsba_get_history(self.h, C.byref(hs)))

        def arr(p, n, dt):
            if n <= 0 or not p:
                return np.zeros(0, dtype=dt)
            return np.ctypeslib.as_array(p, shape=(n,)).astype(dt).copy()

        out = {
            "est": arr(hs.est, hs.n_est, np.float64),
            "est_cycle": arr(hs.est_cycle, hs.n_est, np.int32),
            "est_j": arr(hs.est_j, hs.n_est, np.int32),
            "cycle_m": arr(hs.cycle_m, hs.n_cycles, np.int32).tolist(),
            "cycle_flag": arr(hs.cycle_flag, hs.n_cycles, np.int32).tolist(),
            "cycle_mcur": arr(hs.cycle_mcur, hs.n_cycles, np.int32).tolist(),
            "first_j": hs.first_j,
        }
        s = self._last_s
        j = hs.first_j
        if j > 0:
            rows, cols = (j + 1) * s, j * s
            out["first_H"] = arr(hs.first_H, rows * cols, np.float64).reshape(cols, rows).T.copy()
        out["first_beta"] = arr(hs.first_beta, s * s, np.float64).reshape(s, s).T.copy()
        rows = arr(hs.gram_rows, hs.n_grams, np.int32)
        cols = arr(hs.gram_cols, hs.n_grams, np.int32)
        data = arr(hs.gram_data, int((rows * cols).sum()), np.float64)
        grams, off = [], 0
        for r, c in zip(rows, cols):
            grams.append(data[off:off + r * c].reshape(r, c))
            off += r * c
        out["grams"] = grams
        return out

    # kernel-level entry points -------------------------------------------
    def spmm(self, A: DeviceCSR, V, W):
        d = A.desc()
        _check(self.lib.lsba_spmm(self.h, C.byref(d), C.c_void_p(_ptr(V)), C.c_void_p(_ptr(W)),
                                  V.shape[-1]))

    def gram(self, L, R, G):
        """L: (a, n, s), R: (b, n, s), G: (a*s, b*s) -- all CUDA FP64."""
        a, n, s = L.shape
        b = R.shape[0]
        _check(self.lib.lsba_gram(self.h, C.c_void_p(_ptr(L)), a, C.c_void_p(_ptr(R)), b, n, s,
                                  C.c_void_p(_ptr(G))))

    def gram_df(self, L, R, G, tensor_cores=True):
        """Double-float Gram kernels: L (a, n, s), R (b, n, s) CUDA FP64 -> G (a*s, b*s).
        tensor_cores: False (FP32-pipe kernel), True (tensor-core digit kernel), or
        "stored" (the basis kernel: L_1..L_{a-1} as stored digit planes, R_1 for L_a)."""
        a, n, s = L.shape
        b = R.shape[0]
        mode = 3 if tensor_cores == "stored" else int(bool(tensor_cores))
        _check(self.lib.lsba_gram_df(self.h, C.c_void_p(_ptr(L)), a, C.c_void_p(_ptr(R)), b, n, s,
                                     C.c_void_p(_ptr(G)), mode))

    def gram_fp64tc(self, L, R, G):
        """FP64 Gram on the tensor cores (exact digit products): L (a, n, 8),
        R (b, n, 8) CUDA FP64 -> G (a*8, b*8)."""
        a, n, s = L.shape
        b = R.shape[0]
        _check(self.lib.lsba_gram_fp64tc(self.h, C.c_void_p(_ptr(L)), a, C.c_void_p(_ptr(R)), b, n,
                                         s, C.c_void_p(_ptr(G))))

    def combine_fp64tc(self, inputs, coef1, tri, out1, coef2=None, out2=None):
        """FP64 update on the tensor cores: out1 = ([inputs] coef1) tri^{-1} and
        out2 = [inputs] coef2; inputs (nin, n, 8), coefs (nin*8, 8), tri (8, 8)
        upper or None, outputs (n, 8) -- all CUDA FP64."""
        nin, n, s = inputs.shape
        opt = lambda t: C.c_void_p(_ptr(t)) if t is not None else None  # noqa: E731
        _check(self.lib.lsba_combine_fp64tc(self.h, C.c_void_p(_ptr(inputs)), nin, n, s,
                                            C.c_void_p(_ptr(coef1)), opt(tri), opt(coef2),
                                            C.c_void_p(_ptr(out1)), opt(out2)))

    def combine(self, inputs, coef, tri, out):
        """inputs: (nin, n, s); coef: (nin*s, s); tri: (s, s) upper or None; out: (n, s)."""
        nin, n, s = inputs.shape
        _check(self.lib.lsba_combine(self.h, C.c_void_p(_ptr(inputs)), nin, n, s,
                                     C.c_void_p(_ptr(coef)),
                                     C.c_void_p(_ptr(tri)) if tri is not None else None,
                                     C.c_void_p(_ptr(out))))


def solve(A, B: np.ndarray, m: int, tol: float, skeleton: str = "bcgsi_ls", device: int = 0,
          **opts):
    """Convenience: solve from host arrays on the GPU; returns (X, stats, history or None)."""
    import torch
    dA = DeviceCSR.from_host(A, f"cuda:{device}")
    dB = torch.from_numpy(np.ascontiguousarray(B, dtype=np.float64)).to(f"cuda:{device}")
    dX = torch.empty_like(dB)
    sv = Solver(device, **opts)
    sv._last_s = B.shape[1]
    sv.solve(dA, dB, dX, m, tol, skeleton)
    torch.cuda.synchronize(device)
    st = sv.stats()
    hist = sv.history() if opts.get("record_history") else None
    X = dX.cpu().numpy()
    sv.close()
    return X, st, hist
