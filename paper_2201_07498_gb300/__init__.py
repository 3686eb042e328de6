"""Thin Python binding of the GB300 Top-K sparse eigensolver C ABI.

The arithmetic runs in ``libtopk_eigs.so`` (hand-written CUDA for sm_103a,
declared in ``include/topk_eigs.h``); this module only marshals arguments with
ctypes.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if the library is missing, importing the solver entry points raises.

Method: Sgherzi, Parravicini & Santambrogio, "A Mixed Precision, Multi-GPU
Design for Large-scale Top-K Sparse Eigenproblems" (arXiv 2201.07498):
Lanczos with full reorthogonalisation (Algorithm 1), Jacobi on the
tridiagonal T, Ritz vectors V*Y (Section III), mixed precision (Section III-A).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

from . import _build

__all__ = ["CSR", "Plan", "Server", "TEError", "topk_eigs", "spmv", "lanczos", "tridiag_eigs",
           "spmv_layout", "gram", "quantize", "library_path", "load_library", "PRECISIONS"]

TE_F64, TE_F32, TE_BF16, TE_FP8_E4M3 = 0, 1, 2, 3
TE_DEVICE, TE_HOST = 0, 1
WHICH = {"LM": 0, "LA": 1}
REORTH = {"full": 0, "none": 1, "delayed": 2}
ORDERS = {"keep": 0, "degree": 1}
PRECISIONS = {"ddd": (TE_F64, TE_F64, TE_F64), "fdd": (TE_F32, TE_F64, TE_F64),
              "fdf": (TE_F32, TE_F64, TE_F32),
              "bdf": (TE_BF16, TE_F64, TE_F32), "8df": (TE_FP8_E4M3, TE_F64, TE_F32)}
STATUS = {0: "TE_OK", 1: "TE_ERR_INVALID_ARG", 2: "TE_ERR_OUT_OF_MEMORY", 3: "TE_ERR_CUDA",
          4: "TE_ERR_BREAKDOWN", 5: "TE_ERR_NOT_CONVERGED", 6: "TE_ERR_TIMEOUT",
          7: "TE_ERR_UNSUPPORTED"}


class TEError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class te_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col_idx", ctypes.c_void_p), ("values", ctypes.c_void_p),
                ("row_scale", ctypes.c_void_p), ("where", ctypes.c_int32),
                ("values_f64", ctypes.c_int32)]


class te_precision(ctypes.Structure):
    _fields_ = [("values", ctypes.c_int32), ("arithmetic", ctypes.c_int32),
                ("vectors", ctypes.c_int32)]


class te_options(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("v1", ctypes.c_void_p), ("which", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("device_budget_bytes", ctypes.c_size_t),
                ("reorth", ctypes.c_int32), ("refine", ctypes.c_int32),
                ("matrix_budget_bytes", ctypes.c_size_t), ("autotune", ctypes.c_int32),
                ("order", ctypes.c_int32), ("stall_first_pass", ctypes.c_int32)]


class te_server_options(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int32), ("max_krylov_steps", ctypes.c_int32),
                ("device_budget_bytes", ctypes.c_size_t), ("use_graph", ctypes.c_int32),
                ("autotune", ctypes.c_int32)]


# every symbol the header declares, with its ctypes signature
_SIGS = {
    "te_default_options": (None, [ctypes.c_void_p]),
    "te_last_error": (ctypes.c_char_p, []),
    "te_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "te_workspace_bytes": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                             te_precision]),
    "te_topk_eigs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, te_precision,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]),
    "te_plan_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                      te_precision, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "te_plan_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "te_plan_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p]),
    "te_plan_status": (ctypes.c_int, [ctypes.c_void_p]),
    "te_plan_kernel_count": (ctypes.c_int32, [ctypes.c_void_p]),
    "te_plan_stream_blocks": (ctypes.c_int64, [ctypes.c_void_p]),
    "te_plan_layout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "te_plan_destroy": (None, [ctypes.c_void_p]),
    "te_spmv": (ctypes.c_int, [ctypes.c_void_p, te_precision, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_void_p]),
    "te_lanczos": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, te_precision,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "te_tridiag_eigs": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "te_spmv_noalloc": (ctypes.c_int, [ctypes.c_void_p, te_precision, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "te_plan_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "te_quantize": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p]),
    "te_server_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "te_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                        ctypes.c_int32, te_precision, ctypes.c_uint64,
                                        ctypes.c_void_p]),
    "te_server_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "te_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "te_server_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "te_server_destroy": (None, [ctypes.c_void_p]),
    "te_server_completed": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                           ctypes.c_void_p]),
    "te_server_classes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "te_server_timing": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 6),
    "te_server_analysis": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 7),
    "te_probe_gather": (ctypes.c_int, [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "te_gram": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_void_p]),
    "te_spmv_layout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "te_degree_order": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "te_spmv_layout_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
                              + [ctypes.c_void_p] * 13),
    "te_check_symmetric": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]),
    "te_set_memory_cache": (ctypes.c_int, [ctypes.c_uint64]),
    "te_release_cached_memory": (ctypes.c_int, []),
    "te_memory_cached": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = False):
    """Load libtopk_eigs.so (raises if it is missing, unless asked to build it)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise ImportError(
                f"{_build.LIB} is missing: build it with __graft_entry__.build() "
                "(there is no CPU fallback)")
        _build.build()
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        msg = load_library().te_last_error().decode(errors="replace")
        raise TEError(rc, msg)


def _prec(precision) -> te_precision:
    if isinstance(precision, str):
        v, a, w = PRECISIONS[precision.lower()]
    else:
        v, a, w = precision
    return te_precision(v, a, w)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


@dataclass
class CSR:
    """CSR matrix held in torch tensors (device or host).

    row_ptr: int64 (n+1); col: int32 (nnz); val: float64 (binary64 values,
    which serve every form: the library rounds them to the form's value type
    itself) or float32 (the binary32 values of FDD / FDF).
    """
    n: int
    row_ptr: "object"
    col: "object"
    val: "object"

    @property
    def nnz(self) -> int:
        return int(self.col.numel())

    @property
    def on_device(self) -> bool:
        return bool(self.row_ptr.is_cuda)

    @property
    def values_f64(self) -> bool:
        import torch
        return self.val.dtype == torch.float64

    def to_ctypes(self) -> te_csr:
        for t in (self.row_ptr, self.col, self.val):
            if not t.is_contiguous():
                raise ValueError("CSR tensors must be contiguous")
        return te_csr(self.n, self.nnz, self.row_ptr.data_ptr(), self.col.data_ptr(),
                      self.val.data_ptr(), None, TE_DEVICE if self.on_device else TE_HOST,
                      1 if self.values_f64 else 0)

    @staticmethod
    def from_host(host_csr, precision: str = "ddd", device: str = "cuda", pin: bool = False):
        """Wrap a host CSR (an object with n, row_ptr, col, val as numpy
        arrays) without touching its values.  float64 values are passed as
        binary64 (te_csr.values_f64 = 1: the library rounds them to the form's
        value type and keeps them for refinement); float32 values are the
        binary32 values of FDD / FDF and are refused for other forms."""
        import numpy as np
        import torch
        pv = _prec(precision).values
        val = np.asarray(host_csr.val)
        if val.dtype == np.float32:
            if pv != TE_F32:
                raise ValueError("float32 values serve only the binary32-valued forms "
                                 "(FDD, FDF); pass float64 values")
        elif val.dtype != np.float64:
            raise ValueError(f"values must be float64 or float32, not {val.dtype}")
        rp = torch.from_numpy(np.ascontiguousarray(host_csr.row_ptr, dtype=np.int64))
        ci = torch.from_numpy(np.ascontiguousarray(host_csr.col, dtype=np.int32))
        va = torch.from_numpy(np.ascontiguousarray(val))
        if device == "cpu":
            if pin:
                rp, ci, va = rp.pin_memory(), ci.pin_memory(), va.pin_memory()
            return CSR(int(host_csr.n), rp, ci, va)
        return CSR(int(host_csr.n), rp.to(device), ci.to(device), va.to(device))


def _options(seed=0, v1=None, which="LM", use_graph=True, budget=0, reorth="full",
             refine=False, matrix_budget=0, autotune=False, order="keep",
             stall_first_pass=False) -> te_options:
    o = te_options()
    load_library().te_default_options(ctypes.byref(o))
    o.seed = seed
    o.v1 = None if v1 is None else v1.data_ptr()
    o.which = WHICH[which] if isinstance(which, str) else int(which)
    o.use_graph = 1 if use_graph else 0
    o.device_budget_bytes = budget
    o.reorth = REORTH[reorth] if isinstance(reorth, str) else int(reorth)
    o.refine = 1 if refine else 0
    o.matrix_budget_bytes = matrix_budget
    o.autotune = 1 if autotune else 0
    o.order = ORDERS[order] if isinstance(order, str) else int(order)
    o.stall_first_pass = 1 if stall_first_pass else 0
    return o


def set_memory_cache(keep_bytes: int):
    """Release threshold of the library's device memory pools (bytes kept
    reserved after plans free them; default: all)."""
    _check(load_library().te_set_memory_cache(int(keep_bytes)))


def release_cached_memory():
    """Return the device memory the library keeps for reuse to the driver."""
    _check(load_library().te_release_cached_memory())


def memory_cached(device: int = 0):
    """(reserved, used) bytes of the library's memory pool on `device`."""
    r, u = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load_library().te_memory_cached(device, ctypes.byref(r), ctypes.byref(u)))
    return r.value, u.value


def topk_eigs(csr: CSR, K: int, krylov_steps: int, precision="fdf", *, seed: int = 0, v1=None,
              which="LM", vectors: bool = True, residuals: bool = False, reorth="full",
              refine: bool = False, matrix_budget: int = 0, order="keep", stream=None, out=None):
    """One Top-K solve; returns (eigvals [K] float64 cpu, eigvecs [n, K] float64 or None,
    residuals [K] or None: estimates, or true binary64 residuals with refine).
    Vectors live where the matrix lives unless `out = (eigvals [K], eigvecs
    [K, n] or None)` gives preallocated buffers."""
    import torch
    lib = load_library()
    A = csr.to_ctypes()
    opt = _options(seed, v1, which, reorth=reorth, refine=refine, matrix_budget=matrix_budget,
                   order=order)
    if out is not None:
        ev, U = out
    else:
        ev = torch.empty(K, dtype=torch.float64)
        dev = "cuda" if csr.on_device else "cpu"
        U = torch.empty((K, csr.n), dtype=torch.float64, device=dev) if vectors else None
    res = torch.empty(K, dtype=torch.float64) if residuals else None
    rc = lib.te_topk_eigs(ctypes.byref(A), K, krylov_steps, _prec(precision), ctypes.byref(opt),
                          ctypes.c_void_p(ev.data_ptr()),
                          None if U is None else ctypes.c_void_p(U.data_ptr()),
                          None if res is None else ctypes.c_void_p(res.data_ptr()),
                          _stream_ptr(stream))
    _check(rc)
    return ev, (None if U is None else U.t()), res


class Plan:
    """A reusable solve (row partition, work memory and captured CUDA graph)."""

    def __init__(self, csr: CSR, K: int, krylov_steps: int, precision="fdf", *, seed: int = 0,
                 v1=None, which="LM", use_graph: bool = True, budget: int = 0,
                 reorth="full", refine: bool = False, matrix_budget: int = 0,
                 autotune: bool = False, order="keep", stall_first_pass: bool = False,
                 stream=None):
        """stall_first_pass: test hook of the device-side failure path (the
        first solve's first basis pass times out; see te_options)."""
        self._lib = load_library()
        self.csr, self.K, self.m, self.n = csr, K, krylov_steps, csr.n
        A = csr.to_ctypes()
        opt = _options(seed, v1, which, use_graph, budget, reorth, refine, matrix_budget,
                       autotune, order, stall_first_pass)
        h = ctypes.c_void_p()
        rc = self._lib.te_plan_create(ctypes.byref(A), K, krylov_steps, _prec(precision),
                                      ctypes.byref(opt), _stream_ptr(stream), ctypes.byref(h))
        _check(rc)
        self._h = h

    @property
    def kernel_count(self) -> int:
        return int(self._lib.te_plan_kernel_count(self._h))

    @property
    def layout(self):
        """(window, vmax) of the plan's SpMV layout."""
        w, v = ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.te_plan_layout(self._h, ctypes.byref(w), ctypes.byref(v)))
        return w.value, v.value

    @property
    def stream_blocks(self) -> int:
        """Row blocks each SpMV streams from host memory (0: resident matrix)."""
        return int(self._lib.te_plan_stream_blocks(self._h))

    def solve(self, v1=None, vectors: bool = True, residuals: bool = False, stream=None):
        import torch
        ev = torch.empty(self.K, dtype=torch.float64)
        U = (torch.empty((self.K, self.n), dtype=torch.float64, device="cuda")
             if vectors else None)
        res = torch.empty(self.K, dtype=torch.float64) if residuals else None
        rc = self._lib.te_plan_solve(self._h, None if v1 is None else ctypes.c_void_p(v1.data_ptr()),
                                     ctypes.c_void_p(ev.data_ptr()),
                                     None if U is None else ctypes.c_void_p(U.data_ptr()),
                                     None if res is None else ctypes.c_void_p(res.data_ptr()),
                                     _stream_ptr(stream))
        _check(rc)
        return ev, (None if U is None else U.t()), res

    def launch(self, eigvals_dev, eigvecs_dev=None, v1=None, stream=None):
        """Asynchronous solve into device buffers (eigvecs_dev: (K, n) contiguous or None)."""
        rc = self._lib.te_plan_launch(self._h, None if v1 is None else ctypes.c_void_p(v1.data_ptr()),
                                      ctypes.c_void_p(eigvals_dev.data_ptr()),
                                      None if eigvecs_dev is None
                                      else ctypes.c_void_p(eigvecs_dev.data_ptr()),
                                      _stream_ptr(stream))
        _check(rc)

    def status(self):
        _check(self._lib.te_plan_status(self._h))

    KINDS = ("spmv", "dot", "axpy_dot", "axpy_store", "restart", "jacobi", "ritz", "other",
             "refine")

    def profile(self, stream=None):
        """One un-graphed solve with CUDA events around every kernel:
        {kind: (ms, launches, algorithmic bytes)}."""
        import numpy as np
        nk = len(self.KINDS)
        ms = np.zeros(nk)
        cnt = np.zeros(nk, dtype=np.int32)
        by = np.zeros(nk)
        rc = self._lib.te_plan_profile(self._h, ctypes.c_void_p(ms.ctypes.data),
                                       ctypes.c_void_p(cnt.ctypes.data),
                                       ctypes.c_void_p(by.ctypes.data), _stream_ptr(stream))
        _check(rc)
        return {k: (float(ms[i]), int(cnt[i]), float(by[i])) for i, k in enumerate(self.KINDS)}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.te_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving engine (continuous batching of many small solves on the GPU):
    submit host matrices, call step() repeatedly, poll() finished requests."""

    def __init__(self, max_slots: int = 32, max_krylov_steps: int = 32,
                 budget: int = 4 << 30, use_graph: bool = True, autotune: bool = False):
        self._lib = load_library()
        o = te_server_options(max_slots, max_krylov_steps, budget, 1 if use_graph else 0,
                              1 if autotune else 0)
        h = ctypes.c_void_p()
        _check(self._lib.te_server_create(ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self._meta = {}

    def submit(self, host_csr, K: int, krylov_steps: int, precision="fdf", seed: int = 0) -> int:
        """host_csr: an object with n, row_ptr, col, val (numpy).  Binary32
        values of a binary32-storage request ("fdf") are passed as they are;
        otherwise the values go as binary64 and the library rounds them to
        the form's type."""
        import numpy as np
        rp = np.ascontiguousarray(host_csr.row_ptr, dtype=np.int64)
        ci = np.ascontiguousarray(host_csr.col, dtype=np.int32)
        f32 = np.asarray(host_csr.val).dtype == np.float32 and _prec(precision).values == 1
        va = np.ascontiguousarray(host_csr.val, dtype=np.float32 if f32 else np.float64)
        A = te_csr(int(host_csr.n), len(ci), rp.ctypes.data, ci.ctypes.data, va.ctypes.data,
                   None, TE_HOST, 0 if f32 else 1)
        t = ctypes.c_int64()
        _check(self._lib.te_server_submit(self._h, ctypes.byref(A), K, krylov_steps,
                                          _prec(precision), seed, ctypes.byref(t)))
        # the server reads the arrays at admission: keep them alive until done
        self._meta[t.value] = (int(host_csr.n), K, rp, ci, va)
        return t.value

    def step(self):
        """One engine step; returns (resident, queued)."""
        live, pend = ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.te_server_step(self._h, ctypes.byref(live), ctypes.byref(pend)))
        return live.value, pend.value

    def poll(self, ticket: int, vectors: bool = True, out=None):
        """None while running; else (eigvals [K], eigvecs [n, K] or None,
        residual estimates [K]) as numpy arrays (raises on a failed request).
        out: optional float64 buffer of at least K * n elements (a pinned
        torch tensor, for example) that receives the Ritz vectors instead of
        a new array; the returned eigvecs then view it."""
        import numpy as np
        n, K = self._meta[ticket][:2]
        ev = np.empty(K)
        res = np.empty(K)
        U = None
        if vectors and out is not None:
            flat = out.numpy() if hasattr(out, "numpy") else np.asarray(out)
            if flat.dtype != np.float64 or flat.size < K * n or not flat.flags.c_contiguous:
                raise ValueError("out must be a contiguous float64 buffer of at least K * n")
            U = flat.reshape(-1)[:K * n].reshape(K, n)
        elif vectors:
            U = np.empty((K, n))
        done = ctypes.c_int32()
        rc = self._lib.te_server_poll(self._h, ticket, ctypes.byref(done),
                                      ctypes.c_void_p(ev.ctypes.data),
                                      None if U is None else ctypes.c_void_p(U.ctypes.data),
                                      ctypes.c_void_p(res.ctypes.data))
        if done.value:
            del self._meta[ticket]
        _check(rc)
        if not done.value:
            return None
        return ev, (None if U is None else U.T), res

    def completed(self, cap: int = 4096):
        """Tickets of the requests that finished since the last call (poll
        each once to collect its results)."""
        import numpy as np
        buf = np.empty(cap, dtype=np.int64)
        cnt = ctypes.c_int32()
        _check(self._lib.te_server_completed(self._h, ctypes.c_void_p(buf.ctypes.data), cap,
                                             ctypes.byref(cnt)))
        return [int(t) for t in buf[:cnt.value]]

    def classes(self):
        """{class key: (window, vmax)} chosen by the per-class autotuner."""
        import numpy as np
        cnt = ctypes.c_int32()
        _check(self._lib.te_server_classes(self._h, None, None, None, 0, ctypes.byref(cnt)))
        n = cnt.value
        k, w, v = (np.zeros(max(n, 1), dtype=np.int32) for _ in range(3))
        _check(self._lib.te_server_classes(self._h, ctypes.c_void_p(k.ctypes.data),
                                           ctypes.c_void_p(w.ctypes.data),
                                           ctypes.c_void_p(v.ctypes.data), n, ctypes.byref(cnt)))
        return {int(k[i]): (int(w[i]), int(v[i])) for i in range(min(n, cnt.value))}

    def stats(self):
        live, pend = ctypes.c_int32(), ctypes.c_int32()
        used, peak = ctypes.c_size_t(), ctypes.c_size_t()
        _check(self._lib.te_server_stats(self._h, ctypes.byref(live), ctypes.byref(pend),
                                         ctypes.byref(used), ctypes.byref(peak)))
        return {"live": live.value, "pending": pend.value, "pool_used": used.value,
                "pool_peak": peak.value}

    def timing(self):
        """Cumulative host seconds: wait, admit, launch, submit, and the
        polls' copies and releases."""
        v = [ctypes.c_double() for _ in range(6)]
        _check(self._lib.te_server_timing(self._h, *[ctypes.byref(x) for x in v]))
        return {k: x.value for k, x in zip(("wait_s", "admit_s", "launch_s", "submit_s",
                                            "poll_copy_s", "poll_free_s"), v)}

    def analysis(self):
        """Analysis threads' cumulative seconds (layout, gather into pinned
        memory, copy to the device, staging wait), requests analysed, engine
        steps and the solves they advanced."""
        d = [ctypes.c_double() for _ in range(4)]
        i = [ctypes.c_int64() for _ in range(3)]
        _check(self._lib.te_server_analysis(self._h, *[ctypes.byref(x) for x in d + i]))
        return {"layout_s": d[0].value, "gather_s": d[1].value, "copy_s": d[2].value,
                "stage_wait_s": d[3].value, "analysed": i[0].value,
                "engine_steps": i[1].value, "resident_steps": i[2].value}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.te_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spmv(csr: CSR, x, precision="ddd", stream=None):
    """y = M x (float64 output) with the solver's SpMV kernel."""
    import torch
    lib = load_library()
    A = csr.to_ctypes()
    y = torch.empty(csr.n, dtype=torch.float64, device="cuda")
    rc = lib.te_spmv(ctypes.byref(A), _prec(precision), ctypes.c_void_p(x.data_ptr()),
                     ctypes.c_void_p(y.data_ptr()), _stream_ptr(stream))
    _check(rc)
    return y


def lanczos(csr: CSR, krylov_steps: int, precision="ddd", *, seed: int = 0, v1=None,
            basis: bool = True, reorth="full", order="keep", stream=None):
    """The Lanczos phase: returns (alpha [m], beta [m+1], V [n, m] or None, restarts)."""
    import torch
    lib = load_library()
    A = csr.to_ctypes()
    opt = _options(seed, v1, "LM", False, reorth=reorth, order=order)
    alpha = torch.empty(krylov_steps, dtype=torch.float64)
    beta = torch.empty(krylov_steps + 1, dtype=torch.float64)
    V = (torch.empty((krylov_steps, csr.n), dtype=torch.float64, device="cuda")
         if basis else None)
    restarts = ctypes.c_int32(0)
    rc = lib.te_lanczos(ctypes.byref(A), krylov_steps, _prec(precision), ctypes.byref(opt),
                        ctypes.c_void_p(alpha.data_ptr()), ctypes.c_void_p(beta.data_ptr()),
                        None if V is None else ctypes.c_void_p(V.data_ptr()),
                        ctypes.byref(restarts), _stream_ptr(stream))
    _check(rc)
    return alpha, beta, (None if V is None else V.t()), int(restarts.value)


def spmv_noalloc(csr: CSR, x, y=None, precision="ddd", stream=None):
    """y = M x (float64) through te_spmv_noalloc, which allocates no device
    memory (its work memory is a fixed array inside the library).  Pass a
    preallocated `y` to keep this call free of allocations on the Python side."""
    import torch
    lib = load_library()
    A = csr.to_ctypes()
    if y is None:
        y = torch.empty(csr.n, dtype=torch.float64, device="cuda")
    rc = lib.te_spmv_noalloc(ctypes.byref(A), _prec(precision), ctypes.c_void_p(x.data_ptr()),
                             ctypes.c_void_p(y.data_ptr()), _stream_ptr(stream))
    _check(rc)
    return y


def spmv_layout(row_ptr, nnz: int, window: int = 0, vmax: int = 0):
    """The SELL-C-sigma layout a plan builds for the SpMV (host analysis):
    returns a dict with slice lengths [S], and per lane (32 per slice) the
    output (row, -1 - piece, or INT32_MIN), the first CSR entry and the length
    of its piece, plus the padded entry count and the number of cut rows."""
    import numpy as np
    lib = load_library()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    n = len(rp) - 1
    ns, ne, nl = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    rc = lib.te_spmv_layout(ctypes.c_void_p(rp.ctypes.data), n, nnz, window, vmax,
                            ctypes.byref(ns), ctypes.byref(ne), ctypes.byref(nl), None, None,
                            None, None)
    _check(rc)
    S = ns.value
    slen = np.zeros(S, dtype=np.int32)
    lout = np.zeros(S * 32, dtype=np.int32)
    lsrc = np.zeros(S * 32, dtype=np.int64)
    llen = np.zeros(S * 32, dtype=np.int32)
    rc = lib.te_spmv_layout(ctypes.c_void_p(rp.ctypes.data), n, nnz, window, vmax, None, None,
                            None, ctypes.c_void_p(slen.ctypes.data),
                            ctypes.c_void_p(lout.ctypes.data), ctypes.c_void_p(lsrc.ctypes.data),
                            ctypes.c_void_p(llen.ctypes.data))
    _check(rc)
    return {"slice_len": slen, "lane_out": lout, "lane_src": lsrc, "lane_len": llen,
            "entries": int(ne.value), "long_rows": int(nl.value)}


def spmv_layout_device(row_ptr_dev, nnz: int, window: int = 0, vmax: int = 0, order="keep",
                       stream=None):
    """The SpMV layout (and row order) built on the device from a device
    row_ptr tensor, as plans build it: a dict like spmv_layout's plus perm,
    slice_base, lane_row, long_rows ((row, first, count) per cut row) and
    nbig."""
    import numpy as np
    lib = load_library()
    n = int(row_ptr_dev.numel()) - 1
    od = ORDERS[order] if isinstance(order, str) else int(order)
    ns, ne, nl = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    st = _stream_ptr(stream)
    _check(lib.te_spmv_layout_device(ctypes.c_void_p(row_ptr_dev.data_ptr()), n, nnz, window,
                                     vmax, od, ctypes.byref(ns), ctypes.byref(ne),
                                     ctypes.byref(nl), *([None] * 10), st))
    S, NL = ns.value, nl.value
    out = {"perm": np.zeros(n, dtype=np.int32), "slice_len": np.zeros(S, dtype=np.int32),
           "slice_base": np.zeros(S, dtype=np.int64), "lane_out": np.zeros(S * 32, dtype=np.int32),
           "lane_src": np.zeros(S * 32, dtype=np.int64), "lane_len": np.zeros(S * 32, dtype=np.int32),
           "lane_row": np.zeros(S * 32, dtype=np.int32),
           "long_rows": np.zeros((NL, 3), dtype=np.int32)}
    nb = ctypes.c_int32()
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data)
    _check(lib.te_spmv_layout_device(ctypes.c_void_p(row_ptr_dev.data_ptr()), n, nnz, window,
                                     vmax, od, None, None, None, ptr(out["perm"]),
                                     ptr(out["slice_len"]), ptr(out["slice_base"]),
                                     ptr(out["lane_out"]), ptr(out["lane_src"]),
                                     ptr(out["lane_len"]), ptr(out["lane_row"]),
                                     ptr(out["long_rows"]), ctypes.byref(nb), st))
    out.update({"entries": int(ne.value), "long_rows_count": NL, "nbig": int(nb.value)})
    return out


def check_symmetric(host_csr, tol: float = 0.0):
    """max |a_ij - a_ji| of a host matrix (an object with n, row_ptr, col, val);
    raises TEError when it exceeds tol."""
    csr = CSR.from_host(host_csr, "ddd", device="cpu")
    A = csr.to_ctypes()
    diff = ctypes.c_double()
    _check(load_library().te_check_symmetric(ctypes.byref(A), tol, ctypes.byref(diff)))
    return diff.value


def degree_order(row_ptr, nnz: int):
    """The row order of order="degree" (host): (perm, iperm), perm[r] = the
    caller's row placed at r."""
    import numpy as np
    lib = load_library()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    n = len(rp) - 1
    perm = np.empty(n, dtype=np.int32)
    iperm = np.empty(n, dtype=np.int32)
    _check(lib.te_degree_order(ctypes.c_void_p(rp.ctypes.data), n, nnz,
                               ctypes.c_void_p(perm.ctypes.data), ctypes.c_void_p(iperm.ctypes.data)))
    return perm, iperm


def quantize(csr: CSR, to: str, stream=None):
    """Round the binary64 values of a device CSR (values_f64) to "f32", "bf16"
    (uint16 codes) or "e4m3" (uint8 codes + float32 row scales), in CSR order,
    with the plans' device rounding.  Returns (out, row_scale or None)."""
    import torch
    lib = load_library()
    kinds = {"f32": (TE_F32, torch.float32), "bf16": (TE_BF16, torch.int16),
             "e4m3": (TE_FP8_E4M3, torch.uint8)}
    code, dt = kinds[to]
    out = torch.empty(max(csr.nnz, 1), dtype=dt, device="cuda")
    scale = torch.empty(csr.n, dtype=torch.float32, device="cuda") if to == "e4m3" else None
    A = csr.to_ctypes()
    rc = lib.te_quantize(ctypes.byref(A), code, ctypes.c_void_p(out.data_ptr()),
                         None if scale is None else ctypes.c_void_p(scale.data_ptr()),
                         _stream_ptr(stream))
    _check(rc)
    return out[:csr.nnz], scale


def probe_gather(table_elems: int, stream=None) -> float:
    """Random 4-byte reads per second from a device table (the SpMV's gather
    ceiling)."""
    lib = load_library()
    r = ctypes.c_double()
    _check(lib.te_probe_gather(table_elems, _stream_ptr(stream), ctypes.byref(r)))
    return r.value


def gram(U, stream=None):
    """G = U^T U (float64, K x K numpy) of the columns of U ((n, K) view of a
    contiguous (K, n) device tensor, or a (K, n) contiguous tensor of rows)."""
    import numpy as np
    lib = load_library()
    base = U.t() if (U.dim() == 2 and not U.is_contiguous() and U.t().is_contiguous()) else U
    K, n = base.shape
    G = np.zeros((K, K))
    rc = lib.te_gram(n, K, ctypes.c_void_p(base.data_ptr()), ctypes.c_void_p(G.ctypes.data),
                     _stream_ptr(stream))
    _check(rc)
    return G


def tridiag_eigs(alpha, beta, which="LM", stream=None):
    """Jacobi on tridiag(alpha; beta[1..m-1]) (device tensors); returns
    (theta [m] in selection order, Y [m, m] columns = eigenvectors, sweeps)."""
    import torch
    lib = load_library()
    m = int(alpha.numel())
    theta = torch.empty(m, dtype=torch.float64, device="cuda")
    Y = torch.empty((m, m), dtype=torch.float64, device="cuda")
    sweeps = ctypes.c_int32(0)
    rc = lib.te_tridiag_eigs(m, ctypes.c_void_p(alpha.data_ptr()), ctypes.c_void_p(beta.data_ptr()),
                             WHICH[which] if isinstance(which, str) else int(which),
                             ctypes.c_void_p(theta.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                             ctypes.byref(sweeps), _stream_ptr(stream))
    _check(rc)
    return theta, Y.t(), int(sweeps.value)
