"""Plain FP64 CPU oracle of the Top-K sparse eigensolver.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product path never
imports this package, and this package imports nothing from the product.

The arithmetic lives in ``oracle.c`` (binary64, following Algorithm 1 of
Sgherzi et al., arXiv 2201.07498, and a cyclic Jacobi on T); this module only
compiles it on demand (gcc, OpenMP) and marshals numpy arrays through ctypes.

Every oracle function is pinned by the ``-m "not gpu"`` tests against closed
forms, brute force and invariants; see ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

LARGEST_MAGNITUDE = 0
LARGEST_ALGEBRAIC = 1
BREAKDOWN_TOL = 1e-12
JACOBI_TOL = 1e-16
JACOBI_MAX_SWEEPS = 100

FAULTS = {
    "none": 0,
    "beta_index": 1,
    "alpha_sign": 2,
    "no_reorth": 3,
    "jacobi_sign": 4,
    "ritz_transpose": 5,
    "select_algebraic": 6,
    "spmv_skip_last": 7,
    "no_v1_normalise": 8,
    "refine_no_norm": 9,
    "angle_signed": 10,
    "reorth_ignored": 11,
    "ties_away": 12,
}


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to its source."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        i64, u64, i32, dbl, vp = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32,
                                  ctypes.c_double, ctypes.c_void_p)
        lib.oracle_set_fault.argtypes = [ctypes.c_int]
        lib.oracle_set_fault.restype = None
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
        lib.oracle_set_num_threads.restype = None
        lib.oracle_spmv.argtypes = [i64, vp, vp, vp, vp, vp]
        lib.oracle_spmv.restype = None
        lib.oracle_spmv_row.argtypes = [vp, vp, vp, vp, i64]
        lib.oracle_spmv_row.restype = dbl
        lib.oracle_lanczos.argtypes = [i64, vp, vp, vp, vp, i32, u64, dbl, vp, vp, vp, vp, vp]
        lib.oracle_lanczos.restype = ctypes.c_int
        lib.oracle_jacobi.argtypes = [i32, vp, vp, dbl, i32, vp]
        lib.oracle_jacobi.restype = ctypes.c_int
        lib.oracle_select_topk.argtypes = [i32, vp, i32, i32, vp]
        lib.oracle_select_topk.restype = None
        lib.oracle_ritz.argtypes = [i64, i32, vp, vp, i32, vp, vp]
        lib.oracle_ritz.restype = None
        lib.oracle_topk_eigs.argtypes = [i64, vp, vp, vp, vp, i32, i32, i32, u64, vp, vp, vp,
                                         vp, vp, vp]
        lib.oracle_topk_eigs.restype = ctypes.c_int
        lib.oracle_lanczos_ex.argtypes = [i64, vp, vp, vp, vp, i32, u64, dbl, i32, vp, vp, vp,
                                          vp, vp]
        lib.oracle_lanczos_ex.restype = ctypes.c_int
        lib.oracle_topk_eigs_ex.argtypes = [i64, vp, vp, vp, vp, i32, i32, i32, u64, i32, vp,
                                            vp, vp, vp, vp, vp]
        lib.oracle_topk_eigs_ex.restype = ctypes.c_int
        lib.oracle_refine.argtypes = [i64, vp, vp, vp, i32, vp, vp, vp]
        lib.oracle_refine.restype = None
        lib.oracle_mean_pairwise_angle.argtypes = [i64, i32, vp]
        lib.oracle_mean_pairwise_angle.restype = dbl
        lib.oracle_round_bf16.argtypes = [i64, vp, vp, vp]
        lib.oracle_round_bf16.restype = None
        lib.oracle_quantize_e4m3_rows.argtypes = [i64, vp, vp, vp, vp, vp]
        lib.oracle_quantize_e4m3_rows.restype = None
        lib.oracle_e4m3_value.argtypes = [ctypes.c_uint8]
        lib.oracle_e4m3_value.restype = dbl
        _lib = lib
        return lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _csr_arrays(csr):
    rp = np.ascontiguousarray(csr.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(csr.col, dtype=np.int32)
    val = np.ascontiguousarray(csr.val, dtype=np.float64)
    return int(csr.n), rp, ci, val


class fault:
    """Context manager planting one known mistake in the oracle (tests only)."""

    def __init__(self, name: str):
        self.kind = FAULTS[name]

    def __enter__(self):
        _load().oracle_set_fault(self.kind)
        return self

    def __exit__(self, *exc):
        _load().oracle_set_fault(0)
        return False


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(threads: int) -> None:
    """Thread count of the oracle's OpenMP regions from now on (for timing;
    the results do not depend on it)."""
    _load().oracle_set_num_threads(int(threads))


def spmv(csr, x) -> np.ndarray:
    """y = M x (Algorithm 1, SpMV step)."""
    n, rp, ci, val = _csr_arrays(csr)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(n)
    _load().oracle_spmv(n, _p(rp), _p(ci), _p(val), _p(x), _p(y))
    return y


def spmv_rows(csr, x, rows) -> np.ndarray:
    """(M x)[r] for the sampled rows only."""
    _, rp, ci, val = _csr_arrays(csr)
    x = np.ascontiguousarray(x, dtype=np.float64)
    lib = _load()
    return np.array([lib.oracle_spmv_row(_p(rp), _p(ci), _p(val), _p(x), int(r)) for r in rows])


@dataclass
class LanczosResult:
    alpha: np.ndarray       # m
    beta: np.ndarray        # m + 1; beta[0] = 0, beta[i] = beta_{i+1}
    V: np.ndarray           # n x m (column j = v_{j+1})
    w_last: np.ndarray      # unnormalised last v_nxt (norm beta[m])
    restarts: int

    def T(self) -> np.ndarray:
        m = len(self.alpha)
        return (np.diag(self.alpha) + np.diag(self.beta[1:m], 1)
                + np.diag(self.beta[1:m], -1))


def lanczos(csr, v1_raw, m: int, seed: int = 0, tol: float = BREAKDOWN_TOL,
            reorth: bool = True) -> LanczosResult:
    """Algorithm 1 (reorth=False: the variant without reorthogonalisation)."""
    n, rp, ci, val = _csr_arrays(csr)
    v1 = np.ascontiguousarray(v1_raw, dtype=np.float64)
    alpha = np.empty(m)
    beta = np.empty(m + 1)
    V = np.empty((m, n))  # row j of this array is column j of V
    w = np.empty(n)
    restarts = np.zeros(1, dtype=np.int32)
    rc = _load().oracle_lanczos_ex(n, _p(rp), _p(ci), _p(val), _p(v1), m, seed, tol,
                                   1 if reorth else 0, _p(alpha), _p(beta), _p(V), _p(w),
                                   _p(restarts))
    if rc != 0:
        raise ValueError(f"oracle_lanczos failed with code {rc}")
    return LanczosResult(alpha, beta, V.T.copy(), w, int(restarts[0]))


def jacobi(T, tol: float = JACOBI_TOL, max_sweeps: int = JACOBI_MAX_SWEEPS):
    """Cyclic Jacobi: returns (theta, Y, sweeps, converged); T's diagonal after rotation."""
    T = np.array(T, dtype=np.float64, order="C", copy=True)
    m = T.shape[0]
    Y = np.empty((m, m))
    sweeps = np.zeros(1, dtype=np.int32)
    rc = _load().oracle_jacobi(m, _p(T), _p(Y), tol, max_sweeps, _p(sweeps))
    return np.diag(T).copy(), Y, int(sweeps[0]), rc == 0


def select_topk(theta, K: int, which: int = LARGEST_MAGNITUDE) -> np.ndarray:
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    idx = np.empty(K, dtype=np.int32)
    _load().oracle_select_topk(len(theta), _p(theta), K, which, _p(idx))
    return idx


def ritz(V, Y, idx) -> np.ndarray:
    """U[:, k] = sign_k * V @ Y[:, idx[k]] (n x K)."""
    n, m = V.shape
    Vc = np.ascontiguousarray(V.T, dtype=np.float64)  # column-major V
    Yc = np.ascontiguousarray(Y, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    K = len(idx)
    U = np.empty((K, n))
    _load().oracle_ritz(n, m, _p(Vc), _p(Yc), K, _p(idx), _p(U))
    return U.T.copy()


@dataclass
class TopKResult:
    eigvals: np.ndarray
    eigvecs: np.ndarray | None
    residuals: np.ndarray | None
    alpha: np.ndarray
    beta: np.ndarray
    restarts: int
    sweeps: int
    converged: bool


def refine(csr, U):
    """Rayleigh quotients u'Mu/u'u and residuals ||Mu - theta u|| / ||u|| of the
    columns of U (n x K), in binary64."""
    n, rp, ci, val = _csr_arrays(csr)
    Uc = np.ascontiguousarray(np.asarray(U, dtype=np.float64).T)  # column-major
    K = Uc.shape[0]
    th = np.empty(K)
    res = np.empty(K)
    _load().oracle_refine(n, _p(rp), _p(ci), _p(val), K, _p(Uc), _p(th), _p(res))
    return th, res


def round_bf16(x):
    """bfloat16 rounding (nearest, ties to even): (codes uint16, values float64)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    codes = np.empty(x.shape, dtype=np.uint16)
    deq = np.empty(x.shape)
    _load().oracle_round_bf16(x.size, _p(x), _p(codes), _p(deq))
    return codes, deq


def quantize_e4m3_rows(csr):
    """FP8 E4M3 with one binary32 scale per row: (codes uint8 [nnz],
    scales float32 [n], dequantised values float64 [nnz])."""
    n, rp, ci, val = _csr_arrays(csr)
    codes = np.empty(len(val), dtype=np.uint8)
    scale = np.empty(n, dtype=np.float32)
    deq = np.empty(len(val))
    _load().oracle_quantize_e4m3_rows(n, _p(rp), _p(val), _p(codes), _p(scale), _p(deq))
    return codes, scale, deq


def e4m3_value(code: int) -> float:
    return float(_load().oracle_e4m3_value(code))


def mean_pairwise_angle(U) -> float:
    """Mean sign-free angle (degrees) between the columns of U (n x K)."""
    Uc = np.ascontiguousarray(np.asarray(U, dtype=np.float64).T)
    K, n = Uc.shape
    return float(_load().oracle_mean_pairwise_angle(n, K, _p(Uc)))


def topk_eigs(csr, K: int, m: int, v1_raw, which: int = LARGEST_MAGNITUDE, seed: int = 0,
              want_vectors: bool = True, want_residuals: bool = True,
              reorth: bool = True) -> TopKResult:
    n, rp, ci, val = _csr_arrays(csr)
    v1 = np.ascontiguousarray(v1_raw, dtype=np.float64)
    ev = np.empty(K)
    U = np.empty((K, n)) if want_vectors else None
    res = np.empty(K) if want_residuals else None
    alpha = np.empty(m)
    beta = np.empty(m + 1)
    info = np.zeros(3, dtype=np.int32)
    rc = _load().oracle_topk_eigs_ex(n, _p(rp), _p(ci), _p(val), _p(v1), K, m, which, seed,
                                     1 if reorth else 0, _p(ev), _p(U), _p(res), _p(alpha),
                                     _p(beta), _p(info))
    if rc < 0:
        raise ValueError(f"oracle_topk_eigs failed with code {rc}")
    return TopKResult(ev, None if U is None else U.T.copy(), res, alpha, beta, int(info[0]),
                      int(info[1]), rc == 0)
