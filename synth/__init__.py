"""Seeded synthetic inputs for the Top-K sparse eigensolver.

This package only makes inputs (CSR matrices and raw random vectors); it holds
none of the eigensolver's arithmetic.  Both the CUDA path and the CPU oracle
consume what it produces.  The heavy generators live in ``synth.c`` (C with
OpenMP) and are bound with ctypes; the tiny closed-form test matrices (path and
cycle Laplacians, diagonal matrices) are built here with numpy.

Random numbers: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) addressed by
(seed, stream, index), see ``synth.c``.  Results do not depend on the thread
count or the machine.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``libsynth.so`` next to its source (gcc, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-std=c11", "-o", tmp, _SRC, "-lm"]
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
        lib.synth_rng_u64.argtypes = [u64, u64, u64]
        lib.synth_rng_u64.restype = u64
        lib.synth_uniform_pm1.argtypes = [i64, u64, u64, vp]
        lib.synth_uniform_pm1.restype = None
        lib.synth_uniform_sym.argtypes = [i64, i32, u64]
        lib.synth_uniform_sym.restype = vp
        lib.synth_banded_sym.argtypes = [i64, i32, i32, u64]
        lib.synth_banded_sym.restype = vp
        lib.synth_rmat_sym.argtypes = [i32, i32, dbl, dbl, dbl, u64, ctypes.c_int]
        lib.synth_rmat_sym.restype = vp
        lib.synth_planted_sym.argtypes = [i64, i32, i32, i32, dbl, u64]
        lib.synth_planted_sym.restype = vp
        lib.synth_from_triplets.argtypes = [i64, i64, vp, vp, vp]
        lib.synth_from_triplets.restype = vp
        lib.synth_csr_n.argtypes = [vp]
        lib.synth_csr_n.restype = i64
        lib.synth_csr_nnz.argtypes = [vp]
        lib.synth_csr_nnz.restype = i64
        lib.synth_csr_export.argtypes = [vp, vp, vp, vp]
        lib.synth_csr_export.restype = None
        lib.synth_csr_export_f32.argtypes = [vp, vp]
        lib.synth_csr_export_f32.restype = None
        lib.synth_csr_free.argtypes = [vp]
        lib.synth_csr_free.restype = None
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


@dataclass
class CSR:
    """Host CSR matrix: int64 row pointers, int32 columns, float64 values."""
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        np.add.at(d, (rows, self.col.astype(np.int64)), self.val)
        return d

    def values_f32(self) -> np.ndarray:
        """Values rounded to binary32 (round to nearest even)."""
        return self.val.astype(np.float32)

    def with_f32_values(self) -> "CSR":
        """The same matrix holding binary32 values (rounded to nearest even):
        the input of a caller whose data is binary32 already."""
        return CSR(self.n, self.row_ptr, self.col, self.values_f32())


def _take(handle, out=None) -> CSR:
    lib = _load()
    if not handle:
        raise ValueError("synth: generator rejected its arguments or ran out of memory")
    try:
        n = lib.synth_csr_n(handle)
        nnz = lib.synth_csr_nnz(handle)
        rp = np.empty(n + 1, dtype=np.int64)
        col = np.empty(max(nnz, 0), dtype=np.int32)
        val = np.empty(max(nnz, 0), dtype=np.float64)
        lib.synth_csr_export(handle, _ptr(rp), _ptr(col), _ptr(val))
    finally:
        lib.synth_csr_free(handle)
    return CSR(int(n), rp, col, val)


def rng_u64(seed: int, stream: int, index: int) -> int:
    return int(_load().synth_rng_u64(seed, stream, index))


def uniform_pm1(n: int, seed: int, stream: int = 0) -> np.ndarray:
    """Raw uniform(-1,1) vector (draws 0..n-1 of (seed, stream)); not normalised."""
    out = np.empty(n, dtype=np.float64)
    _load().synth_uniform_pm1(n, seed, stream, _ptr(out))
    return out


def start_vector(n: int, seed: int) -> np.ndarray:
    """The raw start vector the solver normalises: stream 0 of ``seed``."""
    return uniform_pm1(n, seed, 0)


def uniform_sym(n: int, per_row: int, seed: int) -> CSR:
    """``per_row`` uniform-random columns per row, values uniform(0,1), then A + A^T."""
    return _take(_load().synth_uniform_sym(n, per_row, seed))


def banded_sym(n: int, per_row: int, half_width: int, seed: int) -> CSR:
    """``per_row`` columns per row drawn from the ``half_width`` columns right of
    the diagonal, values uniform(0,1), then A + A^T: a banded, mesh-like matrix
    whose SpMV reads x with locality (see ``synth.c``)."""
    return _take(_load().synth_banded_sym(n, per_row, half_width, seed))


def rmat_sym(scale: int, edge_factor: int, seed: int, a: float = 0.57, b: float = 0.19,
             c: float = 0.19, normalized: bool = True) -> CSR:
    """Symmetric R-MAT graph, optionally as D^-1/2 A D^-1/2 (see ``synth.c``)."""
    return _take(_load().synth_rmat_sym(scale, edge_factor, a, b, c, seed, int(normalized)))


def normalize_sym(A: CSR) -> CSR:
    """D^-1/2 W D^-1/2 with the weighted degrees d_i = sum_j |w_ij| (an input
    transformation: rows of weight 0 stay empty)."""
    d = np.add.reduceat(np.abs(A.val), A.row_ptr[:-1]) if A.nnz else np.zeros(A.n)
    d = np.where(np.diff(A.row_ptr) > 0, d, 0.0)
    inv = np.where(d > 0, 1.0 / np.sqrt(np.where(d > 0, d, 1.0)), 0.0)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    return CSR(A.n, A.row_ptr.copy(), A.col.copy(), A.val * inv[rows] * inv[A.col])


def planted_sym(n: int, per_row: int, ncomm: int, smin: int, ratio: float, seed: int) -> CSR:
    """The uniform background of ``uniform_sym`` plus ``ncomm`` disjoint unit
    cliques of sizes round(smin * ratio^k), k = 0 .. ncomm-1, on seeded random
    vertices: ``ncomm`` eigenvalues near the clique sizes minus one stand out
    of the background's spectrum in a geometric progression (see ``synth.c``)."""
    return _take(_load().synth_planted_sym(n, per_row, ncomm, smin, ratio, seed))


def serving_requests(count: int, seed: int):
    """Independent solve requests shaped like a serving mix: n log-uniform in
    [2^10, 2^18], mean degree uniform in [4, 64], half uniform-random (values
    uniform(0,1), symmetrically normalised) and half R-MAT (normalised
    adjacency), K in {4, 8, 16} with m = 2K, binary32 or bfloat16 values.
    Returns a list of (matrix, K, m, precision)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(2.0 ** rng.uniform(10, 18))
        deg = int(rng.integers(4, 65))
        K = int(rng.choice([4, 8, 16]))
        prec = "fdf" if rng.random() < 0.5 else "bdf"
        mseed = int(seed) * 1_000_003 + i
        if rng.random() < 0.5:
            A = normalize_sym(uniform_sym(n, max(1, deg // 2), mseed))
        else:
            A = rmat_sym(max(10, int(round(np.log2(n)))), max(1, deg // 2), mseed)
        out.append((A, K, 2 * K, prec))
    return out


def from_triplets(n: int, rows, cols, vals) -> CSR:
    """CSR from (row, col, value) entries; duplicates summed, columns sorted."""
    r = np.ascontiguousarray(rows, dtype=np.int32)
    c = np.ascontiguousarray(cols, dtype=np.int32)
    v = np.ascontiguousarray(vals, dtype=np.float64)
    return _take(_load().synth_from_triplets(n, len(r), _ptr(r), _ptr(c), _ptr(v)))


def from_dense(d: np.ndarray) -> CSR:
    r, c = np.nonzero(d)
    return from_triplets(d.shape[0], r, c, d[r, c])


# ---------------------------------------------------------------------------
# Closed-form test matrices (tiny; numpy)
# ---------------------------------------------------------------------------

def path_laplacian(n: int) -> CSR:
    """Laplacian of the path graph P_n; eigenvalues 2 - 2 cos(pi k / n), k = 0..n-1."""
    rows, cols, vals = [], [], []
    for i in range(n):
        deg = (1 if i > 0 else 0) + (1 if i < n - 1 else 0)
        rows.append(i); cols.append(i); vals.append(float(deg))
        if i > 0:
            rows.append(i); cols.append(i - 1); vals.append(-1.0)
        if i < n - 1:
            rows.append(i); cols.append(i + 1); vals.append(-1.0)
    return from_triplets(n, rows, cols, vals)


def cycle_laplacian(n: int) -> CSR:
    """Laplacian of the cycle C_n; eigenvalues 2 - 2 cos(2 pi k / n), k = 0..n-1."""
    rows, cols, vals = [], [], []
    for i in range(n):
        rows += [i, i, i]
        cols += [i, (i - 1) % n, (i + 1) % n]
        vals += [2.0, -1.0, -1.0]
    return from_triplets(n, rows, cols, vals)


def diagonal(d) -> CSR:
    d = np.asarray(d, dtype=np.float64)
    idx = np.arange(len(d))
    return from_triplets(len(d), idx, idx, d)


def tridiag_toeplitz(n: int, a: float, b: float) -> CSR:
    """Tridiagonal Toeplitz (a on the diagonal, b off it): a + 2 b cos(pi k/(n+1))."""
    rows, cols, vals = [], [], []
    for i in range(n):
        rows.append(i); cols.append(i); vals.append(a)
        if i > 0:
            rows.append(i); cols.append(i - 1); vals.append(b)
        if i < n - 1:
            rows.append(i); cols.append(i + 1); vals.append(b)
    return from_triplets(n, rows, cols, vals)
