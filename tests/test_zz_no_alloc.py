"""te_spmv_noalloc: the SpMV for callers that cannot allocate device memory.

Such callers (another allocator owns the device memory, or a serving loop
must not pay for allocator locks and latency) get an entry point whose work
memory is a fixed array inside the library.  This test calls it through the
C ABI and checks it against the oracle's SpMV, row by row within the
summation bound the other SpMV parity tests use, on two calls in a row (the
shared array keeps the first call's contents, which must not leak into the
second), and against te_spmv, the allocating entry point.  It covers empty
rows, a hub row that spans many chunks, a matrix without entries, and input
the device rejects (a column outside [0, n), malformed row pointers), after
which the next call works again.  It is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def te():
    import paper_2201_07498_gb300 as te
    te.load_library(build_if_missing=True)
    return te


def _star(n, seed):
    """Symmetric: a hub row of length n-1 (spans many chunks), ragged rows,
    empty rows."""
    rng = np.random.default_rng(seed)
    r, c = [0] * (n - 1), list(range(1, n))
    for i in range(1, n, 3):
        for j in rng.integers(1, n, size=rng.integers(0, 40)):
            r.append(i)
            c.append(int(j))
    v = rng.uniform(0.1, 1.0, size=len(r))
    return synth.from_triplets(n, r + c, c + r, np.concatenate([v, v]))


def _bound(A, x, u):
    """The two sides sum the same products in different orders: a row may
    differ by 2 gamma_k sum_j |a_rj x_j| (gamma_k = k u / (1 - k u))."""
    absprod = oracle.spmv(synth.CSR(A.n, A.row_ptr, A.col, np.abs(A.val)), np.abs(x))
    k = np.maximum(np.diff(A.row_ptr), 1).astype(np.float64)
    return 2 * k * u / (1 - k * u) * absprod + 1e-300


def _call_noalloc(te, csr, x, y, prec, nnz=None):
    lib = te.load_library()
    A = csr.to_ctypes()
    if nnz is not None:
        A.nnz = nnz
    return lib.te_spmv_noalloc(ctypes.byref(A), te._prec(prec), ctypes.c_void_p(x.data_ptr()),
                               ctypes.c_void_p(y.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _inputs(A, prec, call):
    """(host matrix as the CUDA path gets it, the same values in binary64 for
    the oracle, x in binary64, x on the device)."""
    x = synth.uniform_pm1(A.n, 5 + call, 2)
    if prec == "fdf":
        A_in = A.with_f32_values()
        A64 = synth.CSR(A.n, A.row_ptr, A.col, A_in.val.astype(np.float64))
        x32 = x.astype(np.float32)
        return A_in, A64, x32.astype(np.float64), torch.from_numpy(x32).cuda()
    return A, A, x, torch.from_numpy(x).cuda()


@pytest.mark.parametrize("prec", ["ddd", "fdf"])
def test_noalloc_matches_oracle_on_two_calls(te, prec):
    """y = M x against the oracle within the summation bound (binary64, or
    double-float with u = 2^-44 as a margin over its 2^-48), two calls in a
    row on different matrices; also equal to te_spmv within the same bound."""
    mats = [_star(20000, 1), synth.rmat_sym(13, 8, 4)]
    u = 2.0 ** -53 if prec == "ddd" else 2.0 ** -44
    for call, A in enumerate(mats):
        A_in, A64, x, xd = _inputs(A, prec, call)
        csr = te.CSR.from_host(A_in, prec)
        y = torch.full((A.n,), float("nan"), dtype=torch.float64, device="cuda")
        rc = _call_noalloc(te, csr, xd, y, prec)
        assert rc == 0, te.load_library().te_last_error()
        yh = y.cpu().numpy()
        bound = _bound(A64, x, u)
        ref = oracle.spmv(A64, x)
        assert np.all(np.abs(yh - ref) <= bound), (call, np.nanmax(np.abs(yh - ref)))
        y_alloc = te.spmv(csr, xd, prec).cpu().numpy()
        assert np.all(np.abs(yh - y_alloc) <= 2 * bound), call


def test_noalloc_matrix_without_entries(te):
    """nnz = 0: no chunk kernel runs; every row is empty and gets 0."""
    n = 1000
    A = synth.CSR(n, np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32),
                  np.zeros(0, dtype=np.float64))
    rp = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    ci = torch.zeros(1, dtype=torch.int32, device="cuda")
    va = torch.zeros(1, dtype=torch.float64, device="cuda")
    x = torch.from_numpy(synth.uniform_pm1(n, 3, 1)).cuda()
    y = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    lib = te.load_library()
    cA = te.te_csr(n, 0, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), None, 0, 0)
    rc = lib.te_spmv_noalloc(ctypes.byref(cA), te._prec("ddd"), ctypes.c_void_p(x.data_ptr()),
                             ctypes.c_void_p(y.data_ptr()), None)
    assert rc == 0, lib.te_last_error()
    assert np.array_equal(y.cpu().numpy(), oracle.spmv(A, x.cpu().numpy()))


def test_noalloc_rejects_bad_input_then_recovers(te):
    A = synth.uniform_sym(3000, 5, 9)
    x = torch.from_numpy(synth.uniform_pm1(A.n, 1, 1)).cuda()
    y = torch.empty(A.n, dtype=torch.float64, device="cuda")
    bad = synth.CSR(A.n, A.row_ptr, A.col.copy(), A.val)
    bad.col[7] = A.n  # out of range: the kernel's bounds check reports it
    assert _call_noalloc(te, te.CSR.from_host(bad, "ddd"), x, y, "ddd") == 1
    assert b"column index" in te.load_library().te_last_error()
    # row pointers that decrease in the middle (each access stays in bounds)
    rp = A.row_ptr.copy()
    rp[100] = rp[102] + 3
    bad = synth.CSR(A.n, rp, A.col, A.val)
    assert _call_noalloc(te, te.CSR.from_host(bad, "ddd"), x, y, "ddd") == 1
    assert b"row_ptr" in te.load_library().te_last_error()
    # row_ptr[n] != nnz: fewer entries declared than the row pointers span
    good = te.CSR.from_host(A, "ddd")
    assert _call_noalloc(te, good, x, y, "ddd", nnz=A.nnz - 5) == 1
    assert b"row_ptr" in te.load_library().te_last_error()
    # the status word is cleared by the next call
    assert _call_noalloc(te, good, x, y, "ddd") == 0
    ref = oracle.spmv(A, x.cpu().numpy())
    assert np.all(np.abs(y.cpu().numpy() - ref) <= _bound(A, x.cpu().numpy(), 2.0 ** -53))


def test_noalloc_rejects_sizes_beyond_the_scratch(te):
    lib = te.load_library()
    rp = torch.zeros(2, dtype=torch.int64, device="cuda")
    ci = torch.zeros(1, dtype=torch.int32, device="cuda")
    va = torch.zeros(1, dtype=torch.float64, device="cuda")
    # nnz above 131072 * 2048 (the DDD limit); rejected before any kernel runs
    A = te.te_csr(1, 131072 * 2048 + 1, rp.data_ptr(), ci.data_ptr(), va.data_ptr(), None, 0)
    y = torch.empty(1, dtype=torch.float64, device="cuda")
    rc = lib.te_spmv_noalloc(ctypes.byref(A), te._prec("ddd"), ctypes.c_void_p(va.data_ptr()),
                             ctypes.c_void_p(y.data_ptr()), None)
    assert rc == 1
    assert b"exceeds the maximum" in lib.te_last_error()
