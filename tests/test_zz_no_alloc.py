"""te_spmv_noalloc: the SpMV for callers that cannot allocate device memory.

Such callers (another allocator owns the device memory, or a serving loop
must not pay for allocator locks and latency) get an entry point whose work
memory is a fixed array inside the library.  This test calls it through the
C ABI and checks it against te_spmv, the allocating entry point, within the
SpMV summation bound used by the other parity tests, on two calls in a row
(the shared array keeps the first call's contents, which must not leak into
the second).  It is collected last on purpose.
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
    """Two summation orders of the same products differ by at most twice the
    standard bound gamma_k * sum_j |a_rj x_j| per row."""
    absprod = oracle.spmv(synth.CSR(A.n, A.row_ptr, A.col, np.abs(A.val)), np.abs(x))
    k = np.maximum(np.diff(A.row_ptr), 1).astype(np.float64)
    return 4 * k * u / (1 - k * u) * absprod + 1e-300


def _call_noalloc(te, csr, x, y, prec):
    lib = te.load_library()
    A = csr.to_ctypes()
    return lib.te_spmv_noalloc(ctypes.byref(A), te._prec(prec), ctypes.c_void_p(x.data_ptr()),
                               ctypes.c_void_p(y.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("prec", ["ddd", "fdf"])
def test_noalloc_matches_te_spmv_on_two_calls(te, prec):
    mats = [_star(20000, 1), synth.rmat_sym(13, 8, 4)]
    u = 2.0 ** -53 if prec == "ddd" else 2.0 ** -44
    for call, A in enumerate(mats):
        if prec == "fdf":
            A = synth.CSR(A.n, A.row_ptr, A.col, A.val.astype(np.float32).astype(np.float64))
        x = synth.uniform_pm1(A.n, 5 + call, 2)
        if prec == "fdf":
            x = x.astype(np.float32).astype(np.float64)
            xd = torch.from_numpy(x.astype(np.float32)).cuda()
        else:
            xd = torch.from_numpy(x).cuda()
        csr = te.CSR.from_host(A, prec)
        y_ref = te.spmv(csr, xd, prec).cpu().numpy()
        y = torch.full((A.n,), float("nan"), dtype=torch.float64, device="cuda")
        rc = _call_noalloc(te, csr, xd, y, prec)
        assert rc == 0, te.load_library().te_last_error()
        diff = np.abs(y.cpu().numpy() - y_ref)
        assert np.all(diff <= _bound(A, x, u)), (call, np.nanmax(diff))


def test_noalloc_rejects_bad_input_then_recovers(te):
    A = synth.uniform_sym(3000, 5, 9)
    x = torch.from_numpy(synth.uniform_pm1(A.n, 1, 1)).cuda()
    bad = synth.CSR(A.n, A.row_ptr, A.col.copy(), A.val)
    bad.col[7] = A.n  # out of range: the kernel's bounds check reports it
    y = torch.empty(A.n, dtype=torch.float64, device="cuda")
    assert _call_noalloc(te, te.CSR.from_host(bad, "ddd"), x, y, "ddd") == 1
    # the status word is cleared by the next call
    good = te.CSR.from_host(A, "ddd")
    assert _call_noalloc(te, good, x, y, "ddd") == 0
    ref = te.spmv(good, x, "ddd").cpu().numpy()
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
