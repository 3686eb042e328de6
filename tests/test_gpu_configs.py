"""Parity at the other workloads' own sizes, on sampled outputs and on
properties that hold at any size.

* Precision sweep (R-MAT 2^22, edge factor 16, seed 2, normalised adjacency,
  128 M stored non-zeros): the SpMV of every mixed form on sampled rows
  (random, the longest, empty ones) against the oracle's rows on the same
  rounded or quantised values, within the summation bound; the BDF solve
  (K = 16, m = 32, the benchmark's plan options) tied to the bfloat16 matrix
  through the oracle's SpMV: orthonormal basis, T = V^T M V, the Lanczos
  relation, and every returned pair's true residual equal to its estimate,
  all at the binary32 level (64 u32 ||T||).
* Host-streamed (R-MAT 2^25, edge factor 16, seed 3, about 1.07 G stored
  non-zeros, FDD, K = 8, m = 16, 4 GB matrix budget): the streamed solve
  equals the resident solve bit for bit, and the true residual of every
  returned pair (the oracle's SpMV on the binary32-rounded matrix) equals
  its estimate to 1e-9 ||T||.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from test_gpu_parity import spmv_bound

pytestmark = pytest.mark.gpu

LVL32 = 64 * 2.0 ** -24


@pytest.fixture(scope="module")
def te():
    import paper_2201_07498_gb300 as te
    te.load_library(build_if_missing=True)
    return te


@pytest.fixture(scope="module")
def sweep():
    return synth.rmat_sym(22, 16, 2)


def _sample_rows(A, rng):
    deg = np.diff(A.row_ptr)
    rows = list(rng.choice(A.n, size=2000, replace=False))
    rows += list(np.argsort(deg)[-20:])
    rows += list(np.nonzero(deg == 0)[0][:10])
    return np.array(sorted(set(int(r) for r in rows)))


def _stored(A, prec):
    """The matrix a form computes with, as binary64 values."""
    if prec == "fdf":
        return synth.CSR(A.n, A.row_ptr, A.col, A.val.astype(np.float32).astype(np.float64))
    if prec == "bdf":
        return synth.CSR(A.n, A.row_ptr, A.col, oracle.round_bf16(A.val)[1])
    return synth.CSR(A.n, A.row_ptr, A.col, oracle.quantize_e4m3_rows(A)[2])


def _rows_bound(Aq, x, rows, u):
    absref = oracle.spmv_rows(synth.CSR(Aq.n, Aq.row_ptr, Aq.col, np.abs(Aq.val)), np.abs(x),
                              rows)
    k = np.maximum(np.diff(Aq.row_ptr)[rows], 1).astype(np.float64)
    return 2 * k * u / (1 - k * u) * absref + 1e-300


@pytest.mark.parametrize("prec", ["fdf", "bdf", "8df"])
def test_sweep_spmv_sampled_rows(te, sweep, prec):
    A = sweep
    Aq = _stored(A, prec)
    x = synth.uniform_pm1(A.n, 91, 4).astype(np.float32).astype(np.float64)
    rows = _sample_rows(A, np.random.default_rng(1))
    y = te.spmv(te.CSR.from_host(A, prec), torch.from_numpy(x.astype(np.float32)).cuda(), prec)
    y = y[torch.from_numpy(rows).cuda()].cpu().numpy()
    ref = oracle.spmv_rows(Aq, x, rows)
    assert np.all(np.abs(y - ref) <= _rows_bound(Aq, x, rows, 2.0 ** -44))


def test_sweep_bdf_solve_is_valid(te, sweep):
    """The BDF form's basis, T and Ritz pairs, tied to the bfloat16 matrix
    through the oracle's SpMV (see the module docstring)."""
    A = sweep
    Aq = _stored(A, "bdf")
    K, m = 16, 32
    csr = te.CSR.from_host(A, "bdf")
    alpha, beta, V, _ = te.lanczos(csr, m, "bdf", seed=2, reorth="delayed", order="degree")
    Vc = V.t().cpu().numpy()
    del V
    alpha, beta = alpha.numpy(), beta.numpy()
    T = np.diag(alpha) + np.diag(beta[1:m], 1) + np.diag(beta[1:m], -1)
    tn = np.linalg.norm(T, 2)
    assert np.max(np.abs(Vc @ Vc.T - np.eye(m))) <= LVL32
    MV = np.stack([oracle.spmv(Aq, Vc[j]) for j in range(m)])
    assert np.max(np.abs(Vc @ MV.T - T)) <= LVL32 * tn
    for j in range(m - 1):
        r = MV[j] - alpha[j] * Vc[j] - beta[j + 1] * Vc[j + 1]
        if j > 0:
            r -= beta[j] * Vc[j - 1]
        assert np.linalg.norm(r) <= LVL32 * tn, j
    del MV
    plan = te.Plan(csr, K, m, "bdf", seed=2, reorth="delayed", order="degree")
    ev, U, res = plan.solve(residuals=True)
    del plan
    ev, res = ev.numpy(), res.numpy()
    th = np.linalg.eigvalsh(T)
    assert np.all(np.min(np.abs(th[None, :] - ev[:, None]), axis=1) <= 1e-10 * tn)
    Uc = U.t().cpu().numpy()
    del U
    for k in range(K):
        true = np.linalg.norm(oracle.spmv(Aq, Uc[k]) - ev[k] * Uc[k]) / np.linalg.norm(Uc[k])
        assert abs(true - res[k]) <= LVL32 * tn, (k, true, res[k])


def test_streamed_full_size_equals_resident(te):
    A = synth.rmat_sym(25, 16, 3)
    K, m = 8, 16
    host = te.CSR.from_host(A, "fdd", device="cpu", pin=True)
    p_str = te.Plan(host, K, m, "fdd", seed=3, matrix_budget=4 << 30)
    assert p_str.stream_blocks >= 2
    ev1, U1, r1 = p_str.solve(residuals=True)
    del p_str
    p_res = te.Plan(te.CSR.from_host(A, "fdd"), K, m, "fdd", seed=3)
    ev2, U2, r2 = p_res.solve(residuals=True)
    del p_res
    assert torch.equal(ev1, ev2) and torch.equal(r1, r2)
    assert torch.equal(U1.cpu(), U2.cpu())
    del U2, host
    A32 = synth.CSR(A.n, A.row_ptr, A.col, A.val.astype(np.float32).astype(np.float64))
    del A
    Uc = U1.t().cpu().numpy()
    del U1
    ev, res = ev1.numpy(), r1.numpy()
    scale = np.max(np.abs(ev))
    for k in range(K):
        true = np.linalg.norm(oracle.spmv(A32, Uc[k]) - ev[k] * Uc[k]) / np.linalg.norm(Uc[k])
        assert abs(true - res[k]) <= 1e-9 * scale, (k, true, res[k])
