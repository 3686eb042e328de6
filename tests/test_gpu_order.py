"""Rows relabelled by degree (te_options.order = TE_ORDER_DEGREE).

The plan solves P M P^T for the permutation that sorts the rows by length;
the caller must see no difference beyond rounding: the start vector and the
restart draws are indexed by the caller's rows, the Ritz vectors and the
Lanczos basis come back in the caller's row order.  So the FP64 form still
matches the oracle (run on the caller's matrix, in the caller's order) within
the parity tolerances, restart counts included, and the two orders agree.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from test_gpu_parity import SOLVE_CASES, f32_matrix, match_pairs, subspace_angles

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def te():
    import paper_2201_07498_gb300 as te
    te.load_library(build_if_missing=True)
    return te


@pytest.mark.parametrize("name,make,K,m,which", SOLVE_CASES, ids=[c[0] for c in SOLVE_CASES])
@pytest.mark.parametrize("reorth", ["full", "delayed"])
def test_degree_order_ddd_matches_oracle(te, name, make, K, m, which, reorth):
    A = make()
    v1 = synth.start_vector(A.n, 3)
    w = oracle.LARGEST_MAGNITUDE if which == "LM" else oracle.LARGEST_ALGEBRAIC
    ref = oracle.topk_eigs(A, K, m, v1, which=w, seed=3)
    ev, U, res = te.topk_eigs(te.CSR.from_host(A, "ddd"), K, m, "ddd", seed=3,
                              v1=torch.from_numpy(v1).cuda(), which=which, residuals=True,
                              reorth=reorth, order="degree")
    ev = ev.numpy()
    scale = np.max(np.abs(ref.eigvals))
    perm = match_pairs(ev, ref.eigvals, 1e-10 * scale)
    rel = np.abs(ev - ref.eigvals[perm]) / np.maximum(np.abs(ref.eigvals[perm]), 1e-300)
    assert np.max(rel) <= 1e-10, (ev, ref.eigvals)
    ang = subspace_angles(U.cpu().numpy(), ref.eigvecs[:, perm], ref.eigvals[perm])
    assert np.max(ang) <= 1e-8, ang
    assert np.max(np.abs(res.numpy() - ref.residuals[perm])) <= 1e-8 * scale


def test_degree_order_generated_start_vector_and_basis(te):
    """No v1: the start vector is drawn per caller row; te_lanczos returns the
    basis in the caller's order."""
    A = synth.rmat_sym(13, 8, 4)
    m = 16
    ref = oracle.lanczos(A, synth.start_vector(A.n, 21), m, seed=21)
    alpha, beta, V, restarts = te.lanczos(te.CSR.from_host(A, "ddd"), m, "ddd", seed=21,
                                          order="degree")
    tn = np.linalg.norm(ref.T())
    assert restarts == ref.restarts
    assert np.max(np.abs(alpha.numpy() - ref.alpha)) <= 1e-10 * tn
    assert np.max(np.abs(beta.numpy() - ref.beta)) <= 1e-10 * tn
    assert np.max(np.abs(V.cpu().numpy() - ref.V)) <= 1e-8


def test_degree_order_restarts_draw_caller_rows(te):
    """The cycle Laplacian breaks down; each restart vector is drawn per caller
    row, so the restarted process is the oracle's."""
    A = synth.cycle_laplacian(64)
    m = 40
    v1 = synth.start_vector(A.n, 7)
    ref = oracle.lanczos(A, v1, m, seed=7)
    assert ref.restarts > 0
    alpha, beta, V, restarts = te.lanczos(te.CSR.from_host(A, "ddd"), m, "ddd", seed=7,
                                          v1=torch.from_numpy(v1).cuda(), order="degree")
    tn = np.linalg.norm(ref.T())
    assert restarts == ref.restarts
    assert np.max(np.abs(alpha.numpy() - ref.alpha)) <= 1e-10 * tn
    assert np.max(np.abs(beta.numpy() - ref.beta)) <= 1e-10 * tn
    assert np.max(np.abs(V.cpu().numpy() - ref.V)) <= 1e-8


@pytest.mark.parametrize("prec", ["fdf", "bdf", "8df"])
def test_degree_order_reduced_precision(te, prec):
    """The mixed forms: FDF against the oracle on the rounded matrix; every form
    against its own solve in the caller's order (same values, same SpMV sums
    per row; only the sums over rows run in another order)."""
    A = synth.rmat_sym(13, 8, 9)
    K, m = 6, 20
    v1 = torch.from_numpy(synth.start_vector(A.n, 5)).cuda()
    csr = te.CSR.from_host(A, prec)
    ev_k, U_k, _ = te.topk_eigs(csr, K, m, prec, seed=5, v1=v1)
    ev_d, U_d, _ = te.topk_eigs(csr, K, m, prec, seed=5, v1=v1, order="degree")
    ev_k, ev_d = ev_k.numpy(), ev_d.numpy()
    scale = np.max(np.abs(ev_k))
    perm = match_pairs(ev_d, ev_k, 1e-6 * scale)
    ang = subspace_angles(U_d.cpu().numpy(), U_k.cpu().numpy()[:, perm], ev_k[perm])
    assert np.max(ang) <= 1e-3, ang
    if prec == "fdf":
        ref = oracle.topk_eigs(f32_matrix(A), K, m, v1.cpu().numpy(), seed=5)
        match_pairs(ev_d, ref.eigvals, 1e-6 * scale)


def test_degree_order_refinement(te):
    """Refinement runs on the relabelled rows; the refined vectors come back in
    the caller's order and match the refined solve in the caller's order."""
    A = synth.rmat_sym(13, 8, 6)
    K, m = 6, 24
    csr = te.CSR.from_host(A, "fdf")
    ev_k, U_k, r_k = te.topk_eigs(csr, K, m, "fdf", seed=2, refine=True, residuals=True)
    ev_d, U_d, r_d = te.topk_eigs(csr, K, m, "fdf", seed=2, refine=True, residuals=True,
                                  order="degree")
    scale = np.max(np.abs(ev_k.numpy()))
    # each refined value is the Rayleigh quotient of its own vector, within its
    # residual of an eigenvalue: the two orders agree within the residuals
    for v, r in zip(ev_d.numpy(), r_d.numpy()):
        assert np.min(np.abs(ev_k.numpy() - v) - r_k.numpy()) <= r + 1e-12 * scale, (v, r)
    # true binary64 residuals of the returned vectors, in the caller's order
    Ud = U_d.cpu().numpy()
    for k in range(K):
        u = Ud[:, k]
        r = oracle.spmv(A, u) - ev_d.numpy()[k] * u
        assert abs(np.linalg.norm(r) / np.linalg.norm(u) - r_d.numpy()[k]) <= 1e-10 * scale


@pytest.mark.parametrize("graph", [True, False])
def test_degree_order_streamed_equals_resident(te, graph):
    A = synth.rmat_sym(14, 8, 3)
    K, m = 6, 20
    dev = te.CSR.from_host(A, "fdf")
    host = te.CSR.from_host(A, "fdf", device="cpu", pin=True)
    p_res = te.Plan(dev, K, m, "fdf", seed=5, use_graph=graph, order="degree")
    p_str = te.Plan(host, K, m, "fdf", seed=5, use_graph=graph, matrix_budget=96 * 1024,
                    order="degree")
    assert p_str.stream_blocks >= 8
    ev1, U1, r1 = p_res.solve(residuals=True)
    ev2, U2, r2 = p_str.solve(residuals=True)
    assert torch.equal(ev1, ev2) and torch.equal(U1, U2) and torch.equal(r1, r2)


def test_degree_order_graph_replay_and_no_vectors(te):
    A = synth.rmat_sym(13, 8, 8)
    plan = te.Plan(te.CSR.from_host(A, "fdf"), 8, 24, "fdf", seed=4, reorth="delayed",
                   order="degree", autotune=True)
    ev1, U1, _ = plan.solve()
    ev2, U2, _ = plan.solve()
    ev3, U3, _ = plan.solve(vectors=False)
    assert torch.equal(ev1, ev2) and torch.equal(U1, U2) and torch.equal(ev1, ev3)
    assert U3 is None
