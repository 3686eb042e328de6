"""Host-streamed matrix (te_options.matrix_budget_bytes) and the FDD form.

A streamed plan keeps the SpMV layout in pinned host memory and copies it in
row blocks through two device buffers every step.  The blocks run the very
same slice computations as the resident layout, so a streamed solve must equal
the resident one bit for bit, with and without the captured graph.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from test_gpu_parity import f32_matrix, match_pairs, subspace_angles

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def te():
    import paper_2201_07498_gb300 as te
    te.load_library(build_if_missing=True)
    return te


@pytest.mark.parametrize("prec", ["ddd", "fdd", "fdf"])
@pytest.mark.parametrize("graph", [True, False])
def test_streamed_solve_equals_resident(te, prec, graph):
    A = synth.rmat_sym(14, 8, 3)  # ragged rows, cut rows, empty rows
    K, m = 6, 20
    dev = te.CSR.from_host(A, prec)
    host = te.CSR.from_host(A, prec, device="cpu", pin=True)
    p_res = te.Plan(dev, K, m, prec, seed=5, use_graph=graph)
    p_str = te.Plan(host, K, m, prec, seed=5, use_graph=graph, matrix_budget=96 * 1024)
    assert p_res.stream_blocks == 0 and p_str.stream_blocks >= 8
    ev1, U1, r1 = p_res.solve(residuals=True)
    ev2, U2, r2 = p_str.solve(residuals=True)
    assert torch.equal(ev1, ev2) and torch.equal(U1, U2) and torch.equal(r1, r2)
    ev3, U3, _ = p_str.solve()  # the buffers are reused across solves
    assert torch.equal(ev1, ev3) and torch.equal(U1, U3)


def test_streamed_one_shot_solve(te):
    A = synth.uniform_sym(20000, 10, 2)
    host = te.CSR.from_host(A, "fdd", device="cpu", pin=True)
    ev1, U1, _ = te.topk_eigs(host, 8, 16, "fdd", seed=1, matrix_budget=256 * 1024)
    ev2, U2, _ = te.topk_eigs(te.CSR.from_host(A, "fdd"), 8, 16, "fdd", seed=1)
    assert torch.equal(ev1, ev2) and torch.equal(U1.cpu(), U2.cpu())


def test_streaming_limits(te):
    A = synth.uniform_sym(5000, 8, 1)
    dev = te.CSR.from_host(A, "fdf")
    with pytest.raises(te.TEError) as e:  # a device matrix over the budget cannot stream
        te.Plan(dev, 4, 8, "fdf", matrix_budget=64 * 1024)
    assert e.value.status == 2
    host64 = te.CSR.from_host(A, "fdf", device="cpu", pin=True)
    with pytest.raises(te.TEError) as e:
        te.Plan(host64, 4, 8, "fdf", refine=True, matrix_budget=64 * 1024)
    assert e.value.status == 7
    hostb = te.CSR.from_host(A, "bdf", device="cpu", pin=True)
    with pytest.raises(te.TEError) as e:
        te.Plan(hostb, 4, 8, "bdf", matrix_budget=64 * 1024)
    assert e.value.status == 7
    host = te.CSR.from_host(A, "fdf", device="cpu", pin=True)
    with pytest.raises(te.TEError) as e:  # smaller than one slice
        te.Plan(host, 4, 8, "fdf", matrix_budget=1024)
    assert e.value.status == 1
    # a budget above the layout keeps the matrix resident
    p = te.Plan(host, 4, 8, "fdf", matrix_budget=1 << 30)
    assert p.stream_blocks == 0


def test_fdd_matches_oracle(te):
    """binary32 values, binary64 arithmetic and vectors: FP64 accuracy on the
    rounded matrix."""
    A = synth.uniform_sym(10000, 10, 0)
    A32 = f32_matrix(A)
    K, m = 8, 16
    v1 = synth.start_vector(A.n, 3)
    ref = oracle.topk_eigs(A32, K, m, v1, seed=3)
    ev, U, _ = te.topk_eigs(te.CSR.from_host(A, "fdd"), K, m, "fdd", seed=3,
                            v1=torch.from_numpy(v1).cuda())
    ev = ev.numpy()
    scale = np.max(np.abs(ref.eigvals))
    perm = match_pairs(ev, ref.eigvals, 1e-10 * scale)
    assert np.max(np.abs(ev - ref.eigvals[perm]) / np.abs(ref.eigvals[perm])) <= 1e-10
    ang = subspace_angles(U.cpu().numpy(), ref.eigvecs[:, perm], ref.eigvals[perm])
    assert np.max(ang) <= 1e-8
