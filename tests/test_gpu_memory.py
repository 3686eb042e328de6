"""The library's device memory pool (te_mem.cu): plans take their memory from
it and give it back on destruction; a plan built on recycled memory returns
the same bits as one built on fresh memory; the cache can be released."""
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


def test_plan_memory_returns_to_the_pool(te):
    A = synth.rmat_sym(14, 8, 3)
    csr = te.CSR.from_host(A, "fdf")
    torch.cuda.synchronize()
    r0, u0 = te.memory_cached(0)
    plan = te.Plan(csr, 8, 24, "fdf", seed=3, reorth="delayed", order="degree")
    r1, u1 = te.memory_cached(0)
    assert u1 > u0 and r1 >= u1
    plan.close()
    r2, u2 = te.memory_cached(0)
    assert u2 == u0 and r2 >= u1  # kept for the next plan
    te.release_cached_memory()
    r3, u3 = te.memory_cached(0)
    assert u3 == u0 and r3 <= r2


def test_recycled_memory_gives_the_same_bits(te):
    """Every buffer a solve reads is written first: a plan on memory that a
    plan of another matrix has just dirtied returns what a plan on memory
    released to the driver returns, and both match the oracle."""
    A = synth.rmat_sym(13, 8, 5)
    B = synth.uniform_sym(9000, 24, 6)
    K, m = 6, 20
    te.release_cached_memory()
    csr = te.CSR.from_host(A, "ddd")
    ev1, U1, _ = te.Plan(csr, K, m, "ddd", seed=5, reorth="delayed", order="degree").solve()
    junk = te.Plan(te.CSR.from_host(B, "fdf"), 8, 32, "fdf", seed=9, order="degree")
    junk.solve()
    junk.close()
    plan = te.Plan(csr, K, m, "ddd", seed=5, reorth="delayed", order="degree")
    ev2, U2, _ = plan.solve()
    assert torch.equal(ev1, ev2) and torch.equal(U1, U2)
    ref = oracle.topk_eigs(A, K, m, synth.start_vector(A.n, 5), seed=5, want_residuals=False)
    assert np.max(np.abs(np.sort(ev2.numpy()) - np.sort(ref.eigvals))) <= 1e-10


def test_release_threshold(te):
    A = synth.rmat_sym(13, 8, 7)
    csr = te.CSR.from_host(A, "fdf")
    try:
        te.set_memory_cache(0)
        te.release_cached_memory()
        _, u0 = te.memory_cached(0)
        plan = te.Plan(csr, 4, 16, "fdf", seed=7)
        _, u1 = te.memory_cached(0)
        assert u1 > u0
        plan.close()
        torch.cuda.synchronize()
        r2, u2 = te.memory_cached(0)
        assert u2 == u0
    finally:
        te.set_memory_cache(2 ** 64 - 1)
