"""Serving engine (continuous batching): GPU tests through the C ABI.

* a binary32 request served alone matches the oracle on the rounded matrix
  within the FDF tolerance, and so does a bfloat16 request;
* a request's result is bit-identical alone and in a mix of requests of other
  sizes admitted at other steps (each solve's sums do not depend on its
  neighbours), with and without the captured step graph;
* admission waits for pool memory: a small pool serves more requests than fit
  at once, its use never exceeds the budget, and a request larger than the
  whole pool fails with TE_ERR_OUT_OF_MEMORY without stopping the others.
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


def _drain(srv, tickets, vectors=True, max_steps=10000):
    out = {}
    for _ in range(max_steps):
        for t in list(tickets):
            r = srv.poll(t, vectors)
            if r is not None:
                out[t] = r
                tickets.remove(t)
        if not tickets:
            return out
        srv.step()
    raise AssertionError("requests did not finish")


def _mix():
    return [synth.rmat_sym(12, 6, 11), synth.uniform_sym(3000, 5, 12), synth.rmat_sym(10, 16, 13),
            synth.uniform_sym(20000, 3, 14), synth.rmat_sym(14, 4, 15), synth.uniform_sym(700, 9, 16)]


def test_server_request_matches_oracle(te):
    """A binary32 request served by the engine against the oracle run on the
    same binary32-rounded matrix with the same start vector: Ritz values
    within 1e-6 relative, vectors within the Davis-Kahan bound of a 1e-4 ||T||
    perturbation capped at 1e-3 rad (see test_topk_fdf_close_to_oracle),
    residual estimates within 1e-5 |theta_1|."""
    A = synth.uniform_sym(10000, 10, 0)
    K, m = 8, 16
    srv = te.Server(max_slots=4, max_krylov_steps=32, budget=256 << 20)
    t = srv.submit(A, K, m, "fdf", seed=7)
    ev, U, res = _drain(srv, [t])[t]
    ref = oracle.topk_eigs(f32_matrix(A), K, m, synth.start_vector(A.n, 7), seed=7)
    scale = np.max(np.abs(ref.eigvals))
    perm = match_pairs(ev, ref.eigvals, 1e-6 * scale)
    assert np.max(np.abs(ev - ref.eigvals[perm]) / np.abs(ref.eigvals[perm])) <= 1e-6
    T = (np.diag(ref.alpha) + np.diag(ref.beta[1:m], 1) + np.diag(ref.beta[1:m], -1))
    th_all, tn = np.linalg.eigvalsh(T), np.linalg.norm(T, 2)
    ang = subspace_angles(U, ref.eigvecs[:, perm], ref.eigvals[perm])
    gaps = [np.min(np.abs(th_all - v)[np.abs(th_all - v) > 1e-8 * scale])
            for v in ref.eigvals[perm]]
    assert np.all(ang <= np.minimum(1e-3, 1e-4 * tn / np.array(gaps))), (ang, gaps)
    assert np.max(np.abs(res - ref.residuals[perm])) <= 1e-5 * scale


@pytest.mark.parametrize("graph", [True, False])
def test_alone_equals_in_mix(te, graph):
    R = synth.rmat_sym(13, 8, 21)
    srv = te.Server(max_slots=8, max_krylov_steps=32, budget=512 << 20, use_graph=graph)
    t = srv.submit(R, 6, 20, "fdf", seed=3)
    alone = _drain(srv, [t])[t]
    srv.close()
    srv = te.Server(max_slots=8, max_krylov_steps=32, budget=512 << 20, use_graph=graph)
    mix = _mix()
    tickets = [srv.submit(mix[0], 4, 8, "fdf", seed=1), srv.submit(mix[1], 8, 16, "bdf", seed=2)]
    srv.step()
    srv.step()
    tickets.append(srv.submit(mix[2], 4, 12, "fdf", seed=3))
    tr = srv.submit(R, 6, 20, "fdf", seed=3)  # joins while others are mid-solve
    srv.step()
    tickets += [srv.submit(M, 4, 8 + 2 * i, "fdf", seed=5 + i) for i, M in enumerate(mix[3:])]
    got = _drain(srv, tickets + [tr])
    inmix = got[tr]
    for a, b in zip(alone, inmix):
        assert np.array_equal(a, b)


def test_graph_and_direct_steps_agree(te):
    mix = _mix()[:4]
    res = []
    for graph in (True, False):
        srv = te.Server(max_slots=3, max_krylov_steps=32, budget=512 << 20, use_graph=graph)
        ts = [srv.submit(M, 4, 10, "fdf", seed=i) for i, M in enumerate(mix)]
        res.append(_drain(srv, list(ts)))
        srv.close()
    for t0, t1 in zip(sorted(res[0]), sorted(res[1])):
        for a, b in zip(res[0][t0], res[1][t1]):
            assert np.array_equal(a, b)


def test_memory_admission_and_oversize_request(te):
    budget = 24 << 20
    srv = te.Server(max_slots=16, max_krylov_steps=32, budget=budget)
    mats = [synth.uniform_sym(40000, 4, 30 + i) for i in range(6)]  # ~9 MB of pool each
    big = synth.uniform_sym(400000, 8, 40)                          # larger than the pool
    tickets = [srv.submit(M, 4, 12, "fdf", seed=i) for i, M in enumerate(mats)]
    tb = srv.submit(big, 4, 12, "fdf", seed=9)
    queued_while_running = False
    done = {}
    for _ in range(2000):
        live, pend = srv.step()
        st = srv.stats()
        assert st["pool_used"] <= budget and st["pool_peak"] <= budget
        if live >= 1 and pend >= 1:
            queued_while_running = True
        for t in list(tickets):
            r = srv.poll(t, vectors=False)
            if r is not None:
                done[t] = r
                tickets.remove(t)
        if not tickets:
            break
    assert not tickets and queued_while_running
    with pytest.raises(te.TEError) as e:
        for _ in range(100):
            if srv.poll(tb) is not None:
                break
            srv.step()
    assert e.value.status == 2
    # every request equals its own single-solve result
    for i, M in enumerate(mats):
        ev_p, _, _ = te.topk_eigs(te.CSR.from_host(M, "fdf"), 4, 12, "fdf", seed=i, vectors=False)
        ev = done[i + 1][0]
        scale = np.max(np.abs(ev_p.numpy()))
        match_pairs(ev, ev_p.numpy(), 1e-6 * scale)


def test_bf16_request_matches_oracle(te):
    A = synth.uniform_sym(8000, 8, 5)
    Aq = synth.CSR(A.n, A.row_ptr, A.col, oracle.round_bf16(A.val)[1])
    v1 = synth.start_vector(A.n, 11)
    ref = oracle.topk_eigs(Aq, 8, 16, v1, seed=11)
    srv = te.Server(max_slots=2, max_krylov_steps=16, budget=128 << 20)
    t = srv.submit(A, 8, 16, "bdf", seed=11)
    ev, U, _ = _drain(srv, [t])[t]
    scale = np.max(np.abs(ref.eigvals))
    perm = match_pairs(ev, ref.eigvals, 1e-6 * scale)
    assert np.max(np.abs(ev - ref.eigvals[perm])) <= 1e-6 * scale


def test_bad_column_is_rejected_before_the_first_spmv(te):
    A = synth.uniform_sym(3000, 5, 9)
    bad = synth.CSR(A.n, A.row_ptr, A.col.copy(), A.val)
    bad.col[17] = A.n  # outside [0, n): checked on the device at admission
    srv = te.Server(max_slots=4, max_krylov_steps=16, budget=64 << 20)
    tb = srv.submit(bad, 4, 8, "fdf", seed=1)
    tg = srv.submit(A, 4, 8, "fdf", seed=1)
    with pytest.raises(te.TEError) as e:
        for _ in range(50):
            if srv.poll(tb) is not None:
                break
            srv.step()
    assert e.value.status == 1
    ev = _drain(srv, [tg])[tg][0]
    ev_p, _, _ = te.topk_eigs(te.CSR.from_host(A, "fdf"), 4, 8, "fdf", seed=1, vectors=False)
    match_pairs(ev, ev_p.numpy(), 1e-6 * np.max(np.abs(ev_p.numpy())))


def test_completion_queue_reports_every_request_once(te):
    """te_server_completed hands out each finished ticket exactly once, in the
    order the requests finished; polling a reported ticket returns at once."""
    srv = te.Server(max_slots=4, max_krylov_steps=32, budget=256 << 20)
    mats = _mix()
    tickets = [srv.submit(M, 4, 8, "fdf", seed=i) for i, M in enumerate(mats)]
    seen = []
    for _ in range(2000):
        srv.step()
        for t in srv.completed():
            seen.append(t)
            assert srv.poll(t, vectors=False) is not None
        if len(seen) == len(tickets):
            break
    assert sorted(seen) == sorted(tickets) and len(set(seen)) == len(seen)
    assert srv.completed() == []


def test_autotuned_server_matches_oracle(te):
    """With the per-class autotuner on, each class's first request times the
    layout candidates; every request still matches the oracle on its rounded
    matrix (binary32 values) within the FDF tolerance, whichever layout its
    class got."""
    srv = te.Server(max_slots=8, max_krylov_steps=32, budget=512 << 20, autotune=True)
    mats = [synth.rmat_sym(12, 6, 31), synth.rmat_sym(12, 6, 32), synth.uniform_sym(3000, 5, 33),
            synth.uniform_sym(3000, 5, 34), synth.rmat_sym(14, 8, 35)]
    tickets = {srv.submit(M, 4, 12, "fdf", seed=40 + i): i for i, M in enumerate(mats)}
    res = _drain(srv, list(tickets))
    classes = srv.classes()
    assert 1 <= len(classes) <= len(mats)
    for w, v in classes.values():
        assert (w, v) in [(2048, 64), (2048, 32), (2048, 128), (256, 64), (16384, 64)]
    for t, i in tickets.items():
        A = mats[i]
        ev = res[t][0]
        ref = oracle.topk_eigs(f32_matrix(A), 4, 12, synth.start_vector(A.n, 40 + i), seed=40 + i,
                               want_vectors=False)
        scale = np.max(np.abs(ref.eigvals))
        perm = match_pairs(ev, ref.eigvals, 1e-6 * scale)
        assert np.max(np.abs(ev - ref.eigvals[perm])) <= 1e-6 * scale


def test_poll_into_pinned_buffer_and_many_finishing_together(te):
    """Eight requests finish at the same step (their finishing work runs on
    several streams at once): every result collected into a reused pinned
    buffer equals the same request served alone into a new array."""
    mats = _mix()[:4] * 2
    srv = te.Server(max_slots=16, max_krylov_steps=32, budget=1 << 30)
    tickets = [srv.submit(A, 6, 12, "fdf", seed=20 + i) for i, A in enumerate(mats)]
    buf = torch.empty(max(A.n for A in mats) * 6, dtype=torch.float64).pin_memory()
    got, pend = {}, list(tickets)
    for _ in range(10000):
        srv.step()
        for t in list(pend):
            r = srv.poll(t, out=buf)
            if r is not None:
                got[t] = (r[0].copy(), r[1].copy(), r[2].copy())
                pend.remove(t)
        if not pend:
            break
    assert not pend
    srv.close()
    for i, (A, t) in enumerate(zip(mats, tickets)):
        alone = te.Server(max_slots=1, max_krylov_steps=32, budget=256 << 20)
        ta = alone.submit(A, 6, 12, "fdf", seed=20 + i)
        ev, U, res = _drain(alone, [ta])[ta]
        alone.close()
        assert np.array_equal(ev, got[t][0]) and np.array_equal(U, got[t][1])
        assert np.array_equal(res, got[t][2])


def test_server_counters(te):
    """The engine's counters add up: every request is analysed once, each
    step advances between one and max_slots solves, a solve of m steps is
    advanced m times, and the host timers only grow."""
    mats = _mix()[:3]
    srv = te.Server(max_slots=8, max_krylov_steps=32, budget=1 << 30)
    t0 = srv.timing()
    tickets = [srv.submit(A, 4, 10, "fdf", seed=40 + i) for i, A in enumerate(mats)]
    _drain(srv, list(tickets), vectors=True)
    an, t1 = srv.analysis(), srv.timing()
    srv.close()
    assert an["analysed"] == len(mats)
    assert an["engine_steps"] >= 10
    assert an["resident_steps"] == 10 * len(mats)
    assert an["engine_steps"] <= an["resident_steps"] <= 8 * an["engine_steps"]
    for k in ("layout_s", "gather_s", "copy_s", "stage_wait_s"):
        assert an[k] >= 0.0
    for k in t1:
        assert t1[k] >= t0[k] >= 0.0
    assert t1["poll_copy_s"] > 0.0


def test_binary32_values_equal_binary64_submission(te):
    """A binary32-storage request submitted with binary32 values gives the
    same bits as one submitted with binary64 values (the library's rounding
    is round to nearest even, the same as the caller's)."""
    A = synth.rmat_sym(12, 8, 21)
    srv = te.Server(max_slots=4, max_krylov_steps=32, budget=256 << 20)
    t64 = srv.submit(A, 6, 12, "fdf", seed=5)
    t32 = srv.submit(A.with_f32_values(), 6, 12, "fdf", seed=5)
    out = _drain(srv, [t64, t32])
    srv.close()
    for a, b in zip(out[t64], out[t32]):
        assert np.array_equal(a, b)
