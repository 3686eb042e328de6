"""GPU parity: every phase of the CUDA path against the FP64 oracle.

All calls go through the C ABI (``paper_2201_07498_gb300`` only marshals
arguments).  Tolerances:

* SpMV: the two sides sum the same products in different orders, so a row may
  differ by the standard summation bound gamma_k * sum_j |a_rj x_j|
  (gamma_k = k u / (1 - k u), u = 2^-53, k = non-zeros in the row); FDF sums
  exact binary32 products in double-float (about 2^-48), so its bound uses
  u = 2^-44 as a margin.
* DDD solve: relative eigenvalue error <= 1e-10 and eigenvector subspace angle
  <= 1e-8 (clusters of Ritz values closer than 1e-8 |theta_1| are compared as
  subspaces).
* FDF solve against the oracle run on the same binary32-rounded matrix:
  eigenvalues within 1e-6 relative (binary32 Lanczos vectors).
"""
import math

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


def f32_matrix(A):
    """The same matrix with binary32-rounded values (as float64 for the oracle)."""
    return synth.CSR(A.n, A.row_ptr, A.col, A.val.astype(np.float32).astype(np.float64))


def spmv_bound(A, x, u):
    absprod = oracle.spmv(synth.CSR(A.n, A.row_ptr, A.col, np.abs(A.val)), np.abs(x))
    k = np.maximum(np.diff(A.row_ptr), 1).astype(np.float64)
    gam = k * u / (1 - k * u)
    return 2 * gam * absprod + 1e-300


def subspace_angles(U_gpu, U_ref, theta):
    """Largest principal angle per cluster of (nearly) equal Ritz values,
    computed as asin ||(I - Qb Qb^T) Qa||_2 (accurate for tiny angles,
    unlike acos of a cosine close to one)."""
    K = len(theta)
    scale = np.max(np.abs(theta))
    out = []
    k = 0
    while k < K:
        j = k + 1
        while j < K and abs(theta[j] - theta[k]) <= 1e-8 * scale:
            j += 1
        Qa, _ = np.linalg.qr(U_gpu[:, k:j])
        Qb, _ = np.linalg.qr(U_ref[:, k:j])
        s = np.linalg.norm(Qa - Qb @ (Qb.T @ Qa), 2)
        out.append(math.asin(min(1.0, float(s))))
        k = j
    return np.array(out)


def match_pairs(ev_gpu, ev_ref, tol):
    """Pair every selected GPU Ritz value with the nearest unused reference
    value.  Values whose moduli tie within the tolerance (e.g. +1 and -1) may
    come out in either order: the tie is broken in each side's own rounding,
    so only the set is compared.  Returns the permutation of the reference."""
    used = np.zeros(len(ev_ref), dtype=bool)
    perm = []
    for v in ev_gpu:
        d = np.abs(ev_ref - v) + np.where(used, np.inf, 0.0)
        j = int(np.argmin(d))
        assert d[j] <= tol, (v, ev_ref)
        used[j] = True
        perm.append(j)
    return np.array(perm)


def selection_order_valid(ev, which="LM"):
    """The GPU's own output respects the selection key on its own values."""
    key = np.abs(ev) if which == "LM" else ev
    return bool(np.all(np.diff(key) <= 0))


# ---------------------------------------------------------------------------
# matrices
# ---------------------------------------------------------------------------

def star_plus_random(n, seed):
    """Symmetric: one hub row of length n-1 (long-row chunks), ragged random rows,
    empty rows."""
    rng = np.random.default_rng(seed)
    r, c = [0] * (n - 1), list(range(1, n))
    for i in range(1, n, 3):
        for j in rng.integers(1, n, size=rng.integers(0, 40)):
            r.append(i)
            c.append(int(j))
    v = rng.uniform(0.1, 1.0, size=len(r))
    return synth.from_triplets(n, r + c, c + r, np.concatenate([v, v]))


def threshold_rows(symmetric=False):
    """Rows of length exactly around the SpMV's cut length (64) and its
    multiples, plus a row of thousands (plus transposes when `symmetric`)."""
    lens = [0, 1, 31, 32, 33, 63, 64, 65, 127, 128, 129, 4000, 5, 0, 2]
    n = 12000
    rows, cols = [], []
    rng = np.random.default_rng(1)
    for i, L in enumerate(lens):
        cc = rng.choice(np.arange(len(lens), n), size=L, replace=False)
        rows += [i] * L
        cols += [int(x) for x in cc]
    vals = rng.uniform(-1, 1, size=len(rows))
    if symmetric:
        return synth.from_triplets(n, rows + cols, cols + rows, np.concatenate([vals, vals]))
    return synth.from_triplets(n, rows, cols, vals)


SPMV_CASES = {
    "uniform_1e4": lambda: synth.uniform_sym(10000, 10, 0),
    "n1": lambda: synth.from_triplets(1, [0], [0], [2.5]),
    "n7_empty_rows": lambda: synth.from_triplets(7, [1, 3, 3, 6], [3, 1, 6, 3], [1.0, 1.0, -2.0, -2.0]),
    "star_ragged": lambda: star_plus_random(9000, 3),
    "rmat14": lambda: synth.rmat_sym(14, 8, 2),
    "thresholds": lambda: threshold_rows(),
    "banded": lambda: synth.banded_sym(20000, 8, 300, 7),
}


@pytest.mark.parametrize("name", list(SPMV_CASES))
@pytest.mark.parametrize("prec", ["ddd", "fdf"])
def test_spmv_matches_oracle(te, name, prec):
    A = SPMV_CASES[name]()
    x = synth.uniform_pm1(A.n, 11, 5)
    if prec == "fdf":
        A = f32_matrix(A)
        x = x.astype(np.float32).astype(np.float64)
        xd = torch.from_numpy(x.astype(np.float32)).cuda()
        u = 2.0 ** -44
    else:
        xd = torch.from_numpy(x).cuda()
        u = 2.0 ** -53
    y = te.spmv(te.CSR.from_host(A, prec), xd, prec).cpu().numpy()
    ref = oracle.spmv(A, x)
    bound = spmv_bound(A, x, u)
    bad = np.abs(y - ref) > bound
    assert not bad.any(), (name, int(np.argmax(bad)), y[bad][:3], ref[bad][:3])


# ---------------------------------------------------------------------------
# Lanczos phase
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["uniform", "rmat", "cycle_restart"])
def test_lanczos_ddd_matches_oracle(te, case):
    if case == "uniform":
        A, m = synth.uniform_sym(10000, 10, 0), 16
    elif case == "rmat":
        A, m = synth.rmat_sym(13, 8, 3), 24
    else:
        A, m = synth.cycle_laplacian(64), 40
    v1 = synth.start_vector(A.n, 7)
    ref = oracle.lanczos(A, v1, m, seed=7)
    alpha, beta, V, restarts = te.lanczos(te.CSR.from_host(A, "ddd"), m, "ddd", seed=7,
                                          v1=torch.from_numpy(v1).cuda())
    alpha, beta, V = alpha.numpy(), beta.numpy(), V.cpu().numpy()
    tn = np.linalg.norm(ref.T())
    assert restarts == ref.restarts
    assert np.max(np.abs(alpha - ref.alpha)) <= 1e-10 * tn
    assert np.max(np.abs(beta - ref.beta)) <= 1e-10 * tn
    assert np.max(np.abs(V.T @ V - np.eye(m))) <= 1e-12
    # the basis spans the same Krylov space (columns agree up to rounding)
    assert np.max(np.abs(V - ref.V)) <= 1e-8


def test_lanczos_generated_start_vector(te):
    """opt.v1 = NULL draws the start vector from SplitMix64 stream 0 on the GPU."""
    A = synth.uniform_sym(3000, 6, 4)
    v1 = synth.start_vector(A.n, 123)
    ref = oracle.lanczos(A, v1, 8, seed=123)
    alpha, beta, V, _ = te.lanczos(te.CSR.from_host(A, "ddd"), 8, "ddd", seed=123)
    assert np.max(np.abs(V.cpu().numpy()[:, 0] - v1 / np.linalg.norm(v1))) <= 1e-15
    assert np.max(np.abs(alpha.numpy() - ref.alpha)) <= 1e-10 * np.abs(ref.alpha).max()


def test_lanczos_fdf_close_to_oracle(te):
    A = synth.uniform_sym(10000, 10, 0)
    A32 = f32_matrix(A)
    v1 = synth.start_vector(A.n, 0)
    ref = oracle.lanczos(A32, v1, 16)
    alpha, beta, V, _ = te.lanczos(te.CSR.from_host(A, "fdf"), 16, "fdf",
                                   v1=torch.from_numpy(v1).cuda())
    tn = np.linalg.norm(ref.T())
    assert np.max(np.abs(alpha.numpy() - ref.alpha)) <= 1e-6 * tn
    assert np.max(np.abs(beta.numpy() - ref.beta)) <= 1e-6 * tn
    Vh = V.cpu().numpy()
    assert np.max(np.abs(Vh.T @ Vh - np.eye(16))) <= 1e-6


@pytest.mark.parametrize("reorth", ["full", "delayed"])
def test_lanczos_tile_groups_match_oracle(te, reorth):
    """A basis of 7423 tiles of 256 rows (the last one ragged): the passes move
    groups of several tiles per pipeline stage while few columns exist, the
    last group holding fewer tiles than the others."""
    n = 7423 * 256 - 100
    A = synth.uniform_sym(n, 4, 5)
    m = 12
    v1 = synth.start_vector(n, 9)
    ref = oracle.lanczos(A, v1, m, seed=9)
    alpha, beta, V, restarts = te.lanczos(te.CSR.from_host(A, "ddd"), m, "ddd", seed=9,
                                          v1=torch.from_numpy(v1).cuda(), reorth=reorth)
    tn = np.linalg.norm(ref.T())
    assert restarts == ref.restarts == 0
    assert np.max(np.abs(alpha.numpy() - ref.alpha)) <= 1e-10 * tn
    assert np.max(np.abs(beta.numpy() - ref.beta)) <= 1e-10 * tn
    rows = np.r_[0:300, n // 2 - 200:n // 2 + 200, n - 700:n]  # first, middle, ragged end
    Vs = V[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert np.max(np.abs(Vs - ref.V[rows])) <= 1e-8


# ---------------------------------------------------------------------------
# Jacobi phase
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("m", [1, 2, 3, 16, 47, 48, 64])
@pytest.mark.parametrize("which", ["LM", "LA"])
def test_tridiag_jacobi_matches_oracle(te, m, which):
    rng = np.random.default_rng(m)
    alpha = rng.standard_normal(m)
    beta = np.concatenate([[0.0], np.abs(rng.standard_normal(m))])
    T = np.diag(alpha) + np.diag(beta[1:m], 1) + np.diag(beta[1:m], -1)
    theta, Y, sweeps = te.tridiag_eigs(torch.from_numpy(alpha).cuda(),
                                       torch.from_numpy(beta).cuda(), which)
    theta, Y = theta.cpu().numpy(), Y.cpu().numpy()
    th_ref, Y_ref, sw_ref, conv = oracle.jacobi(T)
    w = oracle.LARGEST_MAGNITUDE if which == "LM" else oracle.LARGEST_ALGEBRAIC
    idx = oracle.select_topk(th_ref, m, w)
    tn = np.linalg.norm(T)
    assert np.max(np.abs(theta - th_ref[idx])) <= 1e-13 * max(tn, 1e-300)
    for k in range(m):
        y_ref = Y_ref[:, idx[k]]
        y_ref = y_ref * np.sign(y_ref[np.argmax(np.abs(y_ref))])
        assert np.max(np.abs(Y[:, k] - y_ref)) <= 1e-9
    assert np.max(np.abs(T @ Y - Y * theta)) <= 1e-13 * tn


def test_tridiag_jacobi_toeplitz_closed_form(te):
    m, a, b = 48, 1.5, -0.75
    alpha = np.full(m, a)
    beta = np.concatenate([[0.0], np.full(m, b)])
    theta, _, _ = te.tridiag_eigs(torch.from_numpy(alpha).cuda(), torch.from_numpy(beta).cuda(),
                                  "LA")
    exact = np.sort(a + 2 * b * np.cos(np.pi * np.arange(1, m + 1) / (m + 1)))[::-1]
    assert np.max(np.abs(theta.cpu().numpy() - exact)) <= 1e-13 * 4


# ---------------------------------------------------------------------------
# whole solve
# ---------------------------------------------------------------------------

SOLVE_CASES = [
    ("uniform_1e4_K8_m16", lambda: synth.uniform_sym(10000, 10, 0), 8, 16, "LM"),
    ("rmat13_K6_m20", lambda: synth.rmat_sym(13, 8, 9), 6, 20, "LM"),
    ("star_K4_m12", lambda: star_plus_random(9000, 4), 4, 12, "LM"),
    ("uniform_K_eq_m", lambda: synth.uniform_sym(500, 4, 2), 10, 10, "LA"),
    ("thresholds_K3_m9", lambda: threshold_rows(symmetric=True), 3, 9, "LM"),
]


@pytest.mark.parametrize("name,make,K,m,which", SOLVE_CASES, ids=[c[0] for c in SOLVE_CASES])
def test_topk_ddd_matches_oracle(te, name, make, K, m, which):
    A = make()
    v1 = synth.start_vector(A.n, 3)
    w = oracle.LARGEST_MAGNITUDE if which == "LM" else oracle.LARGEST_ALGEBRAIC
    ref = oracle.topk_eigs(A, K, m, v1, which=w, seed=3)
    ev, U, res = te.topk_eigs(te.CSR.from_host(A, "ddd"), K, m, "ddd", seed=3,
                              v1=torch.from_numpy(v1).cuda(), which=which, residuals=True)
    ev = ev.numpy()
    scale = np.max(np.abs(ref.eigvals))
    assert selection_order_valid(ev, which)
    perm = match_pairs(ev, ref.eigvals, 1e-10 * scale)
    rel = np.abs(ev - ref.eigvals[perm]) / np.maximum(np.abs(ref.eigvals[perm]), 1e-300)
    assert np.max(rel) <= 1e-10, (ev, ref.eigvals)
    ang = subspace_angles(U.cpu().numpy(), ref.eigvecs[:, perm], ref.eigvals[perm])
    assert np.max(ang) <= 1e-8, ang
    # residual estimates = true residuals of the oracle's vectors (Ritz identity)
    assert np.max(np.abs(res.numpy() - ref.residuals[perm])) <= 1e-8 * scale


def test_topk_full_krylov_closed_form(te):
    """m = n on the path Laplacian: all eigenvalues 2 - 2 cos(pi k / n)."""
    n = 40
    A = synth.path_laplacian(n)
    ev, _, _ = te.topk_eigs(te.CSR.from_host(A, "ddd"), n, n, "ddd", seed=5, vectors=False)
    exact = np.sort(2 - 2 * np.cos(np.pi * np.arange(n) / n))
    assert np.max(np.abs(np.sort(ev.numpy()) - exact)) <= 1e-12 * 4


def test_topk_cycle_restarts_recover_multiplicity(te):
    n = 48
    A = synth.cycle_laplacian(n)
    ev, _, _ = te.topk_eigs(te.CSR.from_host(A, "ddd"), n, n, "ddd", seed=2, vectors=False)
    exact = np.sort(2 - 2 * np.cos(2 * np.pi * np.arange(n) / n))
    assert np.max(np.abs(np.sort(ev.numpy()) - exact)) <= 1e-11 * 4


@pytest.mark.parametrize("name,make,K,m,which", SOLVE_CASES[:3], ids=[c[0] for c in SOLVE_CASES[:3]])
def test_topk_fdf_close_to_oracle(te, name, make, K, m, which):
    A = make()
    v1 = synth.start_vector(A.n, 3)
    ref32 = oracle.topk_eigs(f32_matrix(A), K, m, v1, seed=3)
    ref64 = oracle.topk_eigs(A, K, m, v1, seed=3)
    ev, U, _ = te.topk_eigs(te.CSR.from_host(A, "fdf"), K, m, "fdf", seed=3,
                            v1=torch.from_numpy(v1).cuda())
    ev = ev.numpy()
    scale = np.max(np.abs(ref64.eigvals))
    assert selection_order_valid(ev, which)
    perm32 = match_pairs(ev, ref32.eigvals, 1e-6 * scale)
    match_pairs(ev, ref64.eigvals, 1e-6 * scale)
    ang = subspace_angles(U.cpu().numpy(), ref32.eigvecs[:, perm32], ref32.eigvals[perm32])
    # Davis-Kahan: a perturbation eps of the projected problem turns a Ritz
    # vector by at most eps / gap, gap = the distance from its Ritz value to
    # the other Ritz values of T.  FDF stores the basis in binary32 (u32 =
    # 2^-24 per stored vector, over m steps whose Krylov directions amplify
    # it near the clustered eigenvalues of a normalised adjacency): eps =
    # 1e-4 ||T||, and never more than 1e-3 rad.
    m_ = len(ref32.alpha)
    T = (np.diag(ref32.alpha) + np.diag(ref32.beta[1:m_], 1) + np.diag(ref32.beta[1:m_], -1))
    th_all = np.linalg.eigvalsh(T)
    tn = np.linalg.norm(T, 2)
    theta = ref32.eigvals[perm32]
    bounds, k = [], 0
    while k < K:  # one bound per cluster, as subspace_angles groups them
        j = k + 1
        while j < K and abs(theta[j] - theta[k]) <= 1e-8 * scale:
            j += 1
        members = theta[k:j]
        d = np.min(np.abs(th_all[:, None] - members[None, :]), axis=1)
        gap = np.min(d[d > 1e-8 * scale])
        bounds.append(min(1e-3, 1e-4 * tn / gap))
        k = j
    assert np.all(ang <= np.array(bounds)), (ang, bounds)


@pytest.mark.parametrize("order", ["keep", "degree"])
def test_host_outputs_pinned_and_pageable(te, order):
    """Ritz vectors into device memory, into pinned host memory (written by the
    kernels directly) and into pageable host memory (staged): the same bits."""
    A = synth.rmat_sym(13, 8, 3)
    K, m = 6, 20
    csr = te.CSR.from_host(A, "fdf")
    ev_d, U_d, _ = te.topk_eigs(csr, K, m, "fdf", seed=2, order=order)
    outs = []
    for pin in (True, False):
        ev = torch.empty(K, dtype=torch.float64)
        U = torch.empty((K, A.n), dtype=torch.float64)
        if pin:
            ev, U = ev.pin_memory(), U.pin_memory()
        te.topk_eigs(csr, K, m, "fdf", seed=2, order=order, out=(ev, U))
        outs.append((ev, U))
    for ev, U in outs:
        assert torch.equal(ev, ev_d) and torch.equal(U, U_d.t().cpu())


@pytest.mark.parametrize("reorth", ["full", "delayed", "none"])
def test_captured_restarts_equal_uncaptured(te, reorth):
    """The cycle Laplacian breaks down several times in 40 steps: the restart
    passes (captured in the plan's graph, or launched one by one) do the work
    after each breakdown and return at once otherwise.  Same kernels, same
    order: bit-identical results."""
    A = synth.cycle_laplacian(64)
    assert oracle.lanczos(A, synth.start_vector(A.n, 7), 40, seed=7).restarts > 0
    csr = te.CSR.from_host(A, "ddd")
    p_g = te.Plan(csr, 8, 40, "ddd", seed=7, reorth=reorth)
    p_d = te.Plan(csr, 8, 40, "ddd", seed=7, reorth=reorth, use_graph=False)
    ev_g, U_g, r_g = p_g.solve(residuals=True)
    ev_d, U_d, r_d = p_d.solve(residuals=True)
    assert torch.equal(ev_g, ev_d) and torch.equal(U_g, U_d) and torch.equal(r_g, r_d)
    ev_g2, _, _ = p_g.solve()
    assert torch.equal(ev_g, ev_g2)


@pytest.mark.parametrize("prec", ["ddd", "fdf"])
def test_plan_graph_replay_is_deterministic(te, prec):
    A = synth.rmat_sym(12, 8, 1)
    csr = te.CSR.from_host(A, prec)
    plan = te.Plan(csr, 5, 14, prec, seed=9)
    ev1, U1, _ = plan.solve()
    ev2, U2, _ = plan.solve()
    assert torch.equal(ev1, ev2) and torch.equal(U1, U2)
    ev3, U3, _ = te.topk_eigs(csr, 5, 14, prec, seed=9)
    assert torch.equal(ev1, ev3) and torch.equal(U1, U3)
    assert plan.kernel_count > 14 * 4


def test_host_csr_path_equals_device_path(te):
    A = synth.uniform_sym(5000, 8, 6)
    ev_d, U_d, _ = te.topk_eigs(te.CSR.from_host(A, "fdf"), 4, 10, "fdf", seed=1)
    ev_h, U_h, _ = te.topk_eigs(te.CSR.from_host(A, "fdf", device="cpu", pin=True), 4, 10, "fdf",
                                seed=1)
    assert torch.equal(ev_d, ev_h)
    assert torch.equal(U_d.cpu(), U_h)


def test_invalid_csr_is_rejected(te):
    A = synth.uniform_sym(100, 3, 1)
    bad = synth.CSR(A.n, A.row_ptr, A.col.copy(), A.val)
    bad.col[5] = 100  # out of range
    with pytest.raises(te.TEError) as e:
        te.topk_eigs(te.CSR.from_host(bad, "ddd"), 2, 4, "ddd")
    assert e.value.status == 1
