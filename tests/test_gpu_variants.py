"""GPU parity of the solver's variants against the FP64 oracle.

* Binary64 values rounded by the library (values_f64): bit-identical to
  values rounded to binary32 beforehand (the same round-to-nearest-even).
* Rayleigh-quotient refinement (binary64, against the binary64 matrix): for
  DDD the refined values equal the Ritz values (a Ritz value is already the
  Rayleigh quotient of its vector) and the residuals are the oracle's true
  residuals; for FDF the refined values match the oracle's Rayleigh quotients
  of its own Ritz vectors (computed on the same binary32-rounded matrix).
* Without reorthogonalisation (Section IV-D): alpha, beta and the Ritz values
  match the oracle run without reorthogonalisation.
* The Gram matrix behind the orthogonality metric: the mean pairwise angle of
  given vectors matches the oracle's metric.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from test_gpu_parity import f32_matrix, match_pairs, selection_order_valid, subspace_angles

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def te():
    import paper_2201_07498_gb300 as te
    te.load_library(build_if_missing=True)
    return te


def _angle_from_gram(G):
    """Mean sign-free pairwise angle (degrees) from a Gram matrix."""
    K = G.shape[0]
    out = []
    for a in range(K):
        for b in range(a + 1, K):
            c = min(1.0, abs(G[a, b]) / math.sqrt(G[a, a] * G[b, b]))
            out.append(math.degrees(math.acos(c)))
    return float(np.mean(out))


def test_values_f64_rounding_is_round_to_nearest_even(te):
    """The library's binary64 -> binary32 rounding at layout build gives the
    same SpMV, bit for bit, as values rounded by numpy beforehand."""
    A = synth.rmat_sym(13, 8, 4)
    x = torch.from_numpy(synth.uniform_pm1(A.n, 5, 2).astype(np.float32)).cuda()
    y_lib = te.spmv(te.CSR.from_host(A, "fdf"), x, "fdf")
    y_pre = te.spmv(te.CSR.from_host(A.with_f32_values(), "fdf"), x, "fdf")
    assert torch.equal(y_lib, y_pre)


def test_values_f64_solve_equals_prerounded(te):
    A = synth.uniform_sym(5000, 8, 6)
    ev1, U1, _ = te.topk_eigs(te.CSR.from_host(A, "fdf"), 4, 10, "fdf", seed=1)
    ev2, U2, _ = te.topk_eigs(te.CSR.from_host(A.with_f32_values(), "fdf"), 4, 10, "fdf",
                              seed=1)
    assert torch.equal(ev1, ev2) and torch.equal(U1, U2)


def test_refine_ddd_is_the_ritz_value_and_true_residual(te):
    A = synth.uniform_sym(10000, 10, 0)
    K, m = 8, 16
    v1 = synth.start_vector(A.n, 0)
    ref = oracle.topk_eigs(A, K, m, v1, seed=0)
    csr = te.CSR.from_host(A, "ddd")
    ev0, U0, _ = te.topk_eigs(csr, K, m, "ddd", seed=0)
    ev, U, res = te.topk_eigs(csr, K, m, "ddd", seed=0, refine=True, residuals=True)
    scale = np.max(np.abs(ref.eigvals))
    # the Ritz pass is unchanged; the vectors reach the caller through the copy-out
    assert torch.equal(U.cpu(), U0.cpu())
    assert np.max(np.abs(ev.numpy() - ev0.numpy())) <= 1e-12 * scale
    perm = match_pairs(ev.numpy(), ref.eigvals, 1e-10 * scale)
    th_o, res_o = oracle.refine(A, ref.eigvecs[:, perm])
    assert np.max(np.abs(ev.numpy() - th_o)) <= 1e-10 * scale
    assert np.max(np.abs(res.numpy() - res_o)) <= 1e-8 * scale


@pytest.mark.parametrize("plan", [False, True])
def test_refine_fdf_matches_oracle_rayleigh_quotients(te, plan):
    """FDF with refinement against the oracle's Rayleigh quotients of its own
    Ritz vectors, both taken against the binary64 matrix.  The two Krylov
    spaces differ at the 1e-7 level (binary32 vectors), and a Rayleigh
    quotient is stationary at eigenvectors, so the refined values agree much
    more closely than the unrefined ones wherever the pair has converged."""
    A = synth.uniform_sym(10000, 10, 0)
    K, m = 8, 16
    v1 = synth.start_vector(A.n, 0)
    ref32 = oracle.topk_eigs(f32_matrix(A), K, m, v1, seed=0)
    csr = te.CSR.from_host(A, "fdf")
    if plan:
        p = te.Plan(csr, K, m, "fdf", seed=0, refine=True)
        ev, U, res = p.solve(residuals=True)
        ev2, U2, res2 = p.solve(residuals=True)
        assert torch.equal(ev, ev2) and torch.equal(U, U2) and torch.equal(res, res2)
    else:
        ev, U, res = te.topk_eigs(csr, K, m, "fdf", seed=0, refine=True, residuals=True)
    ev, res = ev.numpy(), res.numpy()
    scale = np.max(np.abs(ref32.eigvals))
    perm = match_pairs(ev, ref32.eigvals, 1e-6 * scale)
    th_o, res_o = oracle.refine(A, ref32.eigvecs[:, perm])
    assert np.max(np.abs(ev - th_o)) <= 1e-5 * scale
    assert np.max(np.abs(res - res_o)) <= 1e-5 * scale + 1e-3 * res_o.max()
    # the residuals are the true binary64 residuals of the returned vectors
    Ug = U.cpu().numpy()
    th_g, res_g = oracle.refine(A, Ug)
    assert np.max(np.abs(ev - th_g)) <= 1e-12 * scale
    assert np.max(np.abs(res - res_g)) <= 1e-10 * scale


def test_refine_recovers_fp64_eigenvalues_of_converged_pairs(te):
    """A converged pair of the binary32 matrix sits about u32 |lambda| from
    the binary64 eigenvalue; refinement against the binary64 values moves it
    to within (residual)^2 / gap of it."""
    n = 3000
    d = np.concatenate([[5.0, -4.0, 3.0], np.linspace(-1.0, 1.0, n - 3)])
    d = d + 1e-3 * np.sin(np.arange(n))  # values that do not round exactly to binary32
    A = synth.diagonal(d)
    K, m = 3, 40
    ev, _, res = te.topk_eigs(te.CSR.from_host(A, "fdf"), K, m, "fdf", seed=4,
                              refine=True, residuals=True)
    ev0, _, _ = te.topk_eigs(te.CSR.from_host(A.with_f32_values(), "fdf"), K, m, "fdf", seed=4)
    exact = d[:3]
    perm = match_pairs(ev.numpy(), exact, 1e-5)
    err_ref = np.abs(ev.numpy() - exact[perm])
    err_raw = np.abs(ev0.numpy() - exact[match_pairs(ev0.numpy(), exact, 1e-5)])
    assert np.max(err_ref) <= 1e-12 * 5, err_ref
    assert np.max(err_raw) >= 1e-9, err_raw  # the binary32 values did move them


@pytest.mark.parametrize("prec,tol", [("ddd", 1e-10), ("fdf", 1e-5)])
def test_lanczos_without_reorth_matches_oracle(te, prec, tol):
    A = synth.uniform_sym(10000, 10, 0)
    Ar = A if prec == "ddd" else f32_matrix(A)
    v1 = synth.start_vector(A.n, 0)
    m = 16
    ref = oracle.lanczos(Ar, v1, m, reorth=False)
    alpha, beta, V, _ = te.lanczos(te.CSR.from_host(A, prec), m, prec,
                                   v1=torch.from_numpy(v1).cuda(), reorth="none")
    tn = np.linalg.norm(ref.T())
    assert np.max(np.abs(alpha.numpy() - ref.alpha)) <= tol * tn
    assert np.max(np.abs(beta.numpy() - ref.beta)) <= tol * tn


def test_topk_without_reorth_matches_oracle(te):
    A = synth.uniform_sym(10000, 10, 0)
    K, m = 8, 16
    v1 = synth.start_vector(A.n, 0)
    ref = oracle.topk_eigs(A, K, m, v1, seed=0, reorth=False)
    ev, U, _ = te.topk_eigs(te.CSR.from_host(A, "ddd"), K, m, "ddd", seed=0, reorth="none")
    ev = ev.numpy()
    scale = np.max(np.abs(ref.eigvals))
    assert selection_order_valid(ev)
    perm = match_pairs(ev, ref.eigvals, 1e-9 * scale)
    assert np.max(np.abs(ev - ref.eigvals[perm])) <= 1e-9 * scale
    ang = subspace_angles(U.cpu().numpy(), ref.eigvecs[:, perm], ref.eigvals[perm])
    assert np.max(ang) <= 1e-6, ang


def test_gram_angle_metric_matches_oracle(te):
    n, K = 50000, 12
    U = synth.uniform_pm1(n * K, 11, 3).reshape(K, n).T.copy()
    U[:, 3] += 0.3 * U[:, 1]  # some pairs far from orthogonal
    Ut = torch.from_numpy(np.ascontiguousarray(U.T)).cuda()  # (K, n) rows = vectors
    G = te.gram(Ut)
    assert np.max(np.abs(G - U.T @ U)) <= 1e-10 * np.max(np.abs(G))
    assert abs(_angle_from_gram(G) - oracle.mean_pairwise_angle(U)) <= 1e-9


def test_orthogonality_metric_with_and_without_reorth(te):
    """Section IV-D: with full reorthogonalisation the Ritz vectors stay
    orthogonal (mean angle 90 degrees); without it, a dominant eigenvalue
    converges early and the lost orthogonality shows up as ghost copies,
    exactly as in the oracle run without reorthogonalisation."""
    n = 4000
    d = np.concatenate([[10.0], np.linspace(0.0, 1.0, n - 1)])
    A = synth.diagonal(d)
    K, m = 10, 48
    v1 = synth.start_vector(n, 5)
    csr = te.CSR.from_host(A, "ddd")
    ang = {}
    for mode in ("full", "none"):
        _, U, _ = te.topk_eigs(csr, K, m, "ddd", seed=5, v1=torch.from_numpy(v1).cuda(),
                               reorth=mode)
        ang[mode] = _angle_from_gram(te.gram(U.t().contiguous()))
    ref_none = oracle.topk_eigs(A, K, m, v1, seed=5, reorth=False)
    ang_ref = oracle.mean_pairwise_angle(ref_none.eigvecs)
    assert abs(ang["full"] - 90.0) <= 1e-6, ang
    assert ang["none"] < 89.0 and ang_ref < 89.0, (ang, ang_ref)


# ---------------------------------------------------------------------------
# reduced-precision matrix values (bfloat16, FP8 E4M3 with row scales)
# ---------------------------------------------------------------------------

def _quant_test_matrix():
    """Values over a wide range, exact bfloat16 midpoints, zeros, an all-zero
    row and rows whose largest magnitude is 448 (FP8 scale exactly 1) holding
    exact E4M3 midpoints."""
    rng = np.random.default_rng(21)
    n = 3000
    rows, cols, vals = [], [], []
    for r in range(20, n):  # rows 0..19 hold the crafted entries below only
        k = int(rng.integers(0, 30))
        rows += [r] * k
        cols += [int(c) for c in rng.integers(0, n, k)]
        vals += list(np.exp2(rng.uniform(-30, 30, k)) * rng.choice([-1.0, 1.0], k))
    bf = (np.arange(0x3F00, 0x3F80, dtype=np.uint32) << 16).view(np.float32).astype(float)
    mids_bf = (bf[:-1] + bf[1:]) / 2
    for i, v in enumerate(mids_bf):
        rows.append(5)
        cols.append(i)
        vals.append(v)
    e4 = np.array([(1 + m / 8) * 2.0 ** (e - 7) for e in range(1, 16) for m in range(8)][:-1])
    mids_e4 = (e4[:-1] + e4[1:]) / 2
    for i, v in enumerate(mids_e4):
        rows += [9, 9]
        cols += [2 * i, 2 * i + 1]
        vals += [v, -448.0]
    rows += [11, 11]
    cols += [0, 1]
    vals += [0.0, 0.0]
    return synth.from_triplets(n, rows, cols, np.array(vals))


def test_quantize_is_bit_exact(te):
    A = _quant_test_matrix()
    csr = te.CSR.from_host(A, "ddd")
    codes, _ = te.quantize(csr, "bf16")
    want, _ = oracle.round_bf16(A.val)
    assert np.array_equal(codes.cpu().numpy().view(np.uint16), want)
    f32, _ = te.quantize(csr, "f32")
    assert np.array_equal(f32.cpu().numpy(), A.val.astype(np.float32))
    c8, sc = te.quantize(csr, "e4m3")
    w8, wsc, _ = oracle.quantize_e4m3_rows(A)
    assert np.array_equal(sc.cpu().numpy(), wsc)
    assert np.array_equal(c8.cpu().numpy(), w8)


def _dequantised(A, prec):
    if prec == "bdf":
        return synth.CSR(A.n, A.row_ptr, A.col, oracle.round_bf16(A.val)[1])
    return synth.CSR(A.n, A.row_ptr, A.col, oracle.quantize_e4m3_rows(A)[2])


@pytest.mark.parametrize("prec", ["bdf", "8df"])
def test_spmv_reduced_precision_matches_oracle(te, prec):
    from test_gpu_parity import SPMV_CASES, spmv_bound
    for name in ("uniform_1e4", "thresholds"):
        A = SPMV_CASES[name]()
        Aq = _dequantised(A, prec)
        x = synth.uniform_pm1(A.n, 7, 1).astype(np.float32).astype(np.float64)
        y = te.spmv(te.CSR.from_host(A, prec), torch.from_numpy(x.astype(np.float32)).cuda(),
                    prec).cpu().numpy()
        ref = oracle.spmv(Aq, x)
        assert np.all(np.abs(y - ref) <= spmv_bound(Aq, x, 2.0 ** -44)), name


@pytest.mark.parametrize("prec", ["bdf", "8df"])
def test_topk_reduced_precision_matches_oracle(te, prec):
    """The form's arithmetic is FDF's: against the FP64 oracle run on the same
    rounded matrix the Ritz values agree to the binary32-vector level; with
    refinement they are the binary64 Rayleigh quotients of the vectors."""
    A = synth.uniform_sym(10000, 10, 0)
    Aq = _dequantised(A, prec)
    K, m = 8, 16
    v1 = synth.start_vector(A.n, 0)
    ref = oracle.topk_eigs(Aq, K, m, v1, seed=0)
    csr = te.CSR.from_host(A, prec)
    ev, _, _ = te.topk_eigs(csr, K, m, prec, seed=0)
    ev = ev.numpy()
    scale = np.max(np.abs(ref.eigvals))
    perm = match_pairs(ev, ref.eigvals, 1e-6 * scale)
    assert np.max(np.abs(ev - ref.eigvals[perm])) <= 1e-6 * scale
    evr, Ur, resr = te.topk_eigs(csr, K, m, prec, seed=0, refine=True, residuals=True)
    evr, resr = evr.numpy(), resr.numpy()
    th_o, res_o = oracle.refine(A, ref.eigvecs[:, perm])
    assert np.max(np.abs(evr - th_o)) <= 1e-5 * scale
    th_g, res_g = oracle.refine(A, Ur.cpu().numpy())
    assert np.max(np.abs(evr - th_g)) <= 1e-12 * scale
    assert np.max(np.abs(resr - res_g)) <= 1e-10 * scale


@pytest.mark.parametrize("prec", ["bdf", "8df"])
def test_refine_recovers_diagonal_eigenvalues_from_reduced_values(te, prec):
    """Rounding a diagonal matrix moves its eigenvalues by the rounding error
    but not its eigenvectors; the binary64 Rayleigh quotients of the converged
    Ritz vectors are the exact eigenvalues.  (bfloat16: up to 2^-9 relative;
    FP8: a one-entry row is its own maximum, code 448, so only the binary32
    rounding of the row scale, up to 2^-24, moves it.)"""
    n = 3000
    d = np.concatenate([[5.0, -4.0, 3.0], np.linspace(-1.0, 1.0, n - 3)])
    d = d + 1e-3 * np.sin(np.arange(n))
    A = synth.diagonal(d)
    K, m = 3, 40
    csr = te.CSR.from_host(A, prec)
    ev, _, res = te.topk_eigs(csr, K, m, prec, seed=4, refine=True, residuals=True)
    ev0, _, _ = te.topk_eigs(csr, K, m, prec, seed=4)
    exact = d[:3]
    err_ref = np.abs(ev.numpy() - exact[match_pairs(ev.numpy(), exact, 0.5)])
    err_raw = np.abs(ev0.numpy() - exact[match_pairs(ev0.numpy(), exact, 0.5)])
    assert np.max(err_ref) <= 1e-11 * 5, err_ref
    assert np.max(err_raw) >= (1e-5 if prec == "bdf" else 1e-8), err_raw


@pytest.mark.parametrize("prec,tol", [("ddd", 1e-10), ("fdf", 1e-6)])
def test_autotuned_plan_matches_oracle(te, prec, tol):
    """The autotuner picks one of its candidate layouts; the solve on it
    matches the oracle like the default layout does."""
    from test_gpu_parity import threshold_rows
    for A in (synth.uniform_sym(20000, 8, 7), threshold_rows(symmetric=True)):
        Ar = A if prec == "ddd" else f32_matrix(A)
        v1 = synth.start_vector(A.n, 2)
        ref = oracle.topk_eigs(Ar, 6, 16, v1, seed=2)
        plan = te.Plan(te.CSR.from_host(A, prec), 6, 16, prec, seed=2, autotune=True,
                       v1=torch.from_numpy(v1).cuda())
        assert plan.layout in {(2048, 64), (2048, 32), (2048, 128), (256, 64), (16384, 64)}
        ev, _, _ = plan.solve()
        ev = ev.numpy()
        scale = np.max(np.abs(ref.eigvals))
        perm = match_pairs(ev, ref.eigvals, tol * scale)
        assert np.max(np.abs(ev - ref.eigvals[perm])) <= tol * scale


# ---------------------------------------------------------------------------
# full reorthogonalisation with the second sweep delayed into the next step
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec,tol", [("ddd", 1e-10), ("fdf", 1e-6)])
def test_lanczos_delayed_matches_oracle(te, prec, tol):
    A = synth.uniform_sym(10000, 10, 0)
    Ar = A if prec == "ddd" else f32_matrix(A)
    v1 = synth.start_vector(A.n, 0)
    m = 24
    ref = oracle.lanczos(Ar, v1, m)
    alpha, beta, V, _ = te.lanczos(te.CSR.from_host(A, prec), m, prec,
                                   v1=torch.from_numpy(v1).cuda(), reorth="delayed")
    tn = np.linalg.norm(ref.T())
    assert np.max(np.abs(alpha.numpy() - ref.alpha)) <= tol * tn
    assert np.max(np.abs(beta.numpy() - ref.beta)) <= tol * tn
    Vh = V.cpu().numpy()
    assert np.max(np.abs(Vh.T @ Vh - np.eye(m))) <= (1e-12 if prec == "ddd" else 1e-6)


@pytest.mark.parametrize("prec", ["ddd", "fdf"])
def test_topk_delayed_matches_oracle(te, prec):
    from test_gpu_parity import SOLVE_CASES
    tol = 1e-10 if prec == "ddd" else 1e-6
    for name, make, K, m, which in SOLVE_CASES:
        A = make()
        Ar = A if prec == "ddd" else f32_matrix(A)
        v1 = synth.start_vector(A.n, 3)
        w = oracle.LARGEST_MAGNITUDE if which == "LM" else oracle.LARGEST_ALGEBRAIC
        ref = oracle.topk_eigs(Ar, K, m, v1, which=w, seed=3)
        ev, U, res = te.topk_eigs(te.CSR.from_host(A, prec), K, m, prec, seed=3,
                                  v1=torch.from_numpy(v1).cuda(), which=which, residuals=True,
                                  reorth="delayed")
        ev = ev.numpy()
        scale = np.max(np.abs(ref.eigvals))
        assert selection_order_valid(ev, which), name
        perm = match_pairs(ev, ref.eigvals, tol * scale)
        assert np.max(np.abs(ev - ref.eigvals[perm])) <= tol * scale, name
        if prec == "ddd":
            ang = subspace_angles(U.cpu().numpy(), ref.eigvecs[:, perm], ref.eigvals[perm])
            assert np.max(ang) <= 1e-8, (name, ang)


@pytest.mark.parametrize("prec", ["ddd", "fdf"])
def test_delayed_closed_forms_and_restarts(te, prec):
    """m = n: the path Laplacian's spectrum; the cycle's needs restarts
    (eigenvalues of multiplicity two) and recovers every copy."""
    tol = 1e-11 if prec == "ddd" else 1e-5
    n = 40
    ev, _, _ = te.topk_eigs(te.CSR.from_host(synth.path_laplacian(n), prec), n, n, prec, seed=5,
                            vectors=False, reorth="delayed")
    exact = np.sort(2 - 2 * np.cos(np.pi * np.arange(n) / n))
    assert np.max(np.abs(np.sort(ev.numpy()) - exact)) <= tol * 4
    n = 48
    ev, _, _ = te.topk_eigs(te.CSR.from_host(synth.cycle_laplacian(n), prec), n, n, prec,
                            seed=2, vectors=False, reorth="delayed")
    exact = np.sort(2 - 2 * np.cos(2 * np.pi * np.arange(n) / n))
    assert np.max(np.abs(np.sort(ev.numpy()) - exact)) <= tol * 4


@pytest.mark.parametrize("prec", ["ddd", "fdf"])
def test_delayed_plan_graph_is_deterministic(te, prec):
    A = synth.rmat_sym(12, 8, 1)
    plan = te.Plan(te.CSR.from_host(A, prec), 5, 14, prec, seed=9, reorth="delayed")
    ev1, U1, _ = plan.solve()
    ev2, U2, _ = plan.solve()
    assert torch.equal(ev1, ev2) and torch.equal(U1, U2)
    ev3, _, _ = te.topk_eigs(te.CSR.from_host(A, prec), 5, 14, prec, seed=9)
    scale = np.max(np.abs(ev3.numpy()))
    match_pairs(ev1.numpy(), ev3.numpy(), (1e-10 if prec == "ddd" else 1e-5) * scale)


def test_gather_probe_reports_a_rate(te):
    """The gather-ceiling probe runs and a table that fits on chip serves
    random reads at least as fast as one that does not."""
    small = te.probe_gather(1 << 12)
    big = te.probe_gather(1 << 26)
    assert big > 1e9 and small >= 0.9 * big


# ---------------------------------------------------------------------------
# device-side failure path: a bounded wait that runs out
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec,reorth", [("ddd", "full"), ("fdf", "delayed")])
def test_expired_wait_returns_timeout_then_plan_recovers(te, prec, reorth):
    """The test hook stall_first_pass makes the first basis pass of the plan's
    first solve wait for copies that are never issued: its consumers' bounded
    waits expire, the pass sets TE_ERR_TIMEOUT and every kernel returns (no
    copy is in flight, nothing waits without a limit).  The solve reports the
    status; the context and the plan stay usable, and the next solve of the
    same plan (graph replay) matches the oracle."""
    import time
    A = synth.uniform_sym(10000, 10, 0)
    K, m = 8, 16
    v1 = synth.start_vector(A.n, 0)
    A_ref = A if prec == "ddd" else f32_matrix(A)
    ref = oracle.topk_eigs(A_ref, K, m, v1, seed=0)
    plan = te.Plan(te.CSR.from_host(A, prec), K, m, prec, seed=0, reorth=reorth,
                   stall_first_pass=True)
    t0 = time.perf_counter()
    with pytest.raises(te.TEError) as e:
        plan.solve()
    assert e.value.status == 6, e.value  # TE_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 60.0
    ev, U, _ = plan.solve()
    ev = ev.numpy()
    scale = np.max(np.abs(ref.eigvals))
    tol = 1e-10 if prec == "ddd" else 1e-6
    perm = match_pairs(ev, ref.eigvals, tol * scale)
    assert np.max(np.abs(ev - ref.eigvals[perm]) / np.abs(ref.eigvals[perm])) <= tol
    # a plan without the hook is unaffected
    ev2, _, _ = te.Plan(te.CSR.from_host(A, prec), K, m, prec, seed=0, reorth=reorth).solve()
    assert torch.equal(torch.from_numpy(ev), ev2)


# ---------------------------------------------------------------------------
# Jacobi on a cluster of CTAs: repeated launches give the same bits
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("m", [48, 64])
def test_cluster_jacobi_is_repeatable(te, m):
    """For m >= 40 the Jacobi phase runs on a cluster of eight CTAs that each
    keep a copy of T and push their blocks into the others' copies.  A copy
    overwritten out of order (a missing barrier) would make launches disagree
    with each other under varying schedules; fifty launches must give the same
    bits, matching the oracle."""
    rng = np.random.default_rng(100 + m)
    alpha = rng.standard_normal(m)
    beta = np.concatenate([[0.0], np.abs(rng.standard_normal(m))])
    a_d, b_d = torch.from_numpy(alpha).cuda(), torch.from_numpy(beta).cuda()
    th0, Y0, _ = te.tridiag_eigs(a_d, b_d, "LM")
    for _ in range(49):
        th, Y, _ = te.tridiag_eigs(a_d, b_d, "LM")
        assert torch.equal(th, th0) and torch.equal(Y, Y0)
    T = np.diag(alpha) + np.diag(beta[1:m], 1) + np.diag(beta[1:m], -1)
    th_ref, _, _, _ = oracle.jacobi(T)
    idx = oracle.select_topk(th_ref, m, oracle.LARGEST_MAGNITUDE)
    assert np.max(np.abs(th0.cpu().numpy() - th_ref[idx])) <= 1e-13 * np.linalg.norm(T)
