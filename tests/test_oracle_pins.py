"""Pins of the FP64 oracle against facts fixed outside the oracle itself.

Each pin checks one oracle routine against a closed form, a brute-force
computation, a hand-worked example or an invariant of the mathematics.  The
last test plants, one at a time, a plausible mistake in the oracle and checks
that at least one pin fails for each.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")


def _dense_csr(d):
    return synth.from_dense(np.asarray(d, dtype=np.float64))


# ---------------------------------------------------------------------------
# pin functions: return None when the pin holds, else a message
# ---------------------------------------------------------------------------

def pin_spmv_brute_force():
    """SpMV against a dense mat-vec (brute force), including empty rows."""
    A = synth.uniform_sym(300, 3, seed=7)
    # knock out a few rows/cols to create empty rows
    d = A.to_dense()
    d[[5, 17, 299], :] = 0.0
    d[:, [5, 17, 299]] = 0.0
    B = synth.from_dense(d)
    x = synth.uniform_pm1(300, 3, 0)
    y = oracle.spmv(B, x)
    ref = d @ x
    err = np.max(np.abs(y - ref)) / np.max(np.abs(ref))
    if err > 1e-14:
        return f"spmv rel err {err}"
    rows = [0, 5, 100, 299]
    ys = oracle.spmv_rows(B, x, rows)
    if np.max(np.abs(ys - ref[rows])) > 1e-13:
        return "spmv_rows mismatch"
    return None


def pin_hand_examples():
    """Alpha/beta and eigenvalues of the hand-worked examples."""
    cases = json.load(open(GOLDEN))["cases"]
    for c in cases:
        A = _dense_csr(c["dense"])
        m = c["m"]
        r = oracle.lanczos(A, np.array(c["v1"], dtype=float), m)
        if "alpha" in c:
            if np.max(np.abs(r.alpha - np.array(c["alpha"]))) > 1e-14:
                return f"{c['name']}: alpha {r.alpha}"
            if np.max(np.abs(r.beta - np.array(c["beta"]))) > 1e-14:
                return f"{c['name']}: beta {r.beta}"
        if "alpha_first" in c:
            if abs(r.alpha[0] - c["alpha_first"]) > 1e-14:
                return f"{c['name']}: alpha_1 {r.alpha[0]}"
            if abs(r.alpha.sum() - c["alpha_sum"]) > 1e-13:
                return f"{c['name']}: trace {r.alpha.sum()}"
        res = oracle.topk_eigs(A, m, m, np.array(c["v1"], dtype=float))
        if "eigenvalues_desc" in c:
            got = np.sort(res.eigvals)[::-1]
            if np.max(np.abs(got - np.array(c["eigenvalues_desc"]))) > 1e-13:
                return f"{c['name']}: eigenvalues {got}"
        if "eigenvalues_lm" in c:
            if np.max(np.abs(res.eigvals - np.array(c["eigenvalues_lm"]))) > 1e-13:
                return f"{c['name']}: LM order {res.eigvals}"
    return None


def pin_jacobi_toeplitz():
    """Tridiagonal Toeplitz (a, b): eigenvalues a + 2 b cos(pi k / (m+1))."""
    for m, a, b in [(1, 0.7, 0.0), (2, 1.0, -0.5), (7, 2.0, -1.0), (24, -0.3, 0.9), (48, 1.5, 0.25)]:
        T = np.diag(np.full(m, a)) + np.diag(np.full(m - 1, b), 1) + np.diag(np.full(m - 1, b), -1)
        theta, Y, _, conv = oracle.jacobi(T)
        if not conv:
            return f"jacobi m={m} not converged"
        exact = np.sort(a + 2 * b * np.cos(np.pi * np.arange(1, m + 1) / (m + 1)))
        err = np.max(np.abs(np.sort(theta) - exact))
        if err > 1e-13 * max(1.0, np.linalg.norm(T)):
            return f"jacobi toeplitz m={m} err {err}"
    return None


def pin_jacobi_2x2():
    """2x2 closed form (a+c)/2 +- sqrt(((a-c)/2)^2 + b^2)."""
    for a, b, c in [(2.0, 1.0, 2.0), (1.0, 3.0, -2.0), (5.0, 1e-9, 5.0), (0.0, -1.0, 0.0)]:
        theta, Y, _, _ = oracle.jacobi(np.array([[a, b], [b, c]]))
        mid, rad = (a + c) / 2, math.hypot((a - c) / 2, b)
        if np.max(np.abs(np.sort(theta) - np.array([mid - rad, mid + rad]))) > 1e-14 * (abs(mid) + rad):
            return f"jacobi 2x2 {(a, b, c)} -> {theta}"
        T = np.array([[a, b], [b, c]])
        if np.max(np.abs(T @ Y - Y * theta)) > 1e-14 * (abs(mid) + rad):
            return "jacobi 2x2 eigenvectors"
    return None


def pin_jacobi_random():
    """Random symmetric matrices vs a library eigensolver (test-only)."""
    rng = np.random.default_rng(11)
    for m in [3, 16, 33, 64]:
        G = rng.standard_normal((m, m))
        T = (G + G.T) / 2
        theta, Y, _, conv = oracle.jacobi(T)
        nrm = np.linalg.norm(T)
        if not conv:
            return f"jacobi random m={m} no convergence"
        if np.max(np.abs(np.sort(theta) - np.linalg.eigvalsh(T))) > 1e-13 * nrm:
            return f"jacobi random m={m} eigenvalues"
        if np.max(np.abs(T @ Y - Y * theta)) > 1e-13 * nrm:
            return f"jacobi random m={m} residual"
        if np.max(np.abs(Y.T @ Y - np.eye(m))) > 1e-13:
            return f"jacobi random m={m} orthogonality"
    return None


def pin_lanczos_path_full():
    """Path Laplacian, full Krylov space: 2 - 2 cos(pi k / n)."""
    n = 60
    A = synth.path_laplacian(n)
    v1 = synth.start_vector(n, 5)
    res = oracle.topk_eigs(A, n, n, v1)
    exact = np.sort(2 - 2 * np.cos(np.pi * np.arange(n) / n))
    err = np.max(np.abs(np.sort(res.eigvals) - exact))
    if err > 1e-12 * 4:
        return f"path laplacian err {err}"
    return None


def pin_lanczos_cycle_full():
    """Cycle Laplacian: 2 - 2 cos(2 pi k / n) with multiplicities (needs restarts)."""
    n = 40
    A = synth.cycle_laplacian(n)
    v1 = synth.start_vector(n, 9)
    res = oracle.topk_eigs(A, n, n, v1)
    exact = np.sort(2 - 2 * np.cos(2 * np.pi * np.arange(n) / n))
    err = np.max(np.abs(np.sort(res.eigvals) - exact))
    if res.restarts < 1:
        return "cycle laplacian: no restart happened"
    if err > 1e-12 * 4:
        return f"cycle laplacian err {err}"
    return None


def pin_lanczos_diagonal_trace():
    """Diagonal matrix, m = n: sum(alpha) = trace and Ritz values = diagonal."""
    d = np.linspace(-3.0, 5.0, 50) + 0.01 * np.arange(50) ** 1.5
    A = synth.diagonal(d)
    v1 = synth.start_vector(50, 3)
    r = oracle.lanczos(A, v1, 50)
    if abs(r.alpha.sum() - d.sum()) > 1e-12 * np.abs(d).sum():
        return f"trace {r.alpha.sum()} vs {d.sum()}"
    theta, _, _, _ = oracle.jacobi(r.T())
    if np.max(np.abs(np.sort(theta) - np.sort(d))) > 1e-12 * np.abs(d).max():
        return "diagonal ritz values"
    return None


def pin_lanczos_dense_bruteforce():
    """Random sparse symmetric n <= 200, m = n: eigenvalues, V^T V, residuals."""
    for n, per_row, seed in [(150, 3, 1), (200, 2, 2)]:
        A = synth.uniform_sym(n, per_row, seed)
        d = A.to_dense()
        v1 = synth.start_vector(n, seed)
        res = oracle.topk_eigs(A, n, n, v1)
        lam = np.linalg.eigvalsh(d)
        nrm = np.max(np.abs(lam))
        if np.max(np.abs(np.sort(res.eigvals) - lam)) > 1e-12 * nrm:
            return f"dense brute force n={n}"
        r = oracle.lanczos(A, v1, n)
        if np.max(np.abs(r.V.T @ r.V - np.eye(n))) > 1e-12:
            return f"V^T V n={n}"
        top = np.argsort(-np.abs(res.eigvals))[:8]
        rel = res.residuals[top] / np.abs(res.eigvals[top])
        if np.max(rel) > 1e-10:
            return f"relative residual {np.max(rel)}"
    return None


def pin_lanczos_partial_invariants():
    """m << n: T = V^T A V, A V - V T = w e_m^T, V^T V = I, residual identity, interlacing."""
    n, m = 2000, 20
    A = synth.uniform_sym(n, 5, 21)
    d = A.to_dense()
    v1 = synth.start_vector(n, 21)
    r = oracle.lanczos(A, v1, m)
    V, T = r.V, r.T()
    nrm = np.linalg.norm(d, 2)
    if np.max(np.abs(V[:, 0] - v1 / np.linalg.norm(v1))) > 1e-15:
        return "v_1 is not the normalised start vector"
    if np.max(np.abs(V.T @ d @ V - T)) > 1e-12 * nrm:
        return "T != V^T A V"
    R = d @ V - V @ T
    R[:, -1] -= r.w_last
    if np.max(np.abs(R)) > 1e-12 * nrm:
        return "Lanczos relation"
    if abs(np.linalg.norm(r.w_last) - r.beta[m]) > 1e-14 * nrm:
        return "beta_{m+1} != ||w||"
    if np.max(np.abs(V.T @ V - np.eye(m))) > 1e-12:
        return "orthogonality"
    theta, Y, _, _ = oracle.jacobi(T)
    lam = np.linalg.eigvalsh(d)
    if theta.max() > lam[-1] + 1e-12 * nrm or theta.min() < lam[0] - 1e-12 * nrm:
        return "interlacing"
    res = oracle.topk_eigs(A, 6, m, v1)
    idx = oracle.select_topk(theta, 6)
    for k in range(6):
        ident = r.beta[m] * abs(Y[m - 1, idx[k]])
        if abs(res.residuals[k] - ident) > 1e-10 * nrm:
            return f"residual identity k={k}: {res.residuals[k]} vs {ident}"
    return None


def pin_selection():
    """Largest in modulo: |theta| descending, positive first on ties, then index."""
    theta = np.array([0.5, -2.0, 2.0, 1.0, -1.0, 0.0, -0.5])
    lm = oracle.select_topk(theta, 7, oracle.LARGEST_MAGNITUDE)
    if list(lm) != [2, 1, 3, 4, 0, 6, 5]:
        return f"LM order {list(lm)}"
    la = oracle.select_topk(theta, 7, oracle.LARGEST_ALGEBRAIC)
    if list(la) != [2, 3, 0, 5, 6, 4, 1]:
        return f"LA order {list(la)}"
    return None


def pin_ritz_vectors():
    """Full Krylov: Ritz vectors are eigenvectors (vs a library, up to sign)."""
    n = 80
    A = synth.uniform_sym(n, 4, 33)
    d = A.to_dense()
    v1 = synth.start_vector(n, 33)
    res = oracle.topk_eigs(A, 5, n, v1)
    lam, W = np.linalg.eigh(d)
    for k in range(5):
        u = res.eigvecs[:, k]
        j = np.argmin(np.abs(lam - res.eigvals[k]))
        c = abs(np.dot(u, W[:, j])) / np.linalg.norm(u)
        if abs(c - 1) > 1e-10:
            return f"ritz vector {k} cos {c}"
        if abs(np.linalg.norm(u) - 1) > 1e-12:
            return "ritz vector norm"
    # R9 sign convention on a direct call
    r = oracle.lanczos(A, v1, 10)
    theta, Y, _, _ = oracle.jacobi(r.T())
    idx = oracle.select_topk(theta, 3)
    U = oracle.ritz(r.V, Y, idx)
    for k in range(3):
        y = Y[:, idx[k]]
        s = np.sign(y[np.argmax(np.abs(y))])
        if np.max(np.abs(U[:, k] - s * (r.V @ y))) > 1e-13:
            return "ritz contraction"
    return None


def pin_lanczos_without_reorth():
    """Reorthogonalisation off: the hand-worked examples (exact arithmetic does
    not need it), the three-term relation A V - V T = w e_m^T (which holds
    without reorthogonalisation), and the loss of orthogonality once the
    dominant Ritz value converges (Paige's theory), absent with it on."""
    for c in json.load(open(GOLDEN))["cases"]:
        if "alpha" not in c:
            continue
        r = oracle.lanczos(_dense_csr(c["dense"]), np.array(c["v1"], dtype=float), c["m"],
                           reorth=False)
        if np.max(np.abs(r.alpha - np.array(c["alpha"]))) > 1e-14:
            return f"{c['name']}: alpha without reorth {r.alpha}"
    n, m = 400, 40
    d = np.concatenate([[10.0], np.linspace(0.0, 1.0, n - 1)])
    A = synth.diagonal(d)
    v1 = synth.start_vector(n, 5)
    r0 = oracle.lanczos(A, v1, m, reorth=False)
    r1 = oracle.lanczos(A, v1, m, reorth=True)
    R = np.diag(d) @ r0.V - r0.V @ r0.T()
    R[:, -1] -= r0.w_last
    if np.max(np.abs(R)) > 1e-12 * 10:
        return "three-term relation without reorth"
    lost0 = np.max(np.abs(r0.V.T @ r0.V - np.eye(m)))
    lost1 = np.max(np.abs(r1.V.T @ r1.V - np.eye(m)))
    if not (lost0 > 1e-6 and lost1 < 1e-12):
        return f"orthogonality without / with reorth: {lost0:.2e} / {lost1:.2e}"
    return None


def pin_refine_closed_form():
    """Rayleigh quotient and residual of u = c (e_1 + eps e_2) on diag(d):
    theta = (d1 + eps^2 d2) / (1 + eps^2), residual = |eps (d2 - d1)| / (1 + eps^2);
    an exact eigenvector gives its eigenvalue and residual 0."""
    d = np.array([3.0, -1.5, 0.25, 2.0])
    A = synth.diagonal(d)
    eps, c = 1e-3, 2.5
    u = np.zeros((4, 2))
    u[0, 0], u[1, 0] = c, c * eps
    u[3, 1] = -0.7
    th, res = oracle.refine(A, u)
    th_ref = (d[0] + eps ** 2 * d[1]) / (1 + eps ** 2)
    res_ref = abs(eps * (d[1] - d[0])) / (1 + eps ** 2)
    if abs(th[0] - th_ref) > 1e-15 or abs(res[0] - res_ref) > 1e-15:
        return f"perturbed vector: {th[0]} {res[0]} vs {th_ref} {res_ref}"
    if th[1] != d[3] or res[1] != 0.0:
        return f"exact eigenvector: {th[1]} {res[1]}"
    return None


def pin_pairwise_angle():
    """Orthogonal columns give 90 degrees; cos = +-0.5 gives 60 either sign;
    three vectors at known angles give their mean."""
    Q, _ = np.linalg.qr(synth.uniform_pm1(600, 3, 1).reshape(100, 6))
    if abs(oracle.mean_pairwise_angle(Q) - 90.0) > 1e-9:
        return "orthonormal set"
    a = np.array([1.0, 0.0, 0.0])
    b = np.array([0.5, math.sqrt(3) / 2, 0.0])
    for sgn in (1.0, -1.0):
        if abs(oracle.mean_pairwise_angle(np.stack([a, sgn * b], 1)) - 60.0) > 1e-12:
            return f"60 degrees, sign {sgn}"
    c = np.array([0.0, 0.0, 2.0])
    # angles: (a,b) 60, (a,c) 90, (b,c) 90
    if abs(oracle.mean_pairwise_angle(np.stack([a, -b, c], 1)) - 80.0) > 1e-12:
        return "three vectors"
    return None


def _bf16_table():
    """Every finite non-negative bfloat16 value, by code (brute force)."""
    codes = np.arange(0, 0x7F80, dtype=np.uint32)
    return codes, (codes << 16).view(np.float32).astype(np.float64)


def _e4m3_table():
    """Every finite non-negative E4M3 value, by code, from the format's
    definition: exponent field e (bias 7), 3 fraction bits m; e = 0 is
    subnormal m 2^-9; code 0x7F is NaN."""
    vals = []
    for c in range(0x7F):
        e, m = c >> 3, c & 7
        vals.append(m * 2.0 ** -9 if e == 0 else (1 + m / 8) * 2.0 ** (e - 7))
    return np.arange(0x7F), np.array(vals)


def _check_nearest_even(x, got_codes, got_vals, codes, table, sat=None):
    """got_vals is the nearest table value to |x| (ties: even code), with
    saturation at `sat`; got_codes carry the sign bit of x (zero is +0)."""
    ax = np.abs(x)
    if sat is not None:
        ax = np.minimum(ax, sat)
    j = np.clip(np.searchsorted(table, ax), 1, len(table) - 1)
    lo, hi = table[j - 1], table[j]
    pick = np.where(ax - lo < hi - ax, j - 1, j)
    tie = (ax - lo) == (hi - ax)
    pick = np.where(tie, np.where(codes[j - 1] % 2 == 0, j - 1, j), pick)
    want = table[pick]
    if not np.array_equal(np.abs(got_vals), want):
        k = int(np.argmax(np.abs(got_vals) != want))
        return f"x={x[k]!r}: got {got_vals[k]!r}, nearest-even {want[k]!r}"
    return None


def pin_round_bf16_bruteforce():
    """bfloat16 rounding against the nearest of all 32640 finite magnitudes,
    ties to the even code, including exact midpoints and subnormals."""
    codes, table = _bf16_table()
    rng = np.random.default_rng(12)
    x = np.exp2(rng.uniform(-140, 120, 20000)) * rng.choice([-1.0, 1.0], 20000)
    mids = (table[1:2000:7] + table[2:2001:7]) / 2          # exact midpoints (subnormal)
    mids2 = (table[16000:16400] + table[16001:16401]) / 2   # exact midpoints (normal)
    x = np.concatenate([x, mids, -mids2, mids2, [0.0, -0.0, 1.0, -2.5]])
    got_codes, got = oracle.round_bf16(x)
    msg = _check_nearest_even(x, got_codes, got, codes, table)
    if msg:
        return "bf16 " + msg
    want_sign = (x < 0) & (got != 0)
    if not np.array_equal((got_codes >> 15).astype(bool), want_sign):
        return "bf16 sign bit"
    # the code is the upper half of the binary32 pattern of the value
    if not np.array_equal(((got_codes.astype(np.uint32) << 16).view(np.float32)).astype(float), got):
        return "bf16 code/value mismatch"
    return None


def pin_e4m3_bruteforce():
    """E4M3 rounding at scale 1 (each value shares its row with 448, which
    fixes the scale at 1) against the nearest of all 127 finite magnitudes,
    ties to even; the code table decodes as the format defines.  (With the
    row scale max|a|/448 a scaled value never exceeds 448 (1 + 2^-24), so the
    saturation at 448 cannot be reached from a row.)"""
    codes, table = _e4m3_table()
    for c in range(0x7F):
        if oracle.e4m3_value(c) != table[c] or oracle.e4m3_value(c | 0x80) != -table[c]:
            return f"decode {c:#x}"
    rng = np.random.default_rng(13)
    x = np.concatenate([rng.uniform(-448, 448, 4000),
                        np.exp2(rng.uniform(-12, 8.8, 4000)) * rng.choice([-1.0, 1.0], 4000),
                        (table[:-1] + table[1:]) / 2, [0.0, 448.0, -448.0, 447.9]])
    n = len(x)
    # one row per value, each row padded with +-448 so that its scale is exactly 1
    rp = np.arange(0, 2 * n + 1, 2, dtype=np.int64)
    val = np.empty(2 * n)
    val[0::2] = x
    val[1::2] = 448.0
    col = np.zeros(2 * n, dtype=np.int32)
    col[1::2] = 1
    A = synth.CSR(n, rp, col, val)
    got_codes, scale, deq = oracle.quantize_e4m3_rows(A)
    if not np.all(scale == 1.0):
        return "scale of a row whose largest value is 448"
    msg = _check_nearest_even(x, got_codes[0::2], deq[0::2], codes, table, sat=448.0)
    if msg:
        return "e4m3 " + msg
    return None


def pin_e4m3_row_scales():
    """Per-row scales: binary32(max |a| / 448), 1 for an empty or all-zero
    row; each dequantised value is scale * code value exactly, and a row's
    largest entry maps to the largest code."""
    A = synth.rmat_sym(10, 8, 3)
    val = A.val.copy()
    val[A.row_ptr[7]:A.row_ptr[8]] = 0.0  # an all-zero row
    B = synth.CSR(A.n, A.row_ptr, A.col, val * 3.7)
    codes, scale, deq = oracle.quantize_e4m3_rows(B)
    _, table = _e4m3_table()
    for r in range(B.n):
        a, b = B.row_ptr[r], B.row_ptr[r + 1]
        mx = np.max(np.abs(B.val[a:b])) if b > a else 0.0
        want = np.float32(mx / 448.0) if mx > 0 else np.float32(1.0)
        if scale[r] != want:
            return f"scale of row {r}"
        if b > a:
            dv = np.array([oracle.e4m3_value(int(c)) for c in codes[a:b]])
            if not np.array_equal(deq[a:b], float(scale[r]) * dv):
                return f"dequantised values of row {r}"
            if mx > 0 and np.max(np.abs(dv)) != 448.0:
                return f"row {r} max code"
    return None


PINS = [pin_spmv_brute_force, pin_hand_examples, pin_jacobi_toeplitz, pin_jacobi_2x2,
        pin_jacobi_random, pin_lanczos_path_full, pin_lanczos_cycle_full,
        pin_lanczos_diagonal_trace, pin_lanczos_dense_bruteforce,
        pin_lanczos_partial_invariants, pin_selection, pin_ritz_vectors,
        pin_lanczos_without_reorth, pin_refine_closed_form, pin_pairwise_angle,
        pin_round_bf16_bruteforce, pin_e4m3_bruteforce, pin_e4m3_row_scales]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    msg = pin()
    assert msg is None, msg


@pytest.mark.parametrize("name", [k for k in oracle.FAULTS if k != "none"])
def test_planted_mistake_is_caught(name):
    failures = []
    with oracle.fault(name):
        for pin in PINS:
            try:
                msg = pin()
            except Exception as e:  # a crash also counts as caught
                msg = f"raised {type(e).__name__}"
            if msg is not None:
                failures.append(pin.__name__)
    assert failures, f"planted mistake {name!r} passed every pin"
