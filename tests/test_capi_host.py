"""Host-side checks of the C ABI (no GPU needed).

The library must load, export every function ``include/*.h`` declares,
reject bad arguments before touching the GPU, and partition rows for the
SpMV so that every row and every non-zero is covered exactly once.
"""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def te():
    from paper_2201_07498_gb300 import _build
    _build.build()
    import paper_2201_07498_gb300 as te
    te.load_library()
    return te


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(te_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


def test_every_declared_symbol_is_exported(te):
    names = _declared_functions()
    assert len(names) >= 14, names
    lib = ctypes.CDLL(te.library_path())
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"
    # the Python binding covers every declared function too
    assert set(names) <= set(te._SIGS), set(names) - set(te._SIGS)


def test_status_strings_and_defaults(te):
    lib = te.load_library()
    assert lib.te_status_string(0) == b"TE_OK"
    assert lib.te_status_string(4) == b"TE_ERR_BREAKDOWN"
    o = te.te_options()
    lib.te_default_options(ctypes.byref(o))
    assert o.seed == 0 and o.which == 0 and o.use_graph == 1 and o.device_budget_bytes == 0


def _desc(n, nnz, where=1, scale=None):
    rp = np.zeros(n + 1, dtype=np.int64)
    ci = np.zeros(max(nnz, 1), dtype=np.int32)
    va = np.zeros(max(nnz, 1))
    keep = (rp, ci, va)
    A = __import__("paper_2201_07498_gb300").te_csr(n, nnz, rp.ctypes.data, ci.ctypes.data,
                                                    va.ctypes.data, scale, where)
    return A, keep


@pytest.mark.parametrize("K,m,prec,expect", [
    (0, 4, "ddd", 1),          # K < 1
    (5, 4, "ddd", 1),          # m < K
    (4, 65, "ddd", 7),         # m above the supported maximum
    (4, 11, "ddd", 1),         # m > n (n = 10)
    (2, 4, (1, 1, 1), 7),      # FFF not implemented
    (2, 4, (2, 0, 0), 7),      # BF16 values with binary64 vectors: not a supported form
    (2, 4, (2, 0, 1), 1),      # BDF needs binary64 input values (values_f64)
    (2, 4, (3, 0, 1), 1),      # 8DF likewise
])
def test_argument_validation_before_gpu(te, K, m, prec, expect):
    lib = te.load_library()
    A, keep = _desc(10, 0)
    ev = np.zeros(max(K, 1))
    rc = lib.te_topk_eigs(ctypes.byref(A), K, m, te._prec(prec), None,
                          ctypes.c_void_p(ev.ctypes.data), None, None, None)
    assert rc == expect, (rc, lib.te_last_error())
    assert lib.te_last_error() != b""


def test_option_validation_before_gpu(te):
    """New options are checked before any device work: refinement needs the
    binary64 values, reorth and refine take their documented values only."""
    lib = te.load_library()
    ev = np.zeros(4)
    A, keep = _desc(10, 0)

    def call(A, **kw):
        o = te.te_options()
        lib.te_default_options(ctypes.byref(o))
        assert o.reorth == 0 and o.refine == 0
        for k, v in kw.items():
            setattr(o, k, v)
        return lib.te_topk_eigs(ctypes.byref(A), 2, 4, te._prec("fdf"), ctypes.byref(o),
                                ctypes.c_void_p(ev.ctypes.data), None, None, None)

    assert call(A, refine=1) == 1 and b"binary64" in lib.te_last_error()
    assert call(A, reorth=3) == 1
    assert call(A, refine=3) == 1
    assert call(A, order=2) == 1 and b"order" in lib.te_last_error()
    assert call(A, stall_first_pass=2) == 1 and b"stall_first_pass" in lib.te_last_error()
    A.values_f64 = 2
    assert call(A) == 1
    A.values_f64 = 1
    # noalloc cannot round values (rejected before the pointers are used)
    B, keep2 = _desc(10, 0, where=0)
    B.values_f64 = 1
    assert lib.te_spmv_noalloc(ctypes.byref(B), te._prec("fdf"), ctypes.c_void_p(ev.ctypes.data),
                               ctypes.c_void_p(ev.ctypes.data), None) == 1
    assert b"values_f64" in lib.te_last_error()


def test_server_options_validated_before_gpu(te):
    lib = te.load_library()
    h = ctypes.c_void_p()
    for slots, m, budget in [(0, 16, 1 << 30), (65, 16, 1 << 30), (8, 65, 1 << 30), (8, 16, 1000)]:
        o = te.te_server_options(slots, m, budget, 1)
        assert lib.te_server_create(ctypes.byref(o), ctypes.byref(h)) == 1
    o = te.te_server_options(8, 16, 1 << 30, 1, 2)  # autotune takes 0 or 1
    assert lib.te_server_create(ctypes.byref(o), ctypes.byref(h)) == 1
    assert lib.te_server_create(None, ctypes.byref(h)) == 1


def test_null_and_reserved_arguments(te):
    lib = te.load_library()
    ev = np.zeros(4)
    assert lib.te_topk_eigs(None, 2, 4, te._prec("ddd"), None, ctypes.c_void_p(ev.ctypes.data),
                            None, None, None) == 1
    A, keep = _desc(10, 0, scale=ctypes.c_void_p(ev.ctypes.data).value)
    assert lib.te_topk_eigs(ctypes.byref(A), 2, 4, te._prec("ddd"), None,
                            ctypes.c_void_p(ev.ctypes.data), None, None, None) == 7
    A, keep = _desc(10, 0, where=5)
    assert lib.te_topk_eigs(ctypes.byref(A), 2, 4, te._prec("ddd"), None,
                            ctypes.c_void_p(ev.ctypes.data), None, None, None) == 1


def test_memory_pool_queries_before_gpu(te):
    """The pool queries validate their arguments and report an empty pool
    for a device the library has not allocated on (no CUDA call needed)."""
    lib = te.load_library()
    r, u = ctypes.c_uint64(7), ctypes.c_uint64(7)
    assert lib.te_memory_cached(-1, ctypes.byref(r), ctypes.byref(u)) == 1
    assert lib.te_memory_cached(64, ctypes.byref(r), ctypes.byref(u)) == 1
    assert lib.te_memory_cached(0, None, ctypes.byref(u)) == 1
    assert lib.te_memory_cached(63, ctypes.byref(r), ctypes.byref(u)) == 0
    assert (r.value, u.value) == (0, 0)


def test_workspace_bytes(te):
    lib = te.load_library()
    n = 1 << 24
    A, keep = _desc(1, 0)
    A.n, A.nnz = n, 268_000_000
    b_fdf = lib.te_workspace_bytes(ctypes.byref(A), 24, 48, te._prec("fdf"))
    b_ddd = lib.te_workspace_bytes(ctypes.byref(A), 24, 48, te._prec("ddd"))
    # basis (m+1 columns) + two n-vectors dominate
    assert b_fdf >= n * 49 * 4 + 2 * n * 8
    assert b_ddd >= n * 49 * 8 + 2 * n * 8
    assert b_ddd > b_fdf
    assert lib.te_workspace_bytes(ctypes.byref(A), 0, 48, te._prec("fdf")) == 0


VMAX, C, WINDOW = 64, 32, 2048


def _check_layout(rp, L, VMAX=VMAX, WINDOW=WINDOW):
    """Every entry of every non-empty row is summed by exactly one lane piece;
    short rows are one lane, cut rows are contiguous pieces of <= VMAX; slices
    hold pieces of one window, longest first, padded to their longest piece."""
    n = len(rp) - 1
    lens = np.diff(rp)
    slen, out, src, ln = L["slice_len"], L["lane_out"], L["lane_src"], L["lane_len"]
    S = len(slen)
    assert len(out) == 32 * S
    assert L["entries"] == 32 * int(slen.sum())
    assert np.all(ln <= VMAX)
    cover = np.zeros(int(rp[-1]) + 1, dtype=np.int64)
    seen_rows = np.zeros(n, dtype=np.int64)
    piece_rows = {}
    for s in range(S):
        lanes = slice(32 * s, 32 * s + 32)
        l = ln[lanes]
        assert slen[s] == l.max()
        assert np.all(np.diff(l) <= 0), "lanes of a slice sorted longest first"
        o = out[lanes]
        live = o != np.iinfo(np.int32).min
        rows = []
        for lane in np.nonzero(live)[0]:
            a, b = src[32 * s + lane], src[32 * s + lane] + ln[32 * s + lane]
            assert b > a
            cover[a:b] += 1
            r = int(np.searchsorted(rp, a, side="right") - 1)
            assert rp[r] <= a and b <= rp[r + 1]
            rows.append(r)
            if o[lane] >= 0:
                assert o[lane] == r and a == rp[r] and b == rp[r + 1]
                seen_rows[r] += 1
            else:
                piece_rows.setdefault(r, []).append((-1 - int(o[lane]), a, b))
        assert len({r // WINDOW for r in rows}) <= 1, "a slice stays inside one window"
    assert np.all(cover[: int(rp[-1])] == 1)
    short = (lens > 0) & (lens <= VMAX)
    assert np.all(seen_rows[short] == 1) and np.all(seen_rows[~short] == 0)
    cut = np.nonzero(lens > VMAX)[0]
    assert set(piece_rows) == set(int(r) for r in cut)
    assert L["long_rows"] == len(cut)
    for r, ps in piece_rows.items():
        ps.sort()
        slots = [p[0] for p in ps]
        assert slots == list(range(slots[0], slots[0] + len(slots)))
        assert ps[0][1] == rp[r] and ps[-1][2] == rp[r + 1]
    windows = (n + WINDOW - 1) // WINDOW
    assert L["entries"] <= rp[-1] + windows * 2 * C * VMAX


def test_layout_covers_every_entry_once(te):
    # (scale 18: 128 windows of rows, counted and then written at their
    # offsets by several threads)
    mats = [synth.uniform_sym(5000, 7, 3), synth.rmat_sym(14, 8, 5), synth.rmat_sym(18, 2, 6)]
    # crafted: empty rows, a star (one very long row), rows around the cut length
    n = 20000
    lens = np.zeros(n, dtype=np.int64)
    lens[::7] = 3
    lens[5] = n - 1
    for i, L in enumerate([63, 64, 65, 127, 128, 129, 4000]):
        lens[100 + i] = L
    rp = np.concatenate([[0], np.cumsum(lens)])
    for A in mats:
        _check_layout(A.row_ptr, te.spmv_layout(A.row_ptr, A.nnz))
    L = te.spmv_layout(rp, int(rp[-1]))
    _check_layout(rp, L)
    assert L["long_rows"] == 6


@pytest.mark.parametrize("window,vmax", [(2048, 32), (2048, 128), (256, 64), (16384, 64), (7, 5)])
def test_layout_parameters_cover_every_entry_once(te, window, vmax):
    """The autotuner's candidate layouts (and an odd one) keep every property."""
    for A in (synth.rmat_sym(13, 8, 2), synth.uniform_sym(3000, 6, 3)):
        L = te.spmv_layout(A.row_ptr, A.nnz, window, vmax)
        _check_layout(A.row_ptr, L, VMAX=vmax, WINDOW=window)


def test_layout_rejects_malformed_row_ptr(te):
    with pytest.raises(te.TEError) as e:
        te.spmv_layout(np.array([0, 3, 2, 5]), 5)
    assert e.value.status == 1
    with pytest.raises(te.TEError):
        te.spmv_layout(np.array([1, 3, 4]), 4)
    with pytest.raises(te.TEError):
        te.spmv_layout(np.array([0, 3, 4]), 5)


def test_degree_order_is_the_stable_sort_by_length(te):
    """Against numpy's stable argsort on minus the row lengths; the large
    R-MAT case spreads the histograms over several host threads, the star
    case has one row as long as the matrix."""
    n = 20000
    lens = np.zeros(n, dtype=np.int64)
    lens[::7] = 3
    lens[5] = n - 1
    lens[11::13] = 64
    star = np.concatenate([[0], np.cumsum(lens)])
    for rp in (synth.rmat_sym(20, 4, 1).row_ptr, synth.uniform_sym(3000, 6, 3).row_ptr, star,
               np.array([0, 0, 0]), np.array([0, 5])):
        perm, iperm = te.degree_order(rp, int(rp[-1]))
        ref = np.argsort(-np.diff(rp), kind="stable")
        assert np.array_equal(perm, ref)
        assert np.array_equal(iperm[perm], np.arange(len(rp) - 1))
    with pytest.raises(te.TEError) as e:
        te.degree_order(np.array([0, 3, 2, 5]), 5)
    assert e.value.status == 1


def test_symmetry_check(te):
    for A in (synth.uniform_sym(2000, 5, 1), synth.rmat_sym(12, 8, 2), synth.path_laplacian(30)):
        assert te.check_symmetric(A) == 0.0
    A = synth.uniform_sym(500, 4, 3)
    B = synth.CSR(A.n, A.row_ptr, A.col.copy(), A.val.copy())
    k = int(B.row_ptr[7])  # entry (7, c): its mirror (c, 7) keeps the old value
    B.val[k] += 0.25
    with pytest.raises(te.TEError) as e:
        te.check_symmetric(B)
    assert e.value.status == 1 and "0.25" in str(e.value)
    assert te.check_symmetric(B, tol=0.3) == pytest.approx(0.25)
    # a missing mirror entry counts as zero; duplicates within a row are summed
    C = synth.from_triplets(3, [0, 1, 1], [1, 0, 2], [2.0, 2.0, 5.0])
    with pytest.raises(te.TEError):
        te.check_symmetric(C)
    D = synth.CSR(2, np.array([0, 2, 3]), np.array([1, 1, 0], dtype=np.int32),
                  np.array([1.0, 2.0, 3.0]))
    assert te.check_symmetric(D) == 0.0


def test_product_path_has_no_cpu_fallback():
    """The product package must not import the oracle or the generators."""
    pkg = os.path.join(ROOT, "paper_2201_07498_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True) + \
            glob.glob(os.path.join(pkg, "csrc", "*")):
        src = open(f).read()
        assert "import oracle" not in src and "from oracle" not in src, f
        assert "oracle.h" not in src, f
        assert "import synth" not in src, f


def test_banded_generator_and_its_layout(te):
    """synth.banded_sym: symmetric, every column within the band, no diagonal,
    at most per_row draws above the diagonal per row, reproducible from its
    seed; its SpMV layout keeps every layout property."""
    n, per_row, hw = 3000, 6, 40
    A = synth.banded_sym(n, per_row, hw, 4)
    D = A.to_dense()
    assert np.array_equal(D, D.T)
    rows = np.repeat(np.arange(n), np.diff(A.row_ptr))
    off = A.col.astype(np.int64) - rows
    assert np.all(off != 0) and np.max(np.abs(off)) <= hw
    assert np.all(np.count_nonzero(np.triu(D, 1), axis=1) <= per_row)
    assert np.all((A.val > 0) & (A.val < 2 * per_row))
    B = synth.banded_sym(n, per_row, hw, 4)
    assert np.array_equal(A.row_ptr, B.row_ptr) and np.array_equal(A.col, B.col)
    assert np.array_equal(A.val, B.val)
    assert not np.array_equal(A.col, synth.banded_sym(n, per_row, hw, 5).col)
    _check_layout(A.row_ptr, te.spmv_layout(A.row_ptr, A.nnz))


def _reference_layout(rp, window, vmax):
    """The SELL-C-sigma arrangement written out plainly: per window of rows,
    the pieces in row order (rows longer than vmax cut into pieces of vmax,
    numbered in row order across windows), stably sorted longest first, 32
    per slice, each slice as long as its first piece, empty lanes INT32_MIN."""
    n = len(rp) - 1
    skip = np.iinfo(np.int32).min
    slen, out, src, ln = [], [], [], []
    pieces = 0
    for r0 in range(0, n, window):
        win = []
        for r in range(r0, min(r0 + window, n)):
            L = int(rp[r + 1] - rp[r])
            if L == 0:
                continue
            if L <= vmax:
                win.append((int(rp[r]), L, r))
                continue
            count = (L + vmax - 1) // vmax
            for c in range(count):
                s0 = int(rp[r]) + c * vmax
                win.append((s0, min(vmax, int(rp[r]) + L - s0), -1 - (pieces + c)))
            pieces += count
        win.sort(key=lambda p: -p[1])  # stable
        for i in range(0, len(win), 32):
            part = win[i:i + 32]
            slen.append(part[0][1])
            for lane in range(32):
                if lane < len(part):
                    src.append(part[lane][0]); ln.append(part[lane][1]); out.append(part[lane][2])
                else:
                    src.append(0); ln.append(0); out.append(skip)
    return (np.array(slen, dtype=np.int32), np.array(out, dtype=np.int32),
            np.array(src, dtype=np.int64), np.array(ln, dtype=np.int32))


@pytest.mark.parametrize("window,vmax", [(2048, 64), (2048, 128), (256, 32), (7, 5)])
def test_layout_equals_the_plain_arrangement(te, window, vmax):
    """The threaded two-pass layout build (counts per window, then every window
    written at its offsets) equals the plain sequential arrangement exactly:
    slice lengths, lane outputs and piece slots, piece starts and lengths."""
    n = 6000
    lens = np.zeros(n, dtype=np.int64)
    lens[::5] = 3
    lens[7] = n // 2
    for i, L in enumerate([63, 64, 65, 127, 128, 129, 700]):
        lens[100 + 37 * i] = L
    star = np.concatenate([[0], np.cumsum(lens)])
    for rp in (synth.rmat_sym(13, 8, 4).row_ptr, synth.banded_sym(5000, 6, 50, 2).row_ptr, star):
        L = te.spmv_layout(rp, int(rp[-1]), window, vmax)
        slen, out, src, ln = _reference_layout(rp, window, vmax)
        assert np.array_equal(L["slice_len"], slen)
        assert np.array_equal(L["lane_out"], out)
        assert np.array_equal(L["lane_src"], src)
        assert np.array_equal(L["lane_len"], ln)
        assert L["entries"] == 32 * int(slen.astype(np.int64).sum())


def test_planted_generator_spectrum():
    """synth.planted_sym without a background is a block diagonal of unit
    cliques (zero diagonal) of sizes round(smin * ratio^k): its spectrum is
    s_k - 1 once per clique, -1 with multiplicity sum (s_k - 1), and 0 for
    the vertices outside every clique (dense eigensolver, brute force).  With
    the background it stays symmetric and holds the background's entries."""
    n, ncomm, smin, ratio = 400, 5, 4, 1.5
    A = synth.planted_sym(n, 0, ncomm, smin, ratio, 3)
    D = A.to_dense()
    assert np.array_equal(D, D.T) and np.all(np.diag(D) == 0)
    sizes = [int(np.floor(smin * ratio ** (ncomm - 1 - k) + 0.5)) for k in range(ncomm)]
    assert A.nnz == sum(s * (s - 1) for s in sizes)
    ev = np.sort(np.linalg.eigvalsh(D))
    expect = np.sort(np.concatenate([[s - 1.0 for s in sizes],
                                     -np.ones(sum(s - 1 for s in sizes)),
                                     np.zeros(n - sum(sizes))]))
    assert np.max(np.abs(ev - expect)) <= 1e-12 * max(sizes)
    B = synth.planted_sym(n, 3, ncomm, smin, ratio, 3)
    DB = B.to_dense()
    assert np.array_equal(DB, DB.T)
    bg = synth.uniform_sym(n, 3, 3).to_dense()
    assert np.allclose(DB - bg, D, rtol=0, atol=1e-15)
    assert not np.array_equal(A.col, synth.planted_sym(n, 0, ncomm, smin, ratio, 4).col)


def test_binding_passes_values_through(te):
    """CSR.from_host only marshals: binary64 values for a binary32 form are
    flagged values_f64 (the library rounds them for a narrower form),
    binary32 values pass as they are, and a binary64 form refuses binary32
    values."""
    A = synth.uniform_sym(50, 3, 1)
    c = te.CSR.from_host(A, "fdf", device="cpu")
    assert c.values_f64 and c.to_ctypes().values_f64 == 1
    assert np.array_equal(c.val.numpy(), A.val)
    c32 = te.CSR.from_host(A.with_f32_values(), "fdf", device="cpu")
    assert not c32.values_f64 and c32.to_ctypes().values_f64 == 0
    assert np.array_equal(c32.val.numpy(), A.val.astype(np.float32))
    with pytest.raises(ValueError):
        te.CSR.from_host(A.with_f32_values(), "ddd", device="cpu")
    with pytest.raises(ValueError):
        te.CSR.from_host(A.with_f32_values(), "bdf", device="cpu")
