"""The SpMV layout and the row order built on the device (te_layout_dev.cu)
against a plain arrangement written out in Python, element by element
(integer and index work: bit-exact), and plans built both ways.

The plain arrangement (tests/test_capi_host.py, _reference_layout) takes the
rows in a given order, cuts rows longer than vmax into pieces, sorts each
window's pieces by length (stable, longest first) and packs them 32 per slice.
The row order is numpy's stable sort of the rows by length, longest first.
"""
import numpy as np
import pytest
import torch

import synth
from test_capi_host import _reference_layout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def te():
    import paper_2201_07498_gb300 as te
    te.load_library(build_if_missing=True)
    return te


def _star_lengths(n):
    lens = np.zeros(n, dtype=np.int64)
    lens[::5] = 3
    lens[7] = n // 2
    for i, L in enumerate([63, 64, 65, 127, 128, 129, 700, 1024, 1025, 4097]):
        lens[100 + 37 * i] = L
    return np.concatenate([[0], np.cumsum(lens)])


def _row_ptrs():
    return {
        "rmat13": synth.rmat_sym(13, 8, 4).row_ptr,
        "rmat16": synth.rmat_sym(16, 16, 1).row_ptr,
        "banded": synth.banded_sym(5000, 6, 50, 2).row_ptr,
        "star": _star_lengths(6000),
        "empty_rows": np.zeros(3001, dtype=np.int64),
        "one_row": np.array([0, 5], dtype=np.int64),
        "ragged_tail": synth.uniform_sym(2048 * 3 + 17, 9, 3).row_ptr,
    }


def _expected(rp, window, vmax, order):
    lens = np.diff(rp)
    n = len(lens)
    perm = (np.argsort(-lens, kind="stable") if order == "degree"
            else np.arange(n)).astype(np.int32)
    # the arrangement of the relabelled rows: row r has the length of CSR row
    # perm[r]; its pieces start at that row's first entry
    rp_perm = np.concatenate([[0], np.cumsum(lens[perm])])
    slen, out, src_rel, ln = _reference_layout(rp_perm, window, vmax)
    # map each lane's piece back to the caller's CSR
    rows_of = np.repeat(np.arange(n), lens[perm])
    src = np.zeros_like(src_rel)
    lane_row = np.full(len(out), -1, dtype=np.int32)
    live = ln > 0
    r = rows_of[src_rel[live]]
    src[live] = rp[perm[r]] + (src_rel[live] - rp_perm[r])
    lane_row[live] = perm[r]
    return perm, slen, out, src, ln, lane_row


@pytest.mark.parametrize("order", ["keep", "degree"])
@pytest.mark.parametrize("window,vmax", [(2048, 64), (2048, 128), (2048, 32), (256, 64), (16384, 64),
                                         (256, 32), (7, 5)])
def test_device_layout_equals_the_plain_arrangement(te, order, window, vmax):
    for name, rp in _row_ptrs().items():
        nnz = int(rp[-1])
        L = te.spmv_layout_device(torch.from_numpy(rp).cuda(), nnz, window, vmax, order)
        perm, slen, out, src, ln, lrow = _expected(rp, window, vmax, order)
        assert np.array_equal(L["perm"], perm), name
        assert np.array_equal(L["slice_len"], slen), name
        assert np.array_equal(L["lane_out"], out), name
        assert np.array_equal(L["lane_src"], src), name
        assert np.array_equal(L["lane_len"], ln), name
        assert np.array_equal(L["lane_row"], lrow), name
        sizes = 32 * slen.astype(np.int64)
        bases = np.cumsum(sizes) - sizes
        assert np.array_equal(L["slice_base"], bases), name
        assert L["entries"] == 32 * int(slen.astype(np.int64).sum()), name
        # cut rows: every row longer than vmax once, most pieces first, ties in
        # row order, partial slots numbered in row order
        lens = np.diff(rp)[perm]
        cut = np.nonzero(lens > vmax)[0]
        count = (lens[cut] + vmax - 1) // vmax
        first = np.concatenate([[0], np.cumsum(count)[:-1]])
        o = np.argsort(-count, kind="stable")
        exp = np.stack([cut[o], first[o], count[o]], axis=1) if len(cut) else np.zeros((0, 3))
        assert np.array_equal(L["long_rows"], exp.astype(np.int32)), name
        assert L["nbig"] == int(np.sum(count > 16)), name


def test_device_degree_order_equals_host(te):
    A = synth.rmat_sym(18, 16, 7)
    L = te.spmv_layout_device(torch.from_numpy(A.row_ptr).cuda(), A.nnz, order="degree")
    perm, _ = te.degree_order(A.row_ptr, A.nnz)
    assert np.array_equal(L["perm"], perm)


def test_device_layout_rejects_malformed_row_ptr(te):
    rp = np.array([0, 3, 2, 5], dtype=np.int64)
    with pytest.raises(te.TEError) as e:
        te.spmv_layout_device(torch.from_numpy(rp).cuda(), 5)
    assert e.value.status == 1 and "non-decreasing" in str(e.value)
    with pytest.raises(te.TEError) as e:
        te.spmv_layout_device(torch.from_numpy(np.array([0, 3, 5], dtype=np.int64)).cuda(), 4)
    assert e.value.status == 1


@pytest.mark.parametrize("where", ["device", "host"])
@pytest.mark.parametrize("prec", ["fdf", "bdf", "8df", "ddd"])
def test_plan_with_device_layout_equals_host_layout(te, where, prec):
    """A resident plan builds its layout on the device; a streamed plan of
    the same matrix builds the same layout on the host and runs the same
    slice computations block by block.  Equal layouts give the same bits.
    (bfloat16 and FP8 values cannot be streamed: their device-built plans
    just run.)"""
    A = synth.rmat_sym(14, 8, 3)
    dev = te.CSR.from_host(A, prec, device="cuda" if where == "device" else "cpu",
                           pin=where == "host")
    p1 = te.Plan(dev, 6, 20, prec, seed=5, order="degree")
    ev1, U1, r1 = p1.solve(residuals=True)
    if prec in ("ddd", "fdf"):
        host = te.CSR.from_host(A, prec, device="cpu", pin=True)
        p2 = te.Plan(host, 6, 20, prec, seed=5, order="degree", matrix_budget=96 * 1024)
        assert p2.stream_blocks >= 8
        ev2, U2, r2 = p2.solve(residuals=True)
        assert torch.equal(ev1, ev2) and torch.equal(U1, U2) and torch.equal(r1, r2)
