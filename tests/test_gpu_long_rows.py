"""Compensated summation of outputs with more than 4096 terms (long rows, columns,
fibers and slices) in the binary32 modes.

The data are chosen so that a plain binary32 running sum fails the error gate
(2 log2 n + 2) * 2^-24 of the other GPU tests: every term of the long row has the same
sign and the same low-order bits, so each addition of a running sum rounds the same way
and the errors add up linearly. (Random-sign or cancelling terms would not show the
difference: relative to sum |t|, their running sums stay accurate.) Each test first
shows, on the host, that a plain sequential binary32 sum of the long row's terms taken
in pieces of one work unit misses the gate by a wide margin, and then that the kernel
meets it: rows longer than 4096 nonzeros are accumulated with compensated (Kahan)
summation, or by a summation tree, and pieces of a row are combined in binary64.
"""
import numpy as np
import pytest
import torch

import oracle
import spd_synth
import paper_2207_13901_gb300 as spd
from tests._util import binary32_gate, check_error, row_lengths, small_csr

pytestmark = pytest.mark.gpu

LONG = 10000  # terms of the long output (> 4096)
# per dtype: (value of every long-row entry, value of the dense operand it meets); the
# products are exact in binary32 and their low bits make every running-sum step round
# the same way
DATA = {torch.float32: (1.1, 1.0), torch.bfloat16: (1.3984375, 1.3359375), torch.float64: (1.1, 1.0)}
DTYPES = [torch.float32, torch.bfloat16, torch.float64]


def rounded(a, dtype):
    return torch.as_tensor(np.asarray(a, dtype=np.float64)).to(dtype).to(torch.float64).numpy()


def dev(a, dtype):
    return torch.as_tensor(np.asarray(a, dtype=np.float64)).to(dtype).cuda().contiguous()


def plain_binary32_error(terms, unit):
    """Normalised error of summing `terms` with a binary32 running sum in pieces of
    `unit` terms, the pieces added exactly (the best a piece-wise plain sum can do)."""
    t32 = np.asarray(terms, dtype=np.float32)
    total = 0.0
    for s in range(0, t32.shape[0], unit):
        acc = np.float32(0.0)
        for v in t32[s:s + unit]:
            acc = np.float32(acc + v)
        total += float(acc)
    t64 = t32.astype(np.float64)
    return abs(total - t64.sum()) / np.abs(t64).sum()


def assert_adversarial(terms, unit=2048):
    gate = float(binary32_gate(len(terms)))
    err = plain_binary32_error(terms, unit)
    assert err > 3 * gate, "the data do not defeat a plain running sum (%.3e vs gate %.3e)" % (err, gate)


def long_row_matrix(dtype, seed=3):
    """3000 x 12000: short random rows, empty rows, and row 1234 with LONG entries of the
    same value; returns the matrix and the long row's columns."""
    rng = np.random.default_rng(seed)
    n, m = 3000, 12000
    A = small_csr(rng, n, 400, 0.01)
    rows = np.repeat(np.arange(n), np.diff(A.pos))
    big = np.sort(rng.choice(m, LONG, replace=False))
    v, _ = DATA[dtype]
    A = spd_synth.csr_from_coords(n, m, np.concatenate([rows, np.full(LONG, 1234)]), np.concatenate([A.crd, big]),
                                  vals=np.concatenate([A.vals, np.full(LONG, v)]))
    return A, big


@pytest.mark.parametrize("dtype", DTYPES)
def test_spmv_long_row(dtype):
    A, big = long_row_matrix(dtype)
    v, xv = DATA[dtype]
    rng = np.random.default_rng(1)
    x = rng.uniform(-1, 1, A.ncols)
    x[big] = xv
    vr, xr = rounded(A.vals, dtype), rounded(x, dtype)
    assert_adversarial(np.full(LONG, rounded([v], dtype)[0] * rounded([xv], dtype)[0]))
    ref = oracle.spmv(A.pos, A.crd, vr, xr, accurate=True)
    scale = oracle.spmv(A.pos, A.crd, np.abs(vr), np.abs(xr))
    dA = spd.CSR.from_host(A.pos, A.crd, A.vals, (A.nrows, A.ncols), dtype=dtype)
    for split, tune in [("nnz", None), ("row", None), ("row", {"row_pieces": 3}), ("nnz", {"form": 2}),
                        ("row", {"form": 2, "row_pieces": 3})]:
        y = spd.spmv(dA, dev(x, dtype), split=split, tune=tune)
        check_error(y.double().cpu().numpy(), ref, scale, dtype == torch.float64, row_lengths(A.pos),
                    "spmv long row %s %s %s" % (dtype, split, tune))


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("L", [16, 64, 128])
@pytest.mark.parametrize("lane_groups", [1, 2])
def test_spmm_long_row(dtype, L, lane_groups):
    A, big = long_row_matrix(dtype)
    v, xv = DATA[dtype]
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, (A.ncols, L))
    X[big, :] = xv
    vr, Xr = rounded(A.vals, dtype), rounded(X, dtype)
    sel = np.unique(np.concatenate([rng.integers(0, A.nrows, 300), [1234]]))
    ref = oracle.spmm(A.pos, A.crd, vr, Xr, sel=sel, accurate=True)
    scale = oracle.spmm(A.pos, A.crd, np.abs(vr), np.abs(Xr), sel=sel)
    dA = spd.CSR.from_host(A.pos, A.crd, A.vals, (A.nrows, A.ncols), dtype=dtype)
    dX = dev(X, dtype)
    for split, tune in [("nnz", {}), ("nnz", {"unit_items": 512}), ("row", {})]:
        tune = dict(tune, lane_groups=lane_groups)
        Y = spd.spmm(dA, dX, split=split, tune=tune)
        check_error(Y.double().cpu().numpy()[sel], ref, scale, dtype == torch.float64,
                    row_lengths(A.pos)[sel][:, None], "spmm long row %s L=%d %s %s" % (dtype, L, split, tune))


@pytest.mark.parametrize("dtype", DTYPES)
def test_spmm_t_over_transpose_long_column(dtype):
    """dX = A^T dY as an SpMM over A^T: column 77 of A (a row of A^T) holds LONG entries."""
    rng = np.random.default_rng(4)
    n, m, L = LONG + 500, 300, 32
    v, xv = DATA[dtype]
    rows = np.concatenate([np.arange(LONG), rng.integers(0, n, 3000)])
    cols = np.concatenate([np.full(LONG, 77), rng.integers(0, m, 3000)])
    cols[LONG:][cols[LONG:] == 77] = 78
    vals = np.concatenate([np.full(LONG, v), rng.uniform(-1, 1, 3000)])
    A = spd_synth.csr_from_coords(n, m, rows, cols, vals=vals)
    dY = rng.uniform(-1, 1, (n, L))
    dY[:LONG] = xv
    vr, dYr = rounded(A.vals, dtype), rounded(dY, dtype)
    ref = oracle.spmm_t(A.pos, A.crd, vr, dYr, m, accurate=True)
    scale = oracle.spmm_t(A.pos, A.crd, np.abs(vr), np.abs(dYr), m)
    dA = spd.CSR.from_host(A.pos, A.crd, A.vals, (n, m), dtype=dtype)
    for split in ("nnz", "row"):
        dX = spd.spmm_t(dA, dev(dY, dtype), split=split, method="transpose")
        check_error(dX.double().cpu().numpy(), ref, scale, dtype == torch.float64,
                    np.bincount(A.crd, minlength=m)[:, None], "spmm_t transpose long column %s %s" % (dtype, split))


def long_slice_tensor(dtype, seed=5):
    """CSF 4 x 6000 x 12000: slice 1 holds a fiber of 5000 entries, 40 fibers of 50 and
    1500 fibers of 2 (LONG entries of one value in all); other slices are short."""
    rng = np.random.default_rng(seed)
    v, _ = DATA[dtype]
    ii, jj, kk, vv = [], [], [], []
    def fiber(i, j, ks, val):
        ii.append(np.full(len(ks), i)); jj.append(np.full(len(ks), j)); kk.append(np.sort(ks)); vv.append(val)
    for j in range(0, 30):
        ks = rng.choice(12000, 7, replace=False)
        fiber(0, j, ks, rng.uniform(-1, 1, 7))
    fiber(1, 0, rng.choice(12000, 5000, replace=False), np.full(5000, v))
    for j in range(1, 41):
        fiber(1, j, rng.choice(12000, 50, replace=False), np.full(50, v))
    for j in range(41, 1541):
        fiber(1, j, rng.choice(12000, 2, replace=False), np.full(2, v))
    for j in range(0, 50):
        ks = rng.choice(12000, 5, replace=False)
        fiber(3, j, ks, rng.uniform(-1, 1, 5))
    T = spd_synth.csf3_from_coords((4, 6000, 12000), np.concatenate(ii), np.concatenate(jj), np.concatenate(kk),
                                   np.concatenate(vv))
    assert int(T.pos2[T.pos1[2]] - T.pos2[T.pos1[1]]) == LONG
    return T


@pytest.mark.parametrize("dtype", DTYPES)
def test_spttv_long_fiber(dtype):
    T = long_slice_tensor(dtype)
    v, xv = DATA[dtype]
    c = np.full(T.dims[2], xv)
    vr, cr = rounded(T.vals, dtype), rounded(c, dtype)
    ref = oracle.spttv(T.pos1, T.crd1, T.pos2, T.crd2, vr, cr, accurate=True)
    scale = oracle.spttv(T.pos1, T.crd1, T.pos2, T.crd2, np.abs(vr), np.abs(cr))
    assert_adversarial(np.full(5000, rounded([v], dtype)[0] * rounded([xv], dtype)[0]), unit=2048)
    dT = spd.CSF3.from_host(T.pos1, T.crd1, T.pos2, T.crd2, T.vals, T.dims, dtype=dtype)
    for split, form in (("nnz", 1), ("row", 1), ("nnz", 2), ("row", 2)):
        out = spd.spttv(dT, dev(c, dtype), split=split, tune={"form": form})
        check_error(out.double().cpu().numpy(), ref, scale, dtype == torch.float64, row_lengths(T.pos2),
                    "spttv long fiber %s %s" % (dtype, split))
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("R", [16, 32, 64])
def test_spmttkrp_long_slice(dtype, R):
    T = long_slice_tensor(dtype)
    v, xv = DATA[dtype]
    rng = np.random.default_rng(6)
    C = rng.uniform(-1, 1, (T.dims[1], R))
    C[:1541] = 1.0  # the long slice's fibers meet rows of ones, so every term is v * xv
    D = np.full((T.dims[2], R), xv)
    vr, Cr, Dr = rounded(T.vals, dtype), rounded(C, dtype), rounded(D, dtype)
    assert_adversarial(np.full(LONG, rounded([v], dtype)[0] * rounded([xv], dtype)[0]))
    ref = oracle.spmttkrp(T.pos1, T.crd1, T.pos2, T.crd2, vr, Cr, Dr, accurate=True)
    scale = oracle.spmttkrp(T.pos1, T.crd1, T.pos2, T.crd2, np.abs(vr), np.abs(Cr), np.abs(Dr))
    slice_len = row_lengths(np.asarray(T.pos2, dtype=np.int64)[np.asarray(T.pos1, dtype=np.int64)])
    dT = spd.CSF3.from_host(T.pos1, T.crd1, T.pos2, T.crd2, T.vals, T.dims, dtype=dtype)
    for split, tune in [("nnz", None), ("nnz", {"unit_items": 512}), ("row", None),
                        ("nnz", {"unit_items": 512, "block_threads": 512}), ("row", {"block_threads": 64})]:
        A = spd.spmttkrp(dT, dev(C, dtype), dev(D, dtype), split=split, tune=tune)
        check_error(A.double().cpu().numpy(), ref, scale, dtype == torch.float64, slice_len[:, None],
                    "spmttkrp long slice %s R=%d %s %s" % (dtype, R, split, tune), extra=1)
