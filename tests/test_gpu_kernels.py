"""GPU parity: every CUDA kernel through the C ABI against the CPU oracle.

Sizes span several work pieces and tiles with ragged tails; edge cases cover empty
matrices, empty rows, a row longer than 4096 nonzeros (compensated summation, rows
split across many pieces), all entries in one column, and non-default tunings.

Tolerances, relative to max(|ref|, sum of |terms|) per output entry (the normaliser
of the usual summation error bound):
  binary64 results: 1e-12 against the compensated oracle;
  binary32 / bfloat16 inputs with binary32 accumulation: (2 log2 n + 2) * 2^-24 per
  output of n terms (one more unit for the triple-product statements SDDMM and
  SpMTTKRP) against the compensated oracle run on the same rounded inputs.
Integer, index and structure outputs are compared bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
import spd_synth
import paper_2207_13901_gb300 as spd
from tests._util import check_error, normalized_error, row_lengths, small_csf, small_csr

pytestmark = pytest.mark.gpu

DTYPES = [torch.float64, torch.float32, torch.bfloat16]
SPLITS = ["row", "nnz"]


def rounded(a, dtype):
    """Host values rounded to ``dtype`` and widened back to float64 (what the GPU sees)."""
    return torch.as_tensor(np.asarray(a, dtype=np.float64)).to(dtype).to(torch.float64).numpy()


def dev(a, dtype):
    return torch.as_tensor(np.asarray(a, dtype=np.float64)).to(dtype).cuda().contiguous()


def dev_csr(A, dtype):
    return spd.CSR.from_host(A.pos, A.crd, A.vals, (A.nrows, A.ncols), dtype=dtype)


def dev_csf(T, dtype):
    return spd.CSF3.from_host(T.pos1, T.crd1, T.pos2, T.crd2, T.vals, T.dims, dtype=dtype)


def long_row_csr(seed=5):
    """Many short rows, empty rows, and one row of 10000 nonzeros (> 4096)."""
    rng = np.random.default_rng(seed)
    n, m = 3000, 12000
    A = small_csr(rng, n, 400, 0.01)
    rows = np.repeat(np.arange(n), np.diff(A.pos))
    big_cols = np.sort(rng.choice(m, 10000, replace=False))
    rows = np.concatenate([rows, np.full(10000, 1234)])
    cols = np.concatenate([A.crd, big_cols])
    vals = np.concatenate([A.vals, rng.uniform(-1, 1, 10000)])
    return spd_synth.csr_from_coords(n, m, rows, cols, vals=vals)


def matrices():
    rng = np.random.default_rng(0)
    mats = {
        "uniform4096": spd_synth.uniform_csr(4096, 4096, 16, seed=0),
        "rmat12": spd_synth.rmat_csr(12, 16, seed=1),
        "longrow": long_row_csr(),
        "col0": spd_synth.csr_from_coords(700, 50, np.arange(700), np.zeros(700, dtype=np.int64),
                                          vals=rng.uniform(-1, 1, 700)),
        "empty_rows": small_csr(rng, 5000, 300, 0.002, empty_frac=0.9),
        "no_nnz": spd_synth.csr_from_coords(37, 20, [], [], vals=np.zeros(0)),
        "one_row": small_csr(rng, 1, 9000, 0.6, empty_frac=0.0),
        "banded": spd_synth.banded_csr(20000, 16, seed=4),
    }
    return mats


MATS = None


def get_mats():
    global MATS
    if MATS is None:
        MATS = matrices()
    return MATS


MAT_NAMES = ["uniform4096", "rmat12", "longrow", "col0", "empty_rows", "no_nnz", "one_row", "banded"]


def check(got, ref, scale, dtype, what, nterms, extra=0.0):
    """Error gate of every output: 1e-12 for binary64, binary32_gate(nterms) otherwise."""
    return check_error(got, ref, scale, dtype == torch.float64, nterms, what, extra)


# ------------------------------------------------------------------------------ structure

@pytest.mark.parametrize("name", MAT_NAMES)
def test_partitions_bit_exact(name):
    A = get_mats()[name]
    dA = dev_csr(A, torch.float32)
    T = A.nrows + A.nnz
    for unit in (32, 96, 2048):
        npieces = -(-T // unit)
        if npieces == 0:
            continue
        rows, poss = spd.partition(dA, "nnz", npieces, unit)
        d = np.minimum(np.arange(npieces + 1, dtype=np.int64) * unit, T)
        wr, wp = oracle.merge_path(A.pos, d)
        assert np.array_equal(rows.cpu().numpy(), wr) and np.array_equal(poss.cpu().numpy(), wp)
    for P in (1, 2, 3, 7, 152, 1000):
        rows, poss = spd.partition(dA, "row", P)
        b = oracle.row_split(A.nrows, P)
        assert np.array_equal(rows.cpu().numpy(), b)
        assert np.array_equal(poss.cpu().numpy(), A.pos[b])


def test_validate_detects_planted_faults():
    rng = np.random.default_rng(3)
    A = small_csr(rng, 3000, 200, 0.02)
    cases = [(A.pos, A.crd)]
    p = A.pos.copy(); p[100], p[101] = p[101] + 5, p[100]; cases.append((p, A.crd))
    p = A.pos.copy(); p[-1] -= 1; cases.append((p, A.crd))
    c = A.crd.copy(); c[17] = 200; c[5000 % len(c)] = -3; cases.append((A.pos, c))
    for pos, crd in cases:
        d = spd.CSR.from_host(pos, crd, None, (A.nrows, A.ncols))
        got = spd.validate(d)
        want = oracle.validate_level(A.nrows, A.ncols, pos, crd)
        assert got == want
    T = small_csf(rng, (40, 30, 50), 0.05)
    dT = dev_csf(T, torch.float32)
    assert spd.validate(dT) == (0, -1)
    crd2 = T.crd2.copy(); crd2[7] = 50
    dT2 = spd.CSF3.from_host(T.pos1, T.crd1, T.pos2, crd2, T.vals, T.dims)
    cnt, first = spd.validate(dT2)
    assert cnt == 1 and first == (T.dims[0] + 1 + T.nfib) + (T.nfib + 1) + 7


# ------------------------------------------------------------------------------ SpMV

@pytest.mark.parametrize("name", MAT_NAMES)
@pytest.mark.parametrize("dtype", DTYPES)
def test_spmv(name, dtype):
    A = get_mats()[name]
    rng = np.random.default_rng(11)
    x = rng.uniform(-1, 1, A.ncols)
    vr, xr = rounded(A.vals, dtype), rounded(x, dtype)
    ref = oracle.spmv(A.pos, A.crd, vr, xr, accurate=True)
    scale = oracle.spmv(A.pos, A.crd, np.abs(vr), np.abs(xr))
    dA = dev_csr(A, dtype)
    for split in SPLITS:
        for form in (1, 2):  # block tiles; warp tiles with bulk copies
            y = spd.spmv(dA, dev(x, dtype), split=split, tune={"form": form})
            torch.cuda.synchronize()
            assert y.dtype == spd.result_dtype(dtype)
            check(y.double().cpu().numpy(), ref, scale, dtype, "spmv %s %s %s form %d" % (name, dtype, split, form),
                  row_lengths(A.pos))


@pytest.mark.parametrize("name", ["rmat12", "longrow", "empty_rows", "banded"])
@pytest.mark.parametrize("dtype", DTYPES)
def test_spmv_warp_form_unaligned_operands(name, dtype):
    """crd and vals that do not start on a 16-byte boundary (views one element into
    larger arrays): the warp-tile form falls back from bulk copies to plain loads."""
    A = get_mats()[name]
    rng = np.random.default_rng(18)
    x = rng.uniform(-1, 1, A.ncols)
    vr, xr = rounded(A.vals, dtype), rounded(x, dtype)
    ref = oracle.spmv(A.pos, A.crd, vr, xr, accurate=True)
    scale = oracle.spmv(A.pos, A.crd, np.abs(vr), np.abs(xr))
    crd_big = torch.zeros(A.nnz + 1, dtype=torch.int32, device="cuda")
    crd_big[1:] = torch.as_tensor(A.crd).cuda()
    val_big = torch.zeros(A.nnz + 1, dtype=dtype, device="cuda")
    val_big[1:] = dev(A.vals, dtype)
    dA = spd.CSR(torch.as_tensor(A.pos).cuda(), crd_big[1:], val_big[1:], (A.nrows, A.ncols))
    for split in SPLITS:
        y = spd.spmv(dA, dev(x, dtype), split=split, tune={"form": 2})
        torch.cuda.synchronize()
        check(y.double().cpu().numpy(), ref, scale, dtype, "spmv unaligned %s %s %s" % (name, dtype, split),
              row_lengths(A.pos))


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_spmv_split_invariance_integer_exact(dtype):
    """Integer data: every summation order is exact, so all splits and piece counts give
    bit-identical results equal to the oracle (Section II-D: both distributions
    compute the same statement)."""
    rng = np.random.default_rng(4)
    A = long_row_csr(6)
    vals = rng.integers(-4, 5, A.nnz).astype(np.float64)
    x = rng.integers(-4, 5, A.ncols).astype(np.float64)
    ref = oracle.spmv(A.pos, A.crd, vals, x)
    dA = spd.CSR.from_host(A.pos, A.crd, vals, (A.nrows, A.ncols), dtype=dtype)
    dx = dev(x, dtype)
    for split, tune in [("row", None), ("nnz", None), ("row", {"row_pieces": 1}), ("row", {"row_pieces": 7}),
                        ("row", {"row_pieces": 152}), ("nnz", {"unit_items": 64}), ("nnz", {"form": 2}),
                        ("row", {"form": 2}), ("row", {"form": 2, "row_pieces": 7})]:
        y = spd.spmv(dA, dx, split=split, tune=tune).double().cpu().numpy()
        assert np.array_equal(y, ref), (split, tune)


# ------------------------------------------------------------------------------ SpMM

@pytest.mark.parametrize("name", ["uniform4096", "rmat12", "longrow", "col0", "empty_rows", "no_nnz"])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("L", [1, 7, 16, 32, 48, 64, 128])
def test_spmm(name, dtype, L):
    """L picks the lane shape: vector lanes covering whole tiles (64, 128), narrower
    vectors with idle lanes (16, 32, 48) and scalar lanes (1, 7)."""
    A = get_mats()[name]
    rng = np.random.default_rng(12)
    X = rng.uniform(-1, 1, (A.ncols, L))
    vr, Xr = rounded(A.vals, dtype), rounded(X, dtype)
    sel = None
    if A.nrows > 1500:
        sel = np.unique(np.concatenate([rng.integers(0, A.nrows, 600), np.argsort(np.diff(A.pos))[-20:]]))
    ref = oracle.spmm(A.pos, A.crd, vr, Xr, sel=sel, accurate=True)
    scale = oracle.spmm(A.pos, A.crd, np.abs(vr), np.abs(Xr), sel=sel)
    dA = dev_csr(A, dtype)
    dX = dev(X, dtype)
    for split in SPLITS:
        Y = spd.spmm(dA, dX, split=split)
        torch.cuda.synchronize()
        got = Y.double().cpu().numpy()
        if sel is not None:
            got = got[sel]
        lens = row_lengths(A.pos) if sel is None else row_lengths(A.pos)[sel]
        check(got, ref, scale, dtype, "spmm %s %s L=%d %s" % (name, dtype, L, split), lens[:, None])


@pytest.mark.parametrize("dtype", DTYPES)
def test_spmm_strided_and_tuned(dtype):
    """Leading dimensions larger than L, odd L (scalar lanes, two column tiles) and
    small work units (many pieces per row)."""
    A = get_mats()["longrow"]
    rng = np.random.default_rng(13)
    L = 200
    Xfull = rng.uniform(-1, 1, (A.ncols, 208))
    vr, Xr = rounded(A.vals, dtype), rounded(Xfull[:, :L], dtype)
    sel = np.unique(np.concatenate([rng.integers(0, A.nrows, 300), [1234]]))
    ref = oracle.spmm(A.pos, A.crd, vr, Xr, sel=sel, accurate=True)
    scale = oracle.spmm(A.pos, A.crd, np.abs(vr), np.abs(Xr), sel=sel)
    dA = dev_csr(A, dtype)
    dX = dev(Xfull, dtype)[:, :L]
    Yfull = torch.full((A.nrows, 256), 7.0, dtype=spd.result_dtype(dtype), device="cuda")
    for split, tune in [("nnz", {"unit_items": 32}), ("nnz", {"unit_items": 4096, "block_threads": 128}),
                        ("row", {"row_pieces": 5})]:
        Y = spd.spmm(dA, dX, Y=Yfull[:, :L], split=split, tune=tune)
        torch.cuda.synchronize()
        check(Y.double().cpu().numpy()[sel], ref, scale, dtype, "spmm strided %s %s" % (split, tune),
              row_lengths(A.pos)[sel][:, None])
        assert torch.all(Yfull[:, L:] == 7.0)  # columns beyond L untouched


@pytest.mark.parametrize("name", ["rmat12", "longrow", "empty_rows"])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("L", [16, 32, 64, 128])
@pytest.mark.parametrize("lane_groups", [1, 2])
def test_spmm_lane_shapes(name, dtype, L, lane_groups):
    """Both SpMM lane shapes a caller can force, at every L where they differ:
    lane_groups=1 takes groups of 4, 8 or 16 lanes with one 16-byte vector each, side by
    side on different nonzeros (the library's choice when X fits in 64 MiB);
    lane_groups=2 takes one nonzero per warp step over 32 narrower lanes (its choice for
    larger X, e.g. 8-byte lanes for bfloat16 at L=128 or binary32 at L=64 on the
    2^22-row workload)."""
    A = get_mats()[name]
    rng = np.random.default_rng(17)
    X = rng.uniform(-1, 1, (A.ncols, L))
    vr, Xr = rounded(A.vals, dtype), rounded(X, dtype)
    sel = np.unique(np.concatenate([rng.integers(0, A.nrows, 500), np.argsort(np.diff(A.pos))[-10:]]))
    ref = oracle.spmm(A.pos, A.crd, vr, Xr, sel=sel, accurate=True)
    scale = oracle.spmm(A.pos, A.crd, np.abs(vr), np.abs(Xr), sel=sel)
    dA = dev_csr(A, dtype)
    dX = dev(X, dtype)
    for split, tune in [("nnz", {}), ("nnz", {"unit_items": 256, "inflight": 4}), ("row", {})]:
        tune = dict(tune, lane_groups=lane_groups)
        Y = spd.spmm(dA, dX, split=split, tune=tune)
        torch.cuda.synchronize()
        check(Y.double().cpu().numpy()[sel], ref, scale, dtype, "spmm %s %s L=%d %s %s" % (name, dtype, L, split, tune),
              row_lengths(A.pos)[sel][:, None])


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("block_threads", [64, 512])
def test_warp_kernels_block_sizes(dtype, block_threads):
    """The smallest and largest blocks of the warp-per-unit kernels (the per-warp windows
    live in shared memory sized by the block): SpMM in both lane shapes, SpMM^T, SDDMM
    in both forms and SpMTTKRP, with many pieces per block and a partial last block."""
    A = get_mats()["rmat12"]
    T = get_tens()["zipf"]
    rng = np.random.default_rng(29)
    vr = rounded(A.vals, dtype)
    dA = dev_csr(A, dtype)
    lens = row_lengths(A.pos)
    for split, unit in (("nnz", 96), ("nnz", 2048), ("row", 0)):
        tune = {"block_threads": block_threads}
        if unit:
            tune["unit_items"] = unit
        for L, groups in ((64, 1), (64, 2), (40, 0)):
            X = rng.uniform(-1, 1, (A.ncols, L))
            Xr = rounded(X, dtype)
            ref = oracle.spmm(A.pos, A.crd, vr, Xr, accurate=True)
            scale = oracle.spmm(A.pos, A.crd, np.abs(vr), np.abs(Xr))
            Y = spd.spmm(dA, dev(X, dtype), split=split, tune=dict(tune, lane_groups=groups))
            check(Y.double().cpu().numpy(), ref, scale, dtype, "spmm bt=%d %s L=%d" % (block_threads, tune, L),
                  lens[:, None])
        dY = rng.uniform(-1, 1, (A.nrows, 32))
        dYr = rounded(dY, dtype)
        ref = oracle.spmm_t(A.pos, A.crd, vr, dYr, A.ncols, accurate=True)
        scale = oracle.spmm_t(A.pos, A.crd, np.abs(vr), np.abs(dYr), A.ncols)
        dX = spd.spmm_t(dA, dev(dY, dtype), split=split, tune=tune)
        check(dX.double().cpu().numpy(), ref, scale, dtype, "spmm_t bt=%d %s" % (block_threads, tune),
              np.bincount(A.crd, minlength=A.ncols)[:, None])
        K = 64
        C = rng.standard_normal((A.nrows, K))
        Dnk = rng.standard_normal((A.ncols, K))
        Cr, Dr = rounded(C, dtype), rounded(Dnk, dtype)
        ref = oracle.sddmm(A.pos, A.crd, vr, Cr, Dr, accurate=True)
        scale = oracle.sddmm(A.pos, A.crd, np.abs(vr), np.abs(Cr), np.abs(Dr))
        for form in ((1, 2) if dtype == torch.bfloat16 else (0,)):
            out = spd.sddmm(dA, dev(C, dtype), dev(Dnk, dtype), split=split, tune=dict(tune, form=form))
            check(out.double().cpu().numpy(), ref, scale, dtype, "sddmm bt=%d %s form %d" % (block_threads, tune, form),
                  K, extra=1)
        R = 32
        Cm = rng.standard_normal((T.dims[1], R))
        Dm = rng.standard_normal((T.dims[2], R))
        tv, Cmr, Dmr = rounded(T.vals, dtype), rounded(Cm, dtype), rounded(Dm, dtype)
        ref = oracle.spmttkrp(T.pos1, T.crd1, T.pos2, T.crd2, tv, Cmr, Dmr, accurate=True)
        scale = oracle.spmttkrp(T.pos1, T.crd1, T.pos2, T.crd2, np.abs(tv), np.abs(Cmr), np.abs(Dmr))
        Am = spd.spmttkrp(dev_csf(T, dtype), dev(Cm, dtype), dev(Dm, dtype), split=split, tune=tune)
        check(Am.double().cpu().numpy(), ref, scale, dtype, "spmttkrp bt=%d %s" % (block_threads, tune),
              slice_lengths(T)[:, None], extra=1)


# ------------------------------------------------------------------------------ SpMM^T

@pytest.mark.parametrize("name", ["uniform4096", "rmat12", "longrow", "col0", "empty_rows", "no_nnz"])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("L", [1, 32, 128])
def test_spmm_t(name, dtype, L):
    A = get_mats()[name]
    rng = np.random.default_rng(14)
    dY = rng.uniform(-1, 1, (A.nrows, L))
    vr, dYr = rounded(A.vals, dtype), rounded(dY, dtype)
    ref = oracle.spmm_t(A.pos, A.crd, vr, dYr, A.ncols, accurate=True)
    scale = oracle.spmm_t(A.pos, A.crd, np.abs(vr), np.abs(dYr), A.ncols)
    dA = dev_csr(A, dtype)
    for split in SPLITS:
        dX = spd.spmm_t(dA, dev(dY, dtype), split=split)
        torch.cuda.synchronize()
        check(dX.double().cpu().numpy(), ref, scale, dtype, "spmm_t %s %s L=%d %s" % (name, dtype, L, split),
              np.bincount(A.crd, minlength=A.ncols)[:, None])


# ------------------------------------------------------------------------------ SDDMM

@pytest.mark.parametrize("name", ["uniform4096", "rmat12", "longrow", "col0", "no_nnz"])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("K", [1, 6, 24, 32, 48, 128, 200, 256, 300])
def test_sddmm(name, dtype, K):
    A = get_mats()[name]
    rng = np.random.default_rng(15)
    C = rng.standard_normal((A.nrows, K))
    Dnk = rng.standard_normal((A.ncols, K))
    vr, Cr, Dr = rounded(A.vals, dtype), rounded(C, dtype), rounded(Dnk, dtype)
    sel = None
    if A.nnz > 20000:
        sel = np.unique(rng.integers(0, A.nnz, 4000))
    ref = oracle.sddmm(A.pos, A.crd, vr, Cr, Dr, sel=sel, accurate=True)
    scale = oracle.sddmm(A.pos, A.crd, np.abs(vr), np.abs(Cr), np.abs(Dr), sel=sel)
    dA = dev_csr(A, dtype)
    dC, dD = dev(C, dtype), dev(Dnk, dtype)
    # bfloat16: CUDA cores (form 1) and tensor cores (form 2, used when K is a multiple of 32)
    forms = (1, 2) if dtype == torch.bfloat16 else (0,)
    for split in SPLITS:
        for form in forms:
            out = spd.sddmm(dA, dC, dD, split=split, tune={"form": form})
            torch.cuda.synchronize()
            got = out.double().cpu().numpy()
            if sel is not None:
                got = got[sel]
            check(got, ref, scale, dtype, "sddmm %s %s K=%d %s form %d" % (name, dtype, K, split, form), K, extra=1)
    # the sampling pattern alone (every B value 1)
    ref1 = oracle.sddmm(A.pos, A.crd, None, Cr, Dr, sel=sel, accurate=True)
    scale1 = oracle.sddmm(A.pos, A.crd, None, np.abs(Cr), np.abs(Dr), sel=sel)
    out = spd.sddmm(dA.with_vals(None), dC, dD).double().cpu().numpy()
    check(out if sel is None else out[sel], ref1, scale1, dtype, "sddmm pattern %s" % name, K, extra=1)


@pytest.mark.parametrize("K", [32, 64, 256])
def test_sddmm_tensor_cores_short_rows(K):
    """bfloat16 on the tensor cores where 16 consecutive positions span up to 16 distinct
    rows (rows of 0 to 3 entries): the second pass over the 9th to 16th rows, empty rows,
    and the sampling pattern alone."""
    rng = np.random.default_rng(19)
    A = spd_synth.uniform_csr(5000, 3000, (0, 3), seed=7)
    C = rng.standard_normal((A.nrows, K))
    Dnk = rng.standard_normal((A.ncols, K))
    dt = torch.bfloat16
    vr, Cr, Dr = rounded(A.vals, dt), rounded(C, dt), rounded(Dnk, dt)
    dA = dev_csr(A, dt)
    for vals in (vr, None):
        ref = oracle.sddmm(A.pos, A.crd, vals, Cr, Dr, accurate=True)
        scale = oracle.sddmm(A.pos, A.crd, None if vals is None else np.abs(vals), np.abs(Cr), np.abs(Dr))
        B = dA if vals is not None else dA.with_vals(None)
        for split in SPLITS:
            out = spd.sddmm(B, dev(C, dt), dev(Dnk, dt), split=split, tune={"form": 2})
            torch.cuda.synchronize()
            check(out.double().cpu().numpy(), ref, scale, dt, "sddmm mma short rows K=%d %s" % (K, split), K, extra=1)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("K", [40, 128, 200])
def test_sddmm_strided_operands(dtype, K):
    """C and Dnk as column windows of wider row-major matrices (leading dimension > K,
    starting 16 elements in), for the register-cached and the general forms."""
    A = get_mats()["rmat12"]
    rng = np.random.default_rng(16)
    C = rng.standard_normal((A.nrows, K))
    Dnk = rng.standard_normal((A.ncols, K))
    vr, Cr, Dr = rounded(A.vals, dtype), rounded(C, dtype), rounded(Dnk, dtype)
    ref = oracle.sddmm(A.pos, A.crd, vr, Cr, Dr, accurate=True)
    scale = oracle.sddmm(A.pos, A.crd, np.abs(vr), np.abs(Cr), np.abs(Dr))
    wideC = torch.zeros((A.nrows, K + 48), dtype=dtype, device="cuda")
    wideD = torch.zeros((A.ncols, K + 32), dtype=dtype, device="cuda")
    wideC[:, 16:16 + K] = dev(C, dtype)
    wideD[:, 16:16 + K] = dev(Dnk, dtype)
    dA = dev_csr(A, dtype)
    for split in SPLITS:
        for form in ((1, 2) if dtype == torch.bfloat16 else (0,)):
            out = spd.sddmm(dA, wideC[:, 16:16 + K], wideD[:, 16:16 + K], split=split, tune={"form": form})
            torch.cuda.synchronize()
            check(out.double().cpu().numpy(), ref, scale, dtype, "sddmm strided %s K=%d %s form %d" % (dtype, K, split, form),
                  K, extra=1)


# ------------------------------------------------------------------------------ CSF kernels

def slice_lengths(T):
    """Entries of every slice i of a CSF tensor (the terms summed into row i of SpMTTKRP)."""
    return row_lengths(np.asarray(T.pos2, dtype=np.int64)[np.asarray(T.pos1, dtype=np.int64)])


def tensors():
    rng = np.random.default_rng(21)
    return {
        "zipf": spd_synth.zipf_csf3((1 << 10, 1 << 10, 1 << 10), 200000, seed=0),
        "dense_small": small_csf(rng, (30, 20, 40), 0.3),
        "long_fiber": spd_synth.csf3_from_coords((3, 4, 9000), np.zeros(9000, dtype=np.int64),
                                                 np.full(9000, 2), np.arange(9000), rng.uniform(-1, 1, 9000)),
        "empty_slices": small_csf(rng, (500, 8, 8), 0.02),
    }


TENS = None


def get_tens():
    global TENS
    if TENS is None:
        TENS = tensors()
    return TENS


@pytest.mark.parametrize("name", ["zipf", "dense_small", "long_fiber", "empty_slices"])
@pytest.mark.parametrize("dtype", DTYPES)
def test_spttv(name, dtype):
    T = get_tens()[name]
    rng = np.random.default_rng(22)
    c = rng.standard_normal(T.dims[2])
    vr, cr = rounded(T.vals, dtype), rounded(c, dtype)
    ref = oracle.spttv(T.pos1, T.crd1, T.pos2, T.crd2, vr, cr, accurate=True)
    scale = oracle.spttv(T.pos1, T.crd1, T.pos2, T.crd2, np.abs(vr), np.abs(cr))
    dT = dev_csf(T, dtype)
    for split in SPLITS:
        for form in (1, 2):
            out = spd.spttv(dT, dev(c, dtype), split=split, tune={"form": form})
            torch.cuda.synchronize()
            check(out.double().cpu().numpy(), ref, scale, dtype, "spttv %s %s %s form %d" % (name, dtype, split, form),
                  row_lengths(T.pos2))


@pytest.mark.parametrize("name", ["zipf", "dense_small", "long_fiber", "empty_slices"])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("R", [1, 7, 32, 64])
def test_spmttkrp(name, dtype, R):
    T = get_tens()[name]
    rng = np.random.default_rng(23)
    C = rng.standard_normal((T.dims[1], R))
    D = rng.standard_normal((T.dims[2], R))
    vr, Cr, Dr = rounded(T.vals, dtype), rounded(C, dtype), rounded(D, dtype)
    ref = oracle.spmttkrp(T.pos1, T.crd1, T.pos2, T.crd2, vr, Cr, Dr, accurate=True)
    scale = oracle.spmttkrp(T.pos1, T.crd1, T.pos2, T.crd2, np.abs(vr), np.abs(Cr), np.abs(Dr))
    dT = dev_csf(T, dtype)
    for split, tune in [("row", None), ("nnz", None), ("nnz", {"unit_items": 64})]:
        A = spd.spmttkrp(dT, dev(C, dtype), dev(D, dtype), split=split, tune=tune)
        torch.cuda.synchronize()
        check(A.double().cpu().numpy(), ref, scale, dtype, "spmttkrp %s %s R=%d %s %s" % (name, dtype, R, split, tune),
              slice_lengths(T)[:, None], extra=1)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("R", [32, 40])
def test_spmttkrp_strided_factors(dtype, R):
    """C and D as column windows of wider row-major matrices (leading dimension R + 24,
    starting 8 elements in)."""
    T = get_tens()["zipf"]
    rng = np.random.default_rng(24)
    C = rng.standard_normal((T.dims[1], R))
    D = rng.standard_normal((T.dims[2], R))
    vr, Cr, Dr = rounded(T.vals, dtype), rounded(C, dtype), rounded(D, dtype)
    ref = oracle.spmttkrp(T.pos1, T.crd1, T.pos2, T.crd2, vr, Cr, Dr, accurate=True)
    scale = oracle.spmttkrp(T.pos1, T.crd1, T.pos2, T.crd2, np.abs(vr), np.abs(Cr), np.abs(Dr))
    wideC = torch.zeros((T.dims[1], R + 24), dtype=dtype, device="cuda")
    wideD = torch.zeros((T.dims[2], R + 24), dtype=dtype, device="cuda")
    wideC[:, 8:8 + R] = dev(C, dtype)
    wideD[:, 8:8 + R] = dev(D, dtype)
    dT = dev_csf(T, dtype)
    for split in SPLITS:
        A = spd.spmttkrp(dT, wideC[:, 8:8 + R], wideD[:, 8:8 + R], split=split)
        torch.cuda.synchronize()
        check(A.double().cpu().numpy(), ref, scale, dtype, "spmttkrp strided %s R=%d %s" % (dtype, R, split),
              slice_lengths(T)[:, None], extra=1)


# ------------------------------------------------------------------------------ autograd

def test_spmm_autograd_matches_oracle_gradients_and_finite_differences():
    rng = np.random.default_rng(31)
    A = spd_synth.rmat_csr(8, 4, seed=2)  # 256 rows
    L = 5
    X = rng.uniform(-1, 1, (A.ncols, L))
    W = rng.uniform(-1, 1, (A.nrows, L))  # loss = sum(W * (A X))
    dA = dev_csr(A, torch.float64)
    vals = dA.vals.clone().requires_grad_(True)
    Xt = dev(X, torch.float64).requires_grad_(True)
    Y = spd.autograd.spmm(dA.with_vals(vals), Xt)
    loss = (Y * dev(W, torch.float64)).sum()
    loss.backward()
    gv = vals.grad.cpu().numpy()
    gX = Xt.grad.cpu().numpy()
    # the oracle's gradient loops: dA = SDDMM(pattern, W, X), dX = SpMM^T(A, W)
    ref_gv = oracle.sddmm(A.pos, A.crd, None, W, X, accurate=True)
    ref_gX = oracle.spmm_t(A.pos, A.crd, A.vals, W, A.ncols, accurate=True)
    assert check(gv, ref_gv, oracle.sddmm(A.pos, A.crd, None, np.abs(W), np.abs(X)), torch.float64, "dvals",
                 None) <= 1e-12
    assert check(gX, ref_gX, oracle.spmm_t(A.pos, A.crd, np.abs(A.vals), np.abs(W), A.ncols), torch.float64, "dX",
                 None) <= 1e-12
    # central finite differences of the oracle's forward (the loss is linear in each
    # argument, so h = 1e-6 differences are exact up to rounding)
    h = 1e-6
    f = lambda v, XX: float(np.sum(W * oracle.spmm(A.pos, A.crd, v, XX)))
    for p in rng.integers(0, A.nnz, 25):
        e = np.zeros(A.nnz); e[p] = h
        fd = (f(A.vals + e, X) - f(A.vals - e, X)) / (2 * h)
        assert abs(fd - gv[p]) <= 1e-7 * max(1.0, abs(gv[p]))
    for _ in range(25):
        j, l = rng.integers(0, A.ncols), rng.integers(0, L)
        E = np.zeros_like(X); E[j, l] = h
        fd = (f(A.vals, X + E) - f(A.vals, X - E)) / (2 * h)
        assert abs(fd - gX[j, l]) <= 1e-7 * max(1.0, abs(gX[j, l]))


def test_spmm_autograd_gradcheck():
    A = spd_synth.rmat_csr(6, 3, seed=4)
    dA = dev_csr(A, torch.float64)
    vals = dA.vals.clone().requires_grad_(True)
    X = torch.randn(A.ncols, 3, dtype=torch.float64, device="cuda", requires_grad=True)
    fn = lambda v, XX: spd.autograd.spmm(dA.with_vals(v), XX)
    assert torch.autograd.gradcheck(fn, (vals, X), eps=1e-6, atol=1e-8)


# ------------------------------------------------------------------------------ errors

def test_errors_raise_without_launching():
    A = get_mats()["rmat12"]
    dA = dev_csr(A, torch.float32)
    with pytest.raises(ValueError):
        spd.spmv(dA, torch.zeros(A.ncols + 1, device="cuda"))
    with pytest.raises(TypeError):
        spd.spmv(dA, torch.zeros(A.ncols))  # host tensor: no CPU path
    from paper_2207_13901_gb300 import _abi
    with pytest.raises(_abi.SpdError) as e:
        spd.spmm(dA, torch.zeros(A.ncols, 8, device="cuda"), tune={"unit_items": 33})
    assert e.value.status == 10
