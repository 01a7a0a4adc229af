"""Parity at the largest sizes the level format admits: SPD_MAX_INDEX (2^31 - 2^17 - 1)
entries, rows or fibers. Every kernel forms int32 offsets up to a window, tile or work
unit past its current position; these inputs put positions, rows and fibers at the
limit, with ragged rows (empty rows, a row of 2^27 entries) and ragged fibers.

Values and dense operands are small integers, so every product and partial sum is an
integer far below 2^24 and any summation order is exact: complete outputs are compared
bit for bit with integer sums computed on the host in int64, and sampled rows, positions
and slices with the oracle, run on the sub-structure that holds them (rows and slices
are independent, so the oracle's result for them is the same as on the whole input)."""
import functools

import numpy as np
import pytest
import torch

import oracle
import spd_synth
import paper_2207_13901_gb300 as spd
from paper_2207_13901_gb300 import _abi

pytestmark = pytest.mark.gpu

M = _abi.SPD_MAX_INDEX


def need_memory(host_gb, device_gb):
    avail = 0
    with open("/proc/meminfo") as f:
        for line in f:
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) * 1024
    if avail < host_gb * 2**30:
        pytest.skip("needs %d GiB of free host memory" % host_gb)
    if torch.cuda.mem_get_info()[0] < device_gb * 2**30:
        pytest.skip("needs %d GiB of free device memory" % device_gb)


def small_ints(shape, seed):
    return np.random.default_rng(seed).integers(-3, 4, size=shape).astype(np.int64)


def segment_sums(pos, crd, vals, x, r0, r1):
    """sum_p vals[p] * x[crd[p]] for each row r0 <= r < r1 (int64, exact)."""
    p0, p1 = int(pos[r0]), int(pos[r1])
    cs = np.zeros(p1 - p0 + 1, dtype=np.int64)
    np.cumsum(vals[p0:p1].astype(np.int64) * x[crd[p0:p1]], out=cs[1:])
    return cs[pos[r0 + 1:r1 + 1].astype(np.int64) - p0] - cs[pos[r0:r1].astype(np.int64) - p0]


def row_chunks(pos, entries=1 << 26):
    """Consecutive row ranges of about `entries` entries each (a longer row alone)."""
    n = pos.shape[0] - 1
    r0 = 0
    while r0 < n:
        r1 = int(np.searchsorted(pos, int(pos[r0]) + entries, side="right")) - 1
        r1 = min(max(r1, r0 + 1), n)
        yield r0, r1
        r0 = r1


def sub_rows(pos, crd, vals, rows):
    """The CSR of the given rows alone (pos rebased), values as float64."""
    starts, ends = pos[rows].astype(np.int64), pos[rows + 1].astype(np.int64)
    sp = np.zeros(rows.shape[0] + 1, dtype=np.int64)
    np.cumsum(ends - starts, out=sp[1:])
    idx = np.concatenate([np.arange(a, b) for a, b in zip(starts, ends)]) if rows.shape[0] else np.zeros(0, np.int64)
    return sp.astype(np.int32), crd[idx], vals[idx].astype(np.float64), idx


@functools.lru_cache(maxsize=1)
def limit_entries_matrix():
    """SPD_MAX_INDEX entries over 2^21 ragged rows (one of 2^27 entries), generated once."""
    return spd_synth.limit_csr(1 << 21, 1 << 16, M, seed=11, long_row=1 << 27)


def device_csr(A, dtype):
    vals = torch.from_numpy(A.vals).cuda().to(dtype)
    return spd.CSR(torch.from_numpy(A.pos).cuda(), torch.from_numpy(A.crd).cuda(), vals, (A.nrows, A.ncols))


def test_limit_entries_csr():
    """SPD_MAX_INDEX entries over 2^21 rows: SpMV (both forms, both splits, binary32 and
    bfloat16) on every row, SpMM (L = 8) on sampled rows and on its column sums, SDDMM
    (K = 32) on the positions of sampled rows, the last rows and both ends of the long row."""
    need_memory(48, 48)
    n, m = 1 << 21, 1 << 16
    A = limit_entries_matrix()
    assert A.nnz == M and int(A.pos[-1]) == M
    x = small_ints(m, 12)
    y_dev = {}
    for dtype in (torch.float32, torch.bfloat16):
        dA = device_csr(A, dtype)
        dx = torch.from_numpy(x).cuda().to(dtype)
        for split, form in (("nnz", 1), ("nnz", 2), ("row", 1), ("row", 2)):
            y_dev[(dtype, split, form)] = spd.spmv(dA, dx, split=split, tune={"form": form})
        del dA
    torch.cuda.synchronize()
    for r0, r1 in row_chunks(A.pos):
        want = segment_sums(A.pos, A.crd, A.vals, x, r0, r1).astype(np.float64)
        for key, y in y_dev.items():
            got = y[r0:r1].double().cpu().numpy()
            assert np.array_equal(got, want), ("spmv", key, r0, r1)
    del y_dev

    rng = np.random.default_rng(13)
    long_r = n // 3
    rows = np.unique(np.concatenate([np.arange(5), rng.integers(0, n, 300), np.arange(n - 200, n), [long_r]]))
    dA = device_csr(A, torch.float32)
    L = 8
    X = small_ints((m, L), 14)
    sp, sc, sv, _ = sub_rows(A.pos, A.crd, A.vals, rows)
    want_rows = oracle.spmm(sp, sc, sv, X.astype(np.float64))
    colw = np.zeros(m, dtype=np.float64)  # sum of the values in each column (exact integers)
    for p0 in range(0, M, 1 << 27):
        p1 = min(p0 + (1 << 27), M)
        colw += np.bincount(A.crd[p0:p1], weights=A.vals[p0:p1].astype(np.float64), minlength=m)
    want_colsum = colw @ X.astype(np.float64)
    for split in ("nnz", "row"):
        Y = spd.spmm(dA, torch.from_numpy(X).cuda().float(), split=split).double().cpu().numpy()
        assert np.array_equal(Y[rows], want_rows), ("spmm rows", split)
        assert np.array_equal(Y.sum(axis=0), want_colsum), ("spmm column sums", split)
        del Y

    K = 32
    C = small_ints((n, K), 15)
    Dnk = small_ints((m, K), 16)
    out = spd.sddmm(dA, torch.from_numpy(C).cuda().float(), torch.from_numpy(Dnk).cuda().float(), split="nnz")
    short = rows[rows != long_r]
    sp, sc, sv, idx = sub_rows(A.pos, A.crd, A.vals, short)
    want = oracle.sddmm(sp, sc, sv, C[short].astype(np.float64), Dnk.astype(np.float64))
    got = out[torch.from_numpy(idx).cuda()].double().cpu().numpy()
    assert np.array_equal(got, want), "sddmm sampled rows"
    a, b = int(A.pos[long_r]), int(A.pos[long_r + 1])
    for lo, hi in ((a, a + (1 << 20)), (b - (1 << 20), b)):
        want = oracle.sddmm(np.array([0, hi - lo], dtype=np.int32), A.crd[lo:hi], A.vals[lo:hi].astype(np.float64),
                            C[long_r:long_r + 1].astype(np.float64), Dnk.astype(np.float64))
        assert np.array_equal(out[lo:hi].double().cpu().numpy(), want), ("sddmm long row", lo)


def test_limit_entries_transpose():
    """The transposed structure of the SPD_MAX_INDEX-entry matrix (a stable radix sort of
    2^31 - 2^17 - 1 positions by column) and the SpMM gradient dX = A^T dY (L = 8) by
    atomic scatter and over that structure. Checked as properties, with torch on the
    device: column counts against the host's, every entry of A^T in the right column with
    the right row, positions ascending inside each column; the two dX schedules agree bit
    for bit (integer data) and their column sums equal the row sums of A weighted by dY."""
    need_memory(48, 160)
    A = limit_entries_matrix()
    n, m = A.nrows, A.ncols
    dA = device_csr(A, torch.float32)
    T = spd.transpose(dA)
    counts = np.zeros(m, dtype=np.int64)
    for p0 in range(0, M, 1 << 27):
        counts += np.bincount(A.crd[p0:min(p0 + (1 << 27), M)], minlength=m)
    want_tpos = np.concatenate([[0], np.cumsum(counts)])
    assert np.array_equal(T.t_pos.cpu().numpy().astype(np.int64), want_tpos)
    perm = T.perm.long()
    col = torch.repeat_interleave(torch.arange(m, device="cuda", dtype=torch.int32), torch.from_numpy(counts).cuda())
    assert torch.equal(dA.crd[perm], col)  # every entry of A^T sits in its column
    # stable: A's order inside a column
    assert bool(torch.all((T.perm[1:] > T.perm[:-1]) | (col[1:] != col[:-1])))
    del col
    rows = torch.repeat_interleave(torch.arange(n, device="cuda", dtype=torch.int32),
                                   torch.from_numpy(np.diff(A.pos).astype(np.int64)).cuda())
    assert torch.equal(T.t_crd, rows[perm])  # and carries its row
    del rows, perm
    torch.cuda.empty_cache()
    L = 8
    dY = small_ints((n, L), 17)
    ddY = torch.from_numpy(dY).cuda().float()
    dX_atomic = spd.spmm_t(dA, ddY, split="nnz")
    dX_t = spd.spmm(T.matrix(dA.vals), ddY, split="nnz")  # an SpMM over A^T (65536 rows of about 2^15)
    assert torch.equal(dX_atomic, dX_t)
    rowsum = np.zeros(n, dtype=np.int64)  # sum of the values of each row
    for r0, r1 in row_chunks(A.pos):
        rowsum[r0:r1] = segment_sums(A.pos, A.crd, A.vals, np.ones(m, dtype=np.int64), r0, r1)
    want = rowsum.astype(np.float64) @ dY.astype(np.float64)
    assert np.array_equal(dX_atomic.double().cpu().numpy().sum(axis=0), want)


def union_sizes(ops):
    """Entries of each row of B + C + D for operands whose rows are column runs."""
    lo = np.stack([A.crd[np.minimum(A.pos[:-1], A.nnz - 1)].astype(np.int64) for A in ops], axis=1)
    ln = np.stack([np.diff(A.pos).astype(np.int64) for A in ops], axis=1)
    lo = np.where(ln > 0, lo, 0)
    hi = lo + ln
    order = np.argsort(lo, axis=1, kind="stable")
    lo, hi = np.take_along_axis(lo, order, 1), np.take_along_axis(hi, order, 1)
    size, reach = np.zeros(lo.shape[0], dtype=np.int64), np.full(lo.shape[0], -1, dtype=np.int64)
    for k in range(3):
        start = np.maximum(lo[:, k], reach)
        size += np.where(hi[:, k] > start, hi[:, k] - start, 0)
        reach = np.maximum(reach, hi[:, k])
    return size


def test_limit_spadd3():
    """SpAdd3 with SPD_MAX_INDEX entries in its three operands together, one of them
    holding all but 2^21 (rows of column runs at random offsets, so the three runs of a
    row overlap in part): A's pos against the union sizes computed on the host, sampled
    rows (crd and values) against the oracle, and the sum of A's values against the sum
    of the operands', for both splits."""
    need_memory(48, 96)
    n, m = 1 << 21, 1 << 17
    ops = [spd_synth.limit_interval_csr(n, m, M - (1 << 21), seed=41),
           spd_synth.limit_interval_csr(n, m, 1 << 20, seed=42),
           spd_synth.limit_interval_csr(n, m, 1 << 20, seed=43)]
    want_pos = np.concatenate([[0], np.cumsum(union_sizes(ops))])
    want_sum = sum(int(A.vals.astype(np.int64).sum()) for A in ops)
    rng = np.random.default_rng(44)
    rows = np.unique(np.concatenate([np.arange(3), rng.integers(0, n, 300), np.arange(n - 100, n)]))
    subs = []
    for A in ops:
        sp, sc, sv, _ = sub_rows(A.pos, A.crd, A.vals, rows)
        subs.append(spd_synth.CSR(rows.shape[0], m, sp, sc, sv))
    wp, wc, wv = oracle.spadd3(*subs)
    dops = [device_csr(A, torch.float32) for A in ops]
    for split in ("nnz", "row"):
        S = spd.spadd3(*dops, split=split)
        got_pos = S.pos.cpu().numpy().astype(np.int64)
        assert np.array_equal(got_pos, want_pos), split
        assert float(S.vals.double().sum().item()) == want_sum, split
        got_idx = np.concatenate([np.arange(got_pos[r], got_pos[r + 1]) for r in rows])
        assert np.array_equal(S.crd[torch.from_numpy(got_idx).cuda()].cpu().numpy(), wc), split
        assert np.array_equal(S.vals[torch.from_numpy(got_idx).cuda()].double().cpu().numpy(), wv), split
        del S
        torch.cuda.empty_cache()


def test_limit_rows_csr():
    """SPD_MAX_INDEX rows, 2^22 entries in random rows (the first and last among them):
    SpMV (both forms, both splits) and SpMM (L = 1) on every row that holds entries,
    and zero on all the others."""
    need_memory(48, 64)
    m = 1 << 16
    A = spd_synth.limit_rows_csr(M, m, 1 << 22, seed=21)
    assert A.nrows == M and A.pos.shape[0] == M + 1
    occ = np.flatnonzero(np.diff(A.pos))
    assert occ[0] == 0 and occ[-1] == M - 1
    x = small_ints(m, 22)
    p0 = A.pos[occ].astype(np.int64)
    cs = np.zeros(A.nnz + 1, dtype=np.int64)
    np.cumsum(A.vals.astype(np.int64) * x[A.crd], out=cs[1:])
    want = (cs[A.pos[occ + 1].astype(np.int64)] - cs[p0]).astype(np.float64)
    nonzero = int(np.count_nonzero(want))
    dA = device_csr(A, torch.float32)
    dx = torch.from_numpy(x).cuda().float()
    docc = torch.from_numpy(occ).cuda()
    outs = {}
    for split, form in (("nnz", 1), ("nnz", 2), ("row", 1), ("row", 2)):
        outs[("spmv", split, form)] = spd.spmv(dA, dx, split=split, tune={"form": form})
    outs[("spmm", "nnz", 0)] = spd.spmm(dA, dx[:, None].contiguous(), split="nnz").view(-1)
    for key, y in outs.items():
        assert y.numel() == M
        assert np.array_equal(y[docc].double().cpu().numpy(), want), key
        assert int(torch.count_nonzero(y).item()) == nonzero, key


def test_limit_entries_csf():
    """SPD_MAX_INDEX entries in about 2^30 fibers of 1 to 3 entries over 2^20 slices:
    SpTTV (both forms, both splits) on every fiber, SpMTTKRP (R = 8, both splits) on
    sampled slices, the first and the last ones."""
    need_memory(64, 64)
    dims = (1 << 20, 1 << 16, 1 << 16)
    T = spd_synth.limit_csf3(dims, M, seed=31)
    assert T.nnz == M and int(T.pos2[-1]) == M
    vals = torch.from_numpy(T.vals).cuda().float()
    dT = spd.CSF3(torch.from_numpy(T.pos1).cuda(), torch.from_numpy(T.crd1).cuda(), torch.from_numpy(T.pos2).cuda(),
                  torch.from_numpy(T.crd2).cuda(), vals, dims)
    c = small_ints(dims[2], 32)
    dc = torch.from_numpy(c).cuda().float()
    outs = {}
    for split, form in (("nnz", 1), ("nnz", 2), ("row", 1), ("row", 2)):
        outs[(split, form)] = spd.spttv(dT, dc, split=split, tune={"form": form})
    torch.cuda.synchronize()
    for f0, f1 in row_chunks(T.pos2):
        want = segment_sums(T.pos2, T.crd2, T.vals, c, f0, f1).astype(np.float64)
        for key, o in outs.items():
            assert np.array_equal(o[f0:f1].double().cpu().numpy(), want), ("spttv", key, f0, f1)
    del outs

    R = 8
    Cm, Dm = small_ints((dims[1], R), 33), small_ints((dims[2], R), 34)
    rng = np.random.default_rng(35)
    I = dims[0]
    sl = np.unique(np.concatenate([np.arange(3), rng.integers(0, I, 200), np.arange(I - 100, I)]))
    # the sampled slices as a tensor of their own: fibers and entries rebased
    fpos, fcrd, _, fidx = sub_rows(T.pos1, T.crd1, np.zeros(T.nfib, dtype=np.int8), sl)
    e_lo, e_hi = T.pos2[fidx].astype(np.int64), T.pos2[fidx + 1].astype(np.int64)
    p2 = np.zeros(fidx.shape[0] + 1, dtype=np.int64)
    np.cumsum(e_hi - e_lo, out=p2[1:])
    eidx = np.concatenate([np.arange(a, b) for a, b in zip(e_lo, e_hi)])
    want = oracle.spmttkrp(fpos, fcrd, p2.astype(np.int32), T.crd2[eidx], T.vals[eidx].astype(np.float64),
                           Cm.astype(np.float64), Dm.astype(np.float64))
    dC, dD = torch.from_numpy(Cm).cuda().float(), torch.from_numpy(Dm).cuda().float()
    for split in ("nnz", "row"):
        A = spd.spmttkrp(dT, dC, dD, split=split).double().cpu().numpy()
        assert np.array_equal(A[sl], want), ("spmttkrp", split)
