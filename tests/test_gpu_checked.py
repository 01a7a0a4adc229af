"""Checked mode (spd_set_checked): broken structures are refused with SPD_ERR_STRUCTURE
before any work is launched, valid calls give bit-identical results to unchecked ones,
and a checked call inside a graph capture is refused.

Every planted fault is one that the kernels could not turn into an access outside an
allocation even if the check were missing: a coordinate one past the last column or a
few before the first, read from a dense operand that is a view into a padded buffer, or
a final pos entry one short of nnz (fewer entries processed)."""
import numpy as np
import pytest
import torch

import paper_2207_13901_gb300 as spd
from paper_2207_13901_gb300 import _abi
from tests._util import small_csf, small_csr

pytestmark = pytest.mark.gpu

PAD = 64  # elements (or rows) of padding on both sides of each dense operand


@pytest.fixture
def checked_on():
    spd.set_checked(True)
    try:
        yield
    finally:
        spd.set_checked(False)


def padded_vec(n, seed):
    buf = torch.empty(n + 2 * PAD, device="cuda").uniform_(-1, 1, generator=torch.Generator(device="cuda").manual_seed(seed))
    return buf[PAD:PAD + n]


def padded_mat(n, L, seed):
    buf = torch.empty((n + 2 * PAD, L), device="cuda").uniform_(-1, 1,
                                                                 generator=torch.Generator(device="cuda").manual_seed(seed))
    return buf[PAD:PAD + n]


def faults(A):
    """(name, pos, crd) of broken copies of A's structure and the first bad index."""
    out = []
    c = A.crd.copy(); c[17] = A.ncols
    out.append(("crd past the end", A.pos, c, A.nrows + 1 + 17))
    c = A.crd.copy(); c[5] = -3
    out.append(("negative crd", A.pos, c, A.nrows + 1 + 5))
    p = A.pos.copy(); p[-1] -= 1
    out.append(("short pos", p, A.crd, A.nrows))
    return out


def expect_structure_error(fn, first_bad, name="A"):
    with pytest.raises(_abi.SpdError) as e:
        fn()
    assert e.value.status == 5  # SPD_ERR_STRUCTURE
    msg = str(e.value)
    assert "checked mode: %s " % name in msg and "first at index %d" % first_bad in msg, msg


def test_checked_flag_round_trip():
    assert not spd.checked()
    spd.set_checked(True)
    try:
        assert spd.checked()
    finally:
        spd.set_checked(False)
    assert not spd.checked()


def test_spmv_spmm_sddmm_refuse_broken_structure(checked_on):
    rng = np.random.default_rng(7)
    A = small_csr(rng, 3000, 200, 0.02)
    x = padded_vec(A.ncols, 1)
    X = padded_mat(A.ncols, 32, 2)
    C = padded_mat(A.nrows, 32, 3)
    for what, pos, crd, first in faults(A):
        dA = spd.CSR.from_host(pos, crd, A.vals, (A.nrows, A.ncols))
        y = torch.full((A.nrows,), 7.0, device="cuda")
        Y = torch.full((A.nrows, 32), 7.0, device="cuda")
        out = torch.full((A.nnz,), 7.0, device="cuda")
        for split in ("row", "nnz"):
            expect_structure_error(lambda: spd.spmv(dA, x, y, split=split), first)
            expect_structure_error(lambda: spd.spmm(dA, X, Y, split=split), first)
            expect_structure_error(lambda: spd.spmm_accumulate(dA, X, Y, split=split), first)
            expect_structure_error(lambda: spd.sddmm(dA, C, X, out, split=split), first, name="B")
            expect_structure_error(lambda: spd.partition(dA, split, 4 if split == "row" else
                                                         (A.nrows + A.nnz + 1023) // 1024, 1024), first)
        torch.cuda.synchronize()
        # nothing was launched: the outputs keep their fill
        assert bool((y == 7).all()) and bool((Y == 7).all()) and bool((out == 7).all()), what


def test_spmm_t_transpose_spadd3_batched_refuse_broken_structure(checked_on):
    rng = np.random.default_rng(8)
    A = small_csr(rng, 2000, 300, 0.02)
    p = A.pos.copy(); p[-1] -= 1
    bad = spd.CSR.from_host(p, A.crd, A.vals, (A.nrows, A.ncols))
    good = spd.CSR.from_host(A.pos, A.crd, A.vals, (A.nrows, A.ncols))
    dY = padded_mat(A.nrows, 16, 4)
    expect_structure_error(lambda: spd.spmm_t(bad, dY), A.nrows)
    expect_structure_error(lambda: spd.transpose(bad), A.nrows)
    expect_structure_error(lambda: spd.spadd3(good, bad, good), A.nrows, name="C")
    expect_structure_error(lambda: spd.spadd3(good, good, bad), A.nrows, name="D")
    X = padded_mat(A.ncols, 16, 5)
    expect_structure_error(lambda: spd.SpMMBatch([good, bad], [X, X]), A.nrows, name="a batch matrix")


def test_csf_calls_refuse_broken_structure(checked_on):
    rng = np.random.default_rng(9)
    T = small_csf(rng, (40, 30, 50), 0.05)
    crd2 = T.crd2.copy(); crd2[7] = T.dims[2]
    dT = spd.CSF3.from_host(T.pos1, T.crd1, T.pos2, crd2, T.vals, T.dims)
    first = (T.dims[0] + 1 + T.nfib) + (T.nfib + 1) + 7
    c = padded_vec(T.dims[2], 6)
    Cf = padded_mat(T.dims[1], 8, 7)
    Df = padded_mat(T.dims[2], 8, 8)
    expect_structure_error(lambda: spd.spttv(dT, c), first, name="B")
    expect_structure_error(lambda: spd.spmttkrp(dT, Cf, Df), first, name="B")


def test_checked_results_match_unchecked():
    rng = np.random.default_rng(10)
    A = small_csr(rng, 5000, 700, 0.02, long_rows=2)
    dA = spd.CSR.from_host(A.pos, A.crd, A.vals, (A.nrows, A.ncols))
    x = padded_vec(A.ncols, 11)
    X = padded_mat(A.ncols, 64, 12)
    C = padded_mat(A.nrows, 64, 13)
    T = small_csf(rng, (60, 50, 70), 0.05)
    dT = spd.CSF3.from_host(T.pos1, T.crd1, T.pos2, T.crd2, T.vals, T.dims)
    c = padded_vec(T.dims[2], 14)
    Cf, Df = padded_mat(T.dims[1], 16, 15), padded_mat(T.dims[2], 16, 16)

    def run_all():
        S = spd.spadd3(dA, dA, dA)
        Tr = spd.transpose(dA)
        return [spd.spmv(dA, x), spd.spmm(dA, X), spd.sddmm(dA, C, X), spd.spmm_t(dA, C, method="transpose"),
                spd.spttv(dT, c), spd.spmttkrp(dT, Cf, Df), S.pos, S.crd, S.vals, Tr.t_pos, Tr.t_crd, Tr.perm,
                spd.SpMMBatch([dA, dA], [X, X]).run()[1]]

    plain = run_all()
    spd.set_checked(True)
    try:
        checked = run_all()
    finally:
        spd.set_checked(False)
    torch.cuda.synchronize()
    for a, b in zip(plain, checked):
        assert torch.equal(a, b)


def test_checked_call_refused_inside_graph_capture(checked_on):
    rng = np.random.default_rng(12)
    A = small_csr(rng, 1000, 100, 0.05)
    dA = spd.CSR.from_host(A.pos, A.crd, A.vals, (A.nrows, A.ncols))
    x = padded_vec(A.ncols, 17)
    y = torch.empty(A.nrows, device="cuda")
    need = spd.csr_workspace_size(_abi.SPD_OP_SPMV, dA, "nnz", 0)
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with pytest.raises(_abi.SpdError) as e:
        with torch.cuda.graph(g):
            spd.spmv(dA, x, y, ws=ws)
    assert e.value.status == 10 and "graph capture" in str(e.value)
    spd.set_checked(False)
    g2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g2):
        spd.spmv(dA, x, y, ws=ws)
    g2.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, spd.spmv(dA, x))
