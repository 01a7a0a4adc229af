"""spd_spmv_noalloc: SpMV for callers that cannot allocate device memory.

Some callers cannot hand spd_spmv the workspace it needs: a plugin inside a framework
that owns every device allocation, or a latency-critical path that may not call an
allocator. spd_spmv_noalloc runs the same nnz-split SpMV on a 1 MiB scratch array
compiled into the library. This test calls it through the C ABI twice in a row, on two
different matrices so that the second call starts from the first call's leftover
scratch, and checks each result against the compensated CPU oracle (the error gate of
the other GPU tests) and bit for bit against spd_spmv with the nnz split on the same
inputs (the same kernels and partition).

The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import spd_synth
import paper_2207_13901_gb300 as spd
from paper_2207_13901_gb300 import _abi
from tests._util import check_error, row_lengths

pytestmark = pytest.mark.gpu


def _call_noalloc(A, x, y):
    lib = _abi.load()
    d = A.desc()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = spd.ops._code
    return lib.spd_spmv_noalloc(ctypes.byref(d), ctypes.c_void_p(x.data_ptr()), code(x.dtype),
                                ctypes.c_void_p(y.data_ptr()), code(y.dtype), st)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
def test_noalloc_matches_oracle_and_spmv_on_two_calls_in_a_row(dtype):
    rng = np.random.default_rng(1)
    mats = [spd_synth.rmat_csr(16, 16, seed=5), spd_synth.uniform_csr(3000, 5000, (0, 40), seed=6)]
    for M in mats:
        A = spd.CSR.from_host(M.pos, M.crd, M.vals, (M.nrows, M.ncols), dtype=dtype)
        xh = rng.uniform(-1, 1, M.ncols)
        x = torch.as_tensor(xh).to(dtype).cuda()
        vr = torch.as_tensor(M.vals).to(dtype).double().numpy()
        xr = x.double().cpu().numpy()
        ref = oracle.spmv(M.pos, M.crd, vr, xr, accurate=True)
        scale = oracle.spmv(M.pos, M.crd, np.abs(vr), np.abs(xr))
        y = torch.full((M.nrows,), float("nan"), dtype=spd.result_dtype(dtype), device="cuda")
        assert _call_noalloc(A, x, y) == _abi.SPD_OK, _abi.load().spd_last_error()
        torch.cuda.synchronize()
        got = y.double().cpu().numpy()
        assert np.all(np.isfinite(got))
        check_error(got, ref, scale, dtype == torch.float64, row_lengths(M.pos), "spmv_noalloc %s" % dtype)
        want = spd.spmv(A, x, split="nnz")
        torch.cuda.synchronize()
        assert torch.equal(y, want)


def test_noalloc_runs_the_largest_size_it_accepts():
    """nrows + nnz at the exact limit of the scratch array: accepted and correct; one
    more item is rejected before any launch."""
    from tests.test_abi import noalloc_item_limit
    lib = _abi.load()
    items = noalloc_item_limit(lib)
    nnz = 5000
    n = items - nnz
    lens = torch.zeros(n, dtype=torch.int32, device="cuda")
    lens[7] = 3000
    lens[n - 2] = 2000
    pos = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    pos[1:] = torch.cumsum(lens, 0, dtype=torch.int32)
    del lens
    crd = torch.arange(nnz, dtype=torch.int32, device="cuda") % 4096
    vals = torch.linspace(-1, 1, nnz, dtype=torch.float32, device="cuda")
    A = spd.CSR(pos, crd, vals, (n, 4096))
    x = torch.linspace(-2, 2, 4096, dtype=torch.float32, device="cuda")
    y = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
    assert _call_noalloc(A, x, y) == _abi.SPD_OK, lib.spd_last_error()
    torch.cuda.synchronize()
    v64, x64 = vals.double().cpu().numpy(), x.double().cpu().numpy()
    c64 = crd.cpu().numpy()
    sub_pos = np.array([0, 3000, 5000])  # rows 7 and n - 2 alone
    ref = oracle.spmv(sub_pos, c64, v64, x64, accurate=True)
    scale = oracle.spmv(sub_pos, c64, np.abs(v64), np.abs(x64))
    got = np.array([y[7].item(), y[n - 2].item()])
    check_error(got, ref, scale, False, row_lengths(sub_pos), "spmv_noalloc at the size limit")
    nz = torch.count_nonzero(y).item()
    assert nz == 2 and not torch.isnan(y).any().item()
    big = _abi.spd_csr(n + 1, 4096, nnz, pos.data_ptr(), crd.data_ptr(), vals.data_ptr(), _abi.SPD_F32, 0)
    assert lib.spd_spmv_noalloc(ctypes.byref(big), x.data_ptr(), _abi.SPD_F32, y.data_ptr(), _abi.SPD_F32,
                                None) == _abi.SPD_ERR_SHAPE


def test_noalloc_rejects_inputs_beyond_its_scratch():
    # a descriptor whose partition would need more than 1 MiB of scratch; rejected on the
    # host before anything is launched (the pointers are never dereferenced)
    lib = _abi.load()
    n = 60_000_000
    d = _abi.spd_csr(n, n, 60_000_000, 256, 512, 1024, _abi.SPD_F32, 0)
    assert lib.spd_spmv_noalloc(ctypes.byref(d), 4096, _abi.SPD_F32, 8192, _abi.SPD_F32, None) == _abi.SPD_ERR_SHAPE
    assert b"scratch" in lib.spd_last_error()
