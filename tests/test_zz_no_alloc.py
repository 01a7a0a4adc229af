"""spd_spmv_noalloc: SpMV for callers that cannot allocate device memory.

Some callers (a plugin inside a framework that owns every device allocation, or a
latency-critical path that may not call an allocator) cannot hand spd_spmv the
workspace it needs. spd_spmv_noalloc runs the same nnz-split SpMV on a 1 MiB scratch
array compiled into the library. This test calls it through the C ABI twice in a row,
on two different matrices so that the second call starts from the first call's
leftover scratch, and compares each result with spd_spmv's on the same inputs.

The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import spd_synth
import paper_2207_13901_gb300 as spd
from paper_2207_13901_gb300 import _abi

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-4}  # the tolerances of the other GPU tests


def _call_noalloc(A, x, y):
    lib = _abi.load()
    d = A.desc()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = spd.ops._code
    return lib.spd_spmv_noalloc(ctypes.byref(d), ctypes.c_void_p(x.data_ptr()), code(x.dtype),
                                ctypes.c_void_p(y.data_ptr()), code(y.dtype), st)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_noalloc_matches_spmv_on_two_calls_in_a_row(dtype):
    rng = np.random.default_rng(1)
    mats = [spd_synth.rmat_csr(16, 16, seed=5), spd_synth.uniform_csr(3000, 5000, (0, 40), seed=6)]
    for M in mats:
        A = spd.CSR.from_host(M.pos, M.crd, M.vals, (M.nrows, M.ncols), dtype=dtype)
        x = torch.as_tensor(rng.uniform(-1, 1, M.ncols)).to(dtype).cuda()
        want = spd.spmv(A, x, split="nnz")
        # sum of |terms| per row, the normaliser the other GPU tests use
        scale = spd.spmv(A.with_vals(A.vals.abs()), x.abs(), split="nnz").double().cpu().numpy()
        y = torch.full((M.nrows,), float("nan"), dtype=want.dtype, device="cuda")
        assert _call_noalloc(A, x, y) == _abi.SPD_OK, _abi.load().spd_last_error()
        torch.cuda.synchronize()
        got, ref = y.double().cpu().numpy(), want.double().cpu().numpy()
        assert np.all(np.isfinite(got))
        den = np.maximum(np.abs(ref), scale)
        den[den == 0] = 1.0
        assert np.max(np.abs(got - ref) / den) <= TOL[dtype]


def test_noalloc_rejects_inputs_beyond_its_scratch():
    # a descriptor whose partition would need more than 1 MiB of scratch; rejected on the
    # host before anything is launched (the pointers are never dereferenced)
    lib = _abi.load()
    n = 60_000_000
    d = _abi.spd_csr(n, n, 60_000_000, 256, 512, 1024, _abi.SPD_F32, 0)
    assert lib.spd_spmv_noalloc(ctypes.byref(d), 4096, _abi.SPD_F32, 8192, _abi.SPD_F32, None) == _abi.SPD_ERR_SHAPE
    assert b"scratch" in lib.spd_last_error()
