"""C-ABI checks that need no GPU: the library builds, loads, exports every function
that include/spd.h declares, and rejects bad arguments on the host before any launch."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

from paper_2207_13901_gb300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(spd_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_function():
    lib = _abi.load()
    names = header_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    # the Python binding declares exactly the functions of the headers
    assert sorted(_abi.SIGNATURES) == names


def test_status_strings_and_version():
    lib = _abi.load()
    assert lib.spd_abi_version() == 2
    for s in range(11):
        assert lib.spd_status_str(s)
    assert lib.spd_status_str(99) == b"unknown status"


def test_checked_mode_switch():
    lib = _abi.load()
    assert lib.spd_set_checked(2) == 10
    assert lib.spd_set_checked(1) == 0 and lib.spd_checked() == 1
    try:
        # argument errors are still returned on the host first, before any validation
        bad = _csr(nrows=-1)
        assert lib.spd_spmv(ctypes.byref(bad), None, 1, None, 1, 1, None, None, 0, None) == 2
    finally:
        assert lib.spd_set_checked(0) == 0
    assert lib.spd_checked() == 0


def test_checked_mode_from_environment():
    code = "from paper_2207_13901_gb300 import _abi; print(_abi.load().spd_checked())"
    for value, want in (("1", "1"), ("yes", "1"), ("0", "0"), ("", "0")):
        env = dict(os.environ, SPD_DEBUG=value)
        out = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True,
                             timeout=300)
        assert out.returncode == 0, out.stderr
        assert out.stdout.strip() == want


def _csr(nrows=4, ncols=5, nnz=6, vtype=_abi.SPD_F32):
    # fake, never dereferenced: every check below fails on the host first
    return _abi.spd_csr(nrows, ncols, nnz, 256, 512, 1024, vtype, 0)


def test_index_limit():
    """Every size of a descriptor may reach SPD_MAX_INDEX and no further (the size
    queries check the descriptor on the host; the pointers are never dereferenced)."""
    with open(os.path.join(ROOT, "include", "spd.h")) as f:
        assert "#define SPD_MAX_INDEX %dLL" % _abi.SPD_MAX_INDEX in f.read()
    lib = _abi.load()
    size = ctypes.c_size_t(0)
    M = _abi.SPD_MAX_INDEX
    for nrows, ncols, nnz in ((M, 5, 6), (4, M, 6), (M, M, M)):
        A = _csr(nrows, ncols, nnz)
        for op in (_abi.SPD_OP_SPMV, _abi.SPD_OP_SPMM, _abi.SPD_OP_SDDMM):
            assert lib.spd_csr_workspace_size(op, ctypes.byref(A), _abi.SPD_SPLIT_NNZ, 8, None, ctypes.byref(size)) == 0
    for nrows, ncols, nnz in ((M + 1, 5, 6), (4, M + 1, 6), (4, 5, M + 1), (2**31 - 1, 5, 6)):
        A = _csr(nrows, ncols, nnz)
        assert lib.spd_csr_workspace_size(_abi.SPD_OP_SPMV, ctypes.byref(A), _abi.SPD_SPLIT_NNZ, 0, None,
                                          ctypes.byref(size)) == _abi.SPD_ERR_SHAPE
        assert b"SPD_MAX_INDEX" in lib.spd_last_error()
    full = (M, M, M, M, M)
    B = _abi.spd_csf3(*full, 256, 512, 768, 1024, 2048, _abi.SPD_F32, 0)
    assert lib.spd_csf3_workspace_size(_abi.SPD_OP_SPMTTKRP, ctypes.byref(B), _abi.SPD_SPLIT_NNZ, 8, None,
                                       ctypes.byref(size)) == 0
    for k in range(5):
        dims = list(full)
        dims[k] = M + 1
        B = _abi.spd_csf3(*dims, 256, 512, 768, 1024, 2048, _abi.SPD_F32, 0)
        assert lib.spd_csf3_workspace_size(_abi.SPD_OP_SPTTV, ctypes.byref(B), _abi.SPD_SPLIT_NNZ, 0, None,
                                           ctypes.byref(size)) == _abi.SPD_ERR_SHAPE


def test_host_side_argument_errors():
    lib = _abi.load()
    size = ctypes.c_size_t(0)
    A = _csr()
    # NULL descriptor / output pointer
    assert lib.spd_spmv(None, None, 0, None, 0, 0, None, None, 0, None) == 1
    assert lib.spd_csr_workspace_size(0, ctypes.byref(A), 1, 0, None, None) == 1
    # negative sizes, inconsistent sizes
    bad = _csr(nrows=-1)
    assert lib.spd_csr_workspace_size(0, ctypes.byref(bad), 1, 0, None, ctypes.byref(size)) == 2
    bad = _csr(nrows=0, nnz=3)
    assert lib.spd_csr_workspace_size(0, ctypes.byref(bad), 1, 0, None, ctypes.byref(size)) == 2
    # element type combinations
    assert lib.spd_spmv(ctypes.byref(A), 4096, _abi.SPD_F64, 8192, _abi.SPD_F32, 1, None, None, 0, None) == 3
    assert lib.spd_spmv(ctypes.byref(A), 4096, _abi.SPD_F32, 8192, _abi.SPD_F64, 1, None, None, 0, None) == 3
    assert b"type" in lib.spd_last_error()
    # misaligned values
    mis = _abi.spd_csr(4, 5, 6, 256, 512, 1026, _abi.SPD_F32, 0)
    assert lib.spd_spmv(ctypes.byref(mis), 4096, 1, 8192, 1, 1, None, None, 0, None) == 4
    # unknown split, bad tuning
    assert lib.spd_spmv(ctypes.byref(A), 4096, 1, 8192, 1, 7, None, None, 0, None) == 10
    t = _abi.spd_tune(33, 0, 0, 0)
    assert lib.spd_spmm(ctypes.byref(A), 4096, 8, 8, 1, 8192, 8, 1, 1, ctypes.byref(t), None, 0, None) == 10
    for bt in (544, 1024, 48, 100):  # the warp kernels take 64..512 threads a block, whole warps
        t = _abi.spd_tune(0, 0, bt, 0)
        assert lib.spd_spmm(ctypes.byref(A), 4096, 8, 8, 1, 8192, 8, 1, 1, ctypes.byref(t), None, 0, None) == 10
    # missing or short workspace for the nnz split
    assert lib.spd_spmv(ctypes.byref(A), 4096, 1, 8192, 1, 1, None, None, 0, None) == 6
    assert lib.spd_spmm(ctypes.byref(A), 4096, 8, 4, 1, 8192, 8, 1, 1, None, None, 0, None) == 2  # ldx < L


def test_workspace_sizes():
    lib = _abi.load()
    size = ctypes.c_size_t(0)
    A = _csr(nrows=1000, ncols=1000, nnz=20000)
    assert lib.spd_csr_workspace_size(_abi.SPD_OP_SPMV, ctypes.byref(A), _abi.SPD_SPLIT_ROW, 0, None, ctypes.byref(size)) == 0
    assert size.value == 0  # the row split needs no scratch
    assert lib.spd_csr_workspace_size(_abi.SPD_OP_SPMV, ctypes.byref(A), _abi.SPD_SPLIT_NNZ, 0, None, ctypes.byref(size)) == 0
    pieces = -(-21000 // 2048)
    assert size.value >= 2 * 4 * (pieces + 1) + pieces * (4 + 8)
    assert lib.spd_csr_workspace_size(_abi.SPD_OP_SPMM, ctypes.byref(A), _abi.SPD_SPLIT_NNZ, 128, None, ctypes.byref(size)) == 0
    assert size.value >= pieces * 128 * 8  # binary64 carries, one row per piece
    t = _abi.spd_tune(512, 0, 0, 0)
    assert lib.spd_csr_workspace_size(_abi.SPD_OP_SDDMM, ctypes.byref(A), _abi.SPD_SPLIT_NNZ, 64, ctypes.byref(t), ctypes.byref(size)) == 0
    assert size.value >= 2 * 4 * (-(-21000 // 512) + 1)
    assert lib.spd_csr_workspace_size(_abi.SPD_OP_SPTTV, ctypes.byref(A), 1, 0, None, ctypes.byref(size)) == 10
    B = _abi.spd_csf3(8, 8, 8, 20, 100, 256, 512, 768, 1024, 2048, _abi.SPD_F32, 0)
    assert lib.spd_csf3_workspace_size(_abi.SPD_OP_SPMTTKRP, ctypes.byref(B), 1, 32, None, ctypes.byref(size)) == 0
    assert size.value > 0


def test_transpose_host_checks():
    lib = _abi.load()
    size = ctypes.c_size_t(0)
    A = _csr(nrows=1000, ncols=1000, nnz=20000)
    assert lib.spd_csr_transpose_workspace_size(ctypes.byref(A), ctypes.byref(size)) == 0
    assert size.value >= 3 * 4 * 20000 + 256 * 4 * (-(-20000 // 4096))  # keys x2, payload, digit counts
    assert lib.spd_csr_transpose_workspace_size(ctypes.byref(A), None) == 1
    # NULL outputs, short workspace, misaligned outputs: refused before any launch
    assert lib.spd_csr_transpose(ctypes.byref(A), None, 4096, 8192, 1 << 20, 1 << 30, None) == 1
    assert lib.spd_csr_transpose(ctypes.byref(A), 4096, 8192, 12288, 1 << 20, 16, None) == 6
    assert lib.spd_csr_transpose(ctypes.byref(A), 4098, 8192, 12288, 1 << 20, 1 << 30, None) == 4
    assert lib.spd_gather_vals(-1, 256, 512, 1024, _abi.SPD_F32, None) == 2
    assert lib.spd_gather_vals(10, 256, 512, 1024, 9, None) == 3
    assert lib.spd_gather_vals(10, None, 512, 1024, _abi.SPD_F32, None) == 1
    assert lib.spd_gather_vals(10, 256, 514, 1024, _abi.SPD_F32, None) == 4
    assert lib.spd_gather_vals(0, None, None, None, _abi.SPD_F32, None) == 0  # nothing to do


def test_spadd3_host_checks():
    lib = _abi.load()
    size = ctypes.c_size_t(0)
    A = _csr(nrows=1000, ncols=1000, nnz=20000)
    assert lib.spd_spadd3_workspace_size(ctypes.byref(A), ctypes.byref(A), ctypes.byref(A), 1, None,
                                         ctypes.byref(size)) == 0
    assert size.value >= 4 * 1001 + 2 * 4 * (-(-(1000 + 60000) // 64) + 1)  # pos_sum and the partition
    other = _csr(nrows=1000, ncols=999, nnz=20000)
    assert lib.spd_spadd3_workspace_size(ctypes.byref(A), ctypes.byref(other), ctypes.byref(A), 1, None,
                                         ctypes.byref(size)) == 2
    f64 = _csr(nrows=1000, ncols=1000, nnz=20000, vtype=_abi.SPD_F64)
    assert lib.spd_spadd3_workspace_size(ctypes.byref(A), ctypes.byref(A), ctypes.byref(f64), 1, None,
                                         ctypes.byref(size)) == 3
    nnz = ctypes.c_int64(0)
    assert lib.spd_spadd3_symbolic(ctypes.byref(A), ctypes.byref(A), ctypes.byref(A), 1, None, None,
                                   ctypes.byref(nnz), None, 0, None) == 1
    assert lib.spd_spadd3_symbolic(ctypes.byref(A), ctypes.byref(A), ctypes.byref(A), 1, None, 4096,
                                   ctypes.byref(nnz), None, 0, None) == 6
    assert lib.spd_spadd3_numeric(ctypes.byref(A), ctypes.byref(A), ctypes.byref(A), 1, None, 4096, 10, 8192,
                                  12288, _abi.SPD_F64, None, 0, None) == 3  # binary32 operands give binary32


def test_column_block_host_checks():
    lib = _abi.load()
    size = ctypes.c_size_t(0)
    A = _csr(nrows=1000, ncols=1000, nnz=20000)
    assert lib.spd_csr_column_blocks_workspace_size(ctypes.byref(A), 4, ctypes.byref(size)) == 0
    assert size.value > 0
    assert lib.spd_csr_column_blocks_workspace_size(ctypes.byref(A), 0, ctypes.byref(size)) == 10
    cnt = (ctypes.c_int64 * 4)()
    bad_end = (ctypes.c_int32 * 5)(0, 10, 20, 30, 999)  # must end at ncols
    assert lib.spd_csr_column_blocks(ctypes.byref(A), 4, bad_end, 4096, 8192, 12288, cnt, 1 << 20, 1 << 30, None) == 10
    decreasing = (ctypes.c_int32 * 5)(0, 500, 400, 900, 1000)
    assert lib.spd_csr_column_blocks(ctypes.byref(A), 4, decreasing, 4096, 8192, 12288, cnt, 1 << 20, 1 << 30, None) == 10
    ok = (ctypes.c_int32 * 5)(0, 250, 500, 750, 1000)
    assert lib.spd_csr_column_blocks(ctypes.byref(A), 4, ok, 4096, 8192, 12288, cnt, None, 0, None) == 6
    # the accumulating SpMM checks its arguments like spd_spmm
    assert lib.spd_spmm_accumulate(ctypes.byref(A), 4096, 8, 4, 1, 8192, 8, 1, 1, None, None, 0, None) == 2


def test_product_path_has_no_oracle_dependency():
    """The package never imports or loads the oracle (no CPU fallback)."""
    pkg = os.path.join(ROOT, "paper_2207_13901_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text and "spd_oracle" not in text, f


def test_host_tensors_are_refused():
    """No CPU path: every binding refuses host tensors before calling the library."""
    import torch
    import paper_2207_13901_gb300 as spd
    pos = torch.tensor([0, 1, 2], dtype=torch.int32)
    crd = torch.tensor([0, 1], dtype=torch.int32)
    vals = torch.ones(2)
    with pytest.raises(TypeError, match="no CPU path"):
        spd.CSR(pos, crd, vals, (2, 2))
    with pytest.raises(TypeError, match="no CPU path"):
        spd.CSF3(pos, crd, pos, crd, vals, (2, 2, 2))


def noalloc_item_limit(lib):
    """Largest nrows + nnz whose nnz-split SpMV workspace fits the 1 MiB array of
    spd_spmv_noalloc (from the size query, by bisection)."""
    def ws(items):
        d = _abi.spd_csr(1, 1, items - 1, 256, 512, 1024, _abi.SPD_F32, 0)
        b = ctypes.c_size_t(0)
        assert lib.spd_csr_workspace_size(0, ctypes.byref(d), 1, 0, None, ctypes.byref(b)) == 0
        return b.value

    lo, hi = 1, (1 << 31) - 2
    while hi - lo > 1:
        mid = (lo + hi) // 2
        lo, hi = (mid, hi) if ws(mid) <= (1 << 20) else (lo, mid)
    assert ws(lo) <= (1 << 20) < ws(lo + 1)
    return lo


def test_noalloc_scratch_limit():
    """spd_spmv_noalloc rejects, on the host and before any launch, the first size whose
    workspace exceeds its 1 MiB array (the GPU test runs the largest accepted size)."""
    lib = _abi.load()
    assert lib.spd_checked() == 0
    lo = noalloc_item_limit(lib)
    assert lo > 100_000_000  # the header's "about 107 million"
    d = _abi.spd_csr(1, 1, lo, 256, 512, 1024, _abi.SPD_F32, 0)  # nrows + nnz = lo + 1
    assert lib.spd_spmv_noalloc(ctypes.byref(d), 4096, _abi.SPD_F32, 8192, _abi.SPD_F32, None) == _abi.SPD_ERR_SHAPE
    assert b"scratch" in lib.spd_last_error()
