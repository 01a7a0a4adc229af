"""GPU parity of the value-range column blocks (a universe partition of the Compressed
level): block structure and permutation bit for bit against the oracle, the
accumulating SpMM (Y += A X) and the column-blocked SpMM against the compensated oracle
(tolerances of the other kernels), including empty blocks and blocks of one column."""
import numpy as np
import pytest
import torch

import oracle
import spd_synth
import paper_2207_13901_gb300 as spd
from tests._util import row_lengths
from tests.test_gpu_kernels import DTYPES, check, dev, dev_csr, get_mats, rounded

pytestmark = pytest.mark.gpu

NAMES = ["uniform4096", "rmat12", "longrow", "col0", "empty_rows", "no_nnz", "banded"]


def bounds_sets(m):
    return [[0, m], [0, m // 3, (2 * m) // 3, m], [0, 0, 1, 1, m // 2, m, m], [(b * m) // 16 for b in range(17)]]


@pytest.mark.parametrize("name", NAMES)
def test_column_blocks_bit_exact(name):
    A = get_mats()[name]
    dA = dev_csr(A, torch.float32)
    for bounds in bounds_sets(A.ncols):
        blk_pos, blk_crd, perm, nnz = oracle.column_blocks(A.pos, A.crd, np.array(bounds, dtype=np.int32))
        cb = spd.column_blocks(dA, bounds=bounds)
        torch.cuda.synchronize()
        assert cb.nnz == list(nnz)
        assert np.array_equal(cb.blk_pos.cpu().numpy(), blk_pos), bounds
        assert np.array_equal(cb.blk_crd.cpu().numpy(), blk_crd), bounds
        assert np.array_equal(cb.perm.cpu().numpy(), perm), bounds


@pytest.mark.parametrize("name", ["uniform4096", "rmat12", "longrow", "empty_rows"])
@pytest.mark.parametrize("dtype", DTYPES)
def test_spmm_accumulate(name, dtype):
    A = get_mats()[name]
    rng = np.random.default_rng(51)
    L = 64
    X = rng.uniform(-1, 1, (A.ncols, L))
    Y0 = rng.uniform(-1, 1, (A.nrows, L))
    vr, Xr = rounded(A.vals, dtype), rounded(X, dtype)
    rdt = spd.result_dtype(dtype)
    Y0r = torch.as_tensor(Y0).to(rdt).double().numpy()
    ref = Y0r + oracle.spmm(A.pos, A.crd, vr, Xr, accurate=True)
    scale = np.abs(Y0r) + oracle.spmm(A.pos, A.crd, np.abs(vr), np.abs(Xr))
    dA = dev_csr(A, dtype)
    for split in ("nnz", "row"):
        Y = torch.as_tensor(Y0).to(rdt).cuda()
        spd.spmm_accumulate(dA, dev(X, dtype), Y, split=split)
        torch.cuda.synchronize()
        # Y0 adds one term to every output
        check(Y.double().cpu().numpy(), ref, scale, dtype, "spmm_accumulate %s %s %s" % (name, dtype, split),
              row_lengths(A.pos)[:, None] + 1)


@pytest.mark.parametrize("name", ["rmat12", "longrow", "banded", "no_nnz"])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("L", [64, 128])
def test_spmm_column_blocked(name, dtype, L):
    A = get_mats()[name]
    rng = np.random.default_rng(52)
    X = rng.uniform(-1, 1, (A.ncols, L))
    vr, Xr = rounded(A.vals, dtype), rounded(X, dtype)
    ref = oracle.spmm(A.pos, A.crd, vr, Xr, accurate=True)
    scale = oracle.spmm(A.pos, A.crd, np.abs(vr), np.abs(Xr))
    dA = dev_csr(A, dtype)
    for nblk in (1, 4, 16):
        Y = spd.spmm_column_blocked(dA, dev(X, dtype), nblk=nblk)
        torch.cuda.synchronize()
        check(Y.double().cpu().numpy(), ref, scale, dtype, "column blocked %s %s L=%d nblk=%d" % (name, dtype, L, nblk),
              row_lengths(A.pos)[:, None])
