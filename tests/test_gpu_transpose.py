"""GPU parity of the transposed schedule: A^T's structure and permutation (a stable
radix sort of A's positions by column) bit for bit against the oracle's counting sort,
value gathers bit for bit, and SpMM^T computed as an SpMM over A^T against the
compensated oracle (same tolerances as the other kernels), run to run bit-identical."""
import numpy as np
import pytest
import torch

import oracle
import spd_synth
import paper_2207_13901_gb300 as spd
from tests.test_gpu_kernels import DTYPES, MAT_NAMES, check, dev, dev_csr, get_mats, rounded

pytestmark = pytest.mark.gpu


def extra_mats():
    rng = np.random.default_rng(21)
    wide_cols = np.concatenate([rng.integers(0, 1 << 25, 3000), [(1 << 25) + 2], [0, 0, 1]])
    wide_rows = rng.integers(0, 200, wide_cols.shape[0])
    return {
        # 25-bit column coordinates: four radix passes, an odd number of buffer swaps
        "wide": spd_synth.csr_from_coords(200, (1 << 25) + 3, wide_rows, wide_cols, value_seed=1),
        # one column: every key equal
        "one_col": spd_synth.csr_from_coords(5000, 1, np.arange(5000), np.zeros(5000, dtype=np.int64),
                                             value_seed=2),
        # more than one tile per digit bucket and many tiles (257 columns: two passes)
        "cols257": spd_synth.uniform_csr(20000, 257, 9, seed=3),
    }


ALL = MAT_NAMES + ["wide", "one_col", "cols257"]
_EXTRA = None


def mat(name):
    global _EXTRA
    if name in MAT_NAMES:
        return get_mats()[name]
    if _EXTRA is None:
        _EXTRA = extra_mats()
    return _EXTRA[name]


@pytest.mark.parametrize("name", ALL)
def test_transpose_structure_bit_exact(name):
    A = mat(name)
    t_pos, t_crd, perm = oracle.csr_transpose(A.pos, A.crd, A.ncols)
    dA = dev_csr(A, torch.float32)
    T = spd.transpose(dA)
    torch.cuda.synchronize()
    assert np.array_equal(T.t_pos.cpu().numpy(), t_pos)
    assert np.array_equal(T.t_crd.cpu().numpy(), t_crd)
    assert np.array_equal(T.perm.cpu().numpy(), perm)
    T2 = spd.transpose(dA)  # deterministic: a second run gives the same arrays
    assert torch.equal(T2.perm, T.perm) and torch.equal(T2.t_crd, T.t_crd)


@pytest.mark.parametrize("dtype", DTYPES)
def test_gather_vals_bit_exact(dtype):
    A = mat("rmat12")
    _, _, perm = oracle.csr_transpose(A.pos, A.crd, A.ncols)
    v = dev(A.vals, dtype)
    got = spd.gather_vals(torch.as_tensor(perm).cuda(), v)
    assert torch.equal(got, v[torch.as_tensor(perm, dtype=torch.int64).cuda()])


@pytest.mark.parametrize("name", ["uniform4096", "rmat12", "longrow", "col0", "empty_rows", "no_nnz", "cols257"])
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("L", [1, 32, 128])
def test_spmm_t_over_transpose(name, dtype, L):
    A = mat(name)
    rng = np.random.default_rng(31)
    dY = rng.uniform(-1, 1, (A.nrows, L))
    vr, dYr = rounded(A.vals, dtype), rounded(dY, dtype)
    ref = oracle.spmm_t(A.pos, A.crd, vr, dYr, A.ncols, accurate=True)
    scale = oracle.spmm_t(A.pos, A.crd, np.abs(vr), np.abs(dYr), A.ncols)
    dA = dev_csr(A, dtype)
    ddY = dev(dY, dtype)
    for split in ("nnz", "row"):
        dX = spd.spmm_t(dA, ddY, split=split, method="transpose")
        dX2 = spd.spmm_t(dA, ddY, split=split, method="transpose")
        torch.cuda.synchronize()
        assert torch.equal(dX, dX2), "not run-to-run identical"
        check(dX.double().cpu().numpy(), ref, scale, dtype, "spmm_t transpose %s %s L=%d %s" % (name, dtype, L, split),
              np.bincount(A.crd, minlength=A.ncols)[:, None])


def test_autograd_dx_methods_agree():
    A = mat("rmat12")
    rng = np.random.default_rng(41)
    dA = dev_csr(A, torch.float64)
    X = torch.as_tensor(rng.uniform(-1, 1, (A.ncols, 16))).cuda().requires_grad_(True)
    W = torch.as_tensor(rng.uniform(-1, 1, (A.nrows, 16))).cuda()
    grads = {}
    for dx in ("transpose", "atomic"):
        vals = dA.vals.clone().requires_grad_(True)
        Y = spd.autograd.spmm(dA.with_vals(vals), X, dx=dx)
        (Y * W).sum().backward()
        grads[dx] = (vals.grad.clone(), X.grad.clone())
        X.grad = None
    assert torch.equal(grads["transpose"][0], grads["atomic"][0])
    ref = oracle.spmm_t(A.pos, A.crd, A.vals, W.cpu().numpy(), A.ncols, accurate=True)
    scale = oracle.spmm_t(A.pos, A.crd, np.abs(A.vals), np.abs(W.cpu().numpy()), A.ncols)
    for dx in ("transpose", "atomic"):
        check(grads[dx][1].cpu().numpy(), ref, scale, torch.float64, "dX via %s" % dx, None)
