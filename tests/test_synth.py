"""The input generators: level-format invariants, determinism, and termination on the
small and dense shapes the tests use (no GPU)."""
import numpy as np
import pytest

import oracle
import spd_synth


def _valid(A):
    assert A.pos[0] == 0 and A.pos[-1] == A.nnz and np.all(np.diff(A.pos) >= 0)
    assert oracle.validate_level(A.nrows, A.ncols, A.pos, A.crd) == (0, -1)
    for i in range(min(A.nrows, 300)):
        seg = A.crd[A.pos[i]:A.pos[i + 1]]
        assert np.all(np.diff(seg) > 0)  # sorted, distinct


@pytest.mark.parametrize("shape", [(100, 100, (4, 64)), (50, 64, 64), (4096, 4096, 16), (10, 1, 1), (7, 3, (0, 3))])
def test_uniform_csr_shapes(shape):
    n, m, k = shape
    A = spd_synth.uniform_csr(n, m, k, seed=1)
    _valid(A)
    lens = np.diff(A.pos)
    if isinstance(k, tuple):
        assert lens.min() >= min(k[0], m) and lens.max() <= min(k[1], m)
    else:
        assert np.all(lens == min(k, m))
    B = spd_synth.uniform_csr(n, m, k, seed=1)
    assert np.array_equal(A.crd, B.crd) and np.array_equal(A.vals, B.vals)


def test_batched_small_and_dense():
    mats = spd_synth.batched_uniform_csr(24, 1e2, 3e3, 4, 64, seed=1)
    assert len(mats) == 24
    for A in mats:
        assert A.nrows == A.ncols and 100 <= A.nrows <= 3000
        _valid(A)


def test_rmat_and_zipf_invariants():
    A = spd_synth.rmat_csr(12, 16, seed=1)
    _valid(A)
    assert A.nnz > 0.9 * 16 * 4096 * 0.9
    T = spd_synth.zipf_csf3((1 << 8,) * 3, 20000, seed=2)
    assert T.nnz == 20000
    assert oracle.validate_level(T.dims[0], T.dims[1], T.pos1, T.crd1) == (0, -1)
    assert oracle.validate_level(T.nfib, T.dims[2], T.pos2, T.crd2) == (0, -1)
    assert np.all(np.diff(T.pos2) > 0)  # no empty fibers


def test_banded_structure():
    """Row i holds exactly the columns max(0, i-w) .. min(n-1, i+w), in order."""
    n, w = 50, 3
    A = spd_synth.banded_csr(n, w, seed=1)
    dense = np.zeros((n, n), dtype=bool)
    for i in range(n):
        cols = A.crd[A.pos[i]:A.pos[i + 1]]
        assert np.all(np.diff(cols) == 1)
        dense[i, cols] = True
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    assert np.array_equal(dense, np.abs(ii - jj) <= w)
    assert A.nnz == n * (2 * w + 1) - w * (w + 1)
    assert np.all((A.vals >= -1) & (A.vals < 1))


def test_shifted_csr_rotates_each_row():
    A = spd_synth.rmat_csr(9, 8, seed=2)
    for shift in (1, 2, A.ncols - 1):
        S = spd_synth.shifted_csr(A, shift, seed=3)
        assert np.array_equal(S.pos, A.pos)
        for i in range(A.nrows):
            got = S.crd[S.pos[i]:S.pos[i + 1]]
            assert np.array_equal(got, np.sort((A.crd[A.pos[i]:A.pos[i + 1]] + shift) % A.ncols))


def test_limit_generators_invariants():
    """The size-limit generators at small sizes: exact entry counts, valid level
    format, int8 values in [-3, 3], the long row, the forced first and last rows, and
    fibers of 1 to 3 entries across chunk boundaries of the fiber draw."""
    A = spd_synth.limit_csr(1000, 77, 100000, seed=1, long_row=20000)
    lens = np.diff(A.pos)
    assert A.pos[0] == 0 and A.pos[-1] == 100000 and lens.min() >= 0 and lens[333] >= 20000
    assert 0.05 < np.mean(lens == 0) < 0.2
    assert A.crd.dtype == np.int32 and 0 <= A.crd.min() and A.crd.max() < 77
    assert A.vals.dtype == np.int8 and A.vals.min() == -3 and A.vals.max() == 3
    B = spd_synth.limit_rows_csr(10**6, 50, 5000, seed=2)
    assert B.pos.shape[0] == 10**6 + 1 and B.pos[0] == 0 and B.pos[-1] == 5000 and np.diff(B.pos).min() >= 0
    assert B.pos[1] >= 1 and B.pos[-2] < 5000  # rows 0 and n-1 hold entries
    rows = np.repeat(np.arange(10**6), np.diff(B.pos))
    assert rows.shape[0] == 5000 and np.all(np.diff(rows) >= 0)
    for nnz in (1, 3, 100001, 3 * (1 << 24) + 5):
        T = spd_synth.limit_csf3((500, 40, 60), nnz, seed=3)
        d = np.diff(T.pos2)
        assert T.pos2[0] == 0 and T.pos2[-1] == nnz and d.min() >= 1 and d.max() <= 3
        assert T.pos1[0] == 0 and T.pos1[-1] == T.nfib and np.diff(T.pos1).min() >= 0
        assert T.crd1.max() < 40 and T.crd2.max() < 60 and T.crd2.shape[0] == nnz
    first = spd_synth.limit_csf3((500, 40, 60), 100001, seed=3)
    again = spd_synth.limit_csf3((500, 40, 60), 100001, seed=3)
    for name in ("pos1", "crd1", "pos2", "crd2", "vals"):
        assert np.array_equal(getattr(first, name), getattr(again, name))


def test_limit_interval_csr_rows_are_column_runs():
    A = spd_synth.limit_interval_csr(3000, 64, 150000, seed=4)  # lengths capped at 64 columns
    lens = np.diff(A.pos)
    assert A.pos[-1] == 150000 and lens.max() <= 64 and lens.min() >= 0
    assert oracle.validate_level(A.nrows, A.ncols, A.pos, A.crd) == (0, -1)
    for i in range(A.nrows):
        seg = A.crd[A.pos[i]:A.pos[i + 1]]
        if seg.shape[0]:
            assert np.array_equal(seg, np.arange(seg[0], seg[0] + seg.shape[0]))
    B = spd_synth.limit_interval_csr(1000, 4096, 100000, seed=5)
    assert B.pos[-1] == 100000 and B.vals.dtype == np.int8
