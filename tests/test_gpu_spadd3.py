"""GPU parity of SpAdd3 A = B + C + D with two-phase assembly: A's pos and crd bit for bit
against the oracle (the union of the three patterns), values within the tolerance of
the kernels' arithmetic (binary64: bit for bit, the same (B + C) + D order; binary32 /
bfloat16 inputs summed in binary32: 1e-4 of the sum of magnitudes), both splits and
small work units (pieces that start and end inside rows, runs of equal columns)."""
import numpy as np
import pytest
import torch

import oracle
import spd_synth
import paper_2207_13901_gb300 as spd
from tests._util import check_error, small_csr
from tests.test_gpu_kernels import DTYPES, long_row_csr, rounded

pytestmark = pytest.mark.gpu


def operand_sets():
    rng = np.random.default_rng(3)
    R = spd_synth.rmat_csr(12, 16, seed=1)
    L = long_row_csr()
    E = spd_synth.csr_from_coords(L.nrows, L.ncols, [], [], vals=np.zeros(0))
    one = small_csr(rng, 1, 9000, 0.5, empty_frac=0.0)
    return {
        # the paper's construction: one matrix and its columns shifted by 1 and 2
        "rmat_shifted": (R, spd_synth.shifted_csr(R, 1, seed=2), spd_synth.shifted_csr(R, 2, seed=3)),
        # a row of 10000 entries in every operand: pieces split inside it
        "longrow_shifted": (L, spd_synth.shifted_csr(L, 1, seed=4), spd_synth.shifted_csr(L, 2, seed=5)),
        "independent": tuple(small_csr(rng, 2000, 700, 0.01, empty_frac=0.3, long_rows=2) for _ in range(3)),
        "same_pattern": (L, spd_synth.CSR(L.nrows, L.ncols, L.pos, L.crd, rng.uniform(-1, 1, L.nnz)),
                         spd_synth.CSR(L.nrows, L.ncols, L.pos, L.crd, rng.uniform(-1, 1, L.nnz))),
        "with_empty": (E, L, E),
        "all_empty": (E, E, E),
        "one_row": (one, spd_synth.shifted_csr(one, 1, seed=6), spd_synth.shifted_csr(one, 5, seed=7)),
    }


SETS = None


def get_set(name):
    global SETS
    if SETS is None:
        SETS = operand_sets()
    return SETS[name]


def dev_csr(M, dtype):
    return spd.CSR.from_host(M.pos, M.crd, M.vals, (M.nrows, M.ncols), dtype=dtype)


@pytest.mark.parametrize("name", ["rmat_shifted", "longrow_shifted", "independent", "same_pattern", "with_empty",
                                  "all_empty", "one_row"])
@pytest.mark.parametrize("dtype", DTYPES)
def test_spadd3(name, dtype):
    ops = get_set(name)
    rops = [spd_synth.CSR(M.nrows, M.ncols, M.pos, M.crd, rounded(M.vals, dtype)) for M in ops]
    ap, ac, av = oracle.spadd3(*rops)
    absops = [spd_synth.CSR(M.nrows, M.ncols, M.pos, M.crd, np.abs(M.vals)) for M in rops]
    _, _, scale = oracle.spadd3(*absops)
    dops = [dev_csr(M, dtype) for M in ops]
    for split, tune in [("nnz", None), ("nnz", {"unit_items": 32}), ("nnz", {"unit_items": 4096}),
                        ("row", None), ("row", {"row_pieces": 7})]:
        A = spd.spadd3(*dops, split=split, tune=tune)
        torch.cuda.synchronize()
        what = "spadd3 %s %s %s %s" % (name, dtype, split, tune)
        assert np.array_equal(A.pos.cpu().numpy(), ap), what
        assert np.array_equal(A.crd.cpu().numpy(), ac), what
        got = A.vals.double().cpu().numpy()
        if dtype == torch.float64:
            assert np.array_equal(got, av), what
        else:
            check_error(got, av, scale, False, 3, what)  # at most three terms per entry


def test_spadd3_rejects_mismatched_operands():
    R = get_set("rmat_shifted")[0]
    A = dev_csr(R, torch.float32)
    small = spd_synth.csr_from_coords(10, 10, [1], [2], vals=np.ones(1))
    with pytest.raises(Exception):
        spd.spadd3(A, A, dev_csr(small, torch.float32))
    with pytest.raises(Exception):
        spd.spadd3(A, A, dev_csr(R, torch.float64))
