"""Host-side pieces of bench.py that need no GPU: the algorithmic byte counts behind
the roofline, the lookup of the recorded ncu traffic (valid only for the captured R-MAT
scale, kernel sources and tuning), and the sizing of the CPU oracle sample."""
import numpy as np

import bench
import spd_synth


def test_algorithmic_bytes_formulas():
    n, nnz, L = 1000, 12345, 128
    base = 4 * (n + 1) + 4 * nnz + 4 * nnz
    assert bench.algorithmic_bytes("spmv", n, nnz, 4, 4, 4) == base + 4 * n + 4 * n
    assert bench.algorithmic_bytes("spmm", n, nnz, 4, 4, 4) == base + 4 * n * L + 4 * n * L
    # bfloat16 values and X, binary32 Y
    b16 = 4 * (n + 1) + 4 * nnz + 2 * nnz
    assert bench.algorithmic_bytes("spmm", n, nnz, 2, 2, 4) == b16 + 2 * n * L + 4 * n * L


def test_recorded_traffic_only_for_the_captured_case(monkeypatch):
    tune = {"unit_items": 1024, "block_threads": 128, "inflight": 8}
    got = bench.recorded_traffic(tune, 22)
    assert isinstance(got, int) and got > 10 ** 9
    assert bench.recorded_traffic(tune, 20) is None  # another scale
    assert bench.recorded_traffic(dict(tune, unit_items=2048), 22) is None  # another tuning
    monkeypatch.setattr(bench, "spmm_source_hash", lambda: "0000000000000000")
    assert bench.recorded_traffic(tune, 22) is None  # the kernel sources changed


def test_cpu_sample_is_bounded_and_spans_the_rows():
    A = spd_synth.rmat_csr(12, 16, seed=0)
    per = 1e-6  # seconds per nonzero
    sel, k = bench.cpu_sample(A, 2.0, per)
    assert k >= 1 and sel[0] == 0 and np.all(np.diff(sel) == k)
    snnz = int(np.diff(A.pos)[sel].sum())
    assert snnz * per < 2.0 * 3 or k == 1
    sel_all, k_all = bench.cpu_sample(A, 1e9, per)
    assert k_all == 1 and sel_all.size == A.nrows
    assert bench.host_threads() >= 1


def test_threaded_oracle_runs_every_row():
    A = spd_synth.rmat_csr(10, 8, seed=1)
    x = np.ones(A.ncols)
    X = np.ones((A.ncols, 4))
    sel = np.arange(A.nrows, dtype=np.int64)
    assert bench.oracle_rows_threaded(A, x, X, sel, 3) >= 0.0
