"""Host-side pieces of bench.py that need no GPU: the algorithmic byte counts behind
the roofline, the record and lookup of ncu counters (valid only for the captured case,
kernel sources and tuning), and the sizing of the CPU oracle sample."""
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


def test_recorded_traffic_only_for_the_captured_case(monkeypatch, tmp_path):
    """A record written from an ncu raw CSV is returned for its kernel, case and tuning
    while the kernel's sources are unchanged, and never otherwise."""
    csv_path = tmp_path / "raw.csv"
    csv_path.write_text(
        '"ID","Kernel Name","gpu__time_duration.sum","dram__bytes_read.sum","dram__bytes_write.sum",'
        '"lts__t_sector_hit_rate.pct"\n'
        '"","","usecond","Gbyte","Mbyte","%"\n'
        '"0","spmm_warp_kernel","2,900.5","15.1","480.25","41.5"\n')
    path = str(tmp_path / "traffic.json")
    rec = bench.record_traffic(str(csv_path), "spmm", "rmat22_f32_L128", "1024,128,8", "ncu ...", path=path)
    assert rec["dram_bytes"] == 15_100_000_000 + 480_250_000 and rec["l2_hit_pct"] == 41.5
    got = bench.recorded_traffic("spmm", "rmat22_f32_L128", "1024,128,8", path=path)
    assert got["dram_bytes"] == rec["dram_bytes"]
    assert bench.recorded_traffic("spmm", "rmat20_f32_L128", "1024,128,8", path=path) is None  # another case
    assert bench.recorded_traffic("spmm", "rmat22_f32_L128", "2048,128,8", path=path) is None  # another tuning
    assert bench.recorded_traffic("spmv", "rmat22_f32_L128", "1024,128,8", path=path) is None  # another kernel
    monkeypatch.setattr(bench, "source_hash", lambda kernel: "0000000000000000")
    assert bench.recorded_traffic("spmm", "rmat22_f32_L128", "1024,128,8", path=path) is None  # sources changed
    assert bench.tune_key({"unit_items": 1024, "block_threads": 128, "inflight": 8}) == "1024,128,8"


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
