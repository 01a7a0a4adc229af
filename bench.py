#!/usr/bin/env python
"""Throughput of the SpDISTAL hot path on one GB300: SpMV and SpMM (L = 128) on a
2^22 x 2^22 R-MAT power-law matrix (a = 0.57, b = c = 0.19, 16 samples per row,
duplicates merged), int32 pos/crd, values uniform in [-1, 1).

One step = the whole path once over the matrix: the fused non-zero partition of the
coordinate tree, SpMV y = A x with its binary64 fix-up, and SpMM Y = A X with its
fix-up, in binary32 (values, x and X binary32, binary32 accumulation). Units are
nonzeros processed: each step streams the matrix's nonzeros twice (SpMV and SpMM).

The JSON line also carries, measured in the same run:
  * per-variant results (binary64 / binary32 / bfloat16 x row / nnz split, SpMV and
    SpMM): nonzeros/s, algorithmic-bytes bandwidth and its fraction of the measured
    HBM copy bandwidth, and the error against the compensated binary64 oracle on
    sampled rows (against the same rounded inputs and against the binary64 inputs);
  * the roofline of the dominant kernel (the SpMM call), the CPU oracle timed on the
    host cores on a bounded row sample, an end-to-end figure with host buffers, and
    the SM clocks sampled during the timed region.

``--impl reference`` times the CPU oracle (the reference arm) on bounded row samples.
Multi-GPU: one process per GPU (torchrun); every rank processes its own copy of the
workload (independent problems, no collective on the data path) and the value is the
nonzeros of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L_COLS = 128


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["spd", "reference"], default="spd")
    p.add_argument("--scale", type=int, default=22, help="log2 of the matrix size (22 = the measured workload)")
    p.add_argument("--no-variants", action="store_true", help="skip the per-variant table")
    p.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of CPU oracle work for cpu_baseline")
    p.add_argument("--e2e-steps", type=int, default=20)
    p.add_argument("--fixed-tune", default="",
                   help="UNIT,BLOCK,INFLIGHT: skip the autotuner and run SpMM with this tuning (nnz split)")
    p.add_argument("--rows", default="all",
                   help="comma list of extra hot-path rows to measure: cfg1,sddmm,backward,csf,batched,banded,spadd3,colblock "
                        "(or all, none)")
    p.add_argument("--record-traffic", nargs=5, metavar=("CSV", "KERNEL", "CASE", "TUNE", "COMMAND"),
                   help="store the counters of an ncu raw CSV export in profiles/traffic.json and exit")
    p.add_argument("--case", default="",
                   help="time one kernel case alone and exit (for profiling): spmv:SCALE:DTYPE:FORM, "
                        "banded:0:DTYPE:FORM, spmm:SCALE:DTYPE, sddmm:K:DTYPE:FORM, spttv:0:DTYPE:FORM or "
                        "spmttkrp:R:DTYPE (DTYPE f32, bf16 or f64; nnz split)")
    return p.parse_args(argv)


# ----------------------------------------------------------------------------- distributed

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(backend):
    import torch.distributed as dist
    ws, rank, local = dist_env()
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return ws, rank, local


def aggregate(units_local: float, seconds_local: float):
    """Whole-job throughput: the units of all ranks over the slowest rank's time."""
    import torch
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
        t = torch.tensor([seconds_local], dtype=torch.float64, device=dev)
        u = torch.tensor([units_local], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        return float(u.item()), float(t.item())
    return units_local, seconds_local


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


# ----------------------------------------------------------------------------- workload

def workload(scale: int):
    import spd_synth
    t0 = time.time()
    A = spd_synth.rmat_csr(scale, 16, 0.57, 0.19, 0.19, seed=0)
    n = A.nrows
    x = spd_synth.uniform(n, seed=2, dtype=np.float32)
    X = spd_synth.uniform((n, L_COLS), seed=3, dtype=np.float32)
    return A, x, X, time.time() - t0


# Binary64 fused multiply-add peak of this GPU: 152 SMs x 2 binary64 FMA per clock x 2
# flops x 2.07 GHz. (A run of independent FMA chains on every SM measured 1.3 TFLOP/s in
# binary64 and 77 TFLOP/s in binary32, i.e. 2 and ~124 FMA per clock per SM.)
FP64_FMA_TFLOPS = 1.26
# GB300's nominal HBM3e bandwidth, reported beside the measured copy bandwidth
HBM_NOMINAL_GBS = 7900.0


def workload_name(scale: int) -> str:
    """The benchmarked workload, named the same way by both arms."""
    return ("SpMV + SpMM(L=128) on R-MAT 2^%d (a=.57,b=.19,c=.19, 16 samples/row, dedup), binary32, nnz split "
            "(fused non-zero partition), step = partition + SpMV + fix-up + SpMM + fix-up" % scale)


def algorithmic_bytes(kernel: str, n: int, nnz: int, vbytes: int, xbytes: int, ybytes: int, L: int = L_COLS) -> int:
    """Bytes every kernel must move at least once: pos, crd, values, the dense input
    read once and the output written once."""
    base = 4 * (n + 1) + 4 * nnz + vbytes * nnz
    if kernel == "spmv":
        return base + xbytes * n + ybytes * n
    return base + xbytes * n * L + ybytes * n * L


# Sources each kernel's recorded ncu counters depend on: a record is used only while
# these files are unchanged (their hash is stored with it).
KERNEL_SOURCES = {
    "spmm": ("spd_spmm.cu", "spd_spmm_piece.cuh"),
    "spmv": ("spd_spmv.cu",),
    "spttv": ("spd_spmv.cu",),
    "sddmm": ("spd_sddmm.cu",),
    "spmttkrp": ("spd_mttkrp.cu",),
}
COMMON_SOURCES = ("spd_internal.cuh", "spd_core.cu")
TRAFFIC_JSON = os.path.join(ROOT, "profiles", "traffic.json")


def source_hash(kernel: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[kernel] + COMMON_SOURCES:
        with open(os.path.join(ROOT, "paper_2207_13901_gb300", "csrc", rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, case: str, tune=None, path: str = TRAFFIC_JSON):
    """ncu counters of one launch of `kernel` on `case` (DRAM bytes read + written, L2 hit
    rate) from the committed record, if it was taken on the current kernel sources (and,
    when `tune` is given, with that tuning); otherwise None."""
    try:
        with open(path) as f:
            rec = json.load(f).get("records", {}).get(kernel + "|" + case)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_hash") != source_hash(kernel) or (tune is not None and rec.get("tune") != tune):
        return None
    return {"dram_bytes": int(rec["dram_bytes"]), "l2_hit_pct": rec.get("l2_hit_pct"), "tune": rec.get("tune"),
            "kernel_name": rec.get("kernel_name"), "duration_us_under_ncu": rec.get("duration_us_under_ncu")}


def tune_key(tune) -> str:
    """Tuning of a recorded launch: unit items, threads per block, rows in flight."""
    t = tune or {}
    return "%d,%d,%d" % (t.get("unit_items", 0), t.get("block_threads", 0), t.get("inflight", 0))


def record_traffic(csv_path: str, kernel: str, case: str, tune: str, command: str, path: str = TRAFFIC_JSON) -> dict:
    """Stores the counters of the last launch in an ncu raw CSV export (``ncu -i REPORT
    --page raw --csv``): dram__bytes_read.sum + dram__bytes_write.sum and, when captured,
    lts__t_sector_hit_rate.pct, with the hash of the kernel's sources and the tuning."""
    import csv
    with open(csv_path) as f:
        rows = [r for r in csv.reader(f)]
    hdr, units, last = rows[0], rows[1], rows[-1]
    col = {h: i for i, h in enumerate(hdr)}

    def val(name):
        v = float(last[col[name]].replace(",", ""))
        u = units[col[name]]
        return v * {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}.get(u, 1)

    rec = {"kernel_name": last[col["Kernel Name"]] if "Kernel Name" in col else "",
           "dram_bytes": int(val("dram__bytes_read.sum") + val("dram__bytes_write.sum")),
           "l2_hit_pct": round(val("lts__t_sector_hit_rate.pct"), 2) if "lts__t_sector_hit_rate.pct" in col else None,
           "duration_us_under_ncu": round(val("gpu__time_duration.sum") * {"nsecond": 1e-3, "usecond": 1.0, "msecond": 1e3,
                                                                             "ms": 1e3, "us": 1.0, "ns": 1e-3}.get(
               units[col["gpu__time_duration.sum"]], 1.0), 2),
           "tune": tune, "source_hash": source_hash(kernel), "command": command}
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        data = {}
    data.setdefault("records", {})[kernel + "|" + case] = rec
    data["about"] = ("ncu counters of one launch of each kernel on its workload (one kernel, one launch, "
                     "--clock-control none); bench.py reports them while the kernel's sources are unchanged")
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    return rec


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi SM clock / throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t_start = self.t_stop = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark_start(self):
        self.t_start = time.time()

    def mark_stop(self):
        self.t_stop = time.time()

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = [l for t, l in self.lines if self.t_start is not None and self.t_start - 0.05 <= t <= (self.t_stop or t) + 0.05]
        if not rows:
            rows = [l for _, l in self.lines]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            f = [v.strip() for v in r.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- GPU arm

def error_stats(got, ref, scale):
    den = np.maximum(np.abs(ref), scale)
    den = np.where(den == 0, 1.0, den)
    e = (np.abs(got - ref) / den).ravel()
    return {"max": float(e.max()) if e.size else 0.0, "p99": float(np.quantile(e, 0.99)) if e.size else 0.0}


def run_case(args):
    """One kernel case timed alone (3 untimed calls, then `--steps` calls between CUDA
    events); prints one JSON line. Small enough to run under a profiler. Cases:
      spmv:SCALE:DTYPE:FORM    SpMV on the R-MAT 2^SCALE (16 samples per row), nnz split
      banded:0:DTYPE:FORM      SpMV on the banded matrix (21.2M rows, 33 per row)
      spmm:SCALE:DTYPE         SpMM, L = 128, on the R-MAT 2^SCALE, nnz split, unit 1024,
                               128 threads, 8 rows in flight
      sddmm:K:DTYPE:FORM       SDDMM on the 2^20-row R-MAT with 32 samples per row
      spttv:0:DTYPE:FORM       SpTTV on the Zipf(1.1) CSF tensor (50M nonzeros)
      spmttkrp:R:DTYPE         SpMTTKRP on the same tensor
    (DTYPE f32, bf16 or f64; FORM 0, 1 or 2 as spd_tune.form; nnz split.)"""
    import torch
    import spd_synth
    import paper_2207_13901_gb300 as spd
    parts = args.case.split(":")
    kind, width, dname = parts[0], int(parts[1]), parts[2]
    form = int(parts[3]) if len(parts) > 3 else 0
    dt = {"f32": torch.float32, "bf16": torch.bfloat16, "f64": torch.float64}[dname]
    tune = {"unit_items": 1024, "block_threads": 128}
    if kind in ("spmv", "banded", "spmm"):
        if kind == "banded":
            A = spd_synth.banded_csr(21_212_122, 16, seed=0, value_dtype=np.float32)
            what = "SpMV on the banded matrix, %d nonzeros" % A.nnz
        else:
            A = spd_synth.rmat_csr(width, 16, 0.57, 0.19, 0.19, seed=0)
            what = "%s on R-MAT 2^%d, %d nonzeros" % ("SpMV" if kind == "spmv" else "SpMM L=128", width, A.nnz)
        n = A.nrows
        dA = spd.CSR.from_host(A.pos, A.crd, A.vals, (n, A.ncols), dtype=dt)
        rdt = spd.result_dtype(dt)
        if kind == "spmm":
            tune = dict(tune, inflight=8)
            X = torch.from_numpy(spd_synth.uniform((A.ncols, L_COLS), seed=3, dtype=np.float32)).cuda().to(dt)
            Y = torch.empty((n, L_COLS), dtype=rdt, device="cuda")
            ws = torch.empty(max(spd.csr_workspace_size(1, dA, "nnz", L_COLS, tune), 1), dtype=torch.uint8,
                             device="cuda")
            fn = lambda: spd.spmm(dA, X, Y, split="nnz", tune=tune, ws=ws)
        else:
            tune = {"form": form}
            x = torch.from_numpy(spd_synth.uniform(A.ncols, seed=2, dtype=np.float32)).cuda().to(dt)
            y = torch.empty(n, dtype=rdt, device="cuda")
            ws = torch.empty(max(spd.csr_workspace_size(0, dA, "nnz"), 1), dtype=torch.uint8, device="cuda")
            fn = lambda: spd.spmv(dA, x, y, split="nnz", tune=tune, ws=ws)
        units = A.nnz
    elif kind == "sddmm":
        B = spd_synth.rmat_csr(20, 32, seed=0)
        n = B.nrows
        C = torch.from_numpy(spd_synth.normal((n, width), seed=10 + width, dtype=np.float32)).cuda().to(dt)
        D = torch.from_numpy(spd_synth.normal((n, width), seed=20 + width, dtype=np.float32)).cuda().to(dt)
        dB = spd.CSR.from_host(B.pos, B.crd, B.vals, (n, n), dtype=dt)
        out = torch.empty(B.nnz, dtype=spd.result_dtype(dt), device="cuda")
        tune = dict(tune, form=form)
        fn = lambda: spd.sddmm(dB, C, D, out, split="nnz", tune=tune)
        units, what = B.nnz, "SDDMM K=%d on R-MAT 2^20 (32 samples per row), %d nonzeros" % (width, B.nnz)
    elif kind in ("spmttkrp", "spttv"):
        T = spd_synth.zipf_csf3((1 << 17,) * 3, 50_000_000, 1.1, seed=0)
        dT = spd.CSF3.from_host(T.pos1, T.crd1, T.pos2, T.crd2, T.vals, T.dims, dtype=dt)
        if kind == "spttv":
            tune = {"form": form}
            c = torch.from_numpy(spd_synth.normal(T.dims[2], seed=31, dtype=np.float32)).cuda().to(dt)
            o = torch.empty(T.nfib, dtype=spd.result_dtype(dt), device="cuda")
            fn = lambda: spd.spttv(dT, c, o, split="nnz", tune=tune)
            what = "SpTTV on the Zipf(1.1) CSF 2^17 x 2^17 x 2^17, %d nonzeros" % T.nnz
        else:
            Cf = torch.from_numpy(spd_synth.normal((T.dims[1], width), seed=40 + width, dtype=np.float32)).cuda().to(dt)
            Df = torch.from_numpy(spd_synth.normal((T.dims[2], width), seed=50 + width, dtype=np.float32)).cuda().to(dt)
            Af = torch.empty((T.dims[0], width), dtype=spd.result_dtype(dt), device="cuda")
            fn = lambda: spd.spmttkrp(dT, Cf, Df, Af, split="nnz", tune=tune)
            what = "SpMTTKRP R=%d on the Zipf(1.1) CSF 2^17 x 2^17 x 2^17, %d nonzeros" % (width, T.nnz)
        units = T.nnz
    else:
        raise SystemExit("unknown case %r" % args.case)
    ms = _time_ms(fn, reps=max(1, args.steps), warm=3)
    print(json.dumps({"case": args.case, "workload": what, "dtype": dname, "ms": round(ms, 4),
                      "nnz_per_s": units / (ms * 1e-3), "tune": tune}))


def run_gpu(args):
    import torch
    ws, rank, local = dist_init("nccl")
    torch.cuda.set_device(local)
    import oracle  # CPU baseline and error statements only
    import paper_2207_13901_gb300 as spd
    from paper_2207_13901_gb300 import _abi
    _abi.load()
    dev = torch.device("cuda", local)

    A, x32, X32, gen_s = workload(args.scale)
    n, nnz = A.nrows, A.nnz
    vals64 = A.vals
    stream = torch.cuda.current_stream()

    # ---------------- resident inputs (binary32 step)
    pos_d = torch.from_numpy(A.pos).to(dev)
    crd_d = torch.from_numpy(A.crd).to(dev)
    v32 = torch.from_numpy(vals64).to(torch.float32).to(dev)
    xd = torch.from_numpy(x32).to(dev)
    Xd = torch.from_numpy(X32).to(dev)
    Ad = spd.CSR(pos_d, crd_d, v32, (n, n))
    y = torch.empty(n, dtype=torch.float32, device=dev)
    Y = torch.empty((n, L_COLS), dtype=torch.float32, device=dev)

    # the autotuner picks each call's split and tuning (timed here, outside the timed region)
    from paper_2207_13901_gb300.autotune import Autotuner
    import tempfile
    tuner = Autotuner(path=os.path.join(tempfile.mkdtemp(prefix="spd_tune_"), "autotune.json"))
    if args.fixed_tune:
        u, bt, inf = (int(v) for v in args.fixed_tune.split(","))
        best_spmm = {"split": "nnz", "tune": {"unit_items": u, "block_threads": bt, "inflight": inf}}
        best_spmv = {"split": "nnz", "tune": None}
        spmm_table = spmv_table = "fixed"
    else:
        best_spmm = tuner.spmm(Ad, Xd, Y, force=True)
        spmm_table = tuner.last_table
        best_spmv = tuner.spmv(Ad, xd, y, force=True)
        spmv_table = tuner.last_table
    sp_v, tu_v = best_spmv["split"], best_spmv["tune"]
    sp_m, tu_m = best_spmm["split"], best_spmm["tune"]

    # every call's workspace is allocated once, outside the timed region
    ws_spmv = torch.empty(max(spd.csr_workspace_size(0, Ad, sp_v, 0, tu_v), 1), dtype=torch.uint8, device=dev)
    ws_spmm = torch.empty(max(spd.csr_workspace_size(1, Ad, sp_m, L_COLS, tu_m), 1), dtype=torch.uint8, device=dev)

    ev = lambda: torch.cuda.Event(enable_timing=True)

    def step(marks=None):
        if marks is not None:
            marks[0].record(stream)
        spd.spmv(Ad, xd, y, split=sp_v, tune=tu_v, ws=ws_spmv)
        if marks is not None:
            marks[1].record(stream)
        spd.spmm(Ad, Xd, Y, split=sp_m, tune=tu_m, ws=ws_spmm)
        if marks is not None:
            marks[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    # per-call events on the launching stream for the kernel durations (roofline)
    marks = [[ev(), ev(), ev()] for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    t0, t1 = ev(), ev()
    clocks.mark_start()
    t0.record(stream)
    for k in range(args.steps):
        step(marks[k])
    t1.record(stream)
    torch.cuda.synchronize()
    clocks.mark_stop()
    barrier()
    time.sleep(0.1)
    clocks.stop()
    elapsed = t0.elapsed_time(t1) / 1e3
    spmv_calls = [m[0].elapsed_time(m[1]) for m in marks]
    spmm_calls = [m[1].elapsed_time(m[2]) for m in marks]
    spmv_ms = statistics.mean(spmv_calls)
    spmm_ms = statistics.mean(spmm_calls)
    call_ms = {k: {"mean": round(statistics.mean(v), 4), "median": round(statistics.median(v), 4),
                   "min": round(min(v), 4)} for k, v in (("spmv", spmv_calls), ("spmm", spmm_calls))}
    units_local = 2.0 * nnz * args.steps
    units, secs = aggregate(units_local, elapsed)
    value = units / secs
    ms_per_step = secs * 1e3 / args.steps
    # nnz split: SpMV = partition + tile kernel + fix-up; SpMM = partition + warp kernel +
    # chunk sums + row fix-up. Row split: one kernel each.
    per_call = {("spmv", "nnz"): 3, ("spmm", "nnz"): 4, ("spmv", "row"): 1, ("spmm", "row"): 1}
    launches = args.steps * (per_call[("spmv", sp_v)] + per_call[("spmm", sp_m)])

    hbm, peak_kind = measured_peaks()
    spmm_bytes = algorithmic_bytes("spmm", n, nnz, 4, 4, 4)
    spmv_bytes = algorithmic_bytes("spmv", n, nnz, 4, 4, 4)
    spmm_gbs = spmm_bytes / (spmm_ms * 1e-3) / 1e9
    spmm_rec = (recorded_traffic("spmm", "rmat%d_f32_L%d" % (args.scale, L_COLS), tune_key(tu_m))
                if sp_m == "nnz" else None)
    spmv_rec = (recorded_traffic("spmv", "rmat%d_f32_form%d" % (args.scale, (tu_v or {}).get("form", 1) or 1))
                if sp_v == "nnz" else None)

    # ---------------- errors of the measured step (sampled rows vs the compensated oracle)
    rng = np.random.default_rng(0)
    lens = np.diff(A.pos)
    sel = np.unique(np.concatenate([rng.integers(0, n, 2000), np.argsort(lens)[-4:]])).astype(np.int64)
    torch.cuda.synchronize()

    def errs(dtype_name, yv, Yv):
        vr = torch.from_numpy(vals64).to(getattr(torch, dtype_name)).double().numpy()
        xr = torch.from_numpy(x32).to(getattr(torch, dtype_name)).double().numpy()
        Xs = torch.from_numpy(X32).to(getattr(torch, dtype_name)).double().numpy()
        out = {}
        ref = oracle.spmv(A.pos, A.crd, vr, xr, sel=sel, accurate=True)
        sc = oracle.spmv(A.pos, A.crd, np.abs(vr), np.abs(xr), sel=sel)
        out["spmv"] = error_stats(yv[sel], ref, sc)
        ref64 = oracle.spmv(A.pos, A.crd, vals64, x32.astype(np.float64), sel=sel, accurate=True)
        out["spmv_vs_f64_inputs"] = error_stats(yv[sel], ref64, sc)
        selm = sel[:300]
        refm = oracle.spmm(A.pos, A.crd, vr, Xs, sel=selm, accurate=True)
        scm = oracle.spmm(A.pos, A.crd, np.abs(vr), np.abs(Xs), sel=selm)
        out["spmm"] = error_stats(Yv[selm], refm, scm)
        refm64 = oracle.spmm(A.pos, A.crd, vals64, X32.astype(np.float64), sel=selm, accurate=True)
        out["spmm_vs_f64_inputs"] = error_stats(Yv[selm], refm64, scm)
        return out

    y_h = y.double().cpu().numpy()
    Y_sel = np.zeros((n, L_COLS))
    Y_sel[sel] = Y[torch.from_numpy(sel).to(dev)].double().cpu().numpy()
    step_err = errs("float32", y_h, Y_sel)

    # ---------------- variants (dtype x split), timed outside the headline region
    variants = {}
    if not args.no_variants:
        tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}
        for name, dt in tdt.items():
            vd = torch.from_numpy(vals64).to(dt).to(dev)
            xv = torch.from_numpy(x32).to(dt).to(dev)
            Xv = torch.from_numpy(X32).to(dev).to(dt)
            Av = spd.CSR(pos_d, crd_d, vd, (n, n))
            rt = spd.result_dtype(dt)
            yv = torch.empty(n, dtype=rt, device=dev)
            Yv = torch.empty((n, L_COLS), dtype=rt, device=dev)
            vb = {"f64": 8, "f32": 4, "bf16": 2}[name]
            ob = 8 if name == "f64" else 4
            tuned = tuner.spmm(Av, Xv, Yv, force=True)["tune"] if name != "f32" else tu_m
            for split in ("nnz", "row"):
                tm = tuned if split == "nnz" else None
                wsv = torch.empty(max(spd.csr_workspace_size(0, Av, split), 1), dtype=torch.uint8, device=dev)
                wsm = torch.empty(max(spd.csr_workspace_size(1, Av, split, L_COLS, tm), 1), dtype=torch.uint8, device=dev)
                res = {"spmm_tune": tm}
                for kern, fn, nbytes in (
                        ("spmv", lambda: spd.spmv(Av, xv, yv, split=split, ws=wsv),
                         algorithmic_bytes("spmv", n, nnz, vb, vb, ob)),
                        ("spmm", lambda: spd.spmm(Av, Xv, Yv, split=split, tune=tm, ws=wsm),
                         algorithmic_bytes("spmm", n, nnz, vb, vb, ob))):
                    for _ in range(3):
                        fn()
                    reps = 10
                    e0, e1 = ev(), ev()
                    torch.cuda.synchronize()
                    e0.record(stream)
                    for _ in range(reps):
                        fn()
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1) / reps
                    res[kern] = {"ms": round(ms, 4), "nnz_per_s": nnz / (ms * 1e-3),
                                 "algorithmic_GBps": round(nbytes / (ms * 1e-3) / 1e9, 1),
                                 "hbm_frac": round(nbytes / (ms * 1e-3) / 1e9 / hbm, 4)}
                    if name == "f64" and kern == "spmm":
                        # binary64 SpMM is bound by the FP64 FMA rate, not by memory
                        tf = 2.0 * L_COLS * nnz / (ms * 1e-3) / 1e12
                        res[kern]["alu_roofline"] = {"bound": "alu", "achieved": round(tf, 3),
                                                     "peak": FP64_FMA_TFLOPS, "unit": "TFLOP/s",
                                                     "frac": round(tf / FP64_FMA_TFLOPS, 4)}
                yh = yv.double().cpu().numpy()
                Yh = np.zeros((n, L_COLS))
                Yh[sel] = Yv[torch.from_numpy(sel).to(dev)].double().cpu().numpy()
                tname = {"f64": "float64", "f32": "float32", "bf16": "bfloat16"}[name]
                res["error"] = errs(tname, yh, Yh)
                variants["%s_%s" % (name, split)] = res
            del vd, xv, Xv, yv, Yv, Av
            torch.cuda.empty_cache()

    # ---------------- end to end through the public API with host buffers
    # Every step copies its inputs (the matrix, x and X) in from pinned host memory and its
    # results (y and Y) out. Two device buffer sets and three streams let one step's
    # copies run under its neighbours' copies and kernels (host-to-device and
    # device-to-host copies use separate engines); events keep each set's reuse in order.
    pin = lambda a: torch.from_numpy(a).pin_memory()
    h_pos, h_crd, h_vals = pin(A.pos), pin(A.crd), torch.from_numpy(vals64).to(torch.float32).pin_memory()
    h_x, h_X = pin(x32), pin(X32)
    h_y = torch.empty(n, dtype=torch.float32).pin_memory()
    h_Y = torch.empty((n, L_COLS), dtype=torch.float32).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in (h_pos, h_crd, h_vals, h_x, h_X))
    d2h = h_y.numel() * 4 + h_Y.numel() * 4
    ins = (("pos", h_pos), ("crd", h_crd), ("v", h_vals), ("x", h_x), ("X", h_X))
    bufs = []
    for _ in range(2):
        B = {"pos": torch.empty_like(pos_d), "crd": torch.empty_like(crd_d), "v": torch.empty_like(v32),
             "x": torch.empty_like(xd), "X": torch.empty_like(Xd), "y": torch.empty_like(y), "Y": torch.empty_like(Y)}
        B["A"] = spd.CSR(B["pos"], B["crd"], B["v"], (n, n))
        bufs.append(B)
    s_in, s_comp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev_in, ev_done, ev_free = [ev(), ev()], [ev(), ev()], [ev(), ev()]
    used = [False, False]

    def e2e_step(k):
        b = k % 2
        B = bufs[b]
        with torch.cuda.stream(s_in):
            if used[b]:
                s_in.wait_event(ev_done[b])  # the kernels two steps back have read this set
            for name, h in ins:
                B[name].copy_(h, non_blocking=True)
            ev_in[b].record(s_in)
        with torch.cuda.stream(s_comp):
            s_comp.wait_event(ev_in[b])
            if used[b]:
                s_comp.wait_event(ev_free[b])  # and its results have left the device
            spd.spmv(B["A"], B["x"], B["y"], split=sp_v, tune=tu_v, ws=ws_spmv)
            spd.spmm(B["A"], B["X"], B["Y"], split=sp_m, tune=tu_m, ws=ws_spmm)
            ev_done[b].record(s_comp)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_done[b])
            h_y.copy_(B["y"], non_blocking=True)
            h_Y.copy_(B["Y"], non_blocking=True)
            ev_free[b].record(s_out)
        used[b] = True

    for k in range(2):
        e2e_step(k)
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record(s_in)
    for k in range(args.e2e_steps):
        e2e_step(k)
    e1.record(s_out)  # after the last copy out, which every earlier operation precedes
    torch.cuda.synchronize()
    e2e_s = e0.elapsed_time(e1) / 1e3
    e2e_units, e2e_secs = aggregate(2.0 * nnz * args.e2e_steps, e2e_s)
    del bufs

    # ---------------- CPU oracle on a bounded row sample (rank 0, N = 1 only)
    cpu = cpu_threaded = None
    if rank == 0 and ws == 1:
        cpu, cpu_threaded = cpu_baseline(A, x32, X32, args.cpu_budget)

    rows_out = {}
    wanted = {"cfg1", "sddmm", "backward", "csf", "batched", "banded", "spadd3", "colblock"} if args.rows == "all" else \
        (set() if args.rows == "none" else set(args.rows.split(",")))
    for name, fn in (("cfg1", lambda: row_cfg1(hbm)), ("backward", lambda: row_backward(A, X32, hbm)),
                     ("sddmm", lambda: row_sddmm(hbm)), ("csf", lambda: row_csf(hbm)),
                     ("batched", lambda: row_batched(hbm)), ("banded", lambda: row_banded(hbm)),
                     ("spadd3", lambda: row_spadd3(A, hbm)), ("colblock", lambda: row_colblock(A, X32, hbm))):
        if name not in wanted:
            continue
        if name == "backward":
            del Ad, v32, Xd, Y
            torch.cuda.empty_cache()
        try:
            t_row = time.time()
            rows_out[name] = fn()
            rows_out[name]["wall_s"] = round(time.time() - t_row, 1)
        except Exception as exc:  # a failing row is reported, the headline line still prints
            rows_out[name] = {"failed": "%s: %s" % (type(exc).__name__, exc)}

    clk = clocks.summary()
    props = torch.cuda.get_device_properties(dev)
    sm_count = props.multi_processor_count
    l2_bytes = getattr(props, "L2_cache_size", None)
    # binary32 CUDA-core ridge: 128 FMA lanes per SM, 2 flops each, at the sampled clock
    ridge_mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz")
    fp32_ridge = (2 * 128 * sm_count * ridge_mhz * 1e6 / (hbm * 1e9)) if ridge_mhz else None
    if rank == 0:
        line = {
            "metric": "nonzeros/s",
            "value": value,
            "unit": "nnz/s",
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_per_step,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic",
            "config": {
                "workload": workload_name(args.scale),
                "nrows": n, "nnz": nnz, "L": L_COLS, "split": {"spmv": sp_v, "spmm": sp_m},
                "tune": {"spmv": tu_v, "spmm": tu_m},
                "units": "nonzeros processed (2 x nnz per step)",
                "l2": "inputs larger than L2 (X is %.2f GB, the matrix %.2f GB); no flush" % (X32.nbytes / 1e9, (A.crd.nbytes + nnz * 4) / 1e9),
                "parallelism": "replicas: every rank runs its own problem (no collective)",
                "generate_s": round(gen_s, 1),
            },
            "kernel_ms": {"spmv": round(spmv_ms, 4), "spmm": round(spmm_ms, 4)},
            "call_ms": call_ms,
            "roofline": {
                "bound": "hbm",
                "kernel": "spd_spmm (partition + spmm_warp_kernel + carry fix-up), binary32, %s split" % sp_m,
                "achieved": round(spmm_gbs, 1),
                "peak": hbm,
                "peak_nominal": HBM_NOMINAL_GBS,
                "frac_nominal": round(spmm_gbs / HBM_NOMINAL_GBS, 4),
                "intensity_flop_per_byte": round(2.0 * L_COLS * nnz / spmm_bytes, 3),
                "fp32_ridge_flop_per_byte": round(fp32_ridge, 2) if fp32_ridge else None,
                "sm_count": sm_count,
                "l2_bytes": l2_bytes,
                "peak_kind": peak_kind,
                "unit": "GB/s",
                "frac": round(spmm_gbs / hbm, 4),
                "traffic": (spmm_rec or {}).get("dram_bytes"),
                # the recorded DRAM bytes of the warp kernel over the whole call's mean time
                # (partition and fix-up included, so a lower bound on the kernel's own rate)
                "traffic_achieved": round(spmm_rec["dram_bytes"] / (spmm_ms * 1e-3) / 1e9, 1) if spmm_rec else None,
                "traffic_frac": round(spmm_rec["dram_bytes"] / (spmm_ms * 1e-3) / 1e9 / hbm, 4) if spmm_rec else None,
                "traffic_per_algorithmic_byte": round(spmm_rec["dram_bytes"] / spmm_bytes, 3) if spmm_rec else None,
                "l2_hit_pct": (spmm_rec or {}).get("l2_hit_pct"),
                "traffic_source": "profiles/traffic.json (ncu dram__bytes_read.sum + dram__bytes_write.sum and "
                                  "lts__t_sector_hit_rate.pct of one spmm_warp_kernel launch on this workload)",
                "algorithmic_bytes": spmm_bytes,
                "spmv_achieved": round(spmv_bytes / (spmv_ms * 1e-3) / 1e9, 1),
                "spmv_frac": round(spmv_bytes / (spmv_ms * 1e-3) / 1e9 / hbm, 4),
                "spmv_traffic": (spmv_rec or {}).get("dram_bytes"),
                "spmv_l2_hit_pct": (spmv_rec or {}).get("l2_hit_pct"),
            },
            "error": step_err,
            "e2e": {"value": e2e_units / e2e_secs, "unit": "nnz/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": args.e2e_steps},
            "gpu_launches": launches,
            "clocks": clk,
            "cpu_baseline": cpu,
            "cpu_baseline_threaded": cpu_threaded,
            "variants": variants,
            "autotune": {"spmm": spmm_table, "spmv": spmv_table},
            "rows": rows_out,
        }
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- other rows

def _time_ms(fn, reps=5, warm=2):
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _entry(ms, units, nbytes, hbm, unit_name="nnz"):
    return {"ms": round(ms, 4), unit_name + "_per_s": units / (ms * 1e-3),
            "algorithmic_GBps": round(nbytes / (ms * 1e-3) / 1e9, 1), "hbm_frac": round(nbytes / (ms * 1e-3) / 1e9 / hbm, 4)}


def _rounded(a, dt):
    import torch
    return torch.as_tensor(np.asarray(a)).to(dt).double().numpy()


def row_cfg1(hbm):
    """SpMV on the 4096 x 4096 uniform matrix (16 per row), binary64: latency-bound;
    timed as a replayed CUDA graph of the call."""
    import torch
    import oracle
    import spd_synth
    import paper_2207_13901_gb300 as spd
    A = spd_synth.uniform_csr(4096, 4096, 16, seed=0)
    x = spd_synth.uniform(4096, seed=2)
    dA = spd.CSR.from_host(A.pos, A.crd, A.vals, (4096, 4096), dtype=torch.float64)
    xd = torch.as_tensor(x).cuda()
    out = {}
    for split in ("nnz", "row"):
        y = torch.empty(4096, dtype=torch.float64, device="cuda")
        ws = torch.empty(max(spd.csr_workspace_size(0, dA, split), 1), dtype=torch.uint8, device="cuda")
        spd.spmv(dA, xd, y, split=split, ws=ws)
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            spd.spmv(dA, xd, y, split=split, ws=ws)
        torch.cuda.current_stream().wait_stream(s)
        with torch.cuda.graph(g):
            for _ in range(20):
                spd.spmv(dA, xd, y, split=split, ws=ws)
        ms = _time_ms(lambda: g.replay(), reps=20) / 20
        ref = oracle.spmv(A.pos, A.crd, A.vals, x, accurate=True)
        sc = oracle.spmv(A.pos, A.crd, np.abs(A.vals), np.abs(x))
        e = _entry(ms, A.nnz, algorithmic_bytes("spmv", 4096, A.nnz, 8, 8, 8), hbm)
        e["us"] = round(ms * 1e3, 2)
        e["error"] = error_stats(y.cpu().numpy(), ref, sc)
        out["spmv_f64_" + split] = e
    t = time.perf_counter()
    for _ in range(20):
        oracle.spmv(A.pos, A.crd, A.vals, x)
    dt = (time.perf_counter() - t) / 20
    out["oracle"] = {"nnz_per_s": A.nnz / dt, "cores": 1, "sample": "whole matrix"}
    return out


def row_spadd3(A, hbm):
    """SpAdd3 A = B + C + D on the 2^22 R-MAT: B is the matrix, C and D its columns
    shifted by 1 and 2 (the paper's way of making extra operands) with their own values;
    two-phase assembly, both phases timed (the symbolic one includes its host read of
    nnz(A)); binary32 and binary64; A checked in full against the oracle."""
    import torch
    import oracle
    import spd_synth
    import paper_2207_13901_gb300 as spd
    t0 = time.time()
    n = A.nrows
    ops = [A, spd_synth.shifted_csr(A, 1, seed=11), spd_synth.shifted_csr(A, 2, seed=12)]
    nin = sum(M.nnz for M in ops)
    out = {"inputs_nnz": nin, "generate_s": round(time.time() - t0, 1)}
    for name, dt in (("f32", torch.float32), ("f64", torch.float64)):
        d = [spd.CSR.from_host(M.pos, M.crd, M.vals, (n, n), dtype=dt) for M in ops]
        s = d[0].vals.element_size()
        R = spd.spadd3(*d)  # warm-up, and the result checked below
        ms_total = _time_ms(lambda: spd.spadd3(*d), reps=5, warm=1)
        sym = spd.spadd3_symbolic(*d)
        ms_sym = _time_ms(lambda: spd.spadd3_symbolic(*d), reps=5, warm=1)
        ms_num = _time_ms(lambda: spd.spadd3_numeric(sym, *d), reps=5, warm=1)
        nnz_a = R.nnz
        nbytes = 3 * 4 * (n + 1) + (4 + s) * nin + 4 * (n + 1) + (4 + R.vals.element_size()) * nnz_a
        e = _entry(ms_total, nin, nbytes, hbm)
        e["nnz_A"] = nnz_a
        e["symbolic_ms"] = round(ms_sym, 3)  # counts, scans and the host read of nnz(A)
        e["numeric_ms"] = round(ms_num, 3)
        rops = [spd_synth.CSR(n, n, M.pos, M.crd, _rounded(M.vals, dt)) for M in ops]
        t = time.perf_counter()
        ap, ac, av = oracle.spadd3(*rops)
        t_oracle = time.perf_counter() - t
        _, _, sc = oracle.spadd3(*[spd_synth.CSR(n, n, M.pos, M.crd, np.abs(M.vals)) for M in rops])
        e["structure_bit_exact"] = bool(np.array_equal(R.pos.cpu().numpy(), ap) and np.array_equal(R.crd.cpu().numpy(), ac))
        e["error"] = error_stats(R.vals.double().cpu().numpy(), av, sc)
        out["spadd3_" + name] = e
        out["oracle"] = {"nnz_per_s": nin / t_oracle, "cores": 1, "sample": "the whole problem, binary64"}
        del d, R
        torch.cuda.empty_cache()
    return out


def row_colblock(A, X32, hbm):
    """SpMM (L = 128, binary32) over value-range column blocks of A (a universe partition
    of the Compressed level) against the plain SpMM, on two matrices: the 2^22 R-MAT
    (square: every block costs a pass over Y as large as X) and a wide 2^18 x 2^23 matrix
    with 256 uniform columns per row (X is 4.3 GB, Y 134 MB: blocks of X fit in L2 and
    the extra passes over Y are cheap)."""
    import torch
    import oracle
    import spd_synth
    import paper_2207_13901_gb300 as spd
    t0 = time.time()
    W = spd_synth.uniform_csr(1 << 18, 1 << 23, 256, seed=9)
    XW = spd_synth.uniform((W.ncols, L_COLS), seed=10, dtype=np.float32)
    out = {"wide": {"nrows": W.nrows, "ncols": W.ncols, "nnz": W.nnz}, "generate_s": round(time.time() - t0, 1)}
    rng = np.random.default_rng(8)
    for name, M, Xh, blocks in (("rmat22", A, X32, (4, 32)), ("wide", W, XW, (16, 64))):
        dM = spd.CSR.from_host(M.pos, M.crd, M.vals, (M.nrows, M.ncols), dtype=torch.float32)
        Xd = torch.from_numpy(Xh).cuda()
        Y = torch.empty((M.nrows, L_COLS), dtype=torch.float32, device="cuda")
        nb = 4 * (M.nrows + 1) + 8 * M.nnz + 4 * L_COLS * (M.ncols + M.nrows)  # X read once, Y written once
        res = {"plain": _entry(_time_ms(lambda: spd.spmm(dM, Xd, Y), reps=5), M.nnz, nb, hbm)}
        sel = np.unique(rng.integers(0, M.nrows, 300))
        vr, Xr = _rounded(M.vals, torch.float32), Xh.astype(np.float64)
        ref = oracle.spmm(M.pos, M.crd, vr, Xr, sel=sel, accurate=True)
        sc = oracle.spmm(M.pos, M.crd, np.abs(vr), np.abs(Xr), sel=sel)
        for nblk in blocks:
            t = time.perf_counter()
            spd.column_blocks(dM, nblk=nblk)
            torch.cuda.synchronize()
            build_ms = (time.perf_counter() - t) * 1e3
            ms = _time_ms(lambda: spd.spmm_column_blocked(dM, Xd, Y, nblk=nblk), reps=5)
            e = _entry(ms, M.nnz, nb, hbm)
            e["blocks_build_ms"] = round(build_ms, 1)
            e["error"] = error_stats(Y.double().cpu().numpy()[sel], ref, sc)
            res["blocks%d" % nblk] = e
        out[name] = dict(out.get(name, {}), **res)
        del dM, Xd, Y
        torch.cuda.empty_cache()
    return out


def row_banded(hbm):
    """SpMV on a banded matrix of about 700 million nonzeros (21.2M rows, 33 per row):
    the synthetic workload of the paper's weak-scaling study, with perfect locality of
    the x gathers, so it bounds the HBM fraction the SpMV kernel can reach."""
    import torch
    import oracle
    import spd_synth
    import paper_2207_13901_gb300 as spd
    t0 = time.time()
    n, w = 21_212_122, 16
    A = spd_synth.banded_csr(n, w, seed=0, value_dtype=np.float32)
    x = spd_synth.uniform(n, seed=2, dtype=np.float32)
    out = {"nrows": n, "half_width": w, "nnz": A.nnz, "generate_s": round(time.time() - t0, 1)}
    rng = np.random.default_rng(5)
    sel = np.unique(np.concatenate([rng.integers(0, n, 2000), [0, n - 1]]))
    # the sampled rows as their own CSR (the oracle then reads only those rows)
    lens = (A.pos[sel + 1] - A.pos[sel]).astype(np.int64)
    spos = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    idx = np.concatenate([np.arange(A.pos[r], A.pos[r + 1]) for r in sel])
    scrd, svals = A.crd[idx], A.vals[idx].astype(np.float64)
    for name, dt in (("f32", torch.float32), ("f64", torch.float64), ("bf16", torch.bfloat16)):
        dA = spd.CSR.from_host(A.pos, A.crd, A.vals, (n, n), dtype=dt)
        xd = torch.from_numpy(x).cuda().to(dt)
        y = torch.empty(n, dtype=spd.result_dtype(dt), device="cuda")
        s = dA.vals.element_size()
        for split, form in (("nnz", 1), ("nnz", 2), ("row", 1)):
            tune = {"form": form}
            ms = _time_ms(lambda: spd.spmv(dA, xd, y, split=split, tune=tune), reps=10)
            e = _entry(ms, A.nnz, algorithmic_bytes("spmv", n, A.nnz, s, s, y.element_size()), hbm)
            vr, xr = _rounded(svals, dt), _rounded(x.astype(np.float64), dt)
            ref = oracle.spmv(spos, scrd, vr, xr, accurate=True)
            sc = oracle.spmv(spos, scrd, np.abs(vr), np.abs(xr))
            e["error"] = error_stats(y[torch.from_numpy(sel).cuda()].double().cpu().numpy(), ref, sc)
            e["ncu"] = recorded_traffic("spmv", "banded_%s_form%d" % (name, form)) if split == "nnz" else None
            out["spmv_%s_%s_form%d" % (name, split, form)] = e
        del dA, xd, y
        torch.cuda.empty_cache()
    x64 = x.astype(np.float64)
    t = time.perf_counter()
    for _ in range(20):
        oracle.spmv(spos, scrd, svals, x64)
    out["oracle"] = {"nnz_per_s": 20 * scrd.shape[0] / (time.perf_counter() - t), "cores": 1,
                     "sample": "%d rows (%d nonzeros), binary64" % (sel.size, scrd.shape[0])}
    out["wall_s"] = round(time.time() - t0, 1)
    return out


def row_sddmm(hbm):
    """SDDMM on the 2^20-row R-MAT (32 samples per row), K in {32, 128, 256}, binary32 and
    bfloat16, C and D N(0,1); autotuned split/piece size per case."""
    import torch
    import oracle
    import spd_synth
    import paper_2207_13901_gb300 as spd
    from paper_2207_13901_gb300.autotune import Autotuner
    import tempfile
    B = spd_synth.rmat_csr(20, 32, seed=0)
    n, nnz = B.nrows, B.nnz
    rng = np.random.default_rng(0)
    sel = np.unique(rng.integers(0, nnz, 3000))
    tuner = Autotuner(path=os.path.join(tempfile.mkdtemp(prefix="spd_tune_"), "a.json"), reps=2)
    out = {"nrows": n, "nnz": nnz}
    for K in (32, 128, 256):
        C = spd_synth.normal((n, K), seed=10 + K, dtype=np.float32)
        D = spd_synth.normal((n, K), seed=20 + K, dtype=np.float32)
        for name, dt in (("f32", torch.float32), ("bf16", torch.bfloat16)):
            dB = spd.CSR.from_host(B.pos, B.crd, B.vals, (n, n), dtype=dt)
            Cd, Dd = torch.from_numpy(C).cuda().to(dt), torch.from_numpy(D).cuda().to(dt)
            res = torch.empty(nnz, dtype=torch.float32, device="cuda")
            best = tuner.sddmm(dB, Cd, Dd, force=True)
            wsb = torch.empty(max(spd.csr_workspace_size(3, dB, best["split"], K, best["tune"], vtype=dt), 1),
                              dtype=torch.uint8, device="cuda")
            ms = _time_ms(lambda: spd.sddmm(dB, Cd, Dd, res, split=best["split"], tune=best["tune"], ws=wsb))
            s = 2 if dt == torch.bfloat16 else 4
            nb = 4 * (n + 1) + (4 + s + 4) * nnz + s * 2 * n * K
            e = _entry(ms, nnz, nb, hbm)
            e["tune"] = best
            vr, Cr, Dr = _rounded(B.vals, dt), _rounded(C, dt), _rounded(D, dt)
            ref = oracle.sddmm(B.pos, B.crd, vr, Cr, Dr, sel=sel, accurate=True)
            sc = oracle.sddmm(B.pos, B.crd, np.abs(vr), np.abs(Cr), np.abs(Dr), sel=sel)
            e["error"] = error_stats(res.double().cpu().numpy()[sel], ref, sc)
            e["ncu"] = recorded_traffic("sddmm", "rmat20_k%d_%s" % (K, name))
            out["K%d_%s" % (K, name)] = e
            del dB, Cd, Dd, res
        if K == 128:
            t = time.perf_counter()
            oracle.sddmm(B.pos, B.crd, B.vals, C.astype(np.float64), D.astype(np.float64), sel=sel)
            dt_o = time.perf_counter() - t
            out["oracle_K128"] = {"nnz_per_s": sel.size / dt_o, "cores": 1, "sample": "%d sampled positions" % sel.size}
    torch.cuda.empty_cache()
    return out


def row_backward(A, X32, hbm):
    """SpMM backward on the 2^22 R-MAT with L = 128 in binary32: dvals = SDDMM(pattern,
    dY, X) and dX = SpMM^T(A, dY) (torch.autograd through the hand-written backward; dX
    as an SpMM over A^T, whose structure is built once per pattern, and, for
    comparison, by atomic scatter)."""
    import torch
    import oracle
    import paper_2207_13901_gb300 as spd
    n, nnz, L = A.nrows, A.nnz, X32.shape[1]
    dA = spd.CSR.from_host(A.pos, A.crd, A.vals, (n, n), dtype=torch.float32)
    vals = dA.vals.clone().requires_grad_(True)
    Xd = torch.from_numpy(X32).cuda().requires_grad_(True)
    import spd_synth
    W = torch.from_numpy(spd_synth.uniform((n, L), seed=7, dtype=np.float32)).cuda()
    pattern = dA.with_vals(None)

    def fwd_bwd():
        vals.grad = None
        Xd.grad = None
        Y = spd.autograd.spmm(pattern.with_vals(vals), Xd)
        Y.backward(W)

    ms_transpose = _time_ms(lambda: spd.transpose(dA), reps=3, warm=1)  # once per pattern
    ms_all = _time_ms(fwd_bwd, reps=3, warm=1)  # dX over the cached A^T
    ms_sddmm = _time_ms(lambda: spd.sddmm(pattern, W, Xd.detach()), reps=3, warm=1)
    ms_spmmt = _time_ms(lambda: spd.spmm_t(dA, W), reps=3, warm=1)
    ms_spmmt_tr = _time_ms(lambda: spd.spmm_t(dA, W, method="transpose"), reps=3, warm=1)
    b_sddmm = 4 * (n + 1) + 8 * nnz + 4 * 2 * n * L
    b_spmmt = 4 * (n + 1) + 8 * nnz + 4 * n * L + 4 * n * L
    b_spmmt_tr = b_spmmt + 12 * nnz  # plus the value gather into A^T's order
    out = {"forward_backward_ms": round(ms_all, 3),
           "transpose_build_ms": round(ms_transpose, 3),
           "sddmm_dvals": _entry(ms_sddmm, nnz, b_sddmm, hbm),
           "spmm_t_dX_atomic": _entry(ms_spmmt, nnz, b_spmmt, hbm),
           "spmm_t_dX_transpose": _entry(ms_spmmt_tr, nnz, b_spmmt_tr, hbm)}
    rng = np.random.default_rng(1)
    sel = np.unique(rng.integers(0, nnz, 2000))
    Wh = W.cpu().numpy().astype(np.float64)
    gv = vals.grad.double().cpu().numpy()
    ref = oracle.sddmm(A.pos, A.crd, None, Wh, X32.astype(np.float64), sel=sel, accurate=True)
    sc = oracle.sddmm(A.pos, A.crd, None, np.abs(Wh), np.abs(X32.astype(np.float64)), sel=sel)
    out["sddmm_dvals"]["error"] = error_stats(gv[sel], ref, sc)
    # dX rows j of A^T W, from the oracle's own transposition of A
    t_pos, t_crd, perm = oracle.csr_transpose(A.pos, A.crd, n)
    jsel = np.unique(np.concatenate([rng.integers(0, n, 600), np.argsort(np.diff(t_pos))[-5:]]))
    vr = A.vals.astype(np.float32).astype(np.float64)[perm]
    ref = oracle.spmm(t_pos, t_crd, vr, Wh, sel=jsel, accurate=True)
    sc = oracle.spmm(t_pos, t_crd, np.abs(vr), np.abs(Wh), sel=jsel)
    gx = Xd.grad.double().cpu().numpy()[jsel]
    out["spmm_t_dX_transpose"]["error"] = error_stats(gx, ref, sc)
    t = time.perf_counter()
    oracle.spmm(t_pos, t_crd, vr, Wh, sel=jsel)
    onnz = int(np.diff(t_pos)[jsel].sum())
    out["oracle"] = {"nnz_per_s": onnz / (time.perf_counter() - t), "cores": 1,
                     "sample": "dX rows %d (%d nonzeros of A^T), binary64" % (jsel.size, onnz)}
    del dA, vals, Xd, W
    torch.cuda.empty_cache()
    return out


def row_csf(hbm):
    """SpTTV and SpMTTKRP (R = 32, 64) on the 2^17-cubed Zipf(1.1) CSF tensor with 50M
    nonzeros, binary32 and bfloat16."""
    import torch
    import oracle
    import spd_synth
    import paper_2207_13901_gb300 as spd
    t0 = time.time()
    T = spd_synth.zipf_csf3((1 << 17,) * 3, 50_000_000, 1.1, seed=0)
    out = {"nnz": T.nnz, "nfib": T.nfib, "generate_s": round(time.time() - t0, 1)}
    I, J, K = T.dims
    rng = np.random.default_rng(0)
    fsel = np.unique(np.concatenate([rng.integers(0, T.nfib, 3000), np.argsort(np.diff(T.pos2))[-3:]]))
    ssel = np.unique(rng.integers(2, I, 40))  # slices 0 and 1 hold millions of entries
    c = spd_synth.normal(K, seed=31, dtype=np.float32)
    for name, dt in (("f32", torch.float32), ("bf16", torch.bfloat16)):
        dT = spd.CSF3.from_host(T.pos1, T.crd1, T.pos2, T.crd2, T.vals, T.dims, dtype=dt)
        s = 2 if dt == torch.bfloat16 else 4
        vr = _rounded(T.vals, dt)
        cd = torch.from_numpy(c).cuda().to(dt)
        o = torch.empty(T.nfib, dtype=torch.float32, device="cuda")
        for split in ("nnz", "row"):
            ws = torch.empty(max(spd.csf3_workspace_size(4, dT, split), 1), dtype=torch.uint8, device="cuda")
            ms = _time_ms(lambda: spd.spttv(dT, cd, o, split=split, ws=ws))
            nb = 4 * (T.nfib + 1) + (4 + s) * T.nnz + s * K + 4 * T.nfib
            e = _entry(ms, T.nnz, nb, hbm)
            cr = _rounded(c, dt)
            ref = oracle.spttv(T.pos1, T.crd1, T.pos2, T.crd2, vr, cr, sel=fsel, accurate=True)
            sc = oracle.spttv(T.pos1, T.crd1, T.pos2, T.crd2, np.abs(vr), np.abs(cr), sel=fsel)
            e["error"] = error_stats(o.double().cpu().numpy()[fsel], ref, sc)
            e["ncu"] = recorded_traffic("spttv", "zipf_%s_form1" % name) if split == "nnz" else None
            out["spttv_%s_%s" % (name, split)] = e
        for R in (32, 64):
            C = spd_synth.normal((J, R), seed=40 + R, dtype=np.float32)
            D = spd_synth.normal((K, R), seed=50 + R, dtype=np.float32)
            Cd, Dd = torch.from_numpy(C).cuda().to(dt), torch.from_numpy(D).cuda().to(dt)
            Ao = torch.empty((I, R), dtype=torch.float32, device="cuda")
            for split in ("nnz", "row"):
                ws = torch.empty(max(spd.csf3_workspace_size(5, dT, split, R), 1), dtype=torch.uint8, device="cuda")
                ms = _time_ms(lambda: spd.spmttkrp(dT, Cd, Dd, Ao, split=split, ws=ws))
                nb = 4 * (I + 1) + 4 * T.nfib + 4 * (T.nfib + 1) + (4 + s) * T.nnz + s * (J + K) * R + 4 * I * R
                e = _entry(ms, T.nnz, nb, hbm)
                Cr, Dr = _rounded(C, dt), _rounded(D, dt)
                ref = oracle.spmttkrp(T.pos1, T.crd1, T.pos2, T.crd2, vr, Cr, Dr, sel=ssel, accurate=True)
                sc = oracle.spmttkrp(T.pos1, T.crd1, T.pos2, T.crd2, np.abs(vr), np.abs(Cr), np.abs(Dr), sel=ssel)
                e["error"] = error_stats(Ao.double().cpu().numpy()[ssel], ref, sc)
                e["ncu"] = recorded_traffic("spmttkrp", "zipf_r%d_%s" % (R, name)) if split == "nnz" else None
                out["spmttkrp_R%d_%s_%s" % (R, name, split)] = e
            del Cd, Dd, Ao
        del dT, o
    t = time.perf_counter()
    oracle.spttv(T.pos1, T.crd1, T.pos2, T.crd2, T.vals, c.astype(np.float64), sel=fsel)
    dt_o = time.perf_counter() - t
    snnz = int(np.diff(T.pos2)[fsel].sum())
    out["oracle_spttv"] = {"nnz_per_s": snnz / dt_o, "cores": 1, "sample": "%d fibers" % fsel.size}
    torch.cuda.empty_cache()
    return out


def row_batched(hbm):
    """512 square CSR matrices (rows log-uniform in [1e3, 1e5], 4..64 uniform columns per
    row), L = 64, binary32 and bfloat16: one persistent launch replayed from a CUDA graph
    (policy and piece size autotuned) against 512 plain per-matrix launches."""
    import torch
    import oracle
    import spd_synth
    import paper_2207_13901_gb300 as spd
    t0 = time.time()
    mats = spd_synth.batched_uniform_csr(512, 1e3, 1e5, 4, 64, seed=0)
    L = 64
    rows = sum(A.nrows for A in mats)
    nnz = sum(A.nnz for A in mats)
    out = {"matrices": len(mats), "rows": rows, "nnz": nnz, "generate_s": round(time.time() - t0, 1)}
    rng = np.random.default_rng(0)
    Xh = [spd_synth.uniform((A.ncols, L), seed=1000 + m, dtype=np.float32) for m, A in enumerate(mats)]
    check = sorted(set(rng.integers(0, len(mats), 6).tolist()))
    for name, dt in (("f32", torch.float32), ("bf16", torch.bfloat16)):
        dmats = [spd.CSR.from_host(A.pos, A.crd, A.vals, (A.nrows, A.ncols), dtype=dt) for A in mats]
        Xs = [torch.from_numpy(X).cuda().to(dt) for X in Xh]
        batch = spd.SpMMBatch(dmats, Xs)
        best = batch.autotune(policies=("row", "auto"), units=(512, 1024, 2048), reps=3)
        batch.capture()
        s = 2 if dt == torch.bfloat16 else 4
        nb = sum(4 * (A.nrows + 1) + (4 + s) * A.nnz + (s + 4) * A.nrows * L for A in mats)
        ms_graph = _time_ms(batch.replay, reps=10)
        ms_sep = _time_ms(lambda: batch.run_separately("row"), reps=3)
        e = _entry(ms_graph, nnz, nb, hbm)
        e["tune"] = best
        e["separate_launches_ms"] = round(ms_sep, 3)
        e["speedup_vs_separate"] = round(ms_sep / ms_graph, 3)
        batch.replay()
        torch.cuda.synchronize()
        worst = 0.0
        for m in check:
            A = mats[m]
            sel = np.unique(rng.integers(0, A.nrows, 200))
            vr, Xr = _rounded(A.vals, dt), _rounded(Xh[m], dt)
            ref = oracle.spmm(A.pos, A.crd, vr, Xr, sel=sel, accurate=True)
            sc = oracle.spmm(A.pos, A.crd, np.abs(vr), np.abs(Xr), sel=sel)
            worst = max(worst, error_stats(batch.Ys[m].double().cpu().numpy()[sel], ref, sc)["max"])
        e["error"] = {"max": worst, "matrices_checked": check}
        out[name] = e
        del dmats, Xs, batch
        torch.cuda.empty_cache()
    # the oracle on whole matrices of the batch (one thread)
    t = time.perf_counter()
    onnz = 0
    for m in check:
        A = mats[m]
        oracle.spmm(A.pos, A.crd, A.vals, Xh[m].astype(np.float64))
        onnz += A.nnz
    out["oracle"] = {"nnz_per_s": onnz / (time.perf_counter() - t), "cores": 1,
                     "sample": "%d whole matrices of the batch, binary64" % len(check)}
    return out


# ----------------------------------------------------------------------------- CPU oracle

def cpu_sample(A, budget_s, per_nnz_s):
    """Every k-th row, k chosen so SpMV + SpMM over the sample takes about budget_s."""
    want = max(1000, int(budget_s / max(per_nnz_s, 1e-12)))
    k = max(1, int(round(A.nnz / want)))
    return np.arange(0, A.nrows, k, dtype=np.int64), k


def cpu_calibrate(A, x, X):
    import oracle
    sel = np.arange(0, A.nrows, max(1, A.nrows // 2000), dtype=np.int64)
    snnz = int(np.diff(A.pos)[sel].sum())
    v = A.vals
    t = time.perf_counter()
    oracle.spmv(A.pos, A.crd, v, x, sel=sel)
    oracle.spmm(A.pos, A.crd, v, X, sel=sel)
    return (time.perf_counter() - t) / max(snnz, 1)


def host_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def oracle_rows_threaded(A, x, X, sel, threads):
    """The oracle's SpMV and SpMM over the rows `sel`, dealt round-robin to `threads` host
    threads (the oracle's C loops run without the interpreter lock; every row is summed
    in the same order as in one thread, so the results are the same). Returns seconds."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    parts = [sel[t::threads] for t in range(threads)]

    def work(rows):
        oracle.spmv(A.pos, A.crd, A.vals, x, sel=rows)
        oracle.spmm(A.pos, A.crd, A.vals, X, sel=rows)

    with ThreadPoolExecutor(max_workers=threads) as ex:
        t = time.perf_counter()
        list(ex.map(work, parts))
        return time.perf_counter() - t


def cpu_baseline(A, x32, X32, budget):
    """The oracle on a row sample: one thread (`cpu_baseline`) and, on the same rows, one
    thread per host core (`threaded`)."""
    import oracle
    x = x32.astype(np.float64)
    X = X32.astype(np.float64)
    per = cpu_calibrate(A, x, X)
    sel, k = cpu_sample(A, budget, per)
    snnz = int(np.diff(A.pos)[sel].sum())
    t = time.perf_counter()
    oracle.spmv(A.pos, A.crd, A.vals, x, sel=sel)
    oracle.spmm(A.pos, A.crd, A.vals, X, sel=sel)
    dt = time.perf_counter() - t
    what = "every %d-th row of the matrix (%d rows, %d nonzeros), SpMV + SpMM(L=128) in binary64" % (k, sel.size, snnz)
    T = host_threads()
    dt_t = oracle_rows_threaded(A, x, X, sel, T)
    return ({"value": 2.0 * snnz / dt, "unit": "nnz/s", "cores": 1, "kind": "oracle",
             "sample": "%s, single thread, %.1f s" % (what, dt)},
            {"value": 2.0 * snnz / dt_t, "unit": "nnz/s", "cores": T, "kind": "oracle",
             "sample": "%s, rows dealt to %d host threads, %.1f s" % (what, T, dt_t)})


def run_reference(args):
    ws, rank, local = dist_env()
    if ws > 1 and rank != 0:
        return
    import oracle
    oracle.build()
    A, x32, X32, _ = workload(args.scale)
    x = x32.astype(np.float64)
    X = X32.astype(np.float64)
    per = cpu_calibrate(A, x, X)
    budget = 120.0 / max(1, args.steps + args.warmup)  # whole run within a few minutes
    sel, k = cpu_sample(A, budget, per)
    snnz = int(np.diff(A.pos)[sel].sum())
    T = host_threads()
    for _ in range(args.warmup):
        oracle_rows_threaded(A, x, X, sel, T)
    dt = 0.0
    for _ in range(args.steps):
        dt += oracle_rows_threaded(A, x, X, sel, T)
    value = 2.0 * snnz * args.steps / dt
    sample = ("every %d-th row (%d rows, %d nonzeros) per step, SpMV + SpMM(L=128) in binary64, rows dealt to %d "
              "host threads" % (k, sel.size, snnz, T))
    print(json.dumps({
        "impl": "reference", "metric": "nonzeros/s", "value": value, "unit": "nnz/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.scale), "nrows": A.nrows, "nnz": A.nnz, "L": L_COLS,
                   "units": "nonzeros processed (2 x nnz per step)",
                   "reference": "the CPU oracle (binary64) on a row sample of the workload: " + sample},
        "cpu_baseline": {"value": value, "unit": "nnz/s", "cores": T, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main(argv=None):
    args = parse_args(argv)
    if args.record_traffic:
        csv_path, kernel, case, tune, command = args.record_traffic
        print(json.dumps(record_traffic(csv_path, kernel, case, tune, command)))
    elif args.impl == "reference":
        run_reference(args)
    elif args.case:
        run_case(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
