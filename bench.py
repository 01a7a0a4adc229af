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
    p.add_argument("--e2e-steps", type=int, default=5)
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


def algorithmic_bytes(kernel: str, n: int, nnz: int, vbytes: int, xbytes: int, ybytes: int, L: int = L_COLS) -> int:
    """Bytes every kernel must move at least once: pos, crd, values, the dense input
    read once and the output written once."""
    base = 4 * (n + 1) + 4 * nnz + vbytes * nnz
    if kernel == "spmv":
        return base + xbytes * n + ybytes * n
    return base + xbytes * n * L + ybytes * n * L


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
    spmv_ms = statistics.mean(m[0].elapsed_time(m[1]) for m in marks)
    spmm_ms = statistics.mean(m[1].elapsed_time(m[2]) for m in marks)
    units_local = 2.0 * nnz * args.steps
    units, secs = aggregate(units_local, elapsed)
    value = units / secs
    ms_per_step = secs * 1e3 / args.steps
    per_call = {"nnz": 3, "row": 1}  # partition + kernel + fix-up, or one kernel
    launches = args.steps * (per_call[sp_v] + per_call[sp_m])

    hbm, peak_kind = measured_peaks()
    spmm_bytes = algorithmic_bytes("spmm", n, nnz, 4, 4, 4)
    spmv_bytes = algorithmic_bytes("spmv", n, nnz, 4, 4, 4)
    spmm_gbs = spmm_bytes / (spmm_ms * 1e-3) / 1e9

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
                yh = yv.double().cpu().numpy()
                Yh = np.zeros((n, L_COLS))
                Yh[sel] = Yv[torch.from_numpy(sel).to(dev)].double().cpu().numpy()
                tname = {"f64": "float64", "f32": "float32", "bf16": "bfloat16"}[name]
                res["error"] = errs(tname, yh, Yh)
                variants["%s_%s" % (name, split)] = res
            del vd, xv, Xv, yv, Yv, Av
            torch.cuda.empty_cache()

    # ---------------- end to end through the public API with host buffers
    pin = lambda a: torch.from_numpy(a).pin_memory()
    h_pos, h_crd, h_vals = pin(A.pos), pin(A.crd), torch.from_numpy(vals64).to(torch.float32).pin_memory()
    h_x, h_X = pin(x32), pin(X32)
    h_y = torch.empty(n, dtype=torch.float32).pin_memory()
    h_Y = torch.empty((n, L_COLS), dtype=torch.float32).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in (h_pos, h_crd, h_vals, h_x, h_X))
    d2h = h_y.numel() * 4 + h_Y.numel() * 4

    def e2e_step():
        pos_d.copy_(h_pos, non_blocking=True)
        crd_d.copy_(h_crd, non_blocking=True)
        v32.copy_(h_vals, non_blocking=True)
        xd.copy_(h_x, non_blocking=True)
        Xd.copy_(h_X, non_blocking=True)
        step()
        h_y.copy_(y, non_blocking=True)
        h_Y.copy_(Y, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record(stream)
    for _ in range(args.e2e_steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_s = e0.elapsed_time(e1) / 1e3
    e2e_units, e2e_secs = aggregate(2.0 * nnz * args.e2e_steps, e2e_s)

    # ---------------- CPU oracle on a bounded row sample (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and ws == 1:
        cpu = cpu_baseline(A, x32, X32, args.cpu_budget)

    clk = clocks.summary()
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
                "workload": "SpMV + SpMM(L=128) on R-MAT 2^%d (a=.57,b=.19,c=.19, 16 samples/row, dedup), "
                            "binary32, nnz split (fused non-zero partition), step = partition + SpMV + fix-up + "
                            "SpMM + fix-up" % args.scale,
                "nrows": n, "nnz": nnz, "L": L_COLS, "split": {"spmv": sp_v, "spmm": sp_m},
                "tune": {"spmv": tu_v, "spmm": tu_m},
                "units": "nonzeros processed (2 x nnz per step)",
                "l2": "inputs larger than L2 (X is %.2f GB, the matrix %.2f GB); no flush" % (X32.nbytes / 1e9, (A.crd.nbytes + nnz * 4) / 1e9),
                "parallelism": "replicas: every rank runs its own problem (no collective)",
                "generate_s": round(gen_s, 1),
            },
            "kernel_ms": {"spmv": round(spmv_ms, 4), "spmm": round(spmm_ms, 4)},
            "roofline": {
                "bound": "hbm",
                "kernel": "spd_spmm (partition + spmm_warp_kernel + carry fix-up), binary32, %s split" % sp_m,
                "achieved": round(spmm_gbs, 1),
                "peak": hbm,
                "peak_kind": peak_kind,
                "unit": "GB/s",
                "frac": round(spmm_gbs / hbm, 4),
                "traffic": None,
                "algorithmic_bytes": spmm_bytes,
                "spmv_achieved": round(spmv_bytes / (spmv_ms * 1e-3) / 1e9, 1),
                "spmv_frac": round(spmv_bytes / (spmv_ms * 1e-3) / 1e9 / hbm, 4),
            },
            "error": step_err,
            "e2e": {"value": e2e_units / e2e_secs, "unit": "nnz/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": args.e2e_steps},
            "gpu_launches": launches,
            "clocks": clk,
            "cpu_baseline": cpu,
            "variants": variants,
            "autotune": {"spmm": spmm_table, "spmv": spmv_table},
        }
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


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


def cpu_baseline(A, x32, X32, budget):
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
    return {"value": 2.0 * snnz / dt, "unit": "nnz/s", "cores": 1, "kind": "oracle",
            "sample": "every %d-th row of the matrix (%d rows, %d nonzeros), SpMV + SpMM(L=128) in binary64, "
                      "single thread, %.1f s" % (k, sel.size, snnz, dt)}


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
    for _ in range(args.warmup):
        oracle.spmv(A.pos, A.crd, A.vals, x, sel=sel)
        oracle.spmm(A.pos, A.crd, A.vals, X, sel=sel)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.spmv(A.pos, A.crd, A.vals, x, sel=sel)
        oracle.spmm(A.pos, A.crd, A.vals, X, sel=sel)
    dt = time.perf_counter() - t
    value = 2.0 * snnz * args.steps / dt
    sample = ("every %d-th row (%d rows, %d nonzeros) per step, SpMV + SpMM(L=128) in binary64, single thread"
              % (k, sel.size, snnz))
    print(json.dumps({
        "impl": "reference", "metric": "nonzeros/s", "value": value, "unit": "nnz/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "SpMV + SpMM(L=128) on R-MAT 2^%d, CPU oracle on a row sample" % args.scale},
        "cpu_baseline": {"value": value, "unit": "nnz/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
