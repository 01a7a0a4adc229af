"""Autotuner for the split and tuning of each operation.

For a shape class -- (operation, element type, log2 buckets of rows, nonzeros and the
longest row, dense width, device name) -- every candidate setting (row vs nnz split,
items per work unit, threads per block, rows in flight, SpMM lane shape, SpMV kernel form) is timed with CUDA events on the
caller's operands, and the fastest is kept in a JSON cache (``SPD_AUTOTUNE_CACHE``, by
default ``~/.cache/spd/autotune.json``). Timing runs the real kernels through the C ABI
outside any timed region of the caller; it reads the longest row once with a device
reduction to classify the matrix.
"""
from __future__ import annotations

import json
import math
import os
import threading
from typing import Callable, Dict, List, Optional

import torch

from . import ops

_lock = threading.Lock()


def _bucket(v: int) -> int:
    return 0 if v <= 0 else int(round(math.log2(v)))


def default_cache_path() -> str:
    return os.environ.get("SPD_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "spd", "autotune.json"))


def warp_candidates(include_row: bool = True, inflight: bool = True) -> List[dict]:
    """Settings of the warp-per-unit kernels (SpMM, SpMM^T, SDDMM, SpMTTKRP)."""
    out = []
    for unit in (512, 1024, 2048, 4096):
        for bt in (128, 256, 512):
            for inf in ((4, 8) if inflight else (0,)):
                t = {"unit_items": unit, "block_threads": bt}
                if inf:
                    t["inflight"] = inf
                out.append({"split": "nnz", "tune": t})
    if include_row:
        out.append({"split": "row", "tune": None})
    return out


def spmv_candidates() -> List[dict]:
    """Both splits with both kernel forms of SpMV (block tiles, warp tiles with bulk copies)."""
    return [{"split": split, "tune": {"form": form}} for split in ("nnz", "row") for form in (1, 2)]


class Autotuner:
    def __init__(self, path: Optional[str] = None, reps: int = 3):
        self.path = path or default_cache_path()
        self.reps = reps
        self.cache: Dict[str, dict] = {}
        self.last_table: List[dict] = []
        if os.path.exists(self.path):
            try:
                with open(self.path) as f:
                    self.cache = json.load(f)
            except (OSError, ValueError):
                self.cache = {}

    def save(self) -> None:
        with _lock:
            d = os.path.dirname(self.path)
            if d:
                os.makedirs(d, exist_ok=True)
            tmp = self.path + ".tmp%d" % os.getpid()
            with open(tmp, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)

    @staticmethod
    def shape_key(op: str, A: "ops.CSR", width: int, dtype: torch.dtype) -> str:
        lens = A.pos[1:] - A.pos[:-1]
        maxrow = int(lens.max().item()) if A.shape[0] > 0 else 0
        dev = torch.cuda.get_device_name(A.pos.device)
        return "%s|%s|n%d|nnz%d|max%d|w%d|%s" % (op, str(dtype).replace("torch.", ""), _bucket(A.shape[0]),
                                                _bucket(A.nnz), _bucket(maxrow), width, dev)

    @staticmethod
    def csf_key(op: str, B: "ops.CSF3", width: int, dtype: torch.dtype) -> str:
        """Shape class of a CSF operand: log2 buckets of slices, fibers, entries and the
        largest slice (in entries), with the dense width and the device."""
        ends = B.pos2[B.pos1.long()].long()
        maxsl = int((ends[1:] - ends[:-1]).max().item()) if B.dims[0] > 0 else 0
        dev = torch.cuda.get_device_name(B.pos1.device)
        return "%s|%s|i%d|f%d|nnz%d|max%d|w%d|%s" % (op, str(dtype).replace("torch.", ""), _bucket(B.dims[0]),
                                                     _bucket(B.nfib), _bucket(B.nnz), _bucket(maxsl), width, dev)

    def _time(self, fn: Callable[[], None], reps: int) -> float:
        stream = torch.cuda.current_stream()
        fn()  # warm-up (also allocates the workspace)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def choose(self, key: str, candidates: List[dict], make_fn: Callable[[dict], Callable[[], None]],
               force: bool = False) -> dict:
        """Best candidate for `key` (timed unless cached)."""
        if not force and key in self.cache:
            return self.cache[key]
        table = []
        best = None
        for cand in candidates:
            fn = make_fn(cand)
            reps = 1 if cand["split"] == "row" else self.reps
            ms = self._time(fn, reps)
            table.append({"split": cand["split"], "tune": cand["tune"], "ms": round(ms, 4)})
            if best is None or ms < best["ms"]:
                best = {"split": cand["split"], "tune": cand["tune"], "ms": round(ms, 4)}
        self.last_table = table
        self.cache[key] = best
        self.save()
        return best

    # ---------------------------------------------------------------- operations

    def spmm(self, A: "ops.CSR", X: torch.Tensor, Y: Optional[torch.Tensor] = None, force: bool = False) -> dict:
        Y = Y if Y is not None else torch.empty((A.shape[0], X.shape[1]), dtype=ops.result_dtype(A.dtype), device=X.device)
        key = self.shape_key("spmm", A, X.shape[1], A.dtype)
        cands = warp_candidates(True, inflight=A.dtype != torch.float64)
        if X.shape[1] * X.element_size() < 32 * 16:
            # narrow L: both lane shapes (groups of 16-byte lanes, or 32 narrower lanes)
            cands = [{"split": c["split"], "tune": dict(c["tune"], lane_groups=g) if c["tune"] else None}
                     for c in cands for g in ((1, 2) if c["tune"] else (0,))]
        return self.choose(key, cands, lambda c: (lambda: ops.spmm(A, X, Y, split=c["split"], tune=c["tune"])), force)

    def spmv(self, A: "ops.CSR", x: torch.Tensor, y: Optional[torch.Tensor] = None, force: bool = False) -> dict:
        y = y if y is not None else torch.empty(A.shape[0], dtype=ops.result_dtype(A.dtype), device=x.device)
        key = self.shape_key("spmv", A, 1, A.dtype)
        return self.choose(key, spmv_candidates(),
                           lambda c: (lambda: ops.spmv(A, x, y, split=c["split"], tune=c["tune"])), force)

    def sddmm(self, B: "ops.CSR", C: torch.Tensor, Dnk: torch.Tensor, force: bool = False) -> dict:
        out = torch.empty(B.nnz, dtype=ops.result_dtype(C.dtype), device=C.device)
        key = self.shape_key("sddmm", B, C.shape[1], C.dtype)
        cands = warp_candidates(True, inflight=False)
        if C.dtype == torch.bfloat16:  # CUDA cores or tensor cores
            cands = [{"split": c["split"], "tune": dict(c["tune"] or {}, form=f)} for c in cands for f in (1, 2)]
        return self.choose(key, cands,
                           lambda c: (lambda: ops.sddmm(B, C, Dnk, out, split=c["split"], tune=c["tune"])), force)

    def spmm_t(self, A: "ops.CSR", dY: torch.Tensor, force: bool = False) -> dict:
        dX = torch.empty((A.shape[1], dY.shape[1]), dtype=ops.result_dtype(A.dtype), device=dY.device)
        key = self.shape_key("spmm_t", A, dY.shape[1], A.dtype)
        return self.choose(key, warp_candidates(True, inflight=False),
                           lambda c: (lambda: ops.spmm_t(A, dY, dX, split=c["split"], tune=c["tune"])), force)

    def spttv(self, B: "ops.CSF3", c: torch.Tensor, force: bool = False) -> dict:
        out = torch.empty(B.nfib, dtype=ops.result_dtype(B.dtype), device=c.device)
        key = self.csf_key("spttv", B, 1, B.dtype)
        return self.choose(key, spmv_candidates(),
                           lambda k: (lambda: ops.spttv(B, c, out, split=k["split"], tune=k["tune"])), force)

    def spmttkrp(self, B: "ops.CSF3", C: torch.Tensor, D: torch.Tensor, force: bool = False) -> dict:
        A = torch.empty((B.dims[0], C.shape[1]), dtype=ops.result_dtype(B.dtype), device=C.device)
        key = self.csf_key("spmttkrp", B, C.shape[1], B.dtype)
        return self.choose(key, warp_candidates(True, inflight=False),
                           lambda k: (lambda: ops.spmttkrp(B, C, D, A, split=k["split"], tune=k["tune"])), force)
