"""Batched SpMM: hundreds of independent products Y_m = A_m X_m in one persistent launch.

``SpMMBatch`` plans the batch once (``spd_spmm_batched_plan``: every matrix's pieces laid
end to end, per-matrix split and piece size), then ``run()`` issues the persistent kernel
and the fix-up on the current stream, and ``capture()`` records that run in a CUDA graph
so that ``replay()`` costs one graph launch. ``autotune()`` times the batch under each
candidate policy (split rule x piece size) and keeps the fastest.
"""
from __future__ import annotations

import ctypes
from typing import List, Optional, Sequence

import torch

from . import _abi, ops


def _split_for(A: "ops.CSR", policy: str, long_row: int) -> int:
    if policy == "row":
        return _abi.SPD_SPLIT_ROW
    if policy == "nnz":
        return _abi.SPD_SPLIT_NNZ
    # "auto": the row split unless some row is longer than `long_row` items
    lens = A.pos[1:] - A.pos[:-1]
    return _abi.SPD_SPLIT_NNZ if A.shape[0] and int(lens.max().item()) > long_row else _abi.SPD_SPLIT_ROW


class SpMMBatch:
    """Y_m = A_m X_m for every m, planned once and run as one persistent launch."""

    def __init__(self, mats: Sequence["ops.CSR"], Xs: Sequence[torch.Tensor], Ys: Optional[Sequence[torch.Tensor]] = None,
                 policy: str = "auto", unit_items: int = 1024, block_threads: int = 256, long_row: int = 4096):
        if len(mats) != len(Xs):
            raise ValueError("one X per matrix")
        self.mats = list(mats)
        self.Xs = list(Xs)
        dtype = self.mats[0].dtype if self.mats else torch.float32
        for A, X in zip(self.mats, self.Xs):
            if A.dtype != dtype or X.dtype != dtype or not X.is_cuda or X.stride(1) != 1 or X.shape[0] != A.shape[1]:
                raise ValueError("every matrix and X must share one dtype; X must be a row-major ncols x L CUDA tensor")
        self.L = self.Xs[0].shape[1] if self.Xs else 0
        if any(X.shape[1] != self.L for X in self.Xs):
            raise ValueError("all X must have the same number of columns")
        self.dtype = dtype
        rt = ops.result_dtype(dtype)
        self.Ys = list(Ys) if Ys is not None else [torch.empty((A.shape[0], self.L), dtype=rt, device=X.device)
                                                   for A, X in zip(self.mats, self.Xs)]
        self.graph = None
        self.plan = None
        self.ws = None
        self.configure(policy, unit_items, block_threads, long_row)

    def configure(self, policy: str, unit_items: int, block_threads: int = 256, long_row: int = 4096) -> None:
        """(Re)plan the batch under a split policy ('row', 'nnz' or 'auto') and piece size."""
        lib = _abi.load()
        self.policy, self.unit_items, self.block_threads = policy, unit_items, block_threads
        n = len(self.mats)
        items = (_abi.spd_batch_item * max(n, 1))()
        for m, (A, X, Y) in enumerate(zip(self.mats, self.Xs, self.Ys)):
            items[m] = _abi.spd_batch_item(A.desc(), X.data_ptr(), X.stride(0), Y.data_ptr(), Y.stride(0),
                                           _split_for(A, policy, long_row), unit_items)
        self._items = items
        tune = _abi.spd_tune(unit_items, 0, block_threads, 0)
        size = ctypes.c_size_t(0)
        code = ops._code(self.dtype)
        _abi.check("spd_spmm_batched_workspace_size",
                   lib.spd_spmm_batched_workspace_size(n, items, self.L, code, ctypes.byref(tune), ctypes.byref(size)))
        self.ws = torch.empty(max(size.value, 256), dtype=torch.uint8, device=self.Xs[0].device if n else "cuda")
        self.plan = _abi.spd_batch_plan()
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        _abi.check("spd_spmm_batched_plan",
                   lib.spd_spmm_batched_plan(n, items, self.L, code, ctypes.byref(tune), self.ws.data_ptr(),
                                             self.ws.numel(), ctypes.byref(self.plan), st))
        self.graph = None

    def run(self) -> List[torch.Tensor]:
        lib = _abi.load()
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        _abi.check("spd_spmm_batched_run", lib.spd_spmm_batched_run(ctypes.byref(self.plan), st))
        return self.Ys

    def capture(self) -> "torch.cuda.CUDAGraph":
        """Record one run in a CUDA graph (after a warm-up run on a side stream)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run()
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        self.graph = g
        return g

    def replay(self) -> List[torch.Tensor]:
        if self.graph is None:
            self.capture()
        self.graph.replay()
        return self.Ys

    def run_separately(self, split="auto") -> List[torch.Tensor]:
        """The same products as one spd_spmm launch per matrix (for comparison)."""
        for A, X, Y in zip(self.mats, self.Xs, self.Ys):
            ops.spmm(A, X, Y, split=split)
        return self.Ys

    def autotune(self, policies=("row", "nnz", "auto"), units=(256, 512, 1024, 2048), reps: int = 5) -> dict:
        """Time the batched run under each (policy, piece size) and keep the fastest."""
        table = []
        best = None
        for pol in policies:
            for unit in units:
                self.configure(pol, unit, self.block_threads)
                self.run()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    self.run()
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                table.append({"policy": pol, "unit_items": unit, "ms": round(ms, 4)})
                if best is None or ms < best["ms"]:
                    best = table[-1]
        self.configure(best["policy"], best["unit_items"], self.block_threads)
        self.tuning_table = table
        return best
