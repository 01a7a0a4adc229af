"""Python front end of libspd: torch tensors in, C-ABI calls out.

PyTorch provides device memory and streams only; every step of every operation runs in
the CUDA kernels behind include/spd.h. There is no CPU fallback: inputs must be CUDA
tensors and a missing library raises.

Sparse operands use the level formats of SpDISTAL (Sections II-B, III-B):
``CSR`` = {Dense, Compressed} and ``CSF3`` = {Dense, Compressed, Compressed} with int32
pos/crd arrays.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Tuple

import torch

from . import _abi

_DTYPE_CODE = {torch.float64: _abi.SPD_F64, torch.float32: _abi.SPD_F32, torch.bfloat16: _abi.SPD_BF16}
_SPLIT_CODE = {"row": _abi.SPD_SPLIT_ROW, "nnz": _abi.SPD_SPLIT_NNZ, "auto": _abi.SPD_SPLIT_AUTO}


def result_dtype(dtype: torch.dtype) -> torch.dtype:
    """Type of results for values/dense inputs of ``dtype`` (binary64 stays binary64;
    binary32 and bfloat16 produce binary32)."""
    return torch.float64 if dtype == torch.float64 else torch.float32


def _code(dtype: torch.dtype) -> int:
    if dtype not in _DTYPE_CODE:
        raise TypeError("unsupported element type %s (float64, float32 or bfloat16)" % dtype)
    return _DTYPE_CODE[dtype]


def _split(split) -> int:
    if isinstance(split, int):
        return split
    if split not in _SPLIT_CODE:
        raise ValueError("split must be 'row', 'nnz' or 'auto'")
    return _SPLIT_CODE[split]


def _cuda(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor (there is no CPU path)" % name)
    return t


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _tune(tune) -> Optional[ctypes.POINTER(_abi.spd_tune)]:
    if tune is None:
        return None
    t = _abi.spd_tune(int(tune.get("unit_items", 0)), int(tune.get("row_pieces", 0)),
                      int(tune.get("block_threads", 0)), int(tune.get("inflight", 0)),
                      int(tune.get("lane_groups", 0)), int(tune.get("form", 0)))
    return ctypes.pointer(t)


class CSR:
    """A device CSR matrix: pos int32[nrows+1], crd int32[nnz], vals[nnz]."""

    def __init__(self, pos: torch.Tensor, crd: torch.Tensor, vals: Optional[torch.Tensor], shape: Tuple[int, int],
                 _structure_cache: Optional[dict] = None):
        # results that depend only on the pattern (the transposed structure), shared by
        # every matrix made from this one with with_vals
        self._structure_cache = {} if _structure_cache is None else _structure_cache
        self.pos = _cuda(pos, "pos")
        self.crd = _cuda(crd, "crd")
        self.vals = vals if vals is None else _cuda(vals, "vals")
        if self.pos.dtype != torch.int32 or self.crd.dtype != torch.int32:
            raise TypeError("pos and crd must be int32")
        self.shape = (int(shape[0]), int(shape[1]))
        if self.pos.numel() != self.shape[0] + 1:
            raise ValueError("pos must have nrows + 1 entries")
        if self.vals is not None and self.vals.numel() != self.crd.numel():
            raise ValueError("vals and crd differ in length")
        for t in (self.pos, self.crd) + (() if self.vals is None else (self.vals,)):
            if not t.is_contiguous():
                raise ValueError("pos, crd and vals must be contiguous")

    @property
    def nnz(self) -> int:
        return int(self.crd.numel())

    @property
    def dtype(self) -> torch.dtype:
        return self.vals.dtype if self.vals is not None else torch.float32

    def with_vals(self, vals: Optional[torch.Tensor]) -> "CSR":
        return CSR(self.pos, self.crd, vals, self.shape, self._structure_cache)

    def transposed(self, stream=None) -> "CSRTranspose":
        """A^T's structure (computed once per pattern, then reused)."""
        t = self._structure_cache.get("transpose")
        if t is None:
            t = transpose(self, stream=stream)
            self._structure_cache["transpose"] = t
        return t

    def desc(self, vtype: Optional[torch.dtype] = None) -> _abi.spd_csr:
        vt = vtype if vtype is not None else self.dtype
        return _abi.spd_csr(self.shape[0], self.shape[1], self.nnz, self.pos.data_ptr(),
                            self.crd.data_ptr() if self.nnz else None,
                            self.vals.data_ptr() if (self.vals is not None and self.nnz) else None, _code(vt), 0)

    @classmethod
    def from_host(cls, pos, crd, vals, shape, dtype=torch.float32, device="cuda") -> "CSR":
        """Copy numpy (or CPU torch) arrays to the device; vals are rounded to ``dtype``."""
        p = torch.as_tensor(pos).to(device=device, dtype=torch.int32).contiguous()
        c = torch.as_tensor(crd).to(device=device, dtype=torch.int32).contiguous()
        v = None if vals is None else torch.as_tensor(vals).to(dtype=dtype).to(device).contiguous()
        return cls(p, c, v, shape)


class CSF3:
    """A device CSF 3-tensor: pos1[dim0+1], crd1[nfib], pos2[nfib+1], crd2[nnz], vals[nnz]."""

    def __init__(self, pos1, crd1, pos2, crd2, vals, dims):
        self.pos1, self.crd1 = _cuda(pos1, "pos1"), _cuda(crd1, "crd1")
        self.pos2, self.crd2 = _cuda(pos2, "pos2"), _cuda(crd2, "crd2")
        self.vals = _cuda(vals, "vals")
        self.dims = tuple(int(d) for d in dims)
        for t in (self.pos1, self.crd1, self.pos2, self.crd2):
            if t.dtype != torch.int32 or not t.is_contiguous():
                raise TypeError("pos/crd arrays must be contiguous int32")
        if self.pos1.numel() != self.dims[0] + 1 or self.pos2.numel() != self.crd1.numel() + 1:
            raise ValueError("inconsistent CSF level sizes")

    @property
    def nfib(self) -> int:
        return int(self.crd1.numel())

    @property
    def nnz(self) -> int:
        return int(self.crd2.numel())

    @property
    def dtype(self) -> torch.dtype:
        return self.vals.dtype

    def desc(self) -> _abi.spd_csf3:
        d = self.dims
        return _abi.spd_csf3(d[0], d[1], d[2], self.nfib, self.nnz, self.pos1.data_ptr(),
                             self.crd1.data_ptr() if self.nfib else None, self.pos2.data_ptr(),
                             self.crd2.data_ptr() if self.nnz else None,
                             self.vals.data_ptr() if self.nnz else None, _code(self.dtype), 0)

    @classmethod
    def from_host(cls, pos1, crd1, pos2, crd2, vals, dims, dtype=torch.float32, device="cuda") -> "CSF3":
        t = lambda a: torch.as_tensor(a).to(device=device, dtype=torch.int32).contiguous()
        v = torch.as_tensor(vals).to(dtype=dtype).to(device).contiguous()
        return cls(t(pos1), t(crd1), t(pos2), t(crd2), v, dims)


class CSRTranspose:
    """The structure of A^T for a fixed pattern of A (``spd_csr_transpose``): t_pos
    int32[ncols+1], t_crd int32[nnz] (row coordinates, ascending in each column) and
    perm int32[nnz] (A's position of each entry of A^T)."""

    def __init__(self, t_pos: torch.Tensor, t_crd: torch.Tensor, perm: torch.Tensor, shape: Tuple[int, int]):
        self.t_pos, self.t_crd, self.perm = t_pos, t_crd, perm
        self.shape = shape  # A's shape

    def matrix(self, vals: Optional[torch.Tensor], stream=None) -> CSR:
        """A^T as a CSR matrix (ncols x nrows) carrying ``vals`` (A's values, A's order)."""
        tv = None if vals is None else gather_vals(self.perm, vals, stream=stream)
        return CSR(self.t_pos, self.t_crd, tv, (self.shape[1], self.shape[0]))


# ---------------------------------------------------------------------------- workspace

class Workspace:
    """Caller-side scratch for the compute calls: one growing device buffer per
    (device, stream). Calls on one stream are ordered, so they may share it."""

    def __init__(self):
        self._bufs = {}

    def get(self, nbytes: int, device: torch.device, stream) -> Tuple[Optional[torch.Tensor], int]:
        if nbytes == 0:
            return None, 0
        key = (device.index, stream.value if stream.value is not None else 0)
        buf = self._bufs.get(key)
        if buf is None or buf.numel() < nbytes:
            buf = torch.empty(max(nbytes, 1 << 20), dtype=torch.uint8, device=device)
            self._bufs[key] = buf
        return buf, buf.numel()


_WS = Workspace()


def csr_workspace_size(op: int, A: CSR, split="nnz", width: int = 0, tune=None, vtype=None) -> int:
    lib = _abi.load()
    n = ctypes.c_size_t(0)
    d = A.desc(vtype)
    _abi.check("spd_csr_workspace_size",
               lib.spd_csr_workspace_size(op, ctypes.byref(d), _split(split), int(width), _tune(tune), ctypes.byref(n)))
    return int(n.value)


def csf3_workspace_size(op: int, B: CSF3, split="nnz", width: int = 0, tune=None) -> int:
    lib = _abi.load()
    n = ctypes.c_size_t(0)
    d = B.desc()
    _abi.check("spd_csf3_workspace_size",
               lib.spd_csf3_workspace_size(op, ctypes.byref(d), _split(split), int(width), _tune(tune), ctypes.byref(n)))
    return int(n.value)


def _ws(nbytes, device, stream, ws):
    if ws is not None:
        if ws.numel() * ws.element_size() < nbytes:
            raise ValueError("workspace smaller than %d bytes" % nbytes)
        return ws, ws.numel() * ws.element_size()
    return _WS.get(nbytes, device, stream)


# ---------------------------------------------------------------------------- structure

def validate(T) -> Tuple[int, int]:
    """Level-format check of a CSR or CSF3 (synchronizes the current stream).
    Returns (violations, first bad index or -1)."""
    lib = _abi.load()
    dev = (T.pos if isinstance(T, CSR) else T.pos1).device
    st = _stream(None)
    buf, nb = _WS.get(64, dev, st)
    v = ctypes.c_int64(0)
    f = ctypes.c_int64(0)
    if isinstance(T, CSR):
        d = T.desc(torch.float32 if T.vals is None else None)
        s = lib.spd_csr_validate(ctypes.byref(d), _ptr(buf), nb, ctypes.byref(v), ctypes.byref(f), st)
    else:
        d = T.desc()
        s = lib.spd_csf3_validate(ctypes.byref(d), _ptr(buf), nb, ctypes.byref(v), ctypes.byref(f), st)
    if s not in (_abi.SPD_OK, 5):
        _abi.check("validate", s)
    return int(v.value), int(f.value)


def set_checked(on: bool) -> None:
    """Turns the library's checked mode on or off (``spd_set_checked``): every call that
    takes a sparse operand validates it first and synchronizes its stream afterwards."""
    _abi.check("spd_set_checked", _abi.load().spd_set_checked(1 if on else 0))


def checked() -> bool:
    """True while the library's checked mode is on (``spd_checked``)."""
    return bool(_abi.load().spd_checked())


def fault_status(stream=None) -> int:
    """Synchronizes the stream and returns, then clears, the fault bits that kernels with
    bounded waits recorded (``spd_fault_status``): 0 when none gave up, bit 1 when a wait
    for bulk copies ran out (the outputs of that call are unspecified)."""
    flags = ctypes.c_uint32(0)
    s = _abi.load().spd_fault_status(ctypes.byref(flags), _stream(stream))
    if s not in (0, _abi.SPD_ERR_TIMEOUT):
        _abi.check("spd_fault_status", s)
    return int(flags.value)


def probe_bounded_wait(stream=None) -> None:
    """Runs a kernel whose bounded wait runs out after about 1 s (``spd_probe_bounded_wait``),
    to exercise the fault path: ``fault_status`` reports it afterwards."""
    _abi.check("spd_probe_bounded_wait", _abi.load().spd_probe_bounded_wait(_stream(stream)))


def partition(A: CSR, split: str, npieces: int, unit_items: int = 0):
    """The work partition the kernels use, as two int32 device tensors of npieces + 1."""
    lib = _abi.load()
    dev = A.pos.device
    rows = torch.empty(npieces + 1, dtype=torch.int32, device=dev)
    poss = torch.empty(npieces + 1, dtype=torch.int32, device=dev)
    d = A.desc(torch.float32 if A.vals is None else None)
    _abi.check("spd_csr_partition", lib.spd_csr_partition(ctypes.byref(d), _split(split), int(npieces),
                                                          int(unit_items), _ptr(rows), _ptr(poss), _stream(None)))
    return rows, poss


# ---------------------------------------------------------------------------- kernels

def spmv(A: CSR, x: torch.Tensor, y: Optional[torch.Tensor] = None, split="nnz", tune=None, ws=None, stream=None):
    """y(i) = A(i,j) x(j)."""
    lib = _abi.load()
    _cuda(x, "x")
    n, m = A.shape
    if x.dtype != A.dtype or x.numel() != m or not x.is_contiguous():
        raise ValueError("x must be a contiguous vector of %d elements of %s" % (m, A.dtype))
    if y is None:
        y = torch.empty(n, dtype=result_dtype(A.dtype), device=x.device)
    st = _stream(stream)
    need = csr_workspace_size(_abi.SPD_OP_SPMV, A, split, 0, tune)
    buf, nb = _ws(need, x.device, st, ws)
    d = A.desc()
    _abi.check("spd_spmv", lib.spd_spmv(ctypes.byref(d), _ptr(x), _code(x.dtype), _ptr(y), _code(y.dtype),
                                        _split(split), _tune(tune), _ptr(buf), nb, st))
    return y


def spmm(A: CSR, X: torch.Tensor, Y: Optional[torch.Tensor] = None, split="nnz", tune=None, ws=None, stream=None):
    """Y(i,l) = A(i,j) X(j,l); X is ncols x L (row stride may exceed L)."""
    lib = _abi.load()
    _cuda(X, "X")
    n, m = A.shape
    if X.dim() != 2 or X.shape[0] != m or X.dtype != A.dtype or X.stride(1) != 1:
        raise ValueError("X must be a row-major %d x L matrix of %s" % (m, A.dtype))
    L = X.shape[1]
    if Y is None:
        Y = torch.empty((n, L), dtype=result_dtype(A.dtype), device=X.device)
    st = _stream(stream)
    need = csr_workspace_size(_abi.SPD_OP_SPMM, A, split, L, tune)
    buf, nb = _ws(need, X.device, st, ws)
    d = A.desc()
    _abi.check("spd_spmm", lib.spd_spmm(ctypes.byref(d), _ptr(X), L, X.stride(0), _code(X.dtype), _ptr(Y), Y.stride(0),
                                        _code(Y.dtype), _split(split), _tune(tune), _ptr(buf), nb, st))
    return Y


def spmm_accumulate(A: CSR, X: torch.Tensor, Y: torch.Tensor, split="nnz", tune=None, ws=None, stream=None):
    """Y(i,l) += A(i,j) X(j,l) in place; rows of A without entries leave Y as it is."""
    lib = _abi.load()
    _cuda(X, "X")
    _cuda(Y, "Y")
    n, m = A.shape
    if X.dim() != 2 or X.shape[0] != m or X.dtype != A.dtype or X.stride(1) != 1:
        raise ValueError("X must be a row-major %d x L matrix of %s" % (m, A.dtype))
    L = X.shape[1]
    if Y.shape != (n, L) or Y.dtype != result_dtype(A.dtype) or Y.stride(1) != 1:
        raise ValueError("Y must be a row-major %d x %d matrix of %s" % (n, L, result_dtype(A.dtype)))
    st = _stream(stream)
    need = csr_workspace_size(_abi.SPD_OP_SPMM, A, split, L, tune)
    buf, nb = _ws(need, X.device, st, ws)
    d = A.desc()
    _abi.check("spd_spmm_accumulate", lib.spd_spmm_accumulate(ctypes.byref(d), _ptr(X), L, X.stride(0), _code(X.dtype),
                                                              _ptr(Y), Y.stride(0), _code(Y.dtype), _split(split),
                                                              _tune(tune), _ptr(buf), nb, st))
    return Y


class ColumnBlocks:
    """A's column blocks (``spd_csr_column_blocks``): block b holds the entries with
    bounds[b] <= column < bounds[b+1], as a CSR over blk_pos[b], the slice of blk_crd at
    off[b], and perm into A's positions."""

    def __init__(self, bounds, blk_pos, blk_crd, perm, nnz, shape):
        self.bounds, self.blk_pos, self.blk_crd, self.perm, self.nnz, self.shape = bounds, blk_pos, blk_crd, perm, nnz, shape
        self.off = [0]
        for k in nnz:
            self.off.append(self.off[-1] + k)

    def matrices(self, vals: Optional[torch.Tensor], stream=None):
        """The blocks as CSR matrices of A's shape carrying ``vals`` (A's values, A's order)."""
        bv = None if vals is None else gather_vals(self.perm, vals, stream=stream)
        out = []
        for b in range(len(self.nnz)):
            s, e = self.off[b], self.off[b + 1]
            out.append(CSR(self.blk_pos[b], self.blk_crd[s:e], None if bv is None else bv[s:e], self.shape))
        return out


def column_blocks(A: CSR, nblk: Optional[int] = None, bounds=None, stream=None) -> ColumnBlocks:
    """Split A's columns into value ranges (equal ranges when only nblk is given); cached
    per pattern and bounds."""
    lib = _abi.load()
    n, m = A.shape
    if bounds is None:
        if not nblk or nblk < 1:
            raise ValueError("give nblk >= 1 or bounds")
        bounds = [(b * m) // nblk for b in range(nblk + 1)]
    bounds = [int(v) for v in bounds]
    key = ("column_blocks", tuple(bounds))
    hit = A._structure_cache.get(key)
    if hit is not None:
        return hit
    nb = len(bounds) - 1
    dev = A.pos.device
    st = _stream(stream)
    d = A.desc()
    size = ctypes.c_size_t(0)
    _abi.check("spd_csr_column_blocks_workspace_size",
               lib.spd_csr_column_blocks_workspace_size(ctypes.byref(d), nb, ctypes.byref(size)))
    buf, nbytes = _ws(int(size.value), dev, st, None)
    b_host = (ctypes.c_int32 * (nb + 1))(*bounds)
    blk_pos = torch.empty((nb, n + 1), dtype=torch.int32, device=dev)
    blk_crd = torch.empty(A.nnz, dtype=torch.int32, device=dev)
    perm = torch.empty(A.nnz, dtype=torch.int32, device=dev)
    counts = (ctypes.c_int64 * nb)()
    _abi.check("spd_csr_column_blocks", lib.spd_csr_column_blocks(ctypes.byref(d), nb, b_host, _ptr(blk_pos),
                                                                  _ptr(blk_crd), _ptr(perm), counts, _ptr(buf),
                                                                  nbytes, st))
    cb = ColumnBlocks(bounds, blk_pos, blk_crd, perm, [int(c) for c in counts], A.shape)
    A._structure_cache[key] = cb
    return cb


def spmm_column_blocked(A: CSR, X: torch.Tensor, Y: Optional[torch.Tensor] = None, nblk: Optional[int] = None,
                        bounds=None, split="nnz", tune=None, stream=None):
    """Y = A X as the sum over A's column blocks of A_b X (the first block overwrites Y, the
    others add to it): each product gathers only its block's slab of X."""
    cb = column_blocks(A, nblk=nblk, bounds=bounds, stream=stream)
    mats = cb.matrices(A.vals, stream=stream)
    Y = spmm(mats[0], X, Y, split=split, tune=tune, stream=stream)
    for Ab in mats[1:]:
        if Ab.nnz:
            spmm_accumulate(Ab, X, Y, split=split, tune=tune, stream=stream)
    return Y


def spmm_t(A: CSR, dY: torch.Tensor, dX: Optional[torch.Tensor] = None, split="nnz", tune=None, ws=None,
           stream=None, method: str = "atomic"):
    """dX(j,l) = A(i,j) dY(i,l): the gradient of Y = A X with respect to X.

    method="atomic": walk A's rows and scatter into dX with atomic adds (no extra
    memory; summation order not deterministic). method="transpose": SpMM over A^T,
    whose structure is computed once per pattern (``CSR.transposed``); each row of dX is
    written once in a fixed order, so the result is deterministic."""
    lib = _abi.load()
    _cuda(dY, "dY")
    n, m = A.shape
    if dY.dim() != 2 or dY.shape[0] != n or dY.dtype != A.dtype or dY.stride(1) != 1:
        raise ValueError("dY must be a row-major %d x L matrix of %s" % (n, A.dtype))
    if method == "transpose":
        At = A.transposed(stream=stream).matrix(A.vals, stream=stream)
        return spmm(At, dY, Y=dX, split=split, tune=tune, ws=ws, stream=stream)
    if method != "atomic":
        raise ValueError("method must be 'atomic' or 'transpose'")
    L = dY.shape[1]
    if dX is None:
        dX = torch.empty((m, L), dtype=result_dtype(A.dtype), device=dY.device)
    st = _stream(stream)
    need = csr_workspace_size(_abi.SPD_OP_SPMM_T, A, split, L, tune)
    buf, nb = _ws(need, dY.device, st, ws)
    d = A.desc()
    _abi.check("spd_spmm_t", lib.spd_spmm_t(ctypes.byref(d), _ptr(dY), L, dY.stride(0), _code(dY.dtype), _ptr(dX),
                                            dX.stride(0), _code(dX.dtype), _split(split), _tune(tune), _ptr(buf), nb,
                                            st))
    return dX


def transpose(A: CSR, stream=None, ws=None) -> CSRTranspose:
    """The structure of A^T and the permutation into it (deterministic)."""
    lib = _abi.load()
    n, m = A.shape
    dev = A.pos.device
    st = _stream(stream)
    d = A.desc()
    nb = ctypes.c_size_t(0)
    _abi.check("spd_csr_transpose_workspace_size", lib.spd_csr_transpose_workspace_size(ctypes.byref(d), ctypes.byref(nb)))
    buf, nbytes = _ws(int(nb.value), dev, st, ws)
    t_pos = torch.empty(m + 1, dtype=torch.int32, device=dev)
    t_crd = torch.empty(A.nnz, dtype=torch.int32, device=dev)
    perm = torch.empty(A.nnz, dtype=torch.int32, device=dev)
    _abi.check("spd_csr_transpose", lib.spd_csr_transpose(ctypes.byref(d), _ptr(t_pos), _ptr(t_crd), _ptr(perm),
                                                          _ptr(buf), nbytes, st))
    return CSRTranspose(t_pos, t_crd, perm, A.shape)


def gather_vals(perm: torch.Tensor, vals: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None):
    """out[q] = vals[perm[q]] (A's values in A^T's order)."""
    lib = _abi.load()
    _cuda(perm, "perm")
    _cuda(vals, "vals")
    if perm.dtype != torch.int32 or not perm.is_contiguous() or not vals.is_contiguous():
        raise ValueError("perm must be contiguous int32 and vals contiguous")
    if out is None:
        out = torch.empty(perm.numel(), dtype=vals.dtype, device=vals.device)
    _abi.check("spd_gather_vals", lib.spd_gather_vals(perm.numel(), _ptr(perm), _ptr(vals), _ptr(out),
                                                      _code(vals.dtype), _stream(stream)))
    return out


class Spadd3Symbolic:
    """Result of SpAdd3's symbolic phase: A's pos, nnz(A) and the workspace (holding the
    partition) that the numeric phase reads."""

    def __init__(self, a_pos, nnz, ws, nbytes, split, tune):
        self.a_pos, self.nnz, self.ws, self.nbytes, self.split, self.tune = a_pos, nnz, ws, nbytes, split, tune


def spadd3_symbolic(B: CSR, C: CSR, D: CSR, split="nnz", tune=None, stream=None) -> Spadd3Symbolic:
    """Phase 1 of A = B + C + D: count each row of A (the union of the three patterns)
    and form A's pos; synchronizes the stream to return nnz(A)."""
    lib = _abi.load()
    for M in (C, D):
        if M.shape != B.shape or M.dtype != B.dtype:
            raise ValueError("B, C and D must share shape and value type")
    n = B.shape[0]
    dev = B.pos.device
    st = _stream(stream)
    d = [M.desc() for M in (B, C, D)]
    dp = [ctypes.byref(x) for x in d]
    nb = ctypes.c_size_t(0)
    _abi.check("spd_spadd3_workspace_size", lib.spd_spadd3_workspace_size(*dp, _split(split), _tune(tune), ctypes.byref(nb)))
    # a workspace of its own: it must survive, untouched, until the numeric phase
    nbytes = max(int(nb.value), 1)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    a_pos = torch.empty(n + 1, dtype=torch.int32, device=dev)
    nnz = ctypes.c_int64(0)
    _abi.check("spd_spadd3_symbolic", lib.spd_spadd3_symbolic(*dp, _split(split), _tune(tune), _ptr(a_pos),
                                                              ctypes.byref(nnz), _ptr(ws), nbytes, st))
    return Spadd3Symbolic(a_pos, int(nnz.value), ws, nbytes, split, tune)


def spadd3_numeric(sym: Spadd3Symbolic, B: CSR, C: CSR, D: CSR, stream=None) -> CSR:
    """Phase 2 of A = B + C + D: fill A's crd and vals (sizes from the symbolic phase)."""
    lib = _abi.load()
    dev = B.pos.device
    d = [M.desc() for M in (B, C, D)]
    dp = [ctypes.byref(x) for x in d]
    a_crd = torch.empty(sym.nnz, dtype=torch.int32, device=dev)
    a_vals = torch.empty(sym.nnz, dtype=result_dtype(B.dtype), device=dev)
    _abi.check("spd_spadd3_numeric", lib.spd_spadd3_numeric(*dp, _split(sym.split), _tune(sym.tune), _ptr(sym.a_pos),
                                                            sym.nnz, _ptr(a_crd), _ptr(a_vals), _code(a_vals.dtype),
                                                            _ptr(sym.ws), sym.nbytes, _stream(stream)))
    return CSR(sym.a_pos, a_crd, a_vals, B.shape)


def spadd3(B: CSR, C: CSR, D: CSR, split="nnz", tune=None, stream=None) -> CSR:
    """A = B + C + D on CSR operands of one shape and value type. A's pattern is the union
    of the three (two-phase assembly: row counts and pos first, then crd and vals); the
    call synchronizes the stream once, to learn nnz(A) before allocating it."""
    sym = spadd3_symbolic(B, C, D, split=split, tune=tune, stream=stream)
    return spadd3_numeric(sym, B, C, D, stream=stream)


def sddmm(B: CSR, C: torch.Tensor, Dnk: torch.Tensor, out: Optional[torch.Tensor] = None, split="nnz", tune=None,
          ws=None, stream=None):
    """A(i,j) = B(i,j) C(i,k) D(k,j) on B's pattern; Dnk[j,k] = D(k,j). B.vals None => 1.
    Returns the output values, one per stored position of B (B's pos/crd are the output's)."""
    lib = _abi.load()
    _cuda(C, "C")
    _cuda(Dnk, "Dnk")
    n, m = B.shape
    if C.dim() != 2 or Dnk.dim() != 2 or C.shape[0] != n or Dnk.shape[0] != m or C.shape[1] != Dnk.shape[1]:
        raise ValueError("C must be nrows x K and Dnk ncols x K")
    if C.dtype != Dnk.dtype or (B.vals is not None and B.vals.dtype != C.dtype) or C.stride(1) != 1 or Dnk.stride(1) != 1:
        raise ValueError("C, Dnk (and B's values) must share one dtype and be row-major")
    K = C.shape[1]
    if out is None:
        out = torch.empty(B.nnz, dtype=result_dtype(C.dtype), device=C.device)
    st = _stream(stream)
    need = csr_workspace_size(_abi.SPD_OP_SDDMM, B, split, K, tune, vtype=C.dtype)
    buf, nb = _ws(need, C.device, st, ws)
    d = B.desc(C.dtype)
    _abi.check("spd_sddmm", lib.spd_sddmm(ctypes.byref(d), _ptr(C), K, C.stride(0), _ptr(Dnk), Dnk.stride(0),
                                          _code(C.dtype), _ptr(out), _code(out.dtype), _split(split), _tune(tune),
                                          _ptr(buf), nb, st))
    return out


def spttv(B: CSF3, c: torch.Tensor, out: Optional[torch.Tensor] = None, split="nnz", tune=None, ws=None, stream=None):
    """A(i,j) = B(i,j,k) c(k). Returns one value per fiber; B's pos1/crd1 are the output's."""
    lib = _abi.load()
    _cuda(c, "c")
    if c.dtype != B.dtype or c.numel() != B.dims[2] or not c.is_contiguous():
        raise ValueError("c must be a contiguous vector of dim2 elements of the value type")
    if out is None:
        out = torch.empty(B.nfib, dtype=result_dtype(B.dtype), device=c.device)
    st = _stream(stream)
    need = csf3_workspace_size(_abi.SPD_OP_SPTTV, B, split, 0, tune)
    buf, nb = _ws(need, c.device, st, ws)
    d = B.desc()
    _abi.check("spd_spttv", lib.spd_spttv(ctypes.byref(d), _ptr(c), _code(c.dtype), _ptr(out), _code(out.dtype),
                                          _split(split), _tune(tune), _ptr(buf), nb, st))
    return out


def spmttkrp(B: CSF3, C: torch.Tensor, D: torch.Tensor, A: Optional[torch.Tensor] = None, split="nnz", tune=None,
             ws=None, stream=None):
    """A(i,l) = B(i,j,k) C(j,l) D(k,l); C is dim1 x R, D is dim2 x R."""
    lib = _abi.load()
    _cuda(C, "C")
    _cuda(D, "D")
    if C.dim() != 2 or D.dim() != 2 or C.shape[0] != B.dims[1] or D.shape[0] != B.dims[2] or C.shape[1] != D.shape[1]:
        raise ValueError("C must be dim1 x R and D dim2 x R")
    if C.dtype != B.dtype or D.dtype != B.dtype or C.stride(1) != 1 or D.stride(1) != 1:
        raise ValueError("factors must be row-major and of the value type")
    R = C.shape[1]
    if A is None:
        A = torch.empty((B.dims[0], R), dtype=result_dtype(B.dtype), device=C.device)
    st = _stream(stream)
    need = csf3_workspace_size(_abi.SPD_OP_SPMTTKRP, B, split, R, tune)
    buf, nb = _ws(need, C.device, st, ws)
    d = B.desc()
    _abi.check("spd_spmttkrp", lib.spd_spmttkrp(ctypes.byref(d), _ptr(C), C.stride(0), _ptr(D), D.stride(0), R,
                                                _code(C.dtype), _ptr(A), A.stride(0), _code(A.dtype), _split(split),
                                                _tune(tune), _ptr(buf), nb, st))
    return A
