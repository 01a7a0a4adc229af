"""CPU oracle for the SpDISTAL sparse kernels -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package. The product path (``paper_2207_13901_gb300``) never does, and this
package never imports it: the two share no code. The arithmetic lives in
``spd_oracle.c`` (plain C, binary64, ``-ffp-contract=off``); this module compiles it
with the host C compiler and marshals numpy arrays through ctypes.

Every function takes numpy arrays (int32 structure, values upcast to float64) and
returns float64 results. ``sel`` selects a subset of outputs for sampled checks on
large inputs.

The environment variable ``SPD_ORACLE_LIB`` names a compiled copy of the oracle to load
instead of building this one; the mutation test uses it to run the pins against copies
with a planted mistake.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spd_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libspd_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libspd_oracle.so`` (host gcc)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cc = os.environ.get("CC", "gcc")
    subprocess.check_call([cc, *CFLAGS, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_I64 = ctypes.c_int64
_P = ctypes.c_void_p

_SIGS = {
    "orc_row_split": [_I64, _I64, _P],
    "orc_merge_path": [_I64, _P, _I64, _P, _P, _P],
    "orc_pos_split": [_I64, _P, _I64, _P, _P],
    "orc_spmv": [_I64, _P, _P, _P, _P, _I64, _P, _P],
    "orc_spmv_acc": [_I64, _P, _P, _P, _P, _I64, _P, _P],
    "orc_spmm": [_I64, _I64, _P, _P, _P, _P, _I64, _I64, _P, _P, _I64],
    "orc_spmm_acc": [_I64, _I64, _P, _P, _P, _P, _I64, _I64, _P, _P, _I64],
    "orc_spmm_t": [_I64, _I64, _I64, _P, _P, _P, _P, _I64, _P, _I64],
    "orc_spmm_t_acc": [_I64, _I64, _I64, _P, _P, _P, _P, _I64, _P, _I64],
    "orc_sddmm": [_I64, _I64, _P, _P, _P, _P, _I64, _P, _I64, _I64, _P, _P],
    "orc_sddmm_acc": [_I64, _I64, _P, _P, _P, _P, _I64, _P, _I64, _I64, _P, _P],
    "orc_spttv": [_I64, _P, _P, _P, _P, _P, _P, _I64, _P, _P],
    "orc_spttv_acc": [_I64, _P, _P, _P, _P, _P, _P, _I64, _P, _P],
    "orc_spmttkrp": [_I64, _I64, _P, _P, _P, _P, _P, _P, _I64, _P, _I64, _I64, _P, _P, _I64],
    "orc_spmttkrp_acc": [_I64, _I64, _P, _P, _P, _P, _P, _P, _I64, _P, _I64, _I64, _P, _P, _I64],
    "orc_validate_level": [_I64, _I64, _P, _P, _I64, _P],
    "orc_csr_transpose": [_I64, _I64, _P, _P, _P, _P, _P],
    "orc_spadd3_count": [_I64, _P, _P, _P, _P, _P, _P, _P],
    "orc_spadd3": [_I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P],
    "orc_column_blocks": [_I64, _P, _P, _I64, _P, _P, _P, _P],
}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("SPD_ORACLE_LIB") or build()
            L = ctypes.CDLL(path)
            for name, args in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int64 if name == "orc_validate_level" else None
            _lib = L
    return _lib


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int64)


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def _sel(sel):
    if sel is None:
        return None, 0
    s = _i64(sel)
    return s, s.shape[0]


# ----------------------------------------------------------------------------- partitions

def row_split(n: int, pieces: int) -> np.ndarray:
    """Universe partition bounds floor(c*n/P), c = 0..P."""
    out = np.zeros(pieces + 1, dtype=np.int64)
    lib().orc_row_split(n, pieces, _ptr(out))
    return out


def merge_path(pos, diagonals):
    """(rows, positions) after d items of the row-end/nonzero sequence, per diagonal d."""
    pos = _i32(pos)
    d = _i64(diagonals)
    rows = np.zeros(d.shape[0], dtype=np.int64)
    poss = np.zeros(d.shape[0], dtype=np.int64)
    lib().orc_merge_path(pos.shape[0] - 1, _ptr(pos), d.shape[0], _ptr(d), _ptr(rows), _ptr(poss))
    return rows, poss


def pos_split(pos, positions) -> np.ndarray:
    """Row holding each position (n for position nnz)."""
    pos = _i32(pos)
    q = _i64(positions)
    rows = np.zeros(q.shape[0], dtype=np.int64)
    lib().orc_pos_split(pos.shape[0] - 1, _ptr(pos), q.shape[0], _ptr(q), _ptr(rows))
    return rows


def csr_transpose(pos, crd, ncols: int):
    """A^T's structure (t_pos, t_crd) and perm, perm[q] = A's position of A^T's entry q."""
    pos = _i32(pos)
    crd = _i32(crd)
    nnz = crd.shape[0]
    t_pos = np.zeros(ncols + 1, dtype=np.int32)
    t_crd = np.zeros(nnz, dtype=np.int32)
    perm = np.zeros(nnz, dtype=np.int32)
    lib().orc_csr_transpose(pos.shape[0] - 1, ncols, _ptr(pos), _ptr(crd), _ptr(t_pos), _ptr(t_crd), _ptr(perm))
    return t_pos, t_crd, perm


def spadd3_count(B, C, D) -> np.ndarray:
    """Entries per row of A = B + C + D (the union of the three patterns)."""
    ops = [(_i32(M.pos), _i32(M.crd)) for M in (B, C, D)]
    n = ops[0][0].shape[0] - 1
    out = np.zeros(n, dtype=np.int64)
    lib().orc_spadd3_count(n, *[_ptr(a) for pc in ops for a in pc], _ptr(out))
    return out


def spadd3(B, C, D):
    """(pos, crd, vals) of A = B + C + D; B, C, D are objects with pos/crd/vals (one shape)."""
    ops = [(_i32(M.pos), _i32(M.crd), _f64(M.vals)) for M in (B, C, D)]
    n = ops[0][0].shape[0] - 1
    total = int(sum(M.crd.shape[0] for M in (B, C, D)))
    ap = np.zeros(n + 1, dtype=np.int32)
    ac = np.zeros(max(total, 1), dtype=np.int32)
    av = np.zeros(max(total, 1), dtype=np.float64)
    lib().orc_spadd3(n, *[_ptr(a) for t in ops for a in t], _ptr(ap), _ptr(ac), _ptr(av))
    nnz = int(ap[-1])
    return ap, ac[:nnz].copy(), av[:nnz].copy()


def column_blocks(pos, crd, bounds):
    """Value-range blocks of A's columns: (blk_pos [nblk, n+1], blk_crd, perm, blk_nnz)."""
    pos, crd, bounds = _i32(pos), _i32(crd), _i32(bounds)
    n = pos.shape[0] - 1
    nblk = bounds.shape[0] - 1
    blk_pos = np.zeros((nblk, n + 1), dtype=np.int32)
    blk_crd = np.zeros(max(crd.shape[0], 1), dtype=np.int32)
    perm = np.zeros(max(crd.shape[0], 1), dtype=np.int32)
    lib().orc_column_blocks(n, _ptr(pos), _ptr(crd), nblk, _ptr(bounds), _ptr(blk_pos), _ptr(blk_crd), _ptr(perm))
    total = int(blk_pos[:, -1].sum())
    return blk_pos, blk_crd[:total].copy(), perm[:total].copy(), blk_pos[:, -1].astype(np.int64)


def validate_level(nparent: int, nchild_dim: int, pos, crd):
    """(violation count, first bad index or -1) of one Compressed level."""
    pos = _i32(pos)
    crd = _i32(crd)
    first = np.zeros(1, dtype=np.int64)
    bad = lib().orc_validate_level(nparent, nchild_dim, _ptr(pos), _ptr(crd), crd.shape[0], _ptr(first))
    return int(bad), int(first[0])


# ----------------------------------------------------------------------------- kernels

def spmv(pos, crd, vals, x, sel=None, accurate: bool = False) -> np.ndarray:
    """y(i) = A(i,j) x(j)."""
    pos, crd, vals, x = _i32(pos), _i32(crd), _f64(vals), _f64(x)
    s, ns = _sel(sel)
    n = pos.shape[0] - 1
    y = np.zeros(ns if s is not None else n, dtype=np.float64)
    fn = lib().orc_spmv_acc if accurate else lib().orc_spmv
    fn(n, _ptr(pos), _ptr(crd), _ptr(vals), _ptr(x), ns, _ptr(s), _ptr(y))
    return y


def spmm(pos, crd, vals, X, sel=None, accurate: bool = False) -> np.ndarray:
    """Y(i,l) = A(i,j) X(j,l); X is ncols x L row-major."""
    pos, crd, vals, X = _i32(pos), _i32(crd), _f64(vals), _f64(X)
    s, ns = _sel(sel)
    n = pos.shape[0] - 1
    L = X.shape[1]
    Y = np.zeros((ns if s is not None else n, L), dtype=np.float64)
    fn = lib().orc_spmm_acc if accurate else lib().orc_spmm
    fn(n, L, _ptr(pos), _ptr(crd), _ptr(vals), _ptr(X), L, ns, _ptr(s), _ptr(Y), L)
    return Y


def spmm_t(pos, crd, vals, dY, ncols: int, accurate: bool = False) -> np.ndarray:
    """dX(j,l) = A(i,j) dY(i,l); dY is n x L row-major, result ncols x L."""
    pos, crd, vals, dY = _i32(pos), _i32(crd), _f64(vals), _f64(dY)
    n = pos.shape[0] - 1
    L = dY.shape[1]
    dX = np.zeros((ncols, L), dtype=np.float64)
    fn = lib().orc_spmm_t_acc if accurate else lib().orc_spmm_t
    fn(n, ncols, L, _ptr(pos), _ptr(crd), _ptr(vals), _ptr(dY), L, _ptr(dX), L)
    return dX


def sddmm(pos, crd, vals, C, Dnk, sel=None, accurate: bool = False) -> np.ndarray:
    """A(i,j) = B(i,j) C(i,k) D(k,j) on B's pattern; Dnk[j,k] = D(k,j). vals None => 1."""
    pos, crd, C, Dnk = _i32(pos), _i32(crd), _f64(C), _f64(Dnk)
    v = None if vals is None else _f64(vals)
    s, ns = _sel(sel)
    n = pos.shape[0] - 1
    K = C.shape[1]
    out = np.zeros(ns if s is not None else crd.shape[0], dtype=np.float64)
    fn = lib().orc_sddmm_acc if accurate else lib().orc_sddmm
    fn(n, K, _ptr(pos), _ptr(crd), _ptr(v), _ptr(C), K, _ptr(Dnk), K, ns, _ptr(s), _ptr(out))
    return out


def spttv(pos1, crd1, pos2, crd2, vals, c, sel=None, accurate: bool = False) -> np.ndarray:
    """A(i,j) = B(i,j,k) c(k); one value per fiber of B."""
    pos1, crd1, pos2, crd2 = _i32(pos1), _i32(crd1), _i32(pos2), _i32(crd2)
    vals, c = _f64(vals), _f64(c)
    s, ns = _sel(sel)
    I = pos1.shape[0] - 1
    out = np.zeros(ns if s is not None else crd1.shape[0], dtype=np.float64)
    fn = lib().orc_spttv_acc if accurate else lib().orc_spttv
    fn(I, _ptr(pos1), _ptr(crd1), _ptr(pos2), _ptr(crd2), _ptr(vals), _ptr(c), ns, _ptr(s), _ptr(out))
    return out


def spmttkrp(pos1, crd1, pos2, crd2, vals, C, D, sel=None, accurate: bool = False) -> np.ndarray:
    """A(i,l) = B(i,j,k) C(j,l) D(k,l)."""
    pos1, crd1, pos2, crd2 = _i32(pos1), _i32(crd1), _i32(pos2), _i32(crd2)
    vals, C, D = _f64(vals), _f64(C), _f64(D)
    s, ns = _sel(sel)
    I = pos1.shape[0] - 1
    R = C.shape[1]
    A = np.zeros((ns if s is not None else I, R), dtype=np.float64)
    fn = lib().orc_spmttkrp_acc if accurate else lib().orc_spmttkrp
    fn(I, R, _ptr(pos1), _ptr(crd1), _ptr(pos2), _ptr(crd2), _ptr(vals), _ptr(C), R, _ptr(D), R,
       ns, _ptr(s), _ptr(A), R)
    return A
