"""Seeded synthetic inputs shaped like the paper's workloads (Section VI, Table of tensors).

The paper evaluates on SuiteSparse matrices and FROSTT/Freebase 3-tensors. None of
those datasets ship here, so these generators stand in for them:

* ``rmat_csr``      -- power-law CSR matrices (web/social graphs such as twitter7, sk-2005)
* ``uniform_csr``   -- CSR matrices with a fixed or bounded number of uniform random
                       columns per row
* ``zipf_csf3``     -- 3-tensors whose mode coordinates are Zipf distributed, stored as
                       CSF = {Dense, Compressed, Compressed} (FROSTT / Freebase stand-in)
* ``uniform`` / ``normal`` -- dense operands

This module holds no arithmetic of the sparse kernels themselves: it only draws
coordinates and values and lays them out in the pos/crd level format of Section III-B
(``pos`` holds ``n+1`` offsets; the children of parent entry ``i`` live at
``crd[pos[i]:pos[i+1]]``). It is shared, as the only common code, by the CPU oracle
tests and by the GPU path, so both sides always see bit-identical inputs.

Every generator is deterministic in its ``seed`` (numpy PCG64 streams).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "CSR",
    "CSF3",
    "rmat_csr",
    "uniform_csr",
    "zipf_csf3",
    "batched_uniform_csr",
    "uniform",
    "normal",
    "csr_from_coords",
    "csf3_from_coords",
    "limit_csr",
    "limit_rows_csr",
    "limit_csf3",
    "limit_interval_csr",
]


@dataclasses.dataclass
class CSR:
    """A matrix stored as {Dense, Compressed}: rows dense, columns compressed."""

    nrows: int
    ncols: int
    pos: np.ndarray  # int32 [nrows+1]
    crd: np.ndarray  # int32 [nnz]
    vals: np.ndarray  # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.crd.shape[0])


@dataclasses.dataclass
class CSF3:
    """A 3-tensor stored as {Dense, Compressed, Compressed} (CSF).

    Level 1 (i) is dense; level 2 (j) holds one entry per non-empty fiber (i, j) in
    ``pos1/crd1``; level 3 (k) holds one entry per nonzero in ``pos2/crd2``.
    """

    dims: tuple
    pos1: np.ndarray  # int32 [I+1]
    crd1: np.ndarray  # int32 [F]
    pos2: np.ndarray  # int32 [F+1]
    crd2: np.ndarray  # int32 [nnz]
    vals: np.ndarray  # float64 [nnz]

    @property
    def nfib(self) -> int:
        return int(self.crd1.shape[0])

    @property
    def nnz(self) -> int:
        return int(self.crd2.shape[0])


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(seed))


def _sorted_unique(key: np.ndarray) -> np.ndarray:
    """Sorted distinct values of an int64 array (sort + run mask)."""
    key = np.sort(key, kind="quicksort")
    if key.shape[0] == 0:
        return key
    keep = np.empty(key.shape[0], dtype=bool)
    keep[0] = True
    np.not_equal(key[1:], key[:-1], out=keep[1:])
    return key[keep]


def uniform(shape, seed: int, dtype=np.float64, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Dense array of i.i.d. uniform values in [lo, hi).

    With ``dtype=np.float32`` the values are drawn on the 2^-24 grid of float32, so
    upcasting them to float64 is exact and every precision mode sees the same numbers.
    """
    rng = _rng(seed)
    if dtype == np.float32:
        u = rng.random(shape, dtype=np.float32)
        # (hi-lo)*u + lo with lo=-1, hi=1 is exact on the 2^-24 grid
        return (np.float32(hi - lo) * u + np.float32(lo)).astype(np.float32)
    return rng.uniform(lo, hi, size=shape).astype(dtype)


def normal(shape, seed: int, dtype=np.float64) -> np.ndarray:
    """Dense array of i.i.d. standard normal values."""
    rng = _rng(seed)
    if dtype == np.float32:
        return rng.standard_normal(shape, dtype=np.float32)
    return rng.standard_normal(shape).astype(dtype)


def csr_from_coords(nrows: int, ncols: int, rows: np.ndarray, cols: np.ndarray,
                    vals: Optional[np.ndarray] = None, value_seed: Optional[int] = None) -> CSR:
    """Build a CSR from coordinates: sorts them, merges duplicates, builds pos/crd.

    When ``vals`` is None the values are drawn after de-duplication, in sorted
    coordinate order, uniform in [-1, 1) from the stream ``value_seed``.
    """
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    key = rows * np.int64(ncols) + cols
    if vals is None:
        key = _sorted_unique(key)
    else:
        order = np.argsort(key, kind="stable")
        key = key[order]
        v = np.asarray(vals, dtype=np.float64)[order]
        keep = np.ones(key.shape[0], dtype=bool)
        keep[1:] = key[1:] != key[:-1]
        # duplicates are merged by keeping the first occurrence's value
        key = key[keep]
        vals = v[keep]
    r = key // np.int64(ncols)
    c = key - r * np.int64(ncols)
    counts = np.bincount(r, minlength=nrows).astype(np.int64)
    pos = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(counts, out=pos[1:])
    if vals is None:
        vals = uniform(key.shape[0], value_seed if value_seed is not None else 1)
    return CSR(nrows, ncols, pos.astype(np.int32), c.astype(np.int32), np.asarray(vals, dtype=np.float64))


def rmat_csr(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19,
             c: float = 0.19, seed: int = 0, chunk: int = 1 << 22) -> CSR:
    """R-MAT power-law matrix (Chakrabarti, Zhan, Faloutsos 2004).

    ``edge_factor * 2^scale`` edges are sampled; for every edge and every bit, from the
    most significant down, a quadrant is chosen with probabilities (a, b, c, d=1-a-b-c):
    a = (row bit 0, col bit 0), b = (0, 1), c = (1, 0), d = (1, 1). The choice compares
    one uniform 32-bit draw per edge and bit against the cumulative thresholds
    round(2^32 * (a, a+b, a+b+c)). No noise and no permutation are applied, so the heavy
    rows and columns have small indices. Duplicate edges are merged; values are drawn
    afterwards, uniform in [-1, 1), in sorted order (stream ``seed + 1``).
    """
    n = 1 << scale
    m = edge_factor * n
    rng = _rng(seed)
    ta = np.uint32(min(round(a * 2.0 ** 32), 2 ** 32 - 1))
    tab = np.uint32(min(round((a + b) * 2.0 ** 32), 2 ** 32 - 1))
    tabc = np.uint32(min(round((a + b + c) * 2.0 ** 32), 2 ** 32 - 1))
    key = np.empty(m, dtype=np.int64)
    done = 0
    while done < m:
        cnt = min(chunk, m - done)
        row = np.zeros(cnt, dtype=np.int64)
        col = np.zeros(cnt, dtype=np.int64)
        t1 = np.empty(cnt, dtype=bool)
        t2 = np.empty(cnt, dtype=bool)
        t3 = np.empty(cnt, dtype=bool)
        for bit in range(scale - 1, -1, -1):
            u = rng.integers(0, 1 << 32, size=cnt, dtype=np.uint32)
            np.greater_equal(u, ta, out=t1)
            np.greater_equal(u, tab, out=t2)
            np.greater_equal(u, tabc, out=t3)
            row += t2.astype(np.int64) << bit          # quadrants c, d set the row bit
            np.logical_xor(t1, t2, out=t1)
            np.logical_xor(t1, t3, out=t1)             # quadrants b, d set the column bit
            col += t1.astype(np.int64) << bit
        key[done:done + cnt] = (row << scale) | col
        done += cnt
    key = _sorted_unique(key)
    rows = key >> scale
    cols = key & (n - 1)
    counts = np.bincount(rows, minlength=n).astype(np.int64)
    pos = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=pos[1:])
    vals = uniform(key.shape[0], seed + 1)
    return CSR(n, n, pos.astype(np.int32), cols.astype(np.int32), vals)


def _distinct_sorted_rows(rng: np.random.Generator, ncols: int, ks: np.ndarray):
    """For every row q draw ks[q] distinct columns uniformly at random, sorted.

    Sparse rows (ks[q]^2 <= 4 ncols): whole-row rejection -- a row draws its ks[q] columns
    i.i.d. and rows whose draws repeat a column are drawn again. Dense rows: the first
    ks[q] columns of a random permutation (the order of ncols random keys). Either way
    every row is a uniform random ks[q]-subset. Returns (columns, row offsets)."""
    nrows = ks.shape[0]
    starts = np.zeros(nrows + 1, dtype=np.int64)
    np.cumsum(ks, out=starts[1:])
    kmax = int(ks.max()) if nrows else 0
    out = np.empty((nrows, max(kmax, 1)), dtype=np.int64)
    big = np.iinfo(np.int64).max
    slot = np.arange(max(kmax, 1))[None, :]
    dense = np.flatnonzero(ks * ks > 4 * ncols)
    chunk = max(1, (1 << 24) // max(ncols, 1))
    for c0 in range(0, dense.size, chunk):
        rows_c = dense[c0:c0 + chunk]
        perm = np.argsort(rng.random((rows_c.size, ncols)), axis=1, kind="stable")[:, :max(kmax, 1)]
        perm[slot[:, :perm.shape[1]] >= ks[rows_c][:, None]] = big
        perm.sort(axis=1)
        out[rows_c, :perm.shape[1]] = perm
    todo = np.flatnonzero(ks * ks <= 4 * ncols)
    while todo.size:
        cand = rng.integers(0, ncols, size=(todo.size, max(kmax, 1)), dtype=np.int64)
        cand[slot >= ks[todo][:, None]] = big
        cand.sort(axis=1)
        dup = (cand[:, 1:] == cand[:, :-1]) & (cand[:, 1:] != big)
        bad = dup.any(axis=1)
        good = ~bad
        out[todo[good]] = cand[good]
        todo = todo[bad]
    cols = out[slot < ks[:, None]] if nrows else np.zeros(0, dtype=np.int64)
    return cols, starts


def uniform_csr(nrows: int, ncols: int, nnz_per_row, seed: int = 0,
                value_seed: Optional[int] = None) -> CSR:
    """CSR with uniform random, sorted, distinct columns per row.

    ``nnz_per_row`` is either an int (every row gets exactly that many columns) or a
    (lo, hi) pair (row counts uniform integers in [lo, hi], inclusive).
    """
    rng = _rng(seed)
    if isinstance(nnz_per_row, (tuple, list)):
        lo, hi = nnz_per_row
        ks = rng.integers(lo, hi + 1, size=nrows).astype(np.int64)
    else:
        ks = np.full(nrows, int(nnz_per_row), dtype=np.int64)
    ks = np.minimum(ks, ncols)
    cols, starts = _distinct_sorted_rows(rng, ncols, ks)
    vals = uniform(cols.shape[0], value_seed if value_seed is not None else seed + 1)
    return CSR(nrows, ncols, starts.astype(np.int32), cols.astype(np.int32), vals)


def banded_csr(nrows: int, half_width: int, seed: int = 0, value_dtype=np.float64) -> CSR:
    """Square banded matrix: row i holds every column in [i - w, i + w] inside [0, n)
    (2w + 1 per interior row), values uniform in [-1, 1) from the stream ``seed`` drawn
    in position order (on the binary32 grid when ``value_dtype`` is float32). The
    structure is written directly, row block by row block, with no sorting."""
    n, w = int(nrows), int(half_width)
    i = np.arange(n, dtype=np.int64)
    lo = np.maximum(i - w, 0)
    hi = np.minimum(i + w, n - 1)
    pos = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(hi - lo + 1, out=pos[1:])
    nnz = int(pos[-1])
    crd = np.empty(nnz, dtype=np.int32)
    step = 1 << 20
    for r0 in range(0, n, step):
        r1 = min(n, r0 + step)
        p0, p1 = int(pos[r0]), int(pos[r1])
        # column of position p in row r = lo[r] + (p - pos[r])
        off = np.repeat((lo[r0:r1] - pos[r0:r1]).astype(np.int64), (hi[r0:r1] - lo[r0:r1] + 1))
        crd[p0:p1] = (off + np.arange(p0, p1, dtype=np.int64)).astype(np.int32)
    vals = uniform(nnz, seed, dtype=value_dtype).astype(np.float64) if value_dtype == np.float64 else \
        uniform(nnz, seed, dtype=np.float32)
    return CSR(n, n, pos.astype(np.int32), crd, vals)


def shifted_csr(A: CSR, shift: int, seed: int, value_dtype=np.float64) -> CSR:
    """A's pattern with every column moved by ``shift`` (mod ncols) -- the way the paper
    builds the extra operands of a multi-input statement from one matrix -- and fresh
    values uniform in [-1, 1) from the stream ``seed``. Rows stay sorted: the entries
    that wrap around (a suffix of each sorted row) move to the front."""
    n, m = A.nrows, A.ncols
    crd = A.crd.astype(np.int64)
    lens = np.diff(A.pos).astype(np.int64)
    starts = np.repeat(A.pos[:-1].astype(np.int64), lens)
    off = np.arange(crd.shape[0], dtype=np.int64) - starts  # offset inside the row
    newc = crd + shift
    wrapped = newc >= m
    cw = np.concatenate([[0], np.cumsum(wrapped, dtype=np.int64)])
    w = cw[A.pos[1:]] - cw[A.pos[:-1]]  # wrapped entries per row
    w_e = np.repeat(w, lens)
    len_e = np.repeat(lens, lens)
    dest = starts + np.where(wrapped, off - (len_e - w_e), off + w_e)
    out = np.empty(crd.shape[0], dtype=np.int32)
    out[dest] = (newc % m).astype(np.int32) if m else newc.astype(np.int32)
    vals = uniform(crd.shape[0], seed, dtype=value_dtype)
    if value_dtype != np.float32:
        vals = vals.astype(np.float64)
    return CSR(n, m, A.pos.copy(), out, vals)


def batched_uniform_csr(count: int, rows_lo: float, rows_hi: float, nnz_lo: int, nnz_hi: int,
                        seed: int = 0) -> List[CSR]:
    """``count`` square CSR matrices: rows log-uniform in [rows_lo, rows_hi],
    per-row nnz uniform integers in [nnz_lo, nnz_hi], uniform random columns."""
    rng = _rng(seed)
    u = rng.random(count)
    sizes = np.floor(10.0 ** (np.log10(rows_lo) + u * (np.log10(rows_hi) - np.log10(rows_lo)))).astype(np.int64)
    out = []
    for mi, nm in enumerate(sizes):
        nm = int(max(nm, 1))
        out.append(uniform_csr(nm, nm, (nnz_lo, nnz_hi), seed=seed * 100003 + 2 * mi + 7,
                               value_seed=seed * 100003 + 2 * mi + 8))
    return out


def _zipf_sampler(size: int, s: float):
    """Inverse-CDF table of Zipf(s) truncated to ranks 1..size (rank r -> index r-1)."""
    r = np.arange(1, size + 1, dtype=np.float64)
    pmf = r ** (-s)
    cdf = np.cumsum(pmf)
    cdf /= cdf[-1]
    return cdf


def csf3_from_coords(dims: Sequence[int], i: np.ndarray, j: np.ndarray, k: np.ndarray,
                     vals: np.ndarray) -> CSF3:
    """Build CSF {Dense, Compressed, Compressed} from coordinates that are already
    sorted lexicographically by (i, j, k) and free of duplicates."""
    I, J, K = (int(d) for d in dims)
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    k = np.asarray(k, dtype=np.int64)
    nnz = i.shape[0]
    if nnz:
        newfib = np.ones(nnz, dtype=bool)
        newfib[1:] = (i[1:] != i[:-1]) | (j[1:] != j[:-1])
        fstart = np.flatnonzero(newfib)
    else:
        fstart = np.zeros(0, dtype=np.int64)
    pos2 = np.concatenate([fstart, [nnz]]).astype(np.int64)
    crd1 = j[fstart]
    fslice = i[fstart]
    counts = np.bincount(fslice, minlength=I).astype(np.int64)
    pos1 = np.zeros(I + 1, dtype=np.int64)
    np.cumsum(counts, out=pos1[1:])
    return CSF3((I, J, K), pos1.astype(np.int32), crd1.astype(np.int32), pos2.astype(np.int32),
                k.astype(np.int32), np.asarray(vals, dtype=np.float64))


def zipf_csf3(dims: Sequence[int], nnz: int, s: float = 1.1, seed: int = 0,
              draw_factor: float = 1.6) -> CSF3:
    """3-tensor whose coordinates are independently Zipf(s) on each mode.

    Each coordinate is drawn from Zipf(s) truncated to [0, dim) (rank r maps to index
    r-1, no permutation, so the hot indices are low). Triples are drawn in batches
    until at least ``nnz`` distinct ones exist; if there are more, a seeded uniform
    random subset of exactly ``nnz`` distinct triples is kept. They are sorted
    lexicographically. Values are uniform in [-1, 1), drawn after de-duplication in
    sorted order (stream ``seed + 1``).
    """
    I, J, K = (int(d) for d in dims)
    rng = _rng(seed)
    cdfs = [_zipf_sampler(d, s) for d in (I, J, K)]
    bits_j = max(1, int(math.ceil(math.log2(max(J, 2)))))
    bits_k = max(1, int(math.ceil(math.log2(max(K, 2)))))
    uk = np.zeros(0, dtype=np.int64)
    draw = int(nnz * draw_factor) + 16
    while True:
        coords = []
        for cdf in cdfs:
            u = rng.random(draw)
            coords.append(np.minimum(np.searchsorted(cdf, u, side="right"), cdf.shape[0] - 1).astype(np.int64))
        key = (coords[0] << (bits_j + bits_k)) | (coords[1] << bits_k) | coords[2]
        uk = _sorted_unique(np.concatenate([uk, key]))
        if uk.shape[0] >= nnz:
            break
        draw = max(int((nnz - uk.shape[0]) * 3), 1024)
    if uk.shape[0] > nnz:
        sel = np.sort(rng.choice(uk.shape[0], size=nnz, replace=False))
        uk = uk[sel]
    i = uk >> (bits_j + bits_k)
    j = (uk >> bits_k) & ((1 << bits_j) - 1)
    k = uk & ((1 << bits_k) - 1)
    vals = uniform(uk.shape[0], seed + 1)
    return csf3_from_coords((I, J, K), i, j, k, vals)


# ------------------------------------------------------------------ size-limit inputs
#
# Inputs with as many entries, rows or fibers as the int32 level format admits. Values
# are small integers in [-3, 3], returned as int8 (exact in binary64, binary32 and
# bfloat16): with small integer operands every product and every partial sum is an
# integer far below 2^24, so any summation order gives the exact result and outputs can
# be compared bit for bit. Columns are uniform and not sorted within a row (the level
# format does not require it). Arrays are built without full-size int64 temporaries.


def _small_ints(rng: np.random.Generator, n: int) -> np.ndarray:
    return rng.integers(-3, 4, size=n, dtype=np.int8)


def _ragged_lengths(rng: np.random.Generator, n: int, total: int, empty_frac: float) -> np.ndarray:
    """n non-negative int64 lengths summing to exactly total: lognormal shares, about
    empty_frac of them zero."""
    w = rng.lognormal(0.0, 1.5, n)
    w[rng.random(n) < empty_frac] = 0.0
    if not w.any():
        w[0] = 1.0
    lens = np.floor(w * (total / w.sum())).astype(np.int64)
    short = total - int(lens.sum())  # 0 <= short < number of non-empty entries
    nz = np.flatnonzero(w)
    lens[rng.choice(nz, size=short, replace=short > nz.shape[0])] += 1
    if lens.sum() != total:  # a repeated choice adds more than once; settle the rest on one entry
        lens[nz[0]] += total - int(lens.sum())
    return lens


def limit_csr(nrows: int, ncols: int, nnz: int, seed: int = 0, long_row: int = 0) -> CSR:
    """CSR with exactly ``nnz`` entries over ``nrows`` rows of lognormal lengths (about
    10% empty) and, if ``long_row`` > 0, row nrows // 3 holding ``long_row`` of them;
    int8 values in [-3, 3]."""
    rng = _rng(seed)
    lens = _ragged_lengths(rng, nrows, nnz - long_row, 0.1)
    if long_row:
        lens[nrows // 3] += long_row
    pos = np.zeros(nrows + 1, dtype=np.int32)
    np.cumsum(lens, out=pos[1:], dtype=np.int32)
    crd = rng.integers(0, ncols, size=nnz, dtype=np.int32)
    return CSR(nrows, ncols, pos, crd, _small_ints(rng, nnz))


def limit_rows_csr(nrows: int, ncols: int, nnz: int, seed: int = 0) -> CSR:
    """CSR with ``nrows`` rows (up to the format's limit) and ``nnz`` entries in random
    rows, the first and last row among them; int8 values in [-3, 3]. ``pos`` is built
    as a step function of the occupied rows, with no per-row temporary wider than int32."""
    rng = _rng(seed)
    rows = np.concatenate([[0, nrows - 1], rng.integers(0, nrows, size=nnz - 2)])
    u, cnt = np.unique(rows, return_counts=True)
    # pos[i] = entries in rows < i: 0 up to u[0], then the count before u[k] + 1 ... up to u[k+1]
    values = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int32)
    reps = np.diff(np.concatenate([[-1], u, [nrows]]))
    pos = np.repeat(values, reps)
    crd = rng.integers(0, ncols, size=nnz, dtype=np.int32)
    return CSR(nrows, ncols, pos, crd, _small_ints(rng, nnz))


def limit_csf3(dims: Sequence[int], nnz: int, seed: int = 0) -> CSF3:
    """CSF 3-tensor with exactly ``nnz`` entries in fibers of 1 to 3 entries (about nnz/2
    fibers), the fibers spread over the slices in lognormal counts (about 10% empty
    slices), uniform j per fiber and k per entry (neither sorted nor distinct within its
    parent); int8 values in [-3, 3]."""
    I, J, K = (int(d) for d in dims)
    rng = _rng(seed)
    # fiber ends in chunks of 2^24 fibers until one reaches nnz; that fiber is cut there
    parts = [np.zeros(1, dtype=np.int32)]
    total = 0
    while total < nnz:
        ends = total + np.cumsum(rng.integers(1, 4, size=1 << 24, dtype=np.int64))
        k = int(np.searchsorted(ends, nnz))
        if k < ends.shape[0]:
            ends = ends[:k + 1]
            ends[k] = nnz
        parts.append(ends.astype(np.int32))
        total = int(ends[-1])
    pos2 = np.concatenate(parts)
    del parts
    F = pos2.shape[0] - 1
    pos1 = np.zeros(I + 1, dtype=np.int32)
    np.cumsum(_ragged_lengths(rng, I, F, 0.1), out=pos1[1:], dtype=np.int32)
    crd1 = rng.integers(0, J, size=F, dtype=np.int32)
    crd2 = rng.integers(0, K, size=nnz, dtype=np.int32)
    return CSF3((I, J, K), pos1, crd1, pos2, crd2, _small_ints(rng, nnz))


def limit_interval_csr(nrows: int, ncols: int, nnz: int, seed: int = 0) -> CSR:
    """CSR with exactly ``nnz`` entries whose rows are runs of consecutive columns
    [o_i, o_i + len_i) at a random offset (sorted and distinct, as SpAdd3's operands must
    be): lognormal lengths (about 10% empty rows) capped at ``ncols``; int8 values in
    [-3, 3]. Runs of different operands overlap in part, so a three-way union merges."""
    rng = _rng(seed)
    lens = np.minimum(_ragged_lengths(rng, nrows, nnz, 0.1), ncols)
    short = nnz - int(lens.sum())
    if short > 0:  # the capped excess goes to the first rows with room
        room = np.cumsum(ncols - lens)
        k = int(np.searchsorted(room, short))
        lens[:k] = ncols
        lens[k] += short - (int(room[k - 1]) if k else 0)
    off = (rng.random(nrows) * (ncols - lens + 1)).astype(np.int64)
    pos = np.zeros(nrows + 1, dtype=np.int32)
    np.cumsum(lens, out=pos[1:], dtype=np.int32)
    crd = np.arange(nnz, dtype=np.int32)  # position p of row i gets column o_i + (p - pos[i])
    crd -= np.repeat((pos[:-1].astype(np.int64) - off).astype(np.int32), lens)
    return CSR(nrows, ncols, pos, crd, _small_ints(rng, nnz))
