"""Shared test helpers: small structured inputs, golden-file reader, error metrics."""
import os

import numpy as np

import spd_synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name):
    """Parse a ``key value...`` fixture into a dict of numpy arrays (ints stay ints)."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            arr = np.array([float(v) for v in vals])
            if np.all(arr == np.round(arr)):
                arr = arr.astype(np.int64)
            out[key] = arr
    return out


def small_csr(rng, n, m, density, empty_frac=0.2, long_rows=0, integer=False):
    """A small CSR with some empty rows and optionally a few dense ("long") rows."""
    mask = rng.random((n, m)) < density
    if empty_frac > 0:
        mask[rng.random(n) < empty_frac, :] = False
    for _ in range(long_rows):
        mask[rng.integers(0, n), :] = rng.random(m) < 0.9
    rows, cols = np.nonzero(mask)
    if integer:
        vals = rng.integers(-8, 9, size=rows.shape[0]).astype(np.float64)
    else:
        vals = rng.uniform(-1, 1, size=rows.shape[0])
    return spd_synth.csr_from_coords(n, m, rows, cols, vals=vals)


def small_csf(rng, dims, density, integer=False):
    """A small CSF 3-tensor with some empty slices and fibers of varied length."""
    I, J, K = dims
    mask = rng.random(dims) < density
    mask[rng.random(I) < 0.2] = False
    i, j, k = np.nonzero(mask)  # lexicographic order already
    if integer:
        vals = rng.integers(-8, 9, size=i.shape[0]).astype(np.float64)
    else:
        vals = rng.uniform(-1, 1, size=i.shape[0])
    return spd_synth.csf3_from_coords(dims, i, j, k, vals)


def dense_of_csr(A):
    D = np.zeros((A.nrows, A.ncols))
    for i in range(A.nrows):
        for p in range(A.pos[i], A.pos[i + 1]):
            D[i, A.crd[p]] = A.vals[p]
    return D


def dense_of_csf(T):
    D = np.zeros(T.dims)
    I = T.dims[0]
    for i in range(I):
        for f in range(T.pos1[i], T.pos1[i + 1]):
            for p in range(T.pos2[f], T.pos2[f + 1]):
                D[i, T.crd1[f], T.crd2[p]] = T.vals[p]
    return D


def row_of_positions(pos):
    """Row index of every position (for building per-nonzero coordinates in tests)."""
    n = pos.shape[0] - 1
    return np.repeat(np.arange(n), np.diff(pos))


def normalized_error(got, ref, scale):
    """max |got - ref| / max(|ref|, scale) elementwise, where ``scale`` is the sum of
    the absolute values of the terms of each output (the usual error-bound normaliser)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    denom = np.maximum(np.abs(ref), np.asarray(scale, dtype=np.float64))
    denom = np.where(denom == 0, 1.0, denom)
    return np.abs(got - ref) / denom


U24 = 2.0 ** -24  # unit roundoff of binary32


def binary32_gate(nterms, extra=0.0):
    """Error gate of an output summed from n terms with binary32 accumulation, relative
    to the normaliser of ``normalized_error``: (2 log2 n + 2 + extra) * 2^-24, i.e.
    2 + extra units for a single term. The 2 log2 n units allow a summation tree (a
    per-thread or per-lane run plus a shuffle or scan tree, each about log2 n deep); the
    2 units cover the rounding of each product and of the result; ``extra`` adds units
    for statements whose terms are rounded more than once (triple products)."""
    n = np.maximum(np.asarray(nterms, dtype=np.float64), 1.0)
    return (2.0 * np.log2(n) + 2.0 + extra) * U24


def check_error(got, ref, scale, binary64, nterms, what, extra=0.0):
    """Asserts the normalised error of every output: <= 1e-12 for binary64 results,
    <= binary32_gate(nterms) otherwise (nterms broadcast against the outputs). Returns
    the largest normalised error."""
    err = normalized_error(got, ref, scale)
    if err.size == 0:
        return 0.0
    tol = np.full(err.shape, 1e-12) if binary64 else np.broadcast_to(binary32_gate(nterms, extra), err.shape)
    over = err - tol
    k = int(np.argmax(over))
    assert over.flat[k] <= 0, "%s: normalised error %.3e > gate %.3e at output %s (max error %.3e)" % (
        what, err.flat[k], tol.flat[k], np.unravel_index(k, err.shape), err.max())
    return float(err.max())


def row_lengths(pos):
    """Entries of every row (or fiber) of a Compressed level."""
    return np.diff(np.asarray(pos, dtype=np.int64))
