"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* hand-worked fixtures under tests/golden (integer data, exact)
* dense brute force on small-integer tensors (every sum is exact in binary64, so any
  dropped term, wrong index, wrong sign or transposed operand changes the result)
* closed forms (identity, unit vectors, all-ones operands, empty inputs)
* linearity in the sparse values and in the dense operand
* exact rational arithmetic for the compensated (Dot2) variants
* partition invariants and an independent library cross-check (numpy searchsorted,
  torch.sparse on the CPU)
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import spd_synth
from tests._util import (dense_of_csf, dense_of_csr, normalized_error, read_golden, small_csf,
                         small_csr)

SEEDS = [0, 1, 2, 3]


# ------------------------------------------------------------------------------ golden

def test_golden_spmv():
    g = read_golden("spmv_4x5.txt")
    y = oracle.spmv(g["pos"], g["crd"], g["vals"], g["x"])
    assert np.array_equal(y, g["y"])
    assert np.array_equal(oracle.spmv(g["pos"], g["crd"], g["vals"], g["x"], accurate=True), g["y"])


def test_golden_spmm():
    g = read_golden("spmm_4x5_L2.txt")
    L = int(g["L"][0])
    X = g["X"].reshape(-1, L)
    for acc in (False, True):
        Y = oracle.spmm(g["pos"], g["crd"], g["vals"], X, accurate=acc)
        assert np.array_equal(Y, g["Y"].reshape(-1, L))


def test_golden_spmm_t():
    g = read_golden("spmm_t_4x5_L2.txt")
    L = int(g["L"][0])
    for acc in (False, True):
        dX = oracle.spmm_t(g["pos"], g["crd"], g["vals"], g["dY"].reshape(-1, L), int(g["ncols"][0]), accurate=acc)
        assert np.array_equal(dX, g["dX"].reshape(-1, L))


def test_golden_sddmm():
    g = read_golden("sddmm_4x5_K2.txt")
    K = int(g["K"][0])
    for acc in (False, True):
        out = oracle.sddmm(g["pos"], g["crd"], g["vals"], g["C"].reshape(-1, K), g["Dnk"].reshape(-1, K), accurate=acc)
        assert np.array_equal(out, g["out"])
        # sampled positions give the same values
        sel = np.array([5, 0, 3])
        out_s = oracle.sddmm(g["pos"], g["crd"], g["vals"], g["C"].reshape(-1, K), g["Dnk"].reshape(-1, K), sel=sel, accurate=acc)
        assert np.array_equal(out_s, g["out"][sel])


def test_golden_spttv():
    g = read_golden("spttv_3x3x4.txt")
    for acc in (False, True):
        out = oracle.spttv(g["pos1"], g["crd1"], g["pos2"], g["crd2"], g["vals"], g["c"], accurate=acc)
        assert np.array_equal(out, g["out"])


def test_golden_spmttkrp():
    g = read_golden("spmttkrp_3x3x4_R2.txt")
    R = int(g["R"][0])
    for acc in (False, True):
        A = oracle.spmttkrp(g["pos1"], g["crd1"], g["pos2"], g["crd2"], g["vals"],
                            g["C"].reshape(-1, R), g["D"].reshape(-1, R), accurate=acc)
        assert np.array_equal(A, g["A"].reshape(-1, R))


def test_golden_partitions():
    g = read_golden("partition_4x5.txt")
    rows, poss = oracle.merge_path(g["pos"], g["diag"])
    assert np.array_equal(rows, g["merge_rows"])
    assert np.array_equal(poss, g["merge_pos"])
    assert np.array_equal(oracle.pos_split(g["pos"], g["q"]), g["q_rows"])
    assert np.array_equal(oracle.row_split(4, int(g["pieces"][0])), g["row_bounds"])


def test_golden_transpose():
    g = read_golden("transpose_4x5.txt")
    t_pos, t_crd, perm = oracle.csr_transpose(g["pos"], g["crd"], int(g["ncols"][0]))
    assert np.array_equal(t_pos, g["t_pos"])
    assert np.array_equal(t_crd, g["t_crd"])
    assert np.array_equal(perm, g["perm"])
    assert np.array_equal(g["vals"][perm], g["t_vals"])


def test_golden_spadd3():
    g = read_golden("spadd3_3x4.txt")
    n, m = int(g["nrows"][0]), int(g["ncols"][0])
    B, C, D = [spd_synth.CSR(n, m, g[k + "_pos"], g[k + "_crd"], g[k + "_vals"].astype(np.float64)) for k in "bcd"]
    assert np.array_equal(oracle.spadd3_count(B, C, D), g["row_nnz"])
    ap, ac, av = oracle.spadd3(B, C, D)
    assert np.array_equal(ap, g["a_pos"]) and np.array_equal(ac, g["a_crd"])
    assert np.array_equal(av, g["a_vals"])


def test_golden_column_blocks():
    g = read_golden("column_blocks_4x5.txt")
    blk_pos, blk_crd, perm, nnz = oracle.column_blocks(g["pos"], g["crd"], g["bounds"])
    assert np.array_equal(blk_pos[0], g["blk_pos0"]) and np.array_equal(blk_pos[1], g["blk_pos1"])
    assert np.array_equal(blk_crd, g["blk_crd"]) and np.array_equal(perm, g["perm"])
    assert np.array_equal(nnz, g["blk_nnz"])


# ------------------------------------------------------------------------------ dense brute force

@pytest.mark.parametrize("seed", SEEDS)
def test_spmv_spmm_dense_bruteforce(seed):
    rng = np.random.default_rng(seed)
    n, m = int(rng.integers(1, 48)), int(rng.integers(1, 48))
    A = small_csr(rng, n, m, 0.2, long_rows=1, integer=True)
    D = dense_of_csr(A)
    x = rng.integers(-8, 9, size=m).astype(np.float64)
    X = rng.integers(-8, 9, size=(m, 5)).astype(np.float64)
    for acc in (False, True):
        assert np.array_equal(oracle.spmv(A.pos, A.crd, A.vals, x, accurate=acc), D @ x)
        assert np.array_equal(oracle.spmm(A.pos, A.crd, A.vals, X, accurate=acc), D @ X)
    sel = rng.integers(0, n, size=7)
    assert np.array_equal(oracle.spmv(A.pos, A.crd, A.vals, x, sel=sel), (D @ x)[sel])
    assert np.array_equal(oracle.spmm(A.pos, A.crd, A.vals, X, sel=sel, accurate=True), (D @ X)[sel])


@pytest.mark.parametrize("seed", SEEDS)
def test_spmm_t_dense_bruteforce(seed):
    rng = np.random.default_rng(100 + seed)
    n, m = int(rng.integers(1, 40)), int(rng.integers(1, 40))
    A = small_csr(rng, n, m, 0.25, long_rows=1, integer=True)
    D = dense_of_csr(A)
    dY = rng.integers(-8, 9, size=(n, 3)).astype(np.float64)
    for acc in (False, True):
        assert np.array_equal(oracle.spmm_t(A.pos, A.crd, A.vals, dY, m, accurate=acc), D.T @ dY)


@pytest.mark.parametrize("seed", SEEDS)
def test_sddmm_dense_bruteforce(seed):
    rng = np.random.default_rng(200 + seed)
    n, m, K = int(rng.integers(1, 40)), int(rng.integers(1, 40)), int(rng.integers(1, 9))
    A = small_csr(rng, n, m, 0.25, integer=True)
    Dn = dense_of_csr(A)
    C = rng.integers(-8, 9, size=(n, K)).astype(np.float64)
    Dnk = rng.integers(-8, 9, size=(m, K)).astype(np.float64)
    full = Dn * (C @ Dnk.T)  # B(i,j) * sum_k C(i,k) D(k,j) on every (i,j)
    rows = np.repeat(np.arange(n), np.diff(A.pos))
    want = full[rows, A.crd]
    for acc in (False, True):
        assert np.array_equal(oracle.sddmm(A.pos, A.crd, A.vals, C, Dnk, accurate=acc), want)
    # pattern only: B values are taken as 1
    pat = (C @ Dnk.T)[rows, A.crd]
    assert np.array_equal(oracle.sddmm(A.pos, A.crd, None, C, Dnk), pat)


@pytest.mark.parametrize("seed", SEEDS)
def test_spttv_spmttkrp_dense_bruteforce(seed):
    rng = np.random.default_rng(300 + seed)
    dims = tuple(int(v) for v in rng.integers(1, 12, size=3))
    T = small_csf(rng, dims, 0.3, integer=True)
    Dn = dense_of_csf(T)
    c = rng.integers(-8, 9, size=dims[2]).astype(np.float64)
    R = int(rng.integers(1, 6))
    C = rng.integers(-8, 9, size=(dims[1], R)).astype(np.float64)
    D = rng.integers(-8, 9, size=(dims[2], R)).astype(np.float64)
    full_ttv = np.einsum("ijk,k->ij", Dn, c)
    fib_i = np.repeat(np.arange(dims[0]), np.diff(T.pos1))
    want_ttv = full_ttv[fib_i, T.crd1]
    want_mttkrp = np.einsum("ijk,jl,kl->il", Dn, C, D)
    for acc in (False, True):
        assert np.array_equal(oracle.spttv(T.pos1, T.crd1, T.pos2, T.crd2, T.vals, c, accurate=acc), want_ttv)
        assert np.array_equal(oracle.spmttkrp(T.pos1, T.crd1, T.pos2, T.crd2, T.vals, C, D, accurate=acc),
                              want_mttkrp)


# ------------------------------------------------------------------------------ closed forms

def test_identity_and_unit_vectors():
    n = 17
    I = spd_synth.csr_from_coords(n, n, np.arange(n), np.arange(n), vals=np.ones(n))
    rng = np.random.default_rng(7)
    x = rng.uniform(-1, 1, n)
    X = rng.uniform(-1, 1, (n, 4))
    assert np.array_equal(oracle.spmv(I.pos, I.crd, I.vals, x), x)
    assert np.array_equal(oracle.spmm(I.pos, I.crd, I.vals, X), X)
    assert np.array_equal(oracle.spmm_t(I.pos, I.crd, I.vals, X, n), X)
    # x = e_j extracts column j
    A = small_csr(rng, 9, 11, 0.4)
    Dn = dense_of_csr(A)
    for j in range(11):
        e = np.zeros(11)
        e[j] = 1.0
        assert np.array_equal(oracle.spmv(A.pos, A.crd, A.vals, e), Dn[:, j])


def test_all_ones_and_empty():
    rng = np.random.default_rng(8)
    A = small_csr(rng, 12, 30, 0.3)
    # all-ones values: y_i = sum of x over the row's columns
    x = rng.uniform(-1, 1, 30)
    y = oracle.spmv(A.pos, A.crd, np.ones(A.nnz), x)
    for i in range(12):
        s = 0.0
        for p in range(A.pos[i], A.pos[i + 1]):
            s += x[A.crd[p]]
        assert y[i] == s
    # empty matrix and zero-row matrix
    E = spd_synth.csr_from_coords(5, 6, [], [], vals=np.zeros(0))
    assert np.array_equal(oracle.spmv(E.pos, E.crd, E.vals, np.ones(6)), np.zeros(5))
    assert np.array_equal(oracle.spmm(E.pos, E.crd, E.vals, np.ones((6, 3))), np.zeros((5, 3)))
    Z = spd_synth.csr_from_coords(0, 6, [], [], vals=np.zeros(0))
    assert oracle.spmv(Z.pos, Z.crd, Z.vals, np.ones(6)).shape == (0,)


def test_csf_closed_forms():
    rng = np.random.default_rng(9)
    T = small_csf(rng, (6, 7, 8), 0.3)
    # c = 1: per-fiber sums of the stored values
    out = oracle.spttv(T.pos1, T.crd1, T.pos2, T.crd2, T.vals, np.ones(8))
    for f in range(T.nfib):
        assert out[f] == sum(T.vals[T.pos2[f]:T.pos2[f + 1]].tolist(), 0.0)
    # rank 1, C = D = 1: per-slice sums of the stored values
    A = oracle.spmttkrp(T.pos1, T.crd1, T.pos2, T.crd2, T.vals, np.ones((7, 1)), np.ones((8, 1)), accurate=True)
    for i in range(6):
        lo, hi = T.pos2[T.pos1[i]], T.pos2[T.pos1[i + 1]]
        assert A[i, 0] == pytest.approx(float(sum(Fraction(v) for v in T.vals[lo:hi])), abs=1e-15)


def test_sddmm_k1_closed_form():
    rng = np.random.default_rng(10)
    A = small_csr(rng, 10, 12, 0.4)
    C = rng.uniform(-1, 1, (10, 1))
    Dnk = rng.uniform(-1, 1, (12, 1))
    out = oracle.sddmm(A.pos, A.crd, A.vals, C, Dnk)
    rows = np.repeat(np.arange(10), np.diff(A.pos))
    assert np.array_equal(out, (A.vals * C[rows, 0]) * Dnk[A.crd, 0])


# ------------------------------------------------------------------------------ linearity

@pytest.mark.parametrize("seed", SEEDS)
def test_linearity_integer_exact(seed):
    rng = np.random.default_rng(400 + seed)
    A = small_csr(rng, 20, 25, 0.3, integer=True)
    v2 = rng.integers(-8, 9, size=A.nnz).astype(np.float64)
    x = rng.integers(-8, 9, size=25).astype(np.float64)
    x2 = rng.integers(-8, 9, size=25).astype(np.float64)
    a, b = 3.0, -2.0
    f = lambda v, xx: oracle.spmv(A.pos, A.crd, v, xx)
    assert np.array_equal(f(a * A.vals + b * v2, x), a * f(A.vals, x) + b * f(v2, x))
    assert np.array_equal(f(A.vals, a * x + b * x2), a * f(A.vals, x) + b * f(A.vals, x2))
    T = small_csf(rng, (5, 6, 7), 0.3, integer=True)
    w2 = rng.integers(-8, 9, size=T.nnz).astype(np.float64)
    C = rng.integers(-8, 9, size=(6, 3)).astype(np.float64)
    D = rng.integers(-8, 9, size=(7, 3)).astype(np.float64)
    g = lambda v: oracle.spmttkrp(T.pos1, T.crd1, T.pos2, T.crd2, v, C, D)
    assert np.array_equal(g(a * T.vals + b * w2), a * g(T.vals) + b * g(w2))


# ------------------------------------------------------------------------------ accurate mode vs exact rationals

def _exact_dot(a, b):
    return sum((Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b)), Fraction(0))


@pytest.mark.parametrize("seed", SEEDS)
def test_dot2_against_exact_rationals(seed):
    rng = np.random.default_rng(500 + seed)
    u = 2.0 ** -53
    # one long row with heavy cancellation: terms of size ~1e8 that cancel to ~1
    m = 300
    big = rng.uniform(-1, 1, m // 2) * 1e8
    vals = np.concatenate([big, -big * (1 + 1e-13)]) + rng.uniform(-1, 1, m)
    rng.shuffle(vals)
    x = rng.uniform(0.5, 1.5, m)
    A = spd_synth.csr_from_coords(1, m, np.zeros(m, dtype=np.int64), np.arange(m), vals=vals)
    exact = _exact_dot(A.vals, x[A.crd])
    got = oracle.spmv(A.pos, A.crd, A.vals, x, accurate=True)[0]
    absum = float(sum(abs(Fraction(float(v)) * Fraction(float(w))) for v, w in zip(A.vals, x[A.crd])))
    gamma = (m * u) / (1 - m * u)
    # Dot2 bound (Ogita-Rump-Oishi, Prop. 5.5): |res - s| <= u|s| + gamma_{m}^2 sum|terms|
    assert abs(Fraction(got) - exact) <= Fraction(u) * abs(exact) + Fraction(gamma ** 2 * absum)
    # the plain oracle obeys the recursive-summation bound gamma_m * sum|terms|
    plain = oracle.spmv(A.pos, A.crd, A.vals, x)[0]
    assert abs(Fraction(plain) - exact) <= Fraction(gamma * absum)


def test_triple_product_compensation_against_exact():
    rng = np.random.default_rng(11)
    T = small_csf(rng, (3, 4, 40), 0.9)
    C = rng.uniform(-1, 1, (4, 2)) * 1e3
    D = rng.uniform(-1, 1, (40, 2))
    got = oracle.spmttkrp(T.pos1, T.crd1, T.pos2, T.crd2, T.vals, C, D, accurate=True)
    u = 2.0 ** -53
    for i in range(3):
        for l in range(2):
            ex = Fraction(0)
            ab = Fraction(0)
            for f in range(T.pos1[i], T.pos1[i + 1]):
                j = T.crd1[f]
                for p in range(T.pos2[f], T.pos2[f + 1]):
                    t = Fraction(float(T.vals[p])) * Fraction(float(C[j, l])) * Fraction(float(D[T.crd2[p], l]))
                    ex += t
                    ab += abs(t)
            assert abs(Fraction(got[i, l]) - ex) <= Fraction(2 * u) * abs(ex) + Fraction(1e-28) * ab


def test_triple_product_compensation_under_cancellation():
    # two fibers of one slice whose contributions cancel to a tiny remainder: the
    # compensated result must stay within a few ulps of the exact remainder, which a
    # scheme that drops any second-order term of the triple products cannot do
    rng = np.random.default_rng(14)
    K = 64
    v = rng.uniform(-1, 1, K)
    i = np.zeros(2 * K, dtype=np.int64)
    j = np.repeat([0, 1], K)
    k = np.tile(np.arange(K), 2)
    T = spd_synth.csf3_from_coords((1, 2, K), i, j, k, np.concatenate([v, -v]))
    C = np.array([[1.0 / 3.0], [(1.0 / 3.0) * (1 + 2.0 ** -40)]])
    D = rng.uniform(-1, 1, (K, 1))
    got = oracle.spmttkrp(T.pos1, T.crd1, T.pos2, T.crd2, T.vals, C, D, accurate=True)[0, 0]
    ex = Fraction(0)
    for f, jj in enumerate(T.crd1):
        for p in range(T.pos2[f], T.pos2[f + 1]):
            ex += Fraction(float(T.vals[p])) * Fraction(float(C[jj, 0])) * Fraction(float(D[T.crd2[p], 0]))
    assert abs(Fraction(got) - ex) <= Fraction(4 * 2.0 ** -53) * abs(ex)


# ------------------------------------------------------------------------------ compensated variants under cancellation
#
# Each case below sums terms of size ~1e8 that cancel to a result of order 1, so a
# binary64 running sum loses about 1e-8 per addition: only a compensated sum meets the
# Dot2 bound |res - s| <= u|s| + gamma_m^2 * sum|t| (Ogita, Rump and Oishi 2005, Prop. 5.5;
# u = 2^-53). The exact value is the sum of the rational products of the binary64 inputs.
# A compensated variant that returns only its leading part, drops a low-order fold or an
# error term of a product, or accumulates in the wrong place fails these bounds.

U53 = 2.0 ** -53


def _gamma(m):
    return (m * U53) / (1 - m * U53)


def _cancelling(rng, h, q, big=1e8):
    """h pairs (v, -v(1+d)) of magnitude ~big plus q terms in [-1, 1): the pairs leave
    residues of about big*d, the sum is of order one while partial sums reach ~big."""
    v = rng.uniform(0.5, 1.0, h) * big * rng.choice([-1.0, 1.0], h)
    d = rng.uniform(1e-14, 1e-13, h)
    return v, -v * (1 + d), rng.uniform(-1, 1, q)


def _dot2_ok(got, exact, absum, m, extra=Fraction(0)):
    bound = Fraction(U53) * abs(exact) + Fraction(_gamma(m) ** 2 * absum) + extra
    return abs(Fraction(float(got)) - exact) <= bound


def _fr(a):
    return Fraction(float(a))


@pytest.mark.parametrize("seed", SEEDS)
def test_spmm_acc_against_exact_rationals_under_cancellation(seed):
    rng = np.random.default_rng(600 + seed)
    h, q, L = 120, 24, 3
    m = 2 * h + q
    va, vb, vq = _cancelling(rng, h, q)
    cols = rng.permutation(m)
    ca, cb, cq = cols[:h], cols[h:2 * h], cols[2 * h:]
    vals_of_col = np.empty(m)
    vals_of_col[ca], vals_of_col[cb], vals_of_col[cq] = va, vb, vq
    X = rng.uniform(0.5, 1.5, (m, L))
    X[cb] = X[ca]  # each pair multiplies the same row of X
    # row 1 holds the cancelling sum; rows 0 and 2 are short and well conditioned
    rows = np.concatenate([[0, 0], np.ones(m, dtype=np.int64), [2]])
    cc = np.concatenate([[3, 7], np.arange(m), [5]])
    vv = np.concatenate([[0.25, -0.5], vals_of_col, [0.75]])
    A = spd_synth.csr_from_coords(3, m, rows, cc, vals=vv)
    got = oracle.spmm(A.pos, A.crd, A.vals, X, accurate=True)
    for i in range(3):
        for l in range(L):
            terms = [_fr(A.vals[p]) * _fr(X[A.crd[p], l]) for p in range(A.pos[i], A.pos[i + 1])]
            exact = sum(terms, Fraction(0))
            absum = float(sum(abs(t) for t in terms))
            assert _dot2_ok(got[i, l], exact, absum, len(terms)), (i, l)
    # the plain oracle on row 1 is far from exact (the case is really ill-conditioned)
    plain = oracle.spmm(A.pos, A.crd, A.vals, X)
    ex1 = sum((_fr(A.vals[p]) * _fr(X[A.crd[p], 0]) for p in range(A.pos[1], A.pos[2])), Fraction(0))
    assert abs(Fraction(float(plain[1, 0])) - ex1) > 1e6 * Fraction(U53) * abs(ex1)


@pytest.mark.parametrize("seed", SEEDS)
def test_spmm_t_acc_against_exact_rationals_under_cancellation(seed):
    rng = np.random.default_rng(700 + seed)
    h, q, L = 120, 24, 3
    n = 2 * h + q
    va, vb, vq = _cancelling(rng, h, q)
    rows_perm = rng.permutation(n)
    ra, rb, rq = rows_perm[:h], rows_perm[h:2 * h], rows_perm[2 * h:]
    vals_of_row = np.empty(n)
    vals_of_row[ra], vals_of_row[rb], vals_of_row[rq] = va, vb, vq
    dY = rng.uniform(0.5, 1.5, (n, L))
    dY[rb] = dY[ra]
    # column 1 of A gathers the cancelling entries (one per row); column 0 a few others
    rows = np.concatenate([np.arange(n), [4, 9, 30]])
    cols = np.concatenate([np.ones(n, dtype=np.int64), [0, 0, 0]])
    vals = np.concatenate([vals_of_row, [0.5, -1.25, 0.75]])
    A = spd_synth.csr_from_coords(n, 3, rows, cols, vals=vals)
    got = oracle.spmm_t(A.pos, A.crd, A.vals, dY, 3, accurate=True)
    for j in range(3):
        for l in range(L):
            terms = [_fr(A.vals[p]) * _fr(dY[i, l]) for i in range(n) for p in range(A.pos[i], A.pos[i + 1])
                     if A.crd[p] == j]
            exact = sum(terms, Fraction(0))
            absum = float(sum(abs(t) for t in terms))
            assert _dot2_ok(got[j, l], exact, absum, max(len(terms), 1)), (j, l)
    assert got[2].tolist() == [0.0] * L  # a column without entries


@pytest.mark.parametrize("seed", SEEDS)
def test_sddmm_acc_against_exact_rationals_under_cancellation(seed):
    rng = np.random.default_rng(800 + seed)
    h, q = 100, 20
    K = 2 * h + q
    ks = rng.permutation(K)
    ka, kb, kq = ks[:h], ks[h:2 * h], ks[2 * h:]
    n, m = 3, 4
    C = rng.uniform(-1, 1, (n, K))
    for i in range(n):  # every row of C cancels over k against every row of Dnk
        va, vb, vq = _cancelling(rng, h, q)
        C[i, ka], C[i, kb], C[i, kq] = va, vb, vq
    Dnk = rng.uniform(0.5, 1.5, (m, K))
    Dnk[:, kb] = Dnk[:, ka]
    rows = np.array([0, 0, 1, 2, 2, 2])
    cols = np.array([1, 3, 0, 0, 2, 3])
    b = rng.uniform(0.5, 1.5, rows.shape[0]) * 0.7  # products b*C are inexact in binary64
    B = spd_synth.csr_from_coords(n, m, rows, cols, vals=b)
    got = oracle.sddmm(B.pos, B.crd, B.vals, C, Dnk, accurate=True)
    got_sel = oracle.sddmm(B.pos, B.crd, B.vals, C, Dnk, sel=np.array([4, 0, 2]), accurate=True)
    ri = np.repeat(np.arange(n), np.diff(B.pos))
    for p in range(B.nnz):
        i, j = ri[p], B.crd[p]
        terms = [_fr(B.vals[p]) * _fr(C[i, k]) * _fr(Dnk[j, k]) for k in range(K)]
        exact = sum(terms, Fraction(0))
        absum = float(sum(abs(t) for t in terms))
        # the triple product's second-order term e*c is rounded once: u^2 per term
        extra = Fraction(U53) * abs(exact) + Fraction(2 * U53 * U53 * absum)
        assert _dot2_ok(got[p], exact, absum, K, extra), p
    assert got_sel.tolist() == [got[4], got[0], got[2]]


@pytest.mark.parametrize("seed", SEEDS)
def test_spttv_acc_against_exact_rationals_under_cancellation(seed):
    rng = np.random.default_rng(900 + seed)
    h, q = 120, 24
    m = 2 * h + q
    va, vb, vq = _cancelling(rng, h, q)
    ks = rng.permutation(m)
    ka, kb, kq = ks[:h], ks[h:2 * h], ks[2 * h:]
    vals_of_k = np.empty(m)
    vals_of_k[ka], vals_of_k[kb], vals_of_k[kq] = va, vb, vq
    c = rng.uniform(0.5, 1.5, m)
    c[kb] = c[ka]
    # fiber (0, 1) holds the cancelling sum; fibers (0, 0) and (1, 2) are short
    i = np.concatenate([[0, 0], np.zeros(m, dtype=np.int64), [1, 1]])
    j = np.concatenate([[0, 0], np.ones(m, dtype=np.int64), [2, 2]])
    k = np.concatenate([[4, 9], np.arange(m), [1, 3]])
    v = np.concatenate([[0.5, -0.25], vals_of_k, [1.5, -0.75]])
    T = spd_synth.csf3_from_coords((2, 3, m), i, j, k, v)
    got = oracle.spttv(T.pos1, T.crd1, T.pos2, T.crd2, T.vals, c, accurate=True)
    for f in range(T.nfib):
        terms = [_fr(T.vals[p]) * _fr(c[T.crd2[p]]) for p in range(T.pos2[f], T.pos2[f + 1])]
        exact = sum(terms, Fraction(0))
        absum = float(sum(abs(t) for t in terms))
        assert _dot2_ok(got[f], exact, absum, len(terms)), f
    plain = oracle.spttv(T.pos1, T.crd1, T.pos2, T.crd2, T.vals, c)
    ex1 = sum((_fr(T.vals[p]) * _fr(c[T.crd2[p]]) for p in range(T.pos2[1], T.pos2[2])), Fraction(0))
    assert abs(Fraction(float(plain[1])) - ex1) > 1e6 * Fraction(U53) * abs(ex1)


# ------------------------------------------------------------------------------ partitions

def _random_pos(rng, n, maxlen):
    lens = rng.integers(0, maxlen + 1, size=n)
    lens[rng.random(n) < 0.4] = 0  # many empty rows
    if n:
        lens[rng.integers(0, n)] = maxlen * 20  # one long row
    pos = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=pos[1:])
    return pos.astype(np.int32)


@pytest.mark.parametrize("seed", SEEDS)
def test_merge_path_closed_form(seed):
    rng = np.random.default_rng(600 + seed)
    n = int(rng.integers(0, 200))
    pos = _random_pos(rng, n, 9)
    nnz = int(pos[-1])
    d = np.arange(0, n + nnz + 1)
    rows, poss = oracle.merge_path(pos, d)
    # row r ends at merge index pos[r+1] + r, so the rows completed after d items are
    # those whose end index is below d
    ends = pos[1:].astype(np.int64) + np.arange(n)
    want_rows = np.searchsorted(ends, d, side="left")
    assert np.array_equal(rows, want_rows)
    assert np.array_equal(rows + poss, d)
    # the state is on the path: pos[r] <= p <= pos[r+1] for r < n
    inner = rows < n
    assert np.all(pos[rows[inner]] <= poss[inner]) and np.all(poss[inner] <= pos[rows[inner] + 1])


@pytest.mark.parametrize("seed", SEEDS)
def test_pos_split_and_row_split(seed):
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(1, 300))
    pos = _random_pos(rng, n, 7)
    nnz = int(pos[-1])
    q = np.arange(nnz + 1)
    rows = oracle.pos_split(pos, q)
    assert np.array_equal(rows, np.searchsorted(pos, q, side="right") - 1 if nnz else np.array([n]))
    assert rows[-1] == n
    inner = q < nnz
    assert np.all(pos[rows[inner]] <= q[inner]) and np.all(q[inner] < pos[rows[inner] + 1])
    for P in (1, 2, 3, 7, 152, n + 5):
        b = oracle.row_split(n, P)
        assert b[0] == 0 and b[-1] == n
        sizes = np.diff(b)
        assert sizes.min() >= 0 and sizes.max() - sizes.min() <= 1  # equal pieces up to one row


def test_validate_level_detects_planted_faults():
    rng = np.random.default_rng(12)
    A = small_csr(rng, 30, 20, 0.3)
    assert oracle.validate_level(30, 20, A.pos, A.crd) == (0, -1)
    bad = A.pos.copy()
    bad[5], bad[6] = bad[6] + 1, bad[5]
    cnt, first = oracle.validate_level(30, 20, bad, A.crd)
    assert cnt >= 1 and first in (5, 6)
    short = A.pos.copy()
    short[-1] -= 1
    assert oracle.validate_level(30, 20, short, A.crd)[0] >= 1
    crd = A.crd.copy()
    crd[3] = 20
    cnt, first = oracle.validate_level(30, 20, A.pos, crd)
    assert cnt == 1 and first == 31 + 3


# ------------------------------------------------------------------------------ transposed structure

@pytest.mark.parametrize("seed", SEEDS)
def test_transpose_dense_and_involution(seed):
    """A^T built from (t_pos, t_crd, vals[perm]) equals the dense transpose; transposing
    twice gives A back and the two permutations compose to the identity."""
    rng = np.random.default_rng(seed)
    A = small_csr(rng, 37, 23, 0.15, long_rows=1, integer=True)
    t_pos, t_crd, perm = oracle.csr_transpose(A.pos, A.crd, A.ncols)
    At = spd_synth.CSR(A.ncols, A.nrows, t_pos, t_crd, A.vals[perm])
    assert np.array_equal(dense_of_csr(At), dense_of_csr(A).T)
    assert np.array_equal(np.sort(perm), np.arange(A.nnz))
    b_pos, b_crd, perm2 = oracle.csr_transpose(t_pos, t_crd, A.nrows)
    assert np.array_equal(b_pos, A.pos) and np.array_equal(b_crd, A.crd)
    assert np.array_equal(perm[perm2], np.arange(A.nnz))


def test_transpose_is_the_stable_sort_by_column():
    """perm is numpy's stable sort of A's positions by column (rows ascending within a
    column) and t_crd is sorted within every column."""
    A = spd_synth.rmat_csr(11, 8, seed=4)
    t_pos, t_crd, perm = oracle.csr_transpose(A.pos, A.crd, A.ncols)
    assert np.array_equal(perm, np.argsort(A.crd, kind="stable"))
    assert np.array_equal(t_pos, np.concatenate([[0], np.cumsum(np.bincount(A.crd, minlength=A.ncols))]))
    rows = np.repeat(np.arange(A.nrows), np.diff(A.pos))
    assert np.array_equal(t_crd, rows[perm])
    seg = np.repeat(np.arange(A.ncols), np.diff(t_pos))
    assert np.all((np.diff(t_crd) > 0) | (np.diff(seg) != 0))


def test_transpose_against_scipy_csc():
    sp = pytest.importorskip("scipy.sparse")
    A = spd_synth.rmat_csr(10, 8, seed=6)
    S = sp.csr_matrix((A.vals, A.crd, A.pos), shape=(A.nrows, A.ncols)).tocsc()
    S.sort_indices()
    t_pos, t_crd, perm = oracle.csr_transpose(A.pos, A.crd, A.ncols)
    assert np.array_equal(t_pos, S.indptr) and np.array_equal(t_crd, S.indices)
    assert np.array_equal(A.vals[perm], S.data)


# ------------------------------------------------------------------------------ SpAdd3

def _spadd3_operands(rng, n, m, density, integer):
    return [small_csr(rng, n, m, density, long_rows=1, integer=integer) for _ in range(3)]


@pytest.mark.parametrize("seed", SEEDS)
def test_spadd3_dense_bruteforce_and_union(seed):
    """Values equal the dense sum exactly (small integers); the pattern is the union of
    the three patterns, kept even where values cancel; counts agree with pos."""
    rng = np.random.default_rng(seed)
    B, C, D = _spadd3_operands(rng, 29, 17, 0.2, integer=True)
    C.vals[: C.nnz // 2] = 0.0  # stored zeros stay stored
    ap, ac, av = oracle.spadd3(B, C, D)
    A = spd_synth.CSR(29, 17, ap, ac, av)
    assert np.array_equal(dense_of_csr(A), dense_of_csr(B) + dense_of_csr(C) + dense_of_csr(D))
    for i in range(29):
        want = set(B.crd[B.pos[i]:B.pos[i + 1]]) | set(C.crd[C.pos[i]:C.pos[i + 1]]) | set(D.crd[D.pos[i]:D.pos[i + 1]])
        row = ac[ap[i]:ap[i + 1]]
        assert list(row) == sorted(want)
    assert np.array_equal(oracle.spadd3_count(B, C, D), np.diff(ap))


def test_spadd3_special_cases():
    rng = np.random.default_rng(7)
    B = small_csr(rng, 40, 30, 0.2, long_rows=1)
    E = spd_synth.csr_from_coords(40, 30, [], [], vals=np.zeros(0))
    ap, ac, av = oracle.spadd3(B, E, E)  # adding empty matrices gives B back
    assert np.array_equal(ap, B.pos) and np.array_equal(ac, B.crd) and np.array_equal(av, B.vals)
    ap, ac, av = oracle.spadd3(E, E, B)
    assert np.array_equal(ac, B.crd) and np.array_equal(av, B.vals)
    ap, ac, av = oracle.spadd3(B, B, B)  # same pattern three times: (b + b) + b
    assert np.array_equal(ap, B.pos) and np.array_equal(ac, B.crd) and np.array_equal(av, (B.vals + B.vals) + B.vals)


def test_spadd3_against_scipy():
    sp = pytest.importorskip("scipy.sparse")
    A = spd_synth.rmat_csr(10, 8, seed=8)
    ops = [spd_synth.CSR(A.nrows, A.ncols, A.pos, A.crd, np.abs(A.vals) + 0.5)]
    ops += [spd_synth.shifted_csr(A, s, seed=9 + s) for s in (1, 2)]
    ops[1].vals = np.abs(ops[1].vals) + 0.5  # positive: scipy prunes exact zeros, the oracle keeps them
    ops[2].vals = np.abs(ops[2].vals) + 0.5
    S = [sp.csr_matrix((M.vals, M.crd, M.pos), shape=(A.nrows, A.ncols)) for M in ops]
    R = ((S[0] + S[1]) + S[2]).tocsr()
    R.sort_indices()
    ap, ac, av = oracle.spadd3(*ops)
    assert np.array_equal(ap, R.indptr) and np.array_equal(ac, R.indices)
    assert np.array_equal(av, R.data)


# ------------------------------------------------------------------------------ column blocks

@pytest.mark.parametrize("seed", SEEDS)
def test_column_blocks_partition_the_matrix(seed):
    """The blocks' dense forms add up to A, every block holds only its columns, the
    permutation covers A once, and each row's split points are numpy's searchsorted of
    the bounds in that row; SpMM over the blocks sums to SpMM over A (exact on integers)."""
    rng = np.random.default_rng(seed)
    A = small_csr(rng, 41, 37, 0.2, long_rows=1, integer=True)
    bounds = np.array([0, 5, 6, 20, 37], dtype=np.int32)
    blk_pos, blk_crd, perm, nnz = oracle.column_blocks(A.pos, A.crd, bounds)
    assert np.array_equal(np.sort(perm), np.arange(A.nnz))
    off = np.concatenate([[0], np.cumsum(nnz)])
    total = np.zeros((41, 37))
    X = rng.integers(-4, 5, (37, 3)).astype(np.float64)
    Y = np.zeros((41, 3))
    for b in range(4):
        c = blk_crd[off[b]:off[b + 1]]
        assert np.all((c >= bounds[b]) & (c < bounds[b + 1]))
        Ab = spd_synth.CSR(41, 37, blk_pos[b], c, A.vals[perm[off[b]:off[b + 1]]])
        total += dense_of_csr(Ab)
        Y += oracle.spmm(Ab.pos, Ab.crd, Ab.vals, X)
        for i in range(41):
            row = A.crd[A.pos[i]:A.pos[i + 1]]
            lo, hi = np.searchsorted(row, [bounds[b], bounds[b + 1]])
            assert blk_pos[b][i + 1] - blk_pos[b][i] == hi - lo
    assert np.array_equal(total, dense_of_csr(A))
    assert np.array_equal(Y, oracle.spmm(A.pos, A.crd, A.vals, X))


# ------------------------------------------------------------------------------ library cross-check

def test_torch_sparse_cross_check():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(13)
    A = spd_synth.rmat_csr(10, 8, seed=3)
    X = rng.uniform(-1, 1, (A.ncols, 6))
    S = torch.sparse_csr_tensor(torch.from_numpy(A.pos.astype(np.int64)), torch.from_numpy(A.crd.astype(np.int64)),
                                torch.from_numpy(A.vals), size=(A.nrows, A.ncols), dtype=torch.float64)
    ref = (S @ torch.from_numpy(X)).numpy()
    got = oracle.spmm(A.pos, A.crd, A.vals, X)
    scale = oracle.spmm(A.pos, A.crd, np.abs(A.vals), np.abs(X))
    assert normalized_error(got, ref, scale).max() <= 1e-14
    dY = rng.uniform(-1, 1, (A.nrows, 3))
    ref_t = (S.to_dense().T @ torch.from_numpy(dY)).numpy()
    got_t = oracle.spmm_t(A.pos, A.crd, A.vals, dY, A.ncols)
    scale_t = oracle.spmm_t(A.pos, A.crd, np.abs(A.vals), np.abs(dY), A.ncols)
    assert normalized_error(got_t, ref_t, scale_t).max() <= 1e-14
