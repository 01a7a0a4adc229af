/*
 * spd_oracle.c -- plain, slow, obviously correct CPU oracle for the sparse tensor
 * algebra kernels compiled by SpDISTAL (arXiv 2207.13901).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library's product path may call, link or
 * load this file: only the tests, the smoke check and the benchmark's CPU-baseline
 * leg do. It shares no code, header, table or helper with the CUDA kernels.
 *
 * Conventions (the level format of Section III-B):
 *   * a Compressed level is a pair (pos, crd); the children of parent entry i sit at
 *     positions [pos[i], pos[i+1]) of crd. pos has parent+1 int32 entries.
 *   * CSR = {Dense, Compressed}; CSF = {Dense, Compressed, Compressed}.
 *   * dense matrices are row-major with an explicit leading dimension.
 *   * all arithmetic is IEEE binary64; the file is compiled with
 *     -ffp-contract=off so that no multiply-add is fused behind our back.
 *
 * Every kernel computes its tensor index notation statement (Section II-A: each index
 * variable is a loop, index variables that appear only on the right-hand side are
 * summed) exactly as written, looping over the coordinate tree in ascending position
 * order, i.e. the leaf loop of the generated row-based SpMV in Section IV-C,
 * generalised. Outputs are overwritten (zero-initialised, then accumulated), which is
 * the paper's "a.vals[i] += ..." applied to a zeroed output.
 *
 * The *_acc variants compute the same statements with compensated arithmetic:
 * TwoSum (Knuth), TwoProduct via fma, and the Dot2/Sum2 scheme of Ogita, Rump and
 * Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26(6), 2005. Their result
 * is as accurate as if computed in twice the working precision and then rounded, which
 * makes them the reference for error statements of the GPU kernels.
 *
 * Parity pins (see tests/test_oracle_*.py): dense brute force on small-integer data
 * (exact), closed forms, linearity, exact rational arithmetic for the compensated
 * variants, partition invariants and an independent library cross-check.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------
 * Compensated building blocks (error-free transformations).
 * ------------------------------------------------------------------------------------ */

/* s + e == a + b exactly, s = fl(a + b)  (Knuth's TwoSum, no ordering requirement). */
static void two_sum(double a, double b, double *s, double *e) {
    double x = a + b;
    double z = x - a;
    *s = x;
    *e = (a - (x - z)) + (b - z);
}

/* p + e == a * b exactly, p = fl(a * b)  (TwoProduct with a fused multiply-add). */
static void two_prod(double a, double b, double *p, double *e) {
    double x = a * b;
    *p = x;
    *e = fma(a, b, -x);
}

/* A running compensated sum: value = hi + lo, updated with Sum2 steps. */
typedef struct {
    double hi, lo;
} csum;

static void csum_add_prod(csum *c, double a, double b) {
    double h, r, s, q;
    two_prod(a, b, &h, &r);
    two_sum(c->hi, h, &s, &q);
    c->hi = s;
    c->lo += q + r;
}

/* Adds the triple product a*b*c: a*b = h + e exactly, h*c = h2 + e2 exactly, and e*c
 * is a second-order term whose rounding error is below u^2 |a*b*c|. */
static void csum_add_prod3(csum *cs, double a, double b, double c) {
    double h, e, h2, e2, s, q;
    two_prod(a, b, &h, &e);
    two_prod(h, c, &h2, &e2);
    two_sum(cs->hi, h2, &s, &q);
    cs->hi = s;
    cs->lo += q + (e2 + e * c);
}

static double csum_value(const csum *c) { return c->hi + c->lo; }

/* ------------------------------------------------------------------------------------
 * Work partitions (Sections II-B, III-A, IV-B).
 * ------------------------------------------------------------------------------------ */

/* Universe partition of a Dense level into P pieces: piece c holds coordinates
 * [bounds[c], bounds[c+1]) with bounds[c] = floor(c * n / P). This is the bounds
 * computation of the generated SpMV (Section IV-C) with the remainder distributed
 * instead of dropped. */
void orc_row_split(int64_t n, int64_t P, int64_t *bounds) {
    for (int64_t c = 0; c <= P; ++c) bounds[c] = (c * n) / P;
}

/* Fused non-zero partition of a CSR coordinate tree (coordinate fusion of (i, j) plus a
 * non-zero partition, Section II-B), balanced over rows and nonzeros together.
 *
 * The coordinate tree is flattened into one sequence of items: for every row i, its
 * nonzeros pos[i] .. pos[i+1]-1, followed by one "row end" item. At a state (r, p) the
 * next item is the end of row r when every nonzero of row r has been consumed
 * (pos[r+1] <= p), otherwise it is nonzero p. For each requested diagonal d (ascending)
 * this walks the sequence one item at a time and reports the state after d items:
 * rows_out = number of completed rows, pos_out = number of consumed nonzeros. */
void orc_merge_path(int64_t n, const int32_t *pos, int64_t nd, const int64_t *diag,
                    int64_t *rows_out, int64_t *pos_out) {
    int64_t nnz = pos[n];
    int64_t r = 0, p = 0, done = 0;
    for (int64_t q = 0; q < nd; ++q) {
        int64_t d = diag[q];
        while (done < d) {
            if (r < n && pos[r + 1] <= p) {
                ++r;
            } else if (p < nnz) {
                ++p;
            } else {
                ++r; /* unreachable for d <= n + nnz */
            }
            ++done;
        }
        rows_out[q] = r;
        pos_out[q] = p;
    }
}

/* Non-zero partition of the positions of a Compressed level (Section II-B, Table of
 * level functions: partitionByBounds on crd, then preimage to pos). For every requested
 * position q (ascending, 0 <= q <= nnz) reports the row that holds position q, i.e. the
 * unique r with pos[r] <= q < pos[r+1], found by walking rows; q == nnz maps to n. */
void orc_pos_split(int64_t n, const int32_t *pos, int64_t nq, const int64_t *qs,
                   int64_t *rows_out) {
    int64_t r = 0;
    for (int64_t t = 0; t < nq; ++t) {
        int64_t q = qs[t];
        while (r < n && pos[r + 1] <= q) ++r;
        rows_out[t] = r;
    }
}

/* ------------------------------------------------------------------------------------
 * SpMV  a(i) = B(i,j) * c(j)                                      (Section VI-A)
 * The loop is the generated row-based leaf: for each row, walk its positions.
 * sel == NULL: all rows, y has n entries; otherwise y[t] = row sel[t].
 * ------------------------------------------------------------------------------------ */
void orc_spmv(int64_t n, const int32_t *pos, const int32_t *crd, const double *vals,
              const double *x, int64_t nsel, const int64_t *sel, double *y) {
    int64_t cnt = sel ? nsel : n;
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t i = sel ? sel[t] : t;
        double acc = 0.0;
        for (int64_t jB = pos[i]; jB < pos[i + 1]; ++jB) {
            int64_t j = crd[jB];
            acc += vals[jB] * x[j];
        }
        y[t] = acc;
    }
}

void orc_spmv_acc(int64_t n, const int32_t *pos, const int32_t *crd, const double *vals,
                  const double *x, int64_t nsel, const int64_t *sel, double *y) {
    int64_t cnt = sel ? nsel : n;
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t i = sel ? sel[t] : t;
        csum acc = {0.0, 0.0};
        for (int64_t jB = pos[i]; jB < pos[i + 1]; ++jB) csum_add_prod(&acc, vals[jB], x[crd[jB]]);
        y[t] = csum_value(&acc);
    }
}

/* ------------------------------------------------------------------------------------
 * SpMM  Y(i,l) = A(i,j) * X(j,l)            (Section VI-A: A(i,j) = B(i,k) * C(k,j))
 * X is ncols x L row-major (leading dimension ldx), Y is n x L (leading dimension ldy).
 * ------------------------------------------------------------------------------------ */
void orc_spmm(int64_t n, int64_t L, const int32_t *pos, const int32_t *crd, const double *vals,
              const double *X, int64_t ldx, int64_t nsel, const int64_t *sel, double *Y,
              int64_t ldy) {
    int64_t cnt = sel ? nsel : n;
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t i = sel ? sel[t] : t;
        double *yr = Y + t * ldy;
        for (int64_t l = 0; l < L; ++l) yr[l] = 0.0;
        for (int64_t p = pos[i]; p < pos[i + 1]; ++p) {
            int64_t j = crd[p];
            for (int64_t l = 0; l < L; ++l) yr[l] += vals[p] * X[j * ldx + l];
        }
    }
}

void orc_spmm_acc(int64_t n, int64_t L, const int32_t *pos, const int32_t *crd,
                  const double *vals, const double *X, int64_t ldx, int64_t nsel,
                  const int64_t *sel, double *Y, int64_t ldy) {
    int64_t cnt = sel ? nsel : n;
    csum *acc = (csum *)malloc(sizeof(csum) * (size_t)(L > 0 ? L : 1));
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t i = sel ? sel[t] : t;
        for (int64_t l = 0; l < L; ++l) acc[l].hi = acc[l].lo = 0.0;
        for (int64_t p = pos[i]; p < pos[i + 1]; ++p) {
            int64_t j = crd[p];
            for (int64_t l = 0; l < L; ++l) csum_add_prod(&acc[l], vals[p], X[j * ldx + l]);
        }
        for (int64_t l = 0; l < L; ++l) Y[t * ldy + l] = csum_value(&acc[l]);
    }
    free(acc);
}

/* ------------------------------------------------------------------------------------
 * SpMM^T (the gradient with respect to X of Y = A X):  dX(j,l) = A(i,j) * dY(i,l).
 * Walks A's rows in ascending order and scatters into dX (ncols x L, ld ldx).
 * ------------------------------------------------------------------------------------ */
void orc_spmm_t(int64_t n, int64_t ncols, int64_t L, const int32_t *pos, const int32_t *crd,
                const double *vals, const double *dY, int64_t ldy, double *dX, int64_t ldx) {
    for (int64_t j = 0; j < ncols; ++j)
        for (int64_t l = 0; l < L; ++l) dX[j * ldx + l] = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = pos[i]; p < pos[i + 1]; ++p) {
            int64_t j = crd[p];
            for (int64_t l = 0; l < L; ++l) dX[j * ldx + l] += vals[p] * dY[i * ldy + l];
        }
}

void orc_spmm_t_acc(int64_t n, int64_t ncols, int64_t L, const int32_t *pos, const int32_t *crd,
                    const double *vals, const double *dY, int64_t ldy, double *dX, int64_t ldx) {
    double *lo = (double *)calloc((size_t)(ncols * L > 0 ? ncols * L : 1), sizeof(double));
    for (int64_t j = 0; j < ncols; ++j)
        for (int64_t l = 0; l < L; ++l) dX[j * ldx + l] = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = pos[i]; p < pos[i + 1]; ++p) {
            int64_t j = crd[p];
            for (int64_t l = 0; l < L; ++l) {
                csum c = {dX[j * ldx + l], lo[j * L + l]};
                csum_add_prod(&c, vals[p], dY[i * ldy + l]);
                dX[j * ldx + l] = c.hi;
                lo[j * L + l] = c.lo;
            }
        }
    for (int64_t j = 0; j < ncols; ++j)
        for (int64_t l = 0; l < L; ++l) dX[j * ldx + l] += lo[j * L + l];
    free(lo);
}

/* ------------------------------------------------------------------------------------
 * SDDMM  A(i,j) = B(i,j) * C(i,k) * D(k,j)                        (Section VI-A)
 * The output keeps B's coordinate structure (Section V-B), so only its values are
 * produced, one per position of B. C is n x K (ldc); D is passed transposed, as the
 * ncols x K row-major matrix Dnk with Dnk[j,k] = D(k,j) (ldd). vals == NULL means every
 * stored B value is 1 (the sampling pattern alone). The product is formed left to
 * right as written: (B(i,j) * C(i,k)) * D(k,j), summed over k ascending.
 * sel == NULL: all positions; otherwise out[t] = position sel[t].
 * ------------------------------------------------------------------------------------ */
static int64_t row_of_position(int64_t n, const int32_t *pos, int64_t p) {
    /* the unique i with pos[i] <= p < pos[i+1], by bisection over pos (used only for
     * sampled positions, so a walk from row 0 is not needed) */
    int64_t lo = 0, hi = n; /* invariant: pos[lo] <= p < pos[hi] */
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        if (pos[mid] <= p) lo = mid; else hi = mid;
    }
    return lo;
}

void orc_sddmm(int64_t n, int64_t K, const int32_t *pos, const int32_t *crd, const double *vals,
               const double *C, int64_t ldc, const double *Dnk, int64_t ldd, int64_t nsel,
               const int64_t *sel, double *out) {
    if (!sel) {
        for (int64_t i = 0; i < n; ++i)
            for (int64_t p = pos[i]; p < pos[i + 1]; ++p) {
                int64_t j = crd[p];
                double b = vals ? vals[p] : 1.0;
                double acc = 0.0;
                for (int64_t k = 0; k < K; ++k) acc += (b * C[i * ldc + k]) * Dnk[j * ldd + k];
                out[p] = acc;
            }
        return;
    }
    for (int64_t t = 0; t < nsel; ++t) {
        int64_t p = sel[t];
        int64_t i = row_of_position(n, pos, p);
        int64_t j = crd[p];
        double b = vals ? vals[p] : 1.0;
        double acc = 0.0;
        for (int64_t k = 0; k < K; ++k) acc += (b * C[i * ldc + k]) * Dnk[j * ldd + k];
        out[t] = acc;
    }
}

void orc_sddmm_acc(int64_t n, int64_t K, const int32_t *pos, const int32_t *crd,
                   const double *vals, const double *C, int64_t ldc, const double *Dnk,
                   int64_t ldd, int64_t nsel, const int64_t *sel, double *out) {
    int64_t cnt = sel ? nsel : pos[n];
    int64_t i = 0;
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t p = sel ? sel[t] : t;
        if (sel) i = row_of_position(n, pos, p);
        else while (pos[i + 1] <= p) ++i;
        int64_t j = crd[p];
        double b = vals ? vals[p] : 1.0;
        csum acc = {0.0, 0.0};
        for (int64_t k = 0; k < K; ++k) csum_add_prod3(&acc, b, C[i * ldc + k], Dnk[j * ldd + k]);
        out[t] = csum_value(&acc);
    }
}

/* ------------------------------------------------------------------------------------
 * SpTTV  A(i,j) = B(i,j,k) * c(k)                                 (Section VI-A)
 * B is CSF {Dense, Compressed, Compressed}. The output keeps B's (i,j) coordinate
 * structure (Section V-B): its pos/crd are B's pos1/crd1 and only one value per fiber
 * is produced. sel == NULL: all fibers; otherwise out[t] = fiber sel[t].
 * ------------------------------------------------------------------------------------ */
void orc_spttv(int64_t I, const int32_t *pos1, const int32_t *crd1, const int32_t *pos2,
               const int32_t *crd2, const double *vals, const double *c, int64_t nsel,
               const int64_t *sel, double *out) {
    (void)crd1;
    if (!sel) {
        for (int64_t i = 0; i < I; ++i)
            for (int64_t f = pos1[i]; f < pos1[i + 1]; ++f) {
                double acc = 0.0;
                for (int64_t p = pos2[f]; p < pos2[f + 1]; ++p) acc += vals[p] * c[crd2[p]];
                out[f] = acc;
            }
        return;
    }
    for (int64_t t = 0; t < nsel; ++t) {
        int64_t f = sel[t];
        double acc = 0.0;
        for (int64_t p = pos2[f]; p < pos2[f + 1]; ++p) acc += vals[p] * c[crd2[p]];
        out[t] = acc;
    }
}

void orc_spttv_acc(int64_t I, const int32_t *pos1, const int32_t *crd1, const int32_t *pos2,
                   const int32_t *crd2, const double *vals, const double *c, int64_t nsel,
                   const int64_t *sel, double *out) {
    (void)crd1;
    int64_t cnt = sel ? nsel : pos1[I];
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t f = sel ? sel[t] : t;
        csum acc = {0.0, 0.0};
        for (int64_t p = pos2[f]; p < pos2[f + 1]; ++p) csum_add_prod(&acc, vals[p], c[crd2[p]]);
        out[t] = csum_value(&acc);
    }
}

/* ------------------------------------------------------------------------------------
 * SpMTTKRP  A(i,l) = B(i,j,k) * C(j,l) * D(k,l)                   (Section VI-A)
 * Loop nest i -> j (level 2) -> k (level 3) -> l over the CSF coordinate tree, product
 * formed left to right as written. C is J x R (ldc), D is K x R (ldd), A is I x R (lda).
 * sel == NULL: all slices; otherwise row t of A is slice sel[t].
 * ------------------------------------------------------------------------------------ */
void orc_spmttkrp(int64_t I, int64_t R, const int32_t *pos1, const int32_t *crd1,
                  const int32_t *pos2, const int32_t *crd2, const double *vals,
                  const double *C, int64_t ldc, const double *D, int64_t ldd, int64_t nsel,
                  const int64_t *sel, double *A, int64_t lda) {
    int64_t cnt = sel ? nsel : I;
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t i = sel ? sel[t] : t;
        double *ar = A + t * lda;
        for (int64_t l = 0; l < R; ++l) ar[l] = 0.0;
        for (int64_t f = pos1[i]; f < pos1[i + 1]; ++f) {
            int64_t j = crd1[f];
            for (int64_t p = pos2[f]; p < pos2[f + 1]; ++p) {
                int64_t k = crd2[p];
                for (int64_t l = 0; l < R; ++l) ar[l] += (vals[p] * C[j * ldc + l]) * D[k * ldd + l];
            }
        }
    }
}

void orc_spmttkrp_acc(int64_t I, int64_t R, const int32_t *pos1, const int32_t *crd1,
                      const int32_t *pos2, const int32_t *crd2, const double *vals,
                      const double *C, int64_t ldc, const double *D, int64_t ldd, int64_t nsel,
                      const int64_t *sel, double *A, int64_t lda) {
    int64_t cnt = sel ? nsel : I;
    csum *acc = (csum *)malloc(sizeof(csum) * (size_t)(R > 0 ? R : 1));
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t i = sel ? sel[t] : t;
        for (int64_t l = 0; l < R; ++l) acc[l].hi = acc[l].lo = 0.0;
        for (int64_t f = pos1[i]; f < pos1[i + 1]; ++f) {
            int64_t j = crd1[f];
            for (int64_t p = pos2[f]; p < pos2[f + 1]; ++p) {
                int64_t k = crd2[p];
                for (int64_t l = 0; l < R; ++l)
                    csum_add_prod3(&acc[l], vals[p], C[j * ldc + l], D[k * ldd + l]);
            }
        }
        for (int64_t l = 0; l < R; ++l) A[t * lda + l] = csum_value(&acc[l]);
    }
    free(acc);
}

/* ------------------------------------------------------------------------------------
 * Structure validation of a Compressed level (Section III-B semantics of pos/crd).
 * Returns the number of violations; *first_bad receives the smallest offending index
 * (an index into pos for pos violations, nparent+1+p for a crd violation at position p),
 * or -1 when the level is valid.
 * ------------------------------------------------------------------------------------ */
int64_t orc_validate_level(int64_t nparent, int64_t nchild_dim, const int32_t *pos,
                           const int32_t *crd, int64_t ncrd, int64_t *first_bad) {
    int64_t bad = 0;
    *first_bad = -1;
    if (pos[0] != 0) { ++bad; if (*first_bad < 0) *first_bad = 0; }
    for (int64_t i = 0; i < nparent; ++i)
        if (pos[i + 1] < pos[i]) { ++bad; if (*first_bad < 0) *first_bad = i + 1; }
    if (pos[nparent] != ncrd) { ++bad; if (*first_bad < 0) *first_bad = nparent; }
    for (int64_t p = 0; p < ncrd; ++p)
        if (crd[p] < 0 || crd[p] >= nchild_dim) {
            ++bad;
            if (*first_bad < 0) *first_bad = nparent + 1 + p;
        }
    return bad;
}

/* ------------------------------------------------------------------------------------
 * Transposed structure: A^T in the same {Dense, Compressed} level formats (the CSC
 * encoding of A; Section II-B: CSR's level formats with the dimension order reversed).
 * A counting sort by column that walks A in ascending position order, so the entries
 * of each column keep A's row order.
 *   t_pos[j]  = number of entries of A in columns < j   (ncols + 1 entries)
 *   t_crd[q]  = row of the q-th entry of A^T
 *   perm[q]   = position in A of the q-th entry of A^T
 * ------------------------------------------------------------------------------------ */
void orc_csr_transpose(int64_t n, int64_t ncols, const int32_t *pos, const int32_t *crd,
                       int32_t *t_pos, int32_t *t_crd, int32_t *perm) {
    int64_t *next = (int64_t *)calloc((size_t)(ncols > 0 ? ncols : 1), sizeof(int64_t));
    for (int64_t j = 0; j <= ncols; ++j) t_pos[j] = 0;
    for (int64_t p = 0; p < pos[n]; ++p) t_pos[crd[p] + 1] += 1;   /* column counts */
    for (int64_t j = 0; j < ncols; ++j) t_pos[j + 1] += t_pos[j];  /* running totals */
    for (int64_t j = 0; j < ncols; ++j) next[j] = t_pos[j];
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = pos[i]; p < pos[i + 1]; ++p) {
            const int64_t q = next[crd[p]]++;
            t_crd[q] = (int32_t)i;
            perm[q] = (int32_t)p;
        }
    free(next);
}

/* ------------------------------------------------------------------------------------
 * SpAdd3 A(i,j) = B(i,j) + C(i,j) + D(i,j) (Section VI-A) on CSR operands of one shape.
 * A's structure is not known in advance: it is the union of the three patterns
 * (every coordinate stored in any input is stored in A, even where the values cancel).
 * Assembly in two phases as in Section V-B: orc_spadd3_count writes the number of
 * entries of each row of A (row i's union size), and orc_spadd3 fills A's pos, crd and
 * vals. Rows are merged in ascending column order; a value is formed left to right as
 * the statement is written, (B + C) + D, over the operands that store the coordinate.
 * Each input row must hold ascending, distinct columns.
 * ------------------------------------------------------------------------------------ */
static int64_t spadd3_row(int64_t i, const int32_t *bp, const int32_t *bc, const double *bv,
                          const int32_t *cp, const int32_t *cc, const double *cv,
                          const int32_t *dp, const int32_t *dc, const double *dv,
                          int32_t *out_crd, double *out_val) {
    int64_t pb = bp[i], pc = cp[i], pd = dp[i], k = 0;
    const int64_t eb = bp[i + 1], ec = cp[i + 1], ed = dp[i + 1];
    while (pb < eb || pc < ec || pd < ed) {
        int64_t j = INT64_MAX;  /* smallest column still to merge */
        if (pb < eb && bc[pb] < j) j = bc[pb];
        if (pc < ec && cc[pc] < j) j = cc[pc];
        if (pd < ed && dc[pd] < j) j = dc[pd];
        double v = 0.0;
        int have = 0;
        if (pb < eb && bc[pb] == j) { v = bv ? bv[pb] : 0.0; have = 1; ++pb; }
        if (pc < ec && cc[pc] == j) { double t = cv ? cv[pc] : 0.0; v = have ? v + t : t; have = 1; ++pc; }
        if (pd < ed && dc[pd] == j) { double t = dv ? dv[pd] : 0.0; v = have ? v + t : t; ++pd; }
        if (out_crd) { out_crd[k] = (int32_t)j; out_val[k] = v; }
        ++k;
    }
    return k;
}

void orc_spadd3_count(int64_t n, const int32_t *bp, const int32_t *bc, const int32_t *cp,
                      const int32_t *cc, const int32_t *dp, const int32_t *dc, int64_t *row_nnz) {
    for (int64_t i = 0; i < n; ++i)
        row_nnz[i] = spadd3_row(i, bp, bc, NULL, cp, cc, NULL, dp, dc, NULL, NULL, NULL);
}

void orc_spadd3(int64_t n, const int32_t *bp, const int32_t *bc, const double *bv,
                const int32_t *cp, const int32_t *cc, const double *cv,
                const int32_t *dp, const int32_t *dc, const double *dv,
                int32_t *ap, int32_t *ac, double *av) {
    ap[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t k = spadd3_row(i, bp, bc, bv, cp, cc, cv, dp, dc, dv, ac + ap[i], av + ap[i]);
        ap[i + 1] = (int32_t)(ap[i] + k);
    }
}

/* ------------------------------------------------------------------------------------
 * Universe partition of the Compressed level by coordinate value ranges (the Compressed
 * row of the partitioning table, Section IV-B: partitionByValueRanges on crd, then the
 * preimage in pos). Block b holds A's entries whose column lies in
 * [bounds[b], bounds[b+1]); it is written as its own CSR (the same {Dense, Compressed}
 * format): pos at blk_pos + b*(n+1), coordinates at blk_crd + off_b where off_b is the
 * number of entries of earlier blocks, and perm (same offsets) giving each entry's
 * position in A. Blocks are filled block by block, rows ascending, positions ascending.
 * ------------------------------------------------------------------------------------ */
void orc_column_blocks(int64_t n, const int32_t *pos, const int32_t *crd, int64_t nblk,
                       const int32_t *bounds, int32_t *blk_pos, int32_t *blk_crd, int32_t *perm) {
    int64_t out = 0;
    for (int64_t b = 0; b < nblk; ++b) {
        int32_t *bp = blk_pos + b * (n + 1);
        int64_t k = 0;
        bp[0] = 0;
        for (int64_t i = 0; i < n; ++i) {
            for (int64_t p = pos[i]; p < pos[i + 1]; ++p)
                if (crd[p] >= bounds[b] && crd[p] < bounds[b + 1]) {
                    blk_crd[out + k] = crd[p];
                    perm[out + k] = (int32_t)p;
                    ++k;
                }
            bp[i + 1] = (int32_t)k;
        }
        out += k;
    }
}
