/*
 * spd.h -- C ABI of the GB300 sparse tensor algebra kernels (libspd.so).
 *
 * The library executes the sparse kernels that SpDISTAL (Yadav, Aiken, Kjolstad,
 * "SpDISTAL: Compiling Distributed Sparse Tensor Computations", arXiv 2207.13901)
 * compiles, on one GPU:
 *
 *   SpMV      y(i)   = A(i,j) * x(j)                 Section VI-A
 *   SpMM      Y(i,l) = A(i,j) * X(j,l)               Section VI-A (there A(i,j)=B(i,k)*C(k,j))
 *   SpMM^T    dX(j,l)= A(i,j) * dY(i,l)              gradient of SpMM w.r.t. X (no paper counterpart)
 *   SDDMM     A(i,j) = B(i,j) * C(i,k) * D(k,j)      Section VI-A
 *   SpTTV     A(i,j) = B(i,j,k) * c(k)               Section VI-A
 *   SpMTTKRP  A(i,l) = B(i,j,k) * C(j,l) * D(k,l)    Section VI-A
 *
 * Sparse operands use the Dense/Compressed level formats of Sections II-B and III-B:
 * a Compressed level is a pair (pos, crd) where the children of parent entry i are at
 * positions [pos[i], pos[i+1]) of crd. CSR = {Dense, Compressed};
 * CSF = {Dense, Compressed, Compressed}. pos/crd are int32; pos[0] == 0, pos is
 * non-decreasing, pos[last] == number of children, 0 <= crd < dimension. Coordinates
 * need not be sorted within a segment and duplicates are summed like any other entry.
 *
 * Work is split in one of two ways (Section II-B, IV-B):
 *   SPD_SPLIT_ROW  universe partition of the outer Dense level: piece c of P gets the
 *                  outer coordinates [floor(c*n/P), floor((c+1)*n/P)); the inner levels
 *                  follow by image (partitionFromParent).
 *   SPD_SPLIT_NNZ  coordinate fusion of the levels plus a non-zero partition: the
 *                  coordinate tree is flattened into one sequence of items (each outer
 *                  entry's children followed by one "end of entry" item) and cut into
 *                  pieces of equal item count; the outer level follows by preimage. Outer
 *                  entries cut by a piece boundary are combined afterwards in binary64.
 *   SPD_SPLIT_AUTO picks one of the two from the structure (currently SPD_SPLIT_NNZ).
 *
 * Common conventions for every compute call:
 *   - All array arguments are DEVICE pointers owned by the caller. The library never
 *     frees, retains or allocates them, and the compute calls allocate nothing: the
 *     scratch space they need ("workspace") is passed in by the caller, sized by the
 *     matching *_workspace_size call, and may be reused once the call's work on the
 *     stream has finished.
 *   - Outputs are overwritten (the paper's "+=" into a zeroed output).
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL is the legacy default
 *     stream) except the *_validate calls, which synchronize that stream.
 *   - Argument errors are detected on the host before anything is launched and are
 *     returned as an spd_status; nothing is written in that case. Structure errors
 *     (a pos/crd that breaks the format) are NOT checked by the compute calls: run
 *     spd_csr_validate / spd_csf3_validate once per structure, or turn on checked
 *     mode (spd_set_checked) while debugging.
 *   - Dense matrices are row-major with an explicit leading dimension (in elements).
 *   - Element types: values and dense inputs share one type t; results are binary64
 *     when t is SPD_F64 and binary32 otherwise. SPD_F32/SPD_BF16 accumulate in
 *     binary32, with compensated summation across tiles of one output row; pieces of a
 *     row split across work units are combined in binary64.
 *   - Pointers must be aligned to their element size; wider alignment (16 bytes) of
 *     dense operands and leading dimensions enables vector loads.
 */
#ifndef SPD_H
#define SPD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SPD_ABI_VERSION 2

typedef enum {
    SPD_OK = 0,
    SPD_ERR_NULL = 1,      /* a required pointer is NULL */
    SPD_ERR_SHAPE = 2,     /* a size is negative or sizes are inconsistent */
    SPD_ERR_DTYPE = 3,     /* unsupported element type or type combination */
    SPD_ERR_ALIGN = 4,     /* a pointer or leading dimension is misaligned */
    SPD_ERR_STRUCTURE = 5, /* validate or checked mode: pos/crd break the level format */
    SPD_ERR_WORKSPACE = 6, /* workspace NULL or smaller than the size query returned */
    SPD_ERR_CUDA = 7,      /* a CUDA runtime call or kernel launch failed */
    SPD_ERR_OOM = 8,       /* reserved: the compute calls allocate nothing */
    SPD_ERR_TIMEOUT = 9,   /* a bounded device-side wait gave up */
    SPD_ERR_ARG = 10       /* an enum or tuning value is out of range */
} spd_status;

typedef enum { SPD_F64 = 0, SPD_F32 = 1, SPD_BF16 = 2 } spd_dtype;

typedef enum { SPD_SPLIT_ROW = 0, SPD_SPLIT_NNZ = 1, SPD_SPLIT_AUTO = 2 } spd_split;

typedef enum {
    SPD_OP_SPMV = 0,
    SPD_OP_SPMM = 1,
    SPD_OP_SPMM_T = 2,
    SPD_OP_SDDMM = 3,
    SPD_OP_SPTTV = 4,
    SPD_OP_SPMTTKRP = 5
} spd_op;

/* Largest size of any dimension, count of entries or count of fibers a descriptor may
 * hold: 2^31 - 2^17 - 1. Indices are int32 and the kernels step through them in windows
 * and tiles of up to 2^16 items, so every offset they form stays below 2^31. Larger
 * sizes return SPD_ERR_SHAPE. */
#define SPD_MAX_INDEX 2147352575LL

/* A CSR matrix {Dense, Compressed}: nrows x ncols with nnz stored entries, each size at
 * most SPD_MAX_INDEX.
 * pos: int32[nrows+1], crd: int32[nnz], vals: nnz elements of type vtype (device). */
typedef struct {
    int64_t nrows, ncols, nnz;
    const int32_t *pos;
    const int32_t *crd;
    const void *vals;
    int32_t vtype; /* spd_dtype */
    int32_t reserved;
} spd_csr;

/* A CSF 3-tensor {Dense, Compressed, Compressed} of shape dim0 x dim1 x dim2 with nfib
 * non-empty fibers (i,j) and nnz stored entries, each size at most SPD_MAX_INDEX.
 * pos1: int32[dim0+1], crd1: int32[nfib] (j of each fiber),
 * pos2: int32[nfib+1], crd2: int32[nnz] (k of each entry), vals: nnz elements. */
typedef struct {
    int64_t dim0, dim1, dim2;
    int64_t nfib, nnz;
    const int32_t *pos1;
    const int32_t *crd1;
    const int32_t *pos2;
    const int32_t *crd2;
    const void *vals;
    int32_t vtype; /* spd_dtype */
    int32_t reserved;
} spd_csf3;

/* Optional tuning (NULL = defaults). Zero fields take the default.
 *   unit_items    items (children + end-of-entry marks) per work unit of SPD_SPLIT_NNZ
 *                 for the warp-per-unit kernels (SpMM, SpMM^T, SDDMM, SpMTTKRP);
 *                 must be a multiple of 32 in [32, 65536].
 *   row_pieces    number of pieces P of SPD_SPLIT_ROW (1 <= P <= 2^31-1).
 *   block_threads threads per block for the warp-per-unit kernels: 64..512,
 *                 multiple of 32.
 *   inflight      dense rows a warp keeps in flight per group in SpMM (4 or 8;
 *                 binary64 always uses 4).
 *   lane_groups   lane shape of SpMM when L < 32 vectors of 16 bytes: 1 = groups of
 *                 4, 8 or 16 lanes, one 16-byte vector each, taking different nonzeros
 *                 side by side; 2 = one nonzero per warp step over 32 narrower lanes;
 *                 0 = the library's choice (groups when X is at most 64 MiB, so that its
 *                 rows stay in L2 and the gathers are bound by instruction issue).
 *   form          kernel form, 0 = the library's choice.
 *                 SpMV and SpTTV: 1 = a thread block per piece with tiles of 2048 items
 *                 (little shared memory, so L1 keeps caching the gathered x: the better
 *                 form for power-law columns; the default); 2 = a warp per piece with
 *                 tiles of 256 items whose crd/vals windows arrive by bulk copies (TMA)
 *                 one tile ahead (the better form when x is read locally, e.g. banded
 *                 matrices).
 *                 SDDMM: 1 = CUDA cores (the default); 2 = tensor cores (mma.sync,
 *                 bfloat16 values and dense operands, K a multiple of 32, 16-byte
 *                 aligned rows; other calls take the CUDA cores). */
typedef struct {
    int32_t unit_items;
    int32_t row_pieces;
    int32_t block_threads;
    int32_t inflight;
    int32_t lane_groups;
    int32_t form;
} spd_tune;

/* -------------------------------------------------------------------- misc */

/* SPD_ABI_VERSION of the loaded library. */
int spd_abi_version(void);

/* Static English text for a status code (never NULL). */
const char *spd_status_str(int status);

/* Detail of the last error returned on the calling thread (static buffer of the
 * thread; empty string when there is none). */
const char *spd_last_error(void);

/* Checked mode, for debugging (off by default; on from the start when the environment
 * variable SPD_DEBUG is set to anything but "" or "0"). While it is on, every call that
 * takes a sparse operand (partition, compute, transpose, column blocks, SpAdd3, batched
 * plan) first validates that operand as spd_csr_validate / spd_csf3_validate do, through
 * a status word in device memory, and returns SPD_ERR_STRUCTURE, with the operand's name
 * and first bad index in spd_last_error(), before it launches any work on a broken one.
 * Each call then synchronizes its stream, so that an execution error is returned by the
 * call that caused it (SPD_ERR_CUDA). Checked calls therefore cannot be captured into a
 * CUDA graph: the validation returns SPD_ERR_ARG during a capture (spd_spmm_batched_run,
 * which validates nothing, is still captured; it skips the synchronization then). The
 * validations of concurrent host threads are serialized. `on` is 0 or 1, else
 * SPD_ERR_ARG. Process-wide; not meant to change while calls are in flight. */
spd_status spd_set_checked(int on);

/* 1 while checked mode is on, else 0. */
int spd_checked(void);

/* Device faults of earlier calls: kernels that stage data with bulk copies wait for them
 * with a bounded wait (1 s); one that gives up records bit 1 in a device fault word and
 * leaves its outputs unspecified. This call synchronizes `stream`, stores the OR of the
 * recorded bits in *flags (0 when none), clears them, and returns SPD_ERR_TIMEOUT when any
 * was set. Checked mode performs the same check after every call. Not during a capture. */
spd_status spd_fault_status(uint32_t *flags, void *stream);

/* Diagnostic of the fault path above (no counterpart in the paper): launches on `stream`
 * one kernel that waits, with the same bounded wait, for bulk copies that are never
 * issued, so that the wait gives up after 1 s and records bit 1; spd_fault_status then
 * reports it. The kernel accesses no memory but its own shared memory and leaves no copy
 * in flight, so the context stays usable. Asynchronous; returns SPD_ERR_CUDA only if the
 * launch fails. */
spd_status spd_probe_bounded_wait(void *stream);

/* -------------------------------------------------------------------- sizes */

/* Workspace bytes that `op` on CSR `A` with `split` needs. `width` is L for SpMM and
 * SpMM^T, K for SDDMM, ignored for SpMV. The result may be 0 (any pointer, even NULL,
 * is then accepted as workspace). Host-only, no device access. */
spd_status spd_csr_workspace_size(int op, const spd_csr *A, int split, int64_t width,
                                  const spd_tune *tune, size_t *bytes);

/* Same for the CSF operations (SPD_OP_SPTTV; SPD_OP_SPMTTKRP with width = R). */
spd_status spd_csf3_workspace_size(int op, const spd_csf3 *B, int split, int64_t width,
                                   const spd_tune *tune, size_t *bytes);

/* -------------------------------------------------------------------- structure */

/* Checks the level-format invariants of A (Section III-B): pos[0] == 0, pos
 * non-decreasing, pos[nrows] == nnz, 0 <= crd < ncols. Needs a workspace of at least
 * 64 bytes. Synchronizes `stream`. On return *violations holds the number of violated
 * entries and *first_bad the smallest offending index (an index into pos, or
 * nrows + 1 + p for crd position p), or -1 if there is none. Returns SPD_OK when the
 * structure is valid, SPD_ERR_STRUCTURE when it is not. */
spd_status spd_csr_validate(const spd_csr *A, void *ws, size_t ws_bytes, int64_t *violations,
                            int64_t *first_bad, void *stream);

/* The same checks on both Compressed levels of a CSF tensor: level 2 (pos1/crd1 against
 * dim1, children nfib) then level 3 (pos2/crd2 against dim2, children nnz). first_bad
 * indexes the concatenation pos1 | crd1 | pos2 | crd2. Synchronizes `stream`. */
spd_status spd_csf3_validate(const spd_csf3 *B, void *ws, size_t ws_bytes, int64_t *violations,
                             int64_t *first_bad, void *stream);

/* Writes the work partition the compute calls use (Sections II-B, III-A, IV-C) into two
 * device int32 arrays of length npieces+1:
 *   SPD_SPLIT_ROW: rows_out[c] = floor(c*nrows/P) with P = npieces, pos_out[c] =
 *                  pos[rows_out[c]] (the image of the row piece in crd).
 *   SPD_SPLIT_NNZ: for the diagonals d_c = min(c*unit_items, nrows + nnz) of the
 *                  flattened item sequence, rows_out[c] = number of rows whose end
 *                  item lies before d_c and pos_out[c] = d_c - rows_out[c]; here
 *                  npieces must equal ceil((nrows + nnz) / unit_items).
 * unit_items is ignored for SPD_SPLIT_ROW. Asynchronous. */
spd_status spd_csr_partition(const spd_csr *A, int split, int64_t npieces, int64_t unit_items,
                             int32_t *rows_out, int32_t *pos_out, void *stream);

/* -------------------------------------------------------------------- compute */

/* SpMV y(i) = A(i,j) * x(j).  x: ncols elements of A->vtype; y: nrows elements of
 * y_type (SPD_F64 for F64 values, SPD_F32 otherwise). */
spd_status spd_spmv(const spd_csr *A, const void *x, int x_type, void *y, int y_type, int split,
                    const spd_tune *tune, void *ws, size_t ws_bytes, void *stream);

/* SpMM Y(i,l) = A(i,j) * X(j,l), l < L.  X: ncols x L (leading dimension ldx >= L) of
 * x_type == A->vtype; Y: nrows x L (ldy >= L) of y_type. */
spd_status spd_spmm(const spd_csr *A, const void *X, int64_t L, int64_t ldx, int x_type, void *Y,
                    int64_t ldy, int y_type, int split, const spd_tune *tune, void *ws,
                    size_t ws_bytes, void *stream);

/* Y(i,l) += A(i,j) * X(j,l): as spd_spmm, but the product is added to Y (the generated
 * code's "+=" of Section IV-C on an output that already holds values). Rows of A without
 * entries leave Y untouched. Used to sum the products of column blocks
 * (spd_csr_column_blocks). */
spd_status spd_spmm_accumulate(const spd_csr *A, const void *X, int64_t L, int64_t ldx, int x_type, void *Y,
                               int64_t ldy, int y_type, int split, const spd_tune *tune, void *ws,
                               size_t ws_bytes, void *stream);

/* SpMM^T dX(j,l) = A(i,j) * dY(i,l): the gradient of Y = A X with respect to X, without
 * forming A's transpose (rows of A are walked and scattered with atomic adds, so the
 * summation order is not deterministic).  dY: nrows x L (ldy) of dy_type ==
 * A->vtype; dX: ncols x L (ldx) of dx_type (F64 for F64, F32 otherwise). */
spd_status spd_spmm_t(const spd_csr *A, const void *dY, int64_t L, int64_t ldy, int dy_type,
                      void *dX, int64_t ldx, int dx_type, int split, const spd_tune *tune,
                      void *ws, size_t ws_bytes, void *stream);

/* -------------------------------------------------------------------- transposed schedule
 *
 * A^T in the same {Dense, Compressed} level formats, i.e. A in the CSC encoding (the
 * format language of Section II-B: the level formats of CSR with the dimension order
 * reversed). With it, the SpMM gradient dX = A^T dY is an ordinary spd_spmm over
 * (t_pos, t_crd, gathered values): every row of dX is written once, in a fixed order,
 * with no atomic scatter. The paper's statements do not need it; the structure depends
 * only on A's pattern, so a caller computes it once and reuses it while only the values
 * change. */

/* Workspace bytes of spd_csr_transpose (host only): about 12 bytes per nonzero plus
 * 1 KiB per 4096 nonzeros. */
spd_status spd_csr_transpose_workspace_size(const spd_csr *A, size_t *bytes);

/* The structure of A^T (ncols x nrows) and the permutation into it, all device int32:
 *   t_pos[ncols + 1]: t_pos[j] = number of entries of A in columns < j;
 *   t_crd[nnz]: row coordinates, ascending within each column (entries of a column
 *               keep A's row order: a stable sort of A's positions by column);
 *   perm[nnz]: perm[q] = the position in A of the q-th entry of A^T, so that A^T's
 *              values are vals[perm[q]] (spd_gather_vals).
 * A->vals is not read. Caller-owned outputs; ws of spd_csr_transpose_workspace_size
 * bytes, 256-byte aligned. Asynchronous on `stream`; the result is deterministic.
 * A's structure must be valid (spd_csr_validate): coordinates outside [0, ncols) give
 * an unspecified (but in-bounds) result. */
spd_status spd_csr_transpose(const spd_csr *A, int32_t *t_pos, int32_t *t_crd, int32_t *perm, void *ws,
                             size_t ws_bytes, void *stream);

/* out[q] = in[perm[q]] for q < n: n elements of vtype, device memory, caller-owned.
 * Carries A's values into A^T's order. Asynchronous. */
spd_status spd_gather_vals(int64_t n, const int32_t *perm, const void *in, void *out, int vtype, void *stream);

/* -------------------------------------------------------------------- column blocks
 *
 * Universe partition of A's Compressed level by coordinate value ranges (Section IV-B,
 * the Compressed row of the partitioning table: partitionByValueRanges on crd and its
 * preimage in pos). Block b holds A's entries with bounds[b] <= column < bounds[b+1] and
 * is written as its own CSR of A's shape: pos at blk_pos + b*(nrows+1) (nrows+1 int32,
 * starting at 0), coordinates at blk_crd + off_b, where off_b = blk_nnz[0] + ... +
 * blk_nnz[b-1], and perm (same offsets) holding each entry's position in A, so that the
 * block's values are vals[perm[...]] (spd_gather_vals). Entries keep A's row order and,
 * within a row, column order. Y = A X is then the sum over blocks of A_b X, each of which
 * gathers only rows bounds[b] .. bounds[b+1]-1 of X (spd_spmm for the first block,
 * spd_spmm_accumulate for the others). */

/* Workspace bytes of spd_csr_column_blocks (host only); 1 <= nblk <= 65536. */
spd_status spd_csr_column_blocks_workspace_size(const spd_csr *A, int64_t nblk, size_t *bytes);

/* bounds: host int32[nblk + 1], bounds[0] = 0, bounds[nblk] = ncols, non-decreasing.
 * blk_pos: device int32[nblk * (nrows + 1)]; blk_crd, perm: device int32[nnz]; blk_nnz:
 * host int64[nblk] (entries per block). A->vals is not read. Synchronizes `stream`
 * (the block sizes are returned on the host). */
spd_status spd_csr_column_blocks(const spd_csr *A, int64_t nblk, const int32_t *bounds, int32_t *blk_pos,
                                 int32_t *blk_crd, int32_t *perm, int64_t *blk_nnz, void *ws, size_t ws_bytes,
                                 void *stream);

/* -------------------------------------------------------------------- SpAdd3
 *
 * SpAdd3 A(i,j) = B(i,j) + C(i,j) + D(i,j) (Section VI-A): B, C, D are CSR of one shape
 * and value type, each row with ascending distinct columns. A's pattern is the union
 * of the three patterns (a coordinate stored in any operand is stored in A, even where
 * the values cancel), so A is assembled in two phases (Section V-B): the symbolic call
 * counts each row of A and writes A's pos; the caller then provides crd/vals of the
 * returned size to the numeric call, which fills them. A value is (B + C) + D over the
 * operands that store the coordinate, in binary64 for binary64 operands and in binary32
 * otherwise; A's values have result type (SPD_F64 for F64, SPD_F32 otherwise).
 * split: SPD_SPLIT_ROW (the rows in P = row_pieces or about (nrows + nnz) / unit_items
 * pieces) or SPD_SPLIT_NNZ (pieces of unit_items of the fused rows, entries of B, C and
 * D together; default 64; a piece inside a row takes a column range). Both calls must
 * get the same operands, split, tuning and workspace; the workspace keeps the
 * partition between them and must not be touched in between. */

/* Workspace bytes of the two SpAdd3 calls (host only). */
spd_status spd_spadd3_workspace_size(const spd_csr *B, const spd_csr *C, const spd_csr *D, int split,
                                     const spd_tune *tune, size_t *bytes);

/* Phase 1: a_pos (device int32[nrows + 1], caller-owned) receives A's pos; *nnz_out (host)
 * receives nnz(A) = a_pos[nrows]. Synchronizes `stream` (the size is needed on the host
 * to allocate A). nnz(B) + nnz(C) + nnz(D) must be at most SPD_MAX_INDEX. */
spd_status spd_spadd3_symbolic(const spd_csr *B, const spd_csr *C, const spd_csr *D, int split,
                               const spd_tune *tune, int32_t *a_pos, int64_t *nnz_out, void *ws,
                               size_t ws_bytes, void *stream);

/* Phase 2: writes A's a_nnz coordinates into a_crd (device int32) and values into a_vals
 * (device, a_type = result type), rows in order, columns ascending. a_pos is the
 * symbolic call's output. Asynchronous. */
spd_status spd_spadd3_numeric(const spd_csr *B, const spd_csr *C, const spd_csr *D, int split,
                              const spd_tune *tune, const int32_t *a_pos, int64_t a_nnz, int32_t *a_crd,
                              void *a_vals, int a_type, void *ws, size_t ws_bytes, void *stream);

/* SDDMM A(i,j) = B(i,j) * C(i,k) * D(k,j), k < K. The output keeps B's pattern
 * (Section V-B): out_vals[p] is the value at B's position p, and B's pos/crd serve as
 * the output's. B->vals may be NULL: every B value is then 1 (the sampling pattern).
 * C: nrows x K (ldc); D is passed transposed, as Dnk: ncols x K (ldd) with
 * Dnk[j,k] = D(k,j). C, Dnk (and B's values) have dense_type; out_vals has out_type. */
spd_status spd_sddmm(const spd_csr *B, const void *C, int64_t K, int64_t ldc, const void *Dnk,
                     int64_t ldd, int dense_type, void *out_vals, int out_type, int split,
                     const spd_tune *tune, void *ws, size_t ws_bytes, void *stream);

/* SpTTV A(i,j) = B(i,j,k) * c(k). The output keeps B's (i,j) structure (Section V-B):
 * out_vals[f] belongs to fiber f, and B's pos1/crd1 serve as the output's pos/crd.
 * c: dim2 elements of c_type == B->vtype. */
spd_status spd_spttv(const spd_csf3 *B, const void *c, int c_type, void *out_vals, int out_type,
                     int split, const spd_tune *tune, void *ws, size_t ws_bytes, void *stream);

/* SpMTTKRP A(i,l) = B(i,j,k) * C(j,l) * D(k,l), l < R.  C: dim1 x R (ldc), D: dim2 x R
 * (ldd) of factor_type == B->vtype; A: dim0 x R (lda) of a_type. A row stride of C or D
 * of 4 GiB or more returns SPD_ERR_SHAPE. */
spd_status spd_spmttkrp(const spd_csf3 *B, const void *C, int64_t ldc, const void *D, int64_t ldd,
                        int64_t R, int factor_type, void *A, int64_t lda, int a_type, int split,
                        const spd_tune *tune, void *ws, size_t ws_bytes, void *stream);

/* -------------------------------------------------------------------- batches */

/* One product Y_m = A_m X_m of a batched SpMM (Section VI-A's SpMM statement, applied
 * to many independent matrices). X: A.ncols x L (ldx), Y: A.nrows x L (ldy), both of the
 * batch's value type / result type. split: SPD_SPLIT_ROW or SPD_SPLIT_NNZ for this
 * matrix; unit_items: items per piece for this matrix (multiple of 32 in [32, 65536];
 * 0 = the tuning's unit_items). */
typedef struct {
    spd_csr A;
    const void *X;
    int64_t ldx;
    void *Y;
    int64_t ldy;
    int32_t split;
    int32_t unit_items;
} spd_batch_item;

/* Filled by spd_spmm_batched_plan; owned by the caller; read by spd_spmm_batched_run.
 * It points into the caller's workspace, which must outlive every run of the plan. */
typedef struct {
    int64_t count, total_pieces, L;
    int32_t vtype, epl, group, block_threads, grid, fulltile, has_nnz;
    void *ws;
    size_t off_desc, off_pstart, off_prow, off_ppos, off_crow, off_cval, off_pmat;
} spd_batch_plan;

/* Workspace bytes of a batch (host only). items: host array of count entries. */
spd_status spd_spmm_batched_workspace_size(int64_t count, const spd_batch_item *items, int64_t L, int vtype,
                                           const spd_tune *tune, size_t *bytes);

/* Lays the pieces of every matrix end to end (row split: universe partition of its
 * rows; nnz split: fused non-zero partition computed here on the device) and writes the
 * descriptors into ws. Copies from host memory and synchronizes `stream` before
 * returning. The matrices' structure must not change while the plan is in use (values,
 * X and Y may). */
spd_status spd_spmm_batched_plan(int64_t count, const spd_batch_item *items, int64_t L, int vtype,
                                 const spd_tune *tune, void *ws, size_t ws_bytes, spd_batch_plan *plan,
                                 void *stream);

/* Runs every product of the plan: one persistent kernel whose warps take the global
 * pieces in a static stride, then one fix-up kernel for the nnz-split matrices.
 * Asynchronous; allocates nothing and never synchronizes, so it may be captured in a
 * CUDA graph and replayed. */
spd_status spd_spmm_batched_run(const spd_batch_plan *plan, void *stream);

/* SpMV y(i) = A(i,j) * x(j) for callers that cannot allocate device memory. The paper
 * has no counterpart: this is a calling convention of this library, not a step of the
 * method. Callers such as a plugin inside a host framework that owns all device memory,
 * or a latency-critical path that may not call an allocator, cannot provide the
 * workspace spd_spmv asks for. This entry runs the same nnz-split SpMV (default tuning)
 * on a fixed scratch array compiled into the library: 1 MiB of device memory that every
 * GPU loading the library holds until the process exits. It calls no allocator.
 *   - Limit: the scratch must hold what spd_csr_workspace_size(SPD_OP_SPMV, A,
 *     SPD_SPLIT_NNZ, ...) reports, about 20 bytes per 2048 items, so nrows + nnz up to
 *     about 107 million fits; larger inputs return SPD_ERR_SHAPE before any launch.
 *   - The array exists once per CUDA context that loads the library. The first call
 *     in a context (the current one of the calling thread, e.g. a device's primary
 *     context or a context the caller made current with the driver API) looks up the
 *     array's device address with cudaGetSymbolAddress and caches it under the
 *     context's unique id. Make that first call before any stream capture: while the
 *     stream is being captured it returns SPD_ERR_ARG.
 *   - All calls share the one array, which keeps the last call's contents. Each call
 *     writes every scratch byte before reading it, so no clearing is needed, but calls
 *     whose GPU work overlaps (different streams, or different threads) race on the
 *     array: order them on one stream or synchronise between them.
 *   - Arguments, types, ownership and errors are those of spd_spmv. */
spd_status spd_spmv_noalloc(const spd_csr *A, const void *x, int x_type, void *y, int y_type, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SPD_H */
