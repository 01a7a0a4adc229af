// spd_spmv.cu -- SpMV y(i) = A(i,j) * x(j) and SpTTV A(i,j) = B(i,j,k) * c(k)
// (Section VI-A). SpTTV is the same computation over B's level 3: every fiber (i,j)
// is one output entry (the output keeps B's (i,j) structure, Section V-B).
//
// One thread block consumes one piece of the flattened coordinate tree, tile by tile:
//   1. each row whose end item falls in the tile sets that item's bit in a shared
//      bitmap of the tile (item index = nonzeros before the row end + earlier row
//      ends); a popcount prefix over the bitmap words gives, for any item, the number
//      of row ends before it, i.e. where the merge path crosses that item. The tile's
//      products vals[p] * x[crd[p]] are computed with coalesced crd/vals loads and x
//      gathers into shared memory;
//   2. every thread takes IPT consecutive items of the tile (its start row is one
//      popcount away), sums products and writes the rows it completes;
//   3. a block-wide segmented scan hands each thread the partial sum of the row it
//      started in, and carries the open row into the next tile (compensated when a
//      row spans tiles, i.e. is longer than one tile).
// Row split: piece c = rows [floor(c n/P), floor((c+1) n/P)) (the universe partition of
// the generated code in Section IV-C). Nnz split: pieces of equal item count from the
// partition array; the partial row at each piece end goes to a binary64 carry that a
// fix-up kernel adds to the row (the reduction into the output of Section II-D).
#include "spd_internal.cuh"

namespace spd {

// Shared-memory index with one padding word per 32 entries: each thread consumes IPT
// consecutive entries, so without the skew a warp's 32 threads would fall on only
// 32/IPT banks.
__device__ __forceinline__ int skew(int i) { return i + (i >> 5); }

// Resident blocks per SM: 8 for bfloat16 values; 6 otherwise, which leaves the binary32
// and binary64 tiles enough registers not to spill (measured faster on power-law rows).
template <typename VT, int NT, int IPT>
__global__ void __launch_bounds__(NT, sizeof(VT) == 2 ? 8 : 6) spmv_tile_kernel(
    int64_t n, const int32_t *__restrict__ pos, const int32_t *__restrict__ crd, const VT *__restrict__ vals,
    const VT *__restrict__ x, typename Traits<VT>::out *__restrict__ y,
    const int32_t *__restrict__ prow, const int32_t *__restrict__ ppos,  // nnz split
    int64_t P, int64_t nouter, const int32_t *__restrict__ outer,         // row split
    int32_t *__restrict__ carry_row, double *__restrict__ carry_val) {
    using AT = typename Traits<VT>::acc;
    using OT = typename Traits<VT>::out;
    constexpr int TILE = NT * IPT;
    constexpr int NW = NT / 32;
    constexpr int NWORDS = TILE / 32;  // bitmap words of a tile
    constexpr unsigned FULL = 0xffffffffu;
    static_assert(32 % IPT == 0 && NWORDS == 64, "a thread's items share one bitmap word; warp 0 scans 64 words");
    __shared__ uint32_t s_bits[NWORDS];     // bit k of the tile: item k is a row end
    __shared__ int32_t s_wpre[NWORDS + 1];  // row ends before each word; [NWORDS] = all
    __shared__ AT s_prod[TILE + TILE / 32];
    __shared__ AT s_wv[NW];
    __shared__ int s_wf[NW];
    __shared__ AT s_tv;
    __shared__ int s_tf;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t c = blockIdx.x;
    PieceBounds b;
    if (prow) {
        b = nnz_piece(c, prow, ppos);
    } else if (outer) {
        // SpTTV row split: slices [floor(c I/P), floor((c+1) I/P)) and, by image, their fibers
        int64_t i0 = (c * nouter) / P, i1 = ((c + 1) * nouter) / P;
        b.r0 = __ldg(outer + i0);
        b.r1 = __ldg(outer + i1);
        b.p0 = __ldg(pos + b.r0);
        b.p1 = __ldg(pos + b.r1);
    } else {
        b = row_piece(c, P, n, pos);
    }
    int32_t r = b.r0, p = b.p0;
    AT carry_hi = 0, carry_lo = 0;  // partial of row r accumulated over earlier tiles

    while (true) {
        const int64_t rem_rows = (int64_t)b.r1 - r, rem_nnz = (int64_t)b.p1 - p;
        if (rem_rows + rem_nnz == 0) break;
        const int nr = (int)(rem_rows < TILE ? rem_rows : TILE);
        const int items = (int)((rem_rows + rem_nnz) < TILE ? (rem_rows + rem_nnz) : TILE);
        for (int w = tid; w < NWORDS; w += NT) s_bits[w] = 0u;
        __syncthreads();
        for (int q = tid; q < nr; q += NT) {
            const int e = ld_stream(pos + r + 1 + q) - p + q;  // item index of row q's end
            if (e < items) atomicOr(&s_bits[e >> 5], 1u << (e & 31));
        }
        __syncthreads();
        if (wid == 0) {  // exclusive popcount prefix of the 64 words, two per lane
            const int c0 = __popc(s_bits[2 * lane]), c1 = __popc(s_bits[2 * lane + 1]);
            int inc = c0 + c1;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int t = __shfl_up_sync(FULL, inc, off);
                if (lane >= off) inc += t;
            }
            s_wpre[2 * lane] = inc - c0 - c1;
            s_wpre[2 * lane + 1] = inc - c1;
            if (lane == 31) s_wpre[NWORDS] = inc;
        }
        __syncthreads();
        const int ic = s_wpre[NWORDS];  // row ends in the tile
        const int jc = items - ic;
        // products of the tile's nonzeros: coalesced crd/vals, gathered x
        {
            int32_t cc[IPT];
            AT vv[IPT];
#pragma unroll
            for (int k = 0; k < IPT; ++k) {
                int q = tid + k * NT;
                cc[k] = q < jc ? ld_stream(crd + p + q) : 0;
                vv[k] = q < jc ? (AT)ld_stream(vals + p + q) : (AT)0;
            }
#pragma unroll
            for (int k = 0; k < IPT; ++k) {
                int q = tid + k * NT;
                if (q < jc) s_prod[skew(q)] = vv[k] * (AT)ld_gather(x + cc[k]);
            }
        }
        __syncthreads();
        // this thread's IPT items of the tile
        const int k0 = tid * IPT < items ? tid * IPT : items;
        const int k1 = k0 + IPT < items ? k0 + IPT : items;
        const int word = k0 < TILE ? (k0 >> 5) : NWORDS - 1;
        const int sh = k0 & 31;
        const uint32_t wbits = s_bits[word];
        const uint32_t mine = k0 < TILE ? wbits >> sh : 0u;  // bit k: item k0 + k is a row end
        int i = s_wpre[word] + __popc(sh ? (wbits & ((1u << sh) - 1u)) : 0u);
        int j = k0 - i;
        AT acc = 0, first_val = 0;
        int first_row = -1;
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            if (k0 + k < k1) {
                if ((mine >> k) & 1u) {  // row i ends here: all its children consumed
                    if (first_row < 0) {
                        first_row = i;
                        first_val = acc;
                    } else {
                        y[r + i] = (OT)acc;
                    }
                    acc = 0;
                    ++i;
                } else {
                    acc += s_prod[skew(j)];
                    ++j;
                }
            }
        }
        // block-wide segmented inclusive scan of (ended-a-row, tail partial)
        int f = first_row >= 0;
        AT v = acc;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int pf = __shfl_up_sync(FULL, f, off);
            AT pv = __shfl_up_sync(FULL, v, off);
            if (lane >= off) {
                if (!f) v += pv;
                f |= pf;
            }
        }
        if (lane == 31) {
            s_wf[wid] = f;
            s_wv[wid] = v;
        }
        __syncthreads();
        AT wp_v = 0;
        int wp_f = 0;
        for (int w = 0; w < wid; ++w) {
            if (s_wf[w]) {
                wp_v = s_wv[w];
                wp_f = 1;
            } else {
                wp_v += s_wv[w];
            }
        }
        const AT incl_v = f ? v : wp_v + v;
        const int incl_f = f | wp_f;
        AT ev = __shfl_up_sync(FULL, incl_v, 1);
        int ef = __shfl_up_sync(FULL, incl_f, 1);
        if (lane == 0) {
            ev = wp_v;
            ef = wp_f;
        }
        if (tid == NT - 1) {
            s_tv = incl_v;
            s_tf = incl_f;
        }
        if (first_row >= 0) {
            AT tot = first_val + ev;
            if (!ef) {  // the tile's first completed row is row r: add what earlier tiles carried
                AT hi = carry_hi, lo = carry_lo;
                comp_add(hi, lo, tot);
                tot = hi + lo;
            }
            y[r + first_row] = (OT)tot;
        }
        __syncthreads();
        const AT tv = s_tv;
        const int tf = s_tf;
        if (tf) {
            carry_hi = tv;
            carry_lo = 0;
        } else {
            comp_add(carry_hi, carry_lo, tv);
        }
        r += ic;
        p += jc;
        __syncthreads();
    }
    if (carry_row && tid == 0) {
        // the piece ends inside row r1: hand its partial to the fix-up when it is non-empty
        int32_t start = b.r1 < n ? __ldg(pos + b.r1) : b.p1;
        if (start < b.p0) start = b.p0;
        bool has = b.p1 > start;
        carry_row[c] = has ? b.r1 : -1;
        carry_val[c] = has ? (double)carry_hi + (double)carry_lo : 0.0;
    }
}

// Adds the binary64 carries of consecutive pieces that ended inside the same row to the
// value the completing piece wrote (one thread per run of pieces).
template <typename OT>
__global__ void carry_fixup_scalar_kernel(int64_t npieces, const int32_t *__restrict__ carry_row,
                                          const double *__restrict__ carry_val, OT *__restrict__ y) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= npieces) return;
    int32_t row = carry_row[c];
    if (row < 0) return;
    if (c > 0 && carry_row[c - 1] == row) return;
    double s = 0.0;  // the run in batches of 8 independent loads, summed in piece order
    for (int64_t d = c; d < npieces; d += 8) {
        int32_t tag[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) tag[k] = d + k < npieces ? carry_row[d + k] : -1;
        double v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = tag[k] == row ? carry_val[d + k] : 0.0;
        bool more = true;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            more = more && tag[k] == row;
            if (more) s += v[k];
        }
        if (!more) break;
    }
    y[row] = (OT)((double)y[row] + s);
}

// Shared host path of SpMV (n rows of `pos`) and SpTTV (n = fibers, pos = pos2; the
// row split then partitions the nouter slices of `outer` = pos1).
template <typename VT>
static spd_status launch_spmv(int64_t n, int64_t nnz, const int32_t *pos, const int32_t *crd, const void *vals,
                              const void *x, void *y, int split, const Tuning &tn, int64_t nouter,
                              const int32_t *outer, void *ws, cudaStream_t st) {
    using OT = typename Traits<VT>::out;
    const VT *v = static_cast<const VT *>(vals);
    const VT *xx = static_cast<const VT *>(x);
    OT *yy = static_cast<OT *>(y);
    if (split == SPD_SPLIT_ROW) {
        int64_t P = tn.row_pieces;
        if (P <= 0) P = ceil_div(n + nnz, kSpmvTile);
        if (P < 1) P = 1;
        spmv_tile_kernel<VT, kSpmvThreads, kSpmvIPT><<<(unsigned)P, kSpmvThreads, 0, st>>>(
            n, pos, crd, v, xx, yy, nullptr, nullptr, P, nouter, outer, nullptr, nullptr);
        return check_launch("spmv_tile_kernel(row)");
    }
    WsLayout L = layout_spmv(n, nnz, split);
    char *w = static_cast<char *>(ws);
    int32_t *prow = reinterpret_cast<int32_t *>(w + L.part_row);
    int32_t *ppos = reinterpret_cast<int32_t *>(w + L.part_pos);
    int32_t *crow = reinterpret_cast<int32_t *>(w + L.carry_row);
    double *cval = reinterpret_cast<double *>(w + L.carry_val);
    spd_status s = launch_merge_partition(n, nnz, pos, kSpmvTile, L.npieces, prow, ppos, st);
    if (s) return s;
    spmv_tile_kernel<VT, kSpmvThreads, kSpmvIPT><<<(unsigned)L.npieces, kSpmvThreads, 0, st>>>(
        n, pos, crd, v, xx, yy, prow, ppos, 0, 0, nullptr, crow, cval);
    s = check_launch("spmv_tile_kernel(nnz)");
    if (s) return s;
    carry_fixup_scalar_kernel<OT><<<(unsigned)ceil_div(L.npieces, 256), 256, 0, st>>>(L.npieces, crow, cval, yy);
    return check_launch("carry_fixup_scalar_kernel");
}

static spd_status dispatch_spmv(int vtype, int64_t n, int64_t nnz, const int32_t *pos, const int32_t *crd,
                                const void *vals, const void *x, void *y, int split, const Tuning &tn,
                                int64_t nouter, const int32_t *outer, void *ws, cudaStream_t st) {
    switch (vtype) {
        case SPD_F64: return launch_spmv<double>(n, nnz, pos, crd, vals, x, y, split, tn, nouter, outer, ws, st);
        case SPD_F32: return launch_spmv<float>(n, nnz, pos, crd, vals, x, y, split, tn, nouter, outer, ws, st);
        case SPD_BF16:
            return launch_spmv<__nv_bfloat16>(n, nnz, pos, crd, vals, x, y, split, tn, nouter, outer, ws, st);
        default: return fail(SPD_ERR_DTYPE, "unknown value type %d", vtype);
    }
}

// Nnz-split SpMV with default tuning on a scratch area the caller already owns (laid out
// as layout_spmv describes); used by the entry point that allocates nothing.
spd_status spmv_nnz_on_scratch(const spd_csr *A, const void *x, void *y, void *scratch, cudaStream_t st) {
    Tuning tn;
    read_tune(nullptr, &tn);
    return dispatch_spmv(A->vtype, A->nrows, A->nnz, A->pos, A->crd, A->vals, x, y, SPD_SPLIT_NNZ, tn, 0, nullptr,
                         scratch, st);
}

}  // namespace spd

using namespace spd;

extern "C" {

spd_status spd_spmv(const spd_csr *A, const void *x, int x_type, void *y, int y_type, int split,
                    const spd_tune *tune, void *ws, size_t ws_bytes, void *stream) {
    spd_status s = check_csr(A, true);
    if (s) return s;
    if (x_type != A->vtype) return fail(SPD_ERR_DTYPE, "x type %d differs from the value type %d", x_type, A->vtype);
    if (y_type != result_type(A->vtype)) return fail(SPD_ERR_DTYPE, "y type %d; expected %d", y_type, result_type(A->vtype));
    if (A->ncols > 0 && !x) return fail(SPD_ERR_NULL, "x is NULL");
    if (A->nrows > 0 && !y) return fail(SPD_ERR_NULL, "y is NULL");
    if ((x && !aligned(x, dtype_size(x_type))) || (y && !aligned(y, dtype_size(y_type))))
        return fail(SPD_ERR_ALIGN, "x or y not aligned to its element size");
    Tuning tn;
    if ((s = read_tune(tune, &tn))) return s;
    split = resolve_split(split);
    if (split != SPD_SPLIT_ROW && split != SPD_SPLIT_NNZ) return fail(SPD_ERR_ARG, "unknown split %d", split);
    WsLayout L = layout_spmv(A->nrows, A->nnz, split);
    if ((s = check_ws(L, ws, ws_bytes))) return s;
    cudaStream_t st = as_stream(stream);
    if ((s = checked_csr(A, "A", st))) return s;
    if (A->nrows == 0) return SPD_OK;
    return checked_finish(
        dispatch_spmv(A->vtype, A->nrows, A->nnz, A->pos, A->crd, A->vals, x, y, split, tn, 0, nullptr, ws, st),
        "spd_spmv", st);
}

spd_status spd_spttv(const spd_csf3 *B, const void *c, int c_type, void *out_vals, int out_type, int split,
                     const spd_tune *tune, void *ws, size_t ws_bytes, void *stream) {
    spd_status s = check_csf3(B);
    if (s) return s;
    if (c_type != B->vtype) return fail(SPD_ERR_DTYPE, "c type %d differs from the value type %d", c_type, B->vtype);
    if (out_type != result_type(B->vtype)) return fail(SPD_ERR_DTYPE, "output type %d; expected %d", out_type, result_type(B->vtype));
    if (B->dim2 > 0 && !c) return fail(SPD_ERR_NULL, "c is NULL");
    if (B->nfib > 0 && !out_vals) return fail(SPD_ERR_NULL, "out_vals is NULL");
    if ((c && !aligned(c, dtype_size(c_type))) || (out_vals && !aligned(out_vals, dtype_size(out_type))))
        return fail(SPD_ERR_ALIGN, "c or out_vals not aligned to its element size");
    Tuning tn;
    if ((s = read_tune(tune, &tn))) return s;
    split = resolve_split(split);
    if (split != SPD_SPLIT_ROW && split != SPD_SPLIT_NNZ) return fail(SPD_ERR_ARG, "unknown split %d", split);
    WsLayout L = layout_spmv(B->nfib, B->nnz, split);
    if ((s = check_ws(L, ws, ws_bytes))) return s;
    cudaStream_t st = as_stream(stream);
    if ((s = checked_csf3(B, "B", st))) return s;
    if (B->nfib == 0) return SPD_OK;
    if (split == SPD_SPLIT_ROW && tn.row_pieces <= 0) {
        int64_t P = ceil_div(B->nfib + B->nnz, kSpmvTile);
        tn.row_pieces = P < B->dim0 ? P : B->dim0;
        if (tn.row_pieces < 1) tn.row_pieces = 1;
    }
    return checked_finish(dispatch_spmv(B->vtype, B->nfib, B->nnz, B->pos2, B->crd2, B->vals, c, out_vals, split, tn,
                                        B->dim0, split == SPD_SPLIT_ROW ? B->pos1 : nullptr, ws, st),
                          "spd_spttv", st);
}

}  // extern "C"
