// spd_sddmm.cu -- SDDMM A(i,j) = B(i,j) * C(i,k) * D(k,j) (Section VI-A).
//
// The output keeps B's coordinate structure (Section V-B): one value per stored
// position p of B, so the work is a stream over B's positions with two gathered dense
// rows per position: row i of C and row j of D, with D passed transposed as
// Dnk[j,k] = D(k,j) so that both rows are contiguous. One warp consumes one piece of
// the flattened coordinate tree (rows and positions balanced together); its lanes span
// K in vectors of EPL elements, U positions are in flight at once, and each dot product
// is finished with a butterfly reduction across the warp.
//
// The contraction over k is a dot product per stored position (a matrix-vector shape
// with no reuse of D rows inside a warp), so it stays on the CUDA cores: at about
// 0.5 flop per gathered byte it is bound by the gathers, not by arithmetic.
#include "spd_internal.cuh"

namespace spd {

constexpr unsigned FULLM = 0xffffffffu;

template <typename VT, int EPL, int U>
__global__ void __launch_bounds__(256) sddmm_warp_kernel(
    int64_t n, const int32_t *__restrict__ pos, const int32_t *__restrict__ crd, const VT *__restrict__ vals,
    const VT *__restrict__ C, int64_t ldc, const VT *__restrict__ Dnk, int64_t ldd, int64_t K,
    typename Traits<VT>::out *__restrict__ out, const int32_t *__restrict__ prow, const int32_t *__restrict__ ppos,
    int64_t npieces, int64_t P) {
    using AT = typename Traits<VT>::acc;
    using OT = typename Traits<VT>::out;
    const int lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= (prow ? npieces : P)) return;
    const PieceBounds b = prow ? nnz_piece(c, prow, ppos) : row_piece(c, P, n, pos);
    const int64_t ktiles = (K + 32 * EPL - 1) / (32 * EPL);

    int32_t r = b.r0;
    int32_t rw = r;
    int32_t wend = ((int64_t)rw + lane < n) ? ld_stream(pos + rw + lane + 1) : INT_MAX;
    int32_t cur_end = r < n ? __shfl_sync(FULLM, wend, 0) : INT_MAX;

    for (int32_t pb = b.p0; pb < b.p1; pb += 32) {
        const int cnt = (b.p1 - pb) < 32 ? (b.p1 - pb) : 32;
        int32_t c_l = 0;
        AT v_l = 1;
        if (lane < cnt) {
            c_l = ld_stream(crd + pb + lane);
            if (vals) v_l = (AT)ld_stream(vals + pb + lane);
        }
        for (int j0 = 0; j0 < cnt; j0 += U) {
            int32_t rowu[U], colu[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int j = j0 + u;
                colu[u] = __shfl_sync(FULLM, c_l, j & 31);
                if (j < cnt) {
                    const int32_t pj = pb + j;
                    while (cur_end <= pj) {
                        ++r;
                        if (r - rw == 32) {
                            rw = r;
                            wend = ((int64_t)rw + lane < n) ? ld_stream(pos + rw + lane + 1) : INT_MAX;
                        }
                        cur_end = r < n ? __shfl_sync(FULLM, wend, r - rw) : INT_MAX;
                    }
                }
                rowu[u] = r;
            }
            AT part[U];
#pragma unroll
            for (int u = 0; u < U; ++u) part[u] = 0;
            for (int64_t kt = 0; kt < ktiles; ++kt) {
                const int64_t k = kt * (32 * EPL) + (int64_t)lane * EPL;
                if (k < K) {
                    AT dv[U][EPL], cv[U][EPL];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (j0 + u < cnt) {
                            ld_vec<EPL>(Dnk + (int64_t)colu[u] * ldd + k, dv[u]);
                            ld_vec<EPL>(C + (int64_t)rowu[u] * ldc + k, cv[u]);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (j0 + u < cnt) {
#pragma unroll
                            for (int e = 0; e < EPL; ++e) part[u] = fma(cv[u][e], dv[u][e], part[u]);
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) part[u] += __shfl_xor_sync(FULLM, part[u], off);
            }
            AT mine = 0;
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (lane == u) mine = part[u];
            const AT bv = __shfl_sync(FULLM, v_l, (j0 + lane) & 31);
            if (lane < U && j0 + lane < cnt) __stcs(out + pb + j0 + lane, (OT)(bv * mine));
        }
    }
}

template <typename VT, int EPL>
static spd_status launch_sddmm_epl(const spd_csr *B, const void *C, int64_t K, int64_t ldc, const void *Dnk,
                                   int64_t ldd, void *outv, int split, const Tuning &tn, void *ws, cudaStream_t st) {
    using OT = typename Traits<VT>::out;
    constexpr int U = EPL >= 8 ? 4 : 8;
    const int wpb = tn.block_threads / 32;
    const VT *v = static_cast<const VT *>(B->vals);
    const VT *cc = static_cast<const VT *>(C);
    const VT *dd = static_cast<const VT *>(Dnk);
    OT *o = static_cast<OT *>(outv);
    if (split == SPD_SPLIT_ROW) {
        int64_t P = tn.row_pieces > 0 ? tn.row_pieces : ceil_div(B->nrows + B->nnz, tn.unit_items);
        if (P < 1) P = 1;
        sddmm_warp_kernel<VT, EPL, U><<<(unsigned)ceil_div(P, wpb), tn.block_threads, 0, st>>>(
            B->nrows, B->pos, B->crd, v, cc, ldc, dd, ldd, K, o, nullptr, nullptr, 0, P);
        return check_launch("sddmm_warp_kernel(row)");
    }
    WsLayout Lw = layout_warp(B->nrows, B->nnz, split, tn.unit_items, 0, false);
    char *w = static_cast<char *>(ws);
    int32_t *prow = reinterpret_cast<int32_t *>(w + Lw.part_row);
    int32_t *ppos = reinterpret_cast<int32_t *>(w + Lw.part_pos);
    spd_status s = launch_merge_partition(B->nrows, B->nnz, B->pos, tn.unit_items, Lw.npieces, prow, ppos, st);
    if (s) return s;
    sddmm_warp_kernel<VT, EPL, U><<<(unsigned)ceil_div(Lw.npieces, wpb), tn.block_threads, 0, st>>>(
        B->nrows, B->pos, B->crd, v, cc, ldc, dd, ldd, K, o, prow, ppos, Lw.npieces, 0);
    return check_launch("sddmm_warp_kernel(nnz)");
}

template <typename VT>
static spd_status launch_sddmm(const spd_csr *B, const void *C, int64_t K, int64_t ldc, const void *Dnk, int64_t ldd,
                               void *outv, int split, const Tuning &tn, void *ws, cudaStream_t st) {
    int e1 = pick_epl(K, sizeof(VT), sizeof(VT), C, ldc, nullptr, ldc);
    int e2 = pick_epl(K, sizeof(VT), sizeof(VT), Dnk, ldd, nullptr, ldd);
    int epl = e1 < e2 ? e1 : e2;
    switch (epl) {
        case 1: return launch_sddmm_epl<VT, 1>(B, C, K, ldc, Dnk, ldd, outv, split, tn, ws, st);
        case 2: return launch_sddmm_epl<VT, 2>(B, C, K, ldc, Dnk, ldd, outv, split, tn, ws, st);
        case 4: return launch_sddmm_epl<VT, 4>(B, C, K, ldc, Dnk, ldd, outv, split, tn, ws, st);
        default:
            if constexpr (sizeof(VT) <= 4) return launch_sddmm_epl<VT, 8>(B, C, K, ldc, Dnk, ldd, outv, split, tn, ws, st);
            return launch_sddmm_epl<VT, 4>(B, C, K, ldc, Dnk, ldd, outv, split, tn, ws, st);
    }
}

}  // namespace spd

using namespace spd;

extern "C" spd_status spd_sddmm(const spd_csr *B, const void *C, int64_t K, int64_t ldc, const void *Dnk, int64_t ldd,
                                int dense_type, void *out_vals, int out_type, int split, const spd_tune *tune,
                                void *ws, size_t ws_bytes, void *stream) {
    spd_status s = check_csr(B, false);
    if (s) return s;
    if (K < 0) return fail(SPD_ERR_SHAPE, "K %lld < 0", (long long)K);
    if (dense_type != B->vtype) return fail(SPD_ERR_DTYPE, "dense type %d differs from the value type %d", dense_type, B->vtype);
    if (out_type != result_type(B->vtype)) return fail(SPD_ERR_DTYPE, "output type %d; expected %d", out_type, result_type(B->vtype));
    if ((s = check_dense("C", C, B->nrows, K, ldc, dense_type))) return s;
    if ((s = check_dense("Dnk", Dnk, B->ncols, K, ldd, dense_type))) return s;
    if (B->nnz > 0 && !out_vals) return fail(SPD_ERR_NULL, "out_vals is NULL");
    if (out_vals && !aligned(out_vals, dtype_size(out_type))) return fail(SPD_ERR_ALIGN, "out_vals misaligned");
    Tuning tn;
    if ((s = read_tune(tune, &tn))) return s;
    split = resolve_split(split);
    if (split != SPD_SPLIT_ROW && split != SPD_SPLIT_NNZ) return fail(SPD_ERR_ARG, "unknown split %d", split);
    WsLayout Lw = layout_warp(B->nrows, B->nnz, split, tn.unit_items, 0, false);
    if ((s = check_ws(Lw, ws, ws_bytes))) return s;
    if (B->nnz == 0) return SPD_OK;
    cudaStream_t st = as_stream(stream);
    switch (B->vtype) {
        case SPD_F64: return launch_sddmm<double>(B, C, K, ldc, Dnk, ldd, out_vals, split, tn, ws, st);
        case SPD_F32: return launch_sddmm<float>(B, C, K, ldc, Dnk, ldd, out_vals, split, tn, ws, st);
        case SPD_BF16: return launch_sddmm<__nv_bfloat16>(B, C, K, ldc, Dnk, ldd, out_vals, split, tn, ws, st);
        default: return fail(SPD_ERR_DTYPE, "unknown value type %d", B->vtype);
    }
}
