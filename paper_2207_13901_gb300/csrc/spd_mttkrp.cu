// spd_mttkrp.cu -- SpMTTKRP A(i,l) = B(i,j,k) * C(j,l) * D(k,l) (Section VI-A) on a
// CSF tensor B = {Dense, Compressed, Compressed}.
//
// Per fiber (i,j): t(l) = sum_k B(i,j,k) D(k,l); then A(i,l) += C(j,l) t(l). One warp
// consumes one piece; lanes span R in vectors of EPL elements.
//   Nnz split (the GPU schedule of Section VI-A): coordinate fusion of levels 2 and 3 and
//     a non-zero partition of the fused items (each fiber's entries followed by one
//     "fiber end" item), so pieces balance entries and fibers. The partial fiber at a
//     piece end is folded into the piece's slice partial (by linearity in t), and the
//     slice partial at a piece end goes to a binary64 carry added by the fix-up kernel.
//     Piece c writes the slices [s_c, s_{c+1}) whose last fiber ends inside it, where
//     s_c = #{i : pos1[i+1] <= first fiber of piece c} (s_0 = 0, s_last = I).
//   Row split: universe partition of the slices, [floor(c I/P), floor((c+1) I/P)).
// The contraction per entry is a scaled row of D (no dense reuse within a warp), so the
// work stays on the CUDA cores.
#include "spd_internal.cuh"

namespace spd {

constexpr unsigned FULLK = 0xffffffffu;

template <typename T, int N>
__device__ __forceinline__ void zero_k(T (&a)[N]) {
#pragma unroll
    for (int e = 0; e < N; ++e) a[e] = (T)0;
}

// s_c for every interior piece boundary: the number of slices whose end (pos1[i+1])
// is at or before the piece's first fiber. Binary search over pos1[1..I].
__global__ void slice_partition_kernel(int64_t I, const int32_t *__restrict__ pos1, const int32_t *__restrict__ pfib,
                                       int64_t npieces, int32_t *__restrict__ pslice) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c > npieces) return;
    if (c == 0) {
        pslice[0] = 0;
        return;
    }
    if (c == npieces) {
        pslice[npieces] = (int32_t)I;
        return;
    }
    const int32_t f0 = pfib[c];
    int64_t lo = 0, hi = I;  // count of i in [0, I) with pos1[i+1] <= f0
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (__ldg(pos1 + mid + 1) <= f0) lo = mid + 1;
        else hi = mid;
    }
    pslice[c] = (int32_t)lo;
}

template <typename VT, int EPL, int U>
__global__ void __launch_bounds__(256) spmttkrp_warp_kernel(
    int64_t I, int64_t F, const int32_t *__restrict__ pos1, const int32_t *__restrict__ crd1,
    const int32_t *__restrict__ pos2, const int32_t *__restrict__ crd2, const VT *__restrict__ vals,
    const VT *__restrict__ C, int64_t ldc, const VT *__restrict__ D, int64_t ldd, int64_t R,
    typename Traits<VT>::out *__restrict__ A, int64_t lda, const int32_t *__restrict__ pfib,
    const int32_t *__restrict__ ppos, const int32_t *__restrict__ pslice, int64_t npieces, int64_t P,
    int32_t *__restrict__ carry_row, double *__restrict__ carry_val) {
    using AT = typename Traits<VT>::acc;
    using OT = typename Traits<VT>::out;
    const int lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= (pfib ? npieces : P)) return;
    const int64_t col = (int64_t)blockIdx.y * (32 * EPL) + (int64_t)lane * EPL;
    const bool active = col < R;

    int32_t f0, p0, f1, p1, s0, s1;
    if (pfib) {
        f0 = __ldg(pfib + c);
        p0 = __ldg(ppos + c);
        f1 = __ldg(pfib + c + 1);
        p1 = __ldg(ppos + c + 1);
        s0 = __ldg(pslice + c);
        s1 = __ldg(pslice + c + 1);
    } else {
        s0 = (int32_t)((c * I) / P);
        s1 = (int32_t)(((c + 1) * I) / P);
        f0 = __ldg(pos1 + s0);
        f1 = __ldg(pos1 + s1);
        p0 = __ldg(pos2 + f0);
        p1 = __ldg(pos2 + f1);
    }

    AT t[EPL], a[EPL];
    zero_k(t);
    zero_k(a);
    bool dirty = false;  // a holds contributions not yet written

    // slice-end window: lane q holds pos1[sw + q + 1]
    int32_t i = s0, sw = s0;
    int32_t send = ((int64_t)sw + lane < I) ? __ldg(pos1 + sw + lane + 1) : INT_MAX;
    // fiber windows: lane q holds the end of fiber fw + q and its j coordinate
    int32_t f = f0, fw = f0;
    int32_t fend = ((int64_t)fw + lane < F) ? ld_stream(pos2 + fw + lane + 1) : INT_MAX;
    int32_t fj = ((int64_t)fw + lane < F) ? ld_stream(crd1 + fw + lane) : 0;
    int32_t cur_fend = f < f1 ? __shfl_sync(FULLK, fend, 0) : INT_MAX;

    auto emit_ready = [&]() {  // write every owned slice whose last fiber is done
        while (i < s1) {
            const int32_t e = __shfl_sync(FULLK, send, i - sw);
            if (e > f) break;
            if (active) {
                OT o[EPL];
#pragma unroll
                for (int q = 0; q < EPL; ++q) o[q] = (OT)a[q];
                st_vec(A + (int64_t)i * lda + col, o);
            }
            zero_k(a);
            dirty = false;
            ++i;
            if (i - sw == 32) {
                sw = i;
                send = ((int64_t)sw + lane < I) ? __ldg(pos1 + sw + lane + 1) : INT_MAX;
            }
        }
    };
    auto finish_fiber = [&]() {  // a += C(j,:) * t for the current fiber f
        const int32_t j = __shfl_sync(FULLK, fj, f - fw);
        if (active) {
            AT cv[EPL];
            ld_vec<EPL>(C + (int64_t)j * ldc + col, cv);
#pragma unroll
            for (int q = 0; q < EPL; ++q) a[q] = fma(cv[q], t[q], a[q]);
        }
        zero_k(t);
        dirty = true;
    };
    auto next_fiber = [&]() {
        ++f;
        if (f - fw == 32) {
            fw = f;
            fend = ((int64_t)fw + lane < F) ? ld_stream(pos2 + fw + lane + 1) : INT_MAX;
            fj = ((int64_t)fw + lane < F) ? ld_stream(crd1 + fw + lane) : 0;
        }
        cur_fend = f < f1 ? __shfl_sync(FULLK, fend, f - fw) : INT_MAX;
    };

    emit_ready();
    for (int32_t pb = p0; pb < p1; pb += 32) {
        const int cnt = (p1 - pb) < 32 ? (p1 - pb) : 32;
        int32_t k_l = 0;
        AT v_l = 0;
        if (lane < cnt) {
            k_l = ld_stream(crd2 + pb + lane);
            v_l = (AT)ld_stream(vals + pb + lane);
        }
        for (int j0 = 0; j0 < cnt; j0 += U) {
            AT dv[U][EPL];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int32_t kk = __shfl_sync(FULLK, k_l, (j0 + u) & 31);
                if (active && j0 + u < cnt) ld_vec<EPL>(D + (int64_t)kk * ldd + col, dv[u]);
                else zero_k(dv[u]);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int j = j0 + u;
                const AT vj = __shfl_sync(FULLK, v_l, j & 31);
                if (j < cnt) {
                    const int32_t pj = pb + j;
                    while (cur_fend <= pj) {
                        finish_fiber();
                        next_fiber();
                        emit_ready();
                    }
#pragma unroll
                    for (int q = 0; q < EPL; ++q) t[q] = fma(vj, dv[u][q], t[q]);
                    dirty = true;
                }
            }
        }
    }
    while (f < f1) {  // fibers ending at or after the last entry of the piece
        finish_fiber();
        next_fiber();
        emit_ready();
    }
    if (pfib) {
        // the piece may end inside fiber f1: fold its partial into the slice partial
        const int32_t fstart = f1 < F ? __ldg(pos2 + f1) : p1;
        if (p1 > (fstart > p0 ? fstart : p0)) {
            const int32_t j = __ldg(crd1 + f1);
            if (active) {
                AT cv[EPL];
                ld_vec<EPL>(C + (int64_t)j * ldc + col, cv);
#pragma unroll
                for (int q = 0; q < EPL; ++q) a[q] = fma(cv[q], t[q], a[q]);
            }
            dirty = true;
        }
        const bool has = dirty && i < I;
        if (lane == 0 && blockIdx.y == 0) carry_row[c] = has ? i : -1;
        if (has && active) {
#pragma unroll
            for (int q = 0; q < EPL; ++q) carry_val[c * R + col + q] = (double)a[q];
        }
    }
}

template <typename VT, int EPL>
static spd_status launch_mttkrp_epl(const spd_csf3 *B, const void *C, int64_t ldc, const void *D, int64_t ldd,
                                    int64_t R, void *A, int64_t lda, int split, const Tuning &tn, void *ws,
                                    cudaStream_t st) {
    using OT = typename Traits<VT>::out;
    constexpr int U = 8;
    const int wpb = tn.block_threads / 32;
    const int64_t ctiles = ceil_div(R, 32 * EPL);
    const VT *v = static_cast<const VT *>(B->vals);
    const VT *cc = static_cast<const VT *>(C);
    const VT *dd = static_cast<const VT *>(D);
    OT *aa = static_cast<OT *>(A);
    if (B->nfib == 0) return launch_zero_rows<OT>(B->dim0, R, aa, lda, st);  // every slice is empty
    if (split == SPD_SPLIT_ROW) {
        int64_t P = tn.row_pieces > 0 ? tn.row_pieces : ceil_div(B->nfib + B->nnz, tn.unit_items);
        if (P > B->dim0) P = B->dim0;
        if (P < 1) P = 1;
        dim3 grid((unsigned)ceil_div(P, wpb), (unsigned)ctiles);
        spmttkrp_warp_kernel<VT, EPL, U><<<grid, tn.block_threads, 0, st>>>(
            B->dim0, B->nfib, B->pos1, B->crd1, B->pos2, B->crd2, v, cc, ldc, dd, ldd, R, aa, lda, nullptr, nullptr,
            nullptr, 0, P, nullptr, nullptr);
        return check_launch("spmttkrp_warp_kernel(row)");
    }
    WsLayout Lw = layout_mttkrp(B->nfib, B->nnz, split, tn.unit_items, R);
    char *w = static_cast<char *>(ws);
    int32_t *pfib = reinterpret_cast<int32_t *>(w + Lw.part_row);
    int32_t *ppos = reinterpret_cast<int32_t *>(w + Lw.part_pos);
    int32_t *psl = reinterpret_cast<int32_t *>(w + Lw.part_aux);
    int32_t *crow = reinterpret_cast<int32_t *>(w + Lw.carry_row);
    double *cval = reinterpret_cast<double *>(w + Lw.carry_val);
    spd_status s = launch_merge_partition(B->nfib, B->nnz, B->pos2, tn.unit_items, Lw.npieces, pfib, ppos, st);
    if (s) return s;
    slice_partition_kernel<<<(unsigned)ceil_div(Lw.npieces + 1, 256), 256, 0, st>>>(B->dim0, B->pos1, pfib,
                                                                                     Lw.npieces, psl);
    if ((s = check_launch("slice_partition_kernel"))) return s;
    dim3 grid((unsigned)ceil_div(Lw.npieces, wpb), (unsigned)ctiles);
    spmttkrp_warp_kernel<VT, EPL, U><<<grid, tn.block_threads, 0, st>>>(
        B->dim0, B->nfib, B->pos1, B->crd1, B->pos2, B->crd2, v, cc, ldc, dd, ldd, R, aa, lda, pfib, ppos, psl,
        Lw.npieces, 0, crow, cval);
    if ((s = check_launch("spmttkrp_warp_kernel(nnz)"))) return s;
    return launch_carry_fixup<OT>(Lw.npieces, R, crow, cval, aa, lda, st);
}

template <typename VT>
static spd_status launch_mttkrp(const spd_csf3 *B, const void *C, int64_t ldc, const void *D, int64_t ldd, int64_t R,
                                void *A, int64_t lda, int split, const Tuning &tn, void *ws, cudaStream_t st) {
    using OT = typename Traits<VT>::out;
    int e1 = pick_epl(R, sizeof(VT), sizeof(OT), C, ldc, A, lda);
    int e2 = pick_epl(R, sizeof(VT), sizeof(OT), D, ldd, A, lda);
    int epl = e1 < e2 ? e1 : e2;
    switch (epl) {
        case 1: return launch_mttkrp_epl<VT, 1>(B, C, ldc, D, ldd, R, A, lda, split, tn, ws, st);
        case 2: return launch_mttkrp_epl<VT, 2>(B, C, ldc, D, ldd, R, A, lda, split, tn, ws, st);
        default: return launch_mttkrp_epl<VT, 4>(B, C, ldc, D, ldd, R, A, lda, split, tn, ws, st);
    }
}

}  // namespace spd

using namespace spd;

extern "C" spd_status spd_spmttkrp(const spd_csf3 *B, const void *C, int64_t ldc, const void *D, int64_t ldd,
                                   int64_t R, int factor_type, void *A, int64_t lda, int a_type, int split,
                                   const spd_tune *tune, void *ws, size_t ws_bytes, void *stream) {
    spd_status s = check_csf3(B);
    if (s) return s;
    if (R < 0) return fail(SPD_ERR_SHAPE, "R %lld < 0", (long long)R);
    if (factor_type != B->vtype) return fail(SPD_ERR_DTYPE, "factor type %d differs from the value type %d", factor_type, B->vtype);
    if (a_type != result_type(B->vtype)) return fail(SPD_ERR_DTYPE, "A type %d; expected %d", a_type, result_type(B->vtype));
    if ((s = check_dense("C", C, B->dim1, R, ldc, factor_type))) return s;
    if ((s = check_dense("D", D, B->dim2, R, ldd, factor_type))) return s;
    if ((s = check_dense("A", A, B->dim0, R, lda, a_type))) return s;
    Tuning tn;
    if ((s = read_tune(tune, &tn))) return s;
    split = resolve_split(split);
    if (split != SPD_SPLIT_ROW && split != SPD_SPLIT_NNZ) return fail(SPD_ERR_ARG, "unknown split %d", split);
    WsLayout Lw = layout_mttkrp(B->nfib, B->nnz, split, tn.unit_items, R);
    if ((s = check_ws(Lw, ws, ws_bytes))) return s;
    if (B->dim0 == 0 || R == 0) return SPD_OK;
    cudaStream_t st = as_stream(stream);
    switch (B->vtype) {
        case SPD_F64: return launch_mttkrp<double>(B, C, ldc, D, ldd, R, A, lda, split, tn, ws, st);
        case SPD_F32: return launch_mttkrp<float>(B, C, ldc, D, ldd, R, A, lda, split, tn, ws, st);
        case SPD_BF16: return launch_mttkrp<__nv_bfloat16>(B, C, ldc, D, ldd, R, A, lda, split, tn, ws, st);
        default: return fail(SPD_ERR_DTYPE, "unknown value type %d", B->vtype);
    }
}
