// spd_sddmm.cu -- SDDMM A(i,j) = B(i,j) * C(i,k) * D(k,j) (Section VI-A).
//
// The output keeps B's coordinate structure (Section V-B): one value per stored
// position p of B, so the work is a stream over B's positions with two gathered dense
// rows per position: row i of C and row j of D, with D passed transposed as
// Dnk[j,k] = D(k,j) so that both rows are contiguous.
//
// One warp consumes one piece of the flattened coordinate tree (rows and positions
// balanced together). Positions come in windows of 32: each lane loads one position's
// crd/vals and finds its row with a search over a 32-row window of pos held across the
// lanes; the window for the next rows is fetched while the current window is consumed.
// Lanes form groups of G (G * EPL covers K, EPL elements per 16-byte vector), so a warp
// step covers 32/G positions; U steps are in flight, and the U partial dot products of
// a lane are reduced across the group together by a halving butterfly.
//
// When K fits in one or two k tiles of the group (KT = 1 or 2) a lane keeps its slice of
// the current row of C in registers and loads C only in a warp step whose positions leave
// that row (on the benchmarked R-MAT a row holds about 30 positions), and row addresses are
// a 32-bit row index times a 32-bit byte pitch (one wide multiply-add). KT = 0 is the
// general form for any K or pitch: both rows loaded per position, k tiles in a loop.
//
// The contraction over k is one dot product per stored position (a matrix-vector
// shape, no reuse of D rows inside a warp), so it stays on the CUDA cores: at about
// 0.5 flop per gathered byte it is bound by the gathers, not by arithmetic.
#include "spd_internal.cuh"

namespace spd {

constexpr unsigned FULLM = 0xffffffffu;

template <typename VT, int EPL, int G, int KT>
__global__ void __launch_bounds__(256) sddmm_warp_kernel(
    int64_t n, const int32_t *__restrict__ pos, const int32_t *__restrict__ crd, const VT *__restrict__ vals,
    const VT *__restrict__ C, int64_t ldc, const VT *__restrict__ Dnk, int64_t ldd, int64_t K, uint32_t ldc_b,
    uint32_t ldd_b, typename Traits<VT>::out *__restrict__ out, const int32_t *__restrict__ prow,
    const int32_t *__restrict__ ppos, int64_t npieces, int64_t P) {
    using AT = typename Traits<VT>::acc;
    using OT = typename Traits<VT>::out;
    constexpr int NPG = 32 / G;                             // positions per warp step
    constexpr int U = 4;                                    // warp steps in flight
    __shared__ int32_t s_crd_all[8][32], s_row_all[8][32];  // one window per warp (<= 8 warps)
    __shared__ AT s_val_all[8][32];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid;
    if (c >= (prow ? npieces : P)) return;
    const PieceBounds b = prow ? nnz_piece(c, prow, ppos) : row_piece(c, P, n, pos);
    int32_t *s_crd = s_crd_all[wid];
    int32_t *s_row = s_row_all[wid];
    AT *s_val = s_val_all[wid];
    const int gi = lane / G;  // group of this lane
    const int gl = lane % G;  // lane inside the group
    bool writer;
    const int my_u = reduced_index<G, U>(gl, writer);
    const int64_t ktiles = (K + G * EPL - 1) / (G * EPL);
    // KT > 0: byte offsets of this lane's slice, which k tiles it covers, and the cached
    // slice of row `crow` of C
    constexpr int NKT = KT > 0 ? KT : 1;
    constexpr size_t TB = (size_t)G * EPL * sizeof(VT);
    const char *Cl = reinterpret_cast<const char *>(C) + (size_t)gl * EPL * sizeof(VT);
    const char *Dl = reinterpret_cast<const char *>(Dnk) + (size_t)gl * EPL * sizeof(VT);
    bool kon[NKT];
#pragma unroll
    for (int kt = 0; kt < NKT; ++kt) kon[kt] = (int64_t)kt * G * EPL + (int64_t)gl * EPL < K;
    XVec<VT, EPL> cc[NKT];
    int32_t crow = -1;

    PosRows pr;
    pr.load(b.r0, n, pos, lane);
    for (int32_t pb = b.p0; pb < b.p1; pb += 32) {
        const int cnt = (b.p1 - pb) < 32 ? (b.p1 - pb) : 32;
        const bool valid = lane < cnt;
        const int32_t my_crd = valid ? ld_stream(crd + pb + lane) : 0;
        const AT my_val = (valid && vals) ? (AT)ld_stream(vals + pb + lane) : (AT)1;
        const int32_t my_row = pr.find(pb + lane, valid, n, pos, lane);
        __syncwarp();
        s_crd[lane] = my_crd;
        s_row[lane] = my_row;
        s_val[lane] = my_val;
        __syncwarp();
        // next window starts at the last row of this one (fetched while this one is used)
        const int32_t next_rw = __shfl_sync(FULLM, my_row, cnt - 1);
        if (next_rw != pr.rw) pr.load(next_rw, n, pos, lane);
#pragma unroll 1
        for (int j0 = 0; j0 < cnt; j0 += NPG * U) {
            AT part[U];
#pragma unroll
            for (int u = 0; u < U; ++u) part[u] = 0;
            if constexpr (KT > 0) {
                // rows and columns of the step's positions; a position past the window
                // repeats the last one (its product is zero and never written)
                int32_t rr[U];
                uint32_t dc[U];
                bool ok[U];
                bool same = true;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int j = j0 + u * NPG + gi;
                    ok[u] = j < cnt;
                    const int jc = ok[u] ? j : cnt - 1;
                    rr[u] = s_row[jc];
                    dc[u] = (uint32_t)s_crd[jc];
                    same = same && rr[u] == crow;
                }
#pragma unroll
                for (int kt = 0; kt < KT; ++kt) {
                    if (!kon[kt]) continue;
                    XVec<VT, EPL> dv[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        if (ok[u]) dv[u].load(reinterpret_cast<const VT *>(Dl + kt * TB + (uint64_t)dc[u] * ldd_b));
                        else dv[u].clear();
                    }
                    if (same) {
#pragma unroll
                        for (int u = 0; u < U; ++u) {
#pragma unroll
                            for (int e = 0; e < EPL; ++e)
                                part[u] = fma((AT)cc[kt].at(e), (AT)dv[u].at(e), part[u]);
                        }
                    } else {
                        XVec<VT, EPL> cv[U];
#pragma unroll
                        for (int u = 0; u < U; ++u)
                            cv[u].load(reinterpret_cast<const VT *>(Cl + kt * TB + (uint64_t)(uint32_t)rr[u] * ldc_b));
#pragma unroll
                        for (int u = 0; u < U; ++u) {
#pragma unroll
                            for (int e = 0; e < EPL; ++e)
                                part[u] = fma((AT)cv[u].at(e), (AT)dv[u].at(e), part[u]);
                        }
                        cc[kt] = cv[U - 1];
                    }
                }
                crow = rr[U - 1];
            } else {
#pragma unroll 1
            for (int64_t kt = 0; kt < ktiles; ++kt) {
                const int64_t k = kt * (G * EPL) + (int64_t)gl * EPL;
                if (k < K) {
                    XVec<VT, EPL> cv[U], dv[U];  // bfloat16 stays packed until the multiply
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int j = j0 + u * NPG + gi;
                        if (j < cnt) {
                            cv[u].load(C + (int64_t)s_row[j] * ldc + k);
                            dv[u].load(Dnk + (int64_t)s_crd[j] * ldd + k);
                        } else {
                            cv[u].clear();
                            dv[u].clear();
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
#pragma unroll
                        for (int e = 0; e < EPL; ++e) part[u] = fma((AT)cv[u].at(e), (AT)dv[u].at(e), part[u]);
                    }
                }
            }
            }
            const AT tot = group_reduce<G, U>(part, gl);
            const int j = j0 + my_u * NPG + gi;
            if (writer && j < cnt) __stcs(out + pb + j, (OT)(s_val[j] * tot));
        }
    }
}

template <typename VT, int EPL, int G, int KT>
static spd_status launch_sddmm_g(const spd_csr *B, const void *C, int64_t K, int64_t ldc, const void *Dnk,
                                 int64_t ldd, void *outv, int split, const Tuning &tn, void *ws, cudaStream_t st) {
    using OT = typename Traits<VT>::out;
    const uint32_t ldc_b = (uint32_t)(ldc * (int64_t)sizeof(VT)), ldd_b = (uint32_t)(ldd * (int64_t)sizeof(VT));
    const int threads = tn.block_threads > 256 ? 256 : tn.block_threads;  // shared windows for <= 8 warps
    const int wpb = threads / 32;
    const VT *v = static_cast<const VT *>(B->vals);
    const VT *cc = static_cast<const VT *>(C);
    const VT *dd = static_cast<const VT *>(Dnk);
    OT *o = static_cast<OT *>(outv);
    if (split == SPD_SPLIT_ROW) {
        int64_t P = tn.row_pieces > 0 ? tn.row_pieces : ceil_div(B->nrows + B->nnz, tn.unit_items);
        if (P < 1) P = 1;
        sddmm_warp_kernel<VT, EPL, G, KT><<<(unsigned)ceil_div(P, wpb), threads, 0, st>>>(
            B->nrows, B->pos, B->crd, v, cc, ldc, dd, ldd, K, ldc_b, ldd_b, o, nullptr, nullptr, 0, P);
        return check_launch("sddmm_warp_kernel(row)");
    }
    WsLayout Lw = layout_warp(B->nrows, B->nnz, split, tn.unit_items, 0, false);
    char *w = static_cast<char *>(ws);
    int32_t *prow = reinterpret_cast<int32_t *>(w + Lw.part_row);
    int32_t *ppos = reinterpret_cast<int32_t *>(w + Lw.part_pos);
    spd_status s = launch_merge_partition(B->nrows, B->nnz, B->pos, tn.unit_items, Lw.npieces, prow, ppos, st);
    if (s) return s;
    sddmm_warp_kernel<VT, EPL, G, KT><<<(unsigned)ceil_div(Lw.npieces, wpb), threads, 0, st>>>(
        B->nrows, B->pos, B->crd, v, cc, ldc, dd, ldd, K, ldc_b, ldd_b, o, prow, ppos, Lw.npieces, 0);
    return check_launch("sddmm_warp_kernel(nnz)");
}

// The cached-row form (KT = 1 or 2 k tiles) needs 16-byte vectors and row pitches below
// 4 GiB; anything else takes the general form (KT = 0).
template <typename VT, int EPL, int G>
static spd_status launch_sddmm_kt(const spd_csr *B, const void *C, int64_t K, int64_t ldc, const void *Dnk,
                                  int64_t ldd, void *outv, int split, const Tuning &tn, void *ws, cudaStream_t st) {
    if constexpr (EPL * sizeof(VT) == 16) {
        const int64_t pitch_max = (int64_t)UINT32_MAX / (int64_t)sizeof(VT);
        if (ldc <= pitch_max && ldd <= pitch_max) {
            const int64_t kt = ceil_div(K > 0 ? K : 1, (int64_t)G * EPL);
            if (kt == 1) return launch_sddmm_g<VT, EPL, G, 1>(B, C, K, ldc, Dnk, ldd, outv, split, tn, ws, st);
            if constexpr (G == 32) {
                if (kt == 2) return launch_sddmm_g<VT, EPL, G, 2>(B, C, K, ldc, Dnk, ldd, outv, split, tn, ws, st);
            }
        }
    }
    return launch_sddmm_g<VT, EPL, G, 0>(B, C, K, ldc, Dnk, ldd, outv, split, tn, ws, st);
}

// Group width: the power of two in [4, 32] closest to covering K with EPL-element vectors.
template <typename VT, int EPL>
static spd_status launch_sddmm_epl(const spd_csr *B, const void *C, int64_t K, int64_t ldc, const void *Dnk,
                                   int64_t ldd, void *outv, int split, const Tuning &tn, void *ws, cudaStream_t st) {
    const int64_t lanes = ceil_div(K > 0 ? K : 1, EPL);
    if (lanes <= 4) return launch_sddmm_kt<VT, EPL, 4>(B, C, K, ldc, Dnk, ldd, outv, split, tn, ws, st);
    if (lanes <= 8) return launch_sddmm_kt<VT, EPL, 8>(B, C, K, ldc, Dnk, ldd, outv, split, tn, ws, st);
    if (lanes <= 16) return launch_sddmm_kt<VT, EPL, 16>(B, C, K, ldc, Dnk, ldd, outv, split, tn, ws, st);
    return launch_sddmm_kt<VT, EPL, 32>(B, C, K, ldc, Dnk, ldd, outv, split, tn, ws, st);
}

template <typename VT>
static spd_status launch_sddmm(const spd_csr *B, const void *C, int64_t K, int64_t ldc, const void *Dnk, int64_t ldd,
                               void *outv, int split, const Tuning &tn, void *ws, cudaStream_t st) {
    constexpr int V = 16 / sizeof(VT);  // elements of one 16-byte vector
    const bool vec = K % V == 0 && ldc % V == 0 && ldd % V == 0 && aligned(C, 16) && aligned(Dnk, 16);
    if (vec) return launch_sddmm_epl<VT, V>(B, C, K, ldc, Dnk, ldd, outv, split, tn, ws, st);
    return launch_sddmm_epl<VT, 1>(B, C, K, ldc, Dnk, ldd, outv, split, tn, ws, st);
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
    cudaStream_t st = as_stream(stream);
    if ((s = checked_csr(B, "B", st))) return s;
    if (B->nnz == 0) return SPD_OK;
    switch (B->vtype) {
        case SPD_F64: s = launch_sddmm<double>(B, C, K, ldc, Dnk, ldd, out_vals, split, tn, ws, st); break;
        case SPD_F32: s = launch_sddmm<float>(B, C, K, ldc, Dnk, ldd, out_vals, split, tn, ws, st); break;
        case SPD_BF16: s = launch_sddmm<__nv_bfloat16>(B, C, K, ldc, Dnk, ldd, out_vals, split, tn, ws, st); break;
        default: return fail(SPD_ERR_DTYPE, "unknown value type %d", B->vtype);
    }
    return checked_finish(s, "spd_sddmm", st);
}
