// spd_spmm.cu -- SpMM Y(i,l) = A(i,j) * X(j,l) (Section VI-A) and its gradient with
// respect to X, SpMM^T dX(j,l) = A(i,j) * dY(i,l), without forming A's transpose.
//
// One warp consumes one piece of the flattened coordinate tree of A. The 32 lanes
// span a tile of 32*EPL dense columns, so every nonzero costs one coalesced row of X
// (a 16- or 32-byte vector per lane). crd/vals are streamed 32 at a time and broadcast
// with shuffles; U rows of X are in flight before they are consumed. Row ends come
// from a 32-entry window of pos held one entry per lane. A row is written once, when
// its end item is reached; rows longer than 4096 nonzeros accumulate with Kahan's
// compensated summation in the binary32 modes. In the nnz split the partial row
// at a piece end is stored as binary64 and added by a fix-up kernel.
#include "spd_spmm_piece.cuh"

namespace spd {

constexpr unsigned FULL = kFullMask;

template <typename VT, int EPL, int G, int U, bool FULLTILE, bool ACC>
__global__ void __launch_bounds__(kWarpBlockMax, kSpmmMinBlocks) spmm_warp_kernel(
    int64_t n, const int32_t *__restrict__ pos, const int32_t *__restrict__ crd, const VT *__restrict__ vals,
    const VT *__restrict__ X, uint32_t ldx_bytes, typename Traits<VT>::out *__restrict__ Y, int64_t ldy, int64_t L,
    const int32_t *__restrict__ prow, const int32_t *__restrict__ ppos, int64_t npieces, int64_t P,
    int32_t *__restrict__ carry_row, double *__restrict__ carry_val) {
    using AT = typename Traits<VT>::acc;
    extern __shared__ __align__(16) unsigned char spmm_smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * wpb + wid;
    if (c >= (prow ? npieces : P)) return;  // whole warp
    const PieceBounds b = prow ? nnz_piece(c, prow, ppos) : row_piece(c, P, n, pos);
    int32_t *s_crd = reinterpret_cast<int32_t *>(spmm_smem) + wid * 64;  // [2][32]
    AT *s_val = reinterpret_cast<AT *>(spmm_smem + wpb * 64 * sizeof(int32_t)) + wid * 64;
    int32_t *crow = carry_row ? carry_row + c : nullptr;
    double *cval = carry_row ? carry_val + c * L : nullptr;
    if constexpr (G == 32) {
        const int64_t col = (int64_t)blockIdx.y * (32 * EPL) + (int64_t)lane * EPL;
        spmm_piece<VT, EPL, U, FULLTILE, ACC>(n, pos, crd, vals, X, ldx_bytes, Y, ldy, L, b, col, lane, s_crd, s_val, crow,
                                         blockIdx.y == 0, cval);
    } else {
        const int64_t col = (int64_t)blockIdx.y * (G * EPL) + (int64_t)(lane % G) * EPL;
        AT *s_cmp = reinterpret_cast<AT *>(spmm_smem + wpb * 64 * sizeof(int32_t)) + wpb * 64 + wid * 32 * EPL;
        spmm_piece_grouped<VT, EPL, G, U, FULLTILE, ACC>(n, pos, crd, vals, X, ldx_bytes, Y, ldy, L, b, col, lane, s_crd,
                                                    s_val, s_cmp, crow, blockIdx.y == 0, cval);
    }
}

// dX(j,l) = A(i,j) * dY(i,l): walk A's rows in the piece, keep the current row of dY in
// registers and scatter vals[p] * dY(i,:) into row crd[p] of dX with atomic adds.
template <typename VT, int EPL>
__global__ void __launch_bounds__(kWarpBlockMax) spmm_t_warp_kernel(
    int64_t n, const int32_t *__restrict__ pos, const int32_t *__restrict__ crd, const VT *__restrict__ vals,
    const VT *__restrict__ dY, int64_t ldy, typename Traits<VT>::out *__restrict__ dX, int64_t ldx, int64_t L,
    const int32_t *__restrict__ prow, const int32_t *__restrict__ ppos, int64_t npieces, int64_t P) {
    using AT = typename Traits<VT>::acc;
    const int lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= (prow ? npieces : P)) return;
    const int64_t col = (int64_t)blockIdx.y * (32 * EPL) + (int64_t)lane * EPL;
    const bool active = col < L;
    const PieceBounds b = prow ? nnz_piece(c, prow, ppos) : row_piece(c, P, n, pos);

    int32_t r = b.r0;
    RowWindow win;
    win.load(r, n, pos, lane);
    int32_t cur_end = r < n ? win.end_of(r) : INT_MAX;
    int32_t loaded = -1;  // row of dY held in dy
    AT dy[EPL];
    zero(dy);
    for (int32_t pb = b.p0; pb < b.p1; pb += 32) {
        const int cnt = (b.p1 - pb) < 32 ? (b.p1 - pb) : 32;
        int32_t c_l = 0;
        AT v_l = 0;
        if (lane < cnt) {
            c_l = ld_stream(crd + pb + lane);
            v_l = (AT)ld_stream(vals + pb + lane);
        }
        for (int j = 0; j < cnt; ++j) {
            const int32_t pj = pb + j;
            while (cur_end <= pj) {
                ++r;
                if (r - win.rw == 32) win.load(r, n, pos, lane);
                cur_end = r < n ? win.end_of(r) : INT_MAX;
            }
            if (loaded != r) {
                if (active) ld_vec<EPL>(dY + (int64_t)r * ldy + col, dy);
                loaded = r;
            }
            const int32_t cj = __shfl_sync(FULL, c_l, j);
            const AT vj = __shfl_sync(FULL, v_l, j);
            if (active) {
                auto *dst = dX + (int64_t)cj * ldx + col;
                if constexpr (sizeof(AT) == 4 && EPL % 4 == 0) {
#pragma unroll
                    for (int q = 0; q < EPL / 4; ++q)
                        atomicAdd(reinterpret_cast<float4 *>(dst) + q,
                                  make_float4(vj * dy[4 * q], vj * dy[4 * q + 1], vj * dy[4 * q + 2], vj * dy[4 * q + 3]));
                } else if constexpr (sizeof(AT) == 4 && EPL == 2) {
                    atomicAdd(reinterpret_cast<float2 *>(dst), make_float2(vj * dy[0], vj * dy[1]));
                } else {
#pragma unroll
                    for (int e = 0; e < EPL; ++e) atomicAdd(dst + e, vj * dy[e]);
                }
            }
        }
    }
}

// ------------------------------------------------------------------ host side

static int64_t default_row_pieces(int64_t n, int64_t nnz, int64_t unit) {
    int64_t P = ceil_div(n + nnz, unit);
    return P < 1 ? 1 : P;
}

template <typename VT, int EPL, int G, int U, bool FULLTILE, bool ACC>
static spd_status launch_spmm_shape(const spd_csr *A, const void *X, int64_t L, int64_t ldx, void *Y, int64_t ldy,
                                    int split, const Tuning &tn, void *ws, cudaStream_t st) {
    using OT = typename Traits<VT>::out;
    const int wpb = tn.block_threads / 32;
    const int64_t ctiles = ceil_div(L, G * EPL);
    const size_t smem = (size_t)wpb * spmm_warp_smem<VT>(EPL, G);
    const VT *v = static_cast<const VT *>(A->vals);
    const VT *x = static_cast<const VT *>(X);
    OT *y = static_cast<OT *>(Y);
    if (split == SPD_SPLIT_ROW) {
        const int64_t P = tn.row_pieces > 0 ? tn.row_pieces : default_row_pieces(A->nrows, A->nnz, tn.unit_items);
        dim3 grid((unsigned)ceil_div(P, wpb), (unsigned)ctiles);
        spmm_warp_kernel<VT, EPL, G, U, FULLTILE, ACC><<<grid, tn.block_threads, smem, st>>>(
            A->nrows, A->pos, A->crd, v, x, (uint32_t)(ldx * sizeof(VT)), y, ldy, L, nullptr, nullptr, 0, P, nullptr,
            nullptr);
        return check_launch("spmm_warp_kernel(row)");
    }
    WsLayout Lw = layout_warp(A->nrows, A->nnz, split, tn.unit_items, L, true);
    char *w = static_cast<char *>(ws);
    int32_t *prow = reinterpret_cast<int32_t *>(w + Lw.part_row);
    int32_t *ppos = reinterpret_cast<int32_t *>(w + Lw.part_pos);
    int32_t *crow = reinterpret_cast<int32_t *>(w + Lw.carry_row);
    double *cval = reinterpret_cast<double *>(w + Lw.carry_val);
    spd_status s = launch_merge_partition(A->nrows, A->nnz, A->pos, tn.unit_items, Lw.npieces, prow, ppos, st);
    if (s) return s;
    dim3 grid((unsigned)ceil_div(Lw.npieces, wpb), (unsigned)ctiles);
    spmm_warp_kernel<VT, EPL, G, U, FULLTILE, ACC><<<grid, tn.block_threads, smem, st>>>(
        A->nrows, A->pos, A->crd, v, x, (uint32_t)(ldx * sizeof(VT)), y, ldy, L, prow, ppos, Lw.npieces, 0, crow,
        cval);
    if ((s = check_launch("spmm_warp_kernel(nnz)"))) return s;
    return launch_carry_fixup<OT>(Lw.npieces, L, crow, cval, reinterpret_cast<int32_t *>(w + Lw.chunk_row),
                                  reinterpret_cast<double *>(w + Lw.chunk_val), y, ldy, st);
}

// Rows in flight per group: the tuning's 4 or 8 for one entry per warp step in the
// binary32 modes; 4 for binary64 (8 would spill) and for lane groups.
template <typename VT, int EPL, int G, bool ACC>
static spd_status launch_spmm_u(const spd_csr *A, const void *X, int64_t L, int64_t ldx, void *Y, int64_t ldy,
                                int split, const Tuning &tn, void *ws, cudaStream_t st) {
    const bool full = L % (G * EPL) == 0;
    if constexpr (sizeof(VT) == 8 || G < 32) {
        return full ? launch_spmm_shape<VT, EPL, G, 4, true, ACC>(A, X, L, ldx, Y, ldy, split, tn, ws, st)
                    : launch_spmm_shape<VT, EPL, G, 4, false, ACC>(A, X, L, ldx, Y, ldy, split, tn, ws, st);
    } else {
        if (tn.inflight == 4)
            return full ? launch_spmm_shape<VT, EPL, G, 4, true, ACC>(A, X, L, ldx, Y, ldy, split, tn, ws, st)
                        : launch_spmm_shape<VT, EPL, G, 4, false, ACC>(A, X, L, ldx, Y, ldy, split, tn, ws, st);
        return full ? launch_spmm_shape<VT, EPL, G, 8, true, ACC>(A, X, L, ldx, Y, ldy, split, tn, ws, st)
                    : launch_spmm_shape<VT, EPL, G, 8, false, ACC>(A, X, L, ldx, Y, ldy, split, tn, ws, st);
    }
}

template <typename VT>
static spd_status launch_spmm(const spd_csr *A, const void *X, int64_t L, int64_t ldx, void *Y, int64_t ldy,
                              int split, const Tuning &tn, void *ws, cudaStream_t st, bool accumulate) {
    using OT = typename Traits<VT>::out;
    const SpmmShape sh = pick_spmm_shape(L, sizeof(VT), sizeof(OT), X, ldx, Y, ldy, tn.lane_groups,
                                         (uint64_t)A->ncols * (uint64_t)ldx * sizeof(VT));
    return with_lane_shape<VT>(sh.epl, sh.group, [&](auto shape) {
        constexpr int E = decltype(shape)::epl, G = decltype(shape)::group;
        return accumulate ? launch_spmm_u<VT, E, G, true>(A, X, L, ldx, Y, ldy, split, tn, ws, st)
                          : launch_spmm_u<VT, E, G, false>(A, X, L, ldx, Y, ldy, split, tn, ws, st);
    });
}

template <typename VT, int EPL>
static spd_status launch_spmm_t_epl(const spd_csr *A, const void *dY, int64_t L, int64_t ldy, void *dX, int64_t ldx,
                                    int split, const Tuning &tn, void *ws, cudaStream_t st) {
    using OT = typename Traits<VT>::out;
    const int wpb = tn.block_threads / 32;
    const int64_t ctiles = ceil_div(L, 32 * EPL);
    const VT *v = static_cast<const VT *>(A->vals);
    const VT *g = static_cast<const VT *>(dY);
    OT *d = static_cast<OT *>(dX);
    {
        spd_status s = launch_zero_rows<OT>(A->ncols, L, d, ldx, st);
        if (s) return s;
    }
    if (A->nrows == 0 || A->nnz == 0) return SPD_OK;
    if (split == SPD_SPLIT_ROW) {
        const int64_t P = tn.row_pieces > 0 ? tn.row_pieces : default_row_pieces(A->nrows, A->nnz, tn.unit_items);
        dim3 grid((unsigned)ceil_div(P, wpb), (unsigned)ctiles);
        spmm_t_warp_kernel<VT, EPL><<<grid, tn.block_threads, 0, st>>>(A->nrows, A->pos, A->crd, v, g, ldy, d, ldx, L,
                                                                       nullptr, nullptr, 0, P);
        return check_launch("spmm_t_warp_kernel(row)");
    }
    WsLayout Lw = layout_warp(A->nrows, A->nnz, split, tn.unit_items, L, false);
    char *w = static_cast<char *>(ws);
    int32_t *prow = reinterpret_cast<int32_t *>(w + Lw.part_row);
    int32_t *ppos = reinterpret_cast<int32_t *>(w + Lw.part_pos);
    spd_status s = launch_merge_partition(A->nrows, A->nnz, A->pos, tn.unit_items, Lw.npieces, prow, ppos, st);
    if (s) return s;
    dim3 grid((unsigned)ceil_div(Lw.npieces, wpb), (unsigned)ctiles);
    spmm_t_warp_kernel<VT, EPL><<<grid, tn.block_threads, 0, st>>>(A->nrows, A->pos, A->crd, v, g, ldy, d, ldx, L,
                                                                   prow, ppos, Lw.npieces, 0);
    return check_launch("spmm_t_warp_kernel(nnz)");
}

template <typename VT>
static spd_status launch_spmm_t(const spd_csr *A, const void *dY, int64_t L, int64_t ldy, void *dX, int64_t ldx,
                                int split, const Tuning &tn, void *ws, cudaStream_t st) {
    using OT = typename Traits<VT>::out;
    int epl = pick_epl(L, sizeof(VT), sizeof(OT), dY, ldy, dX, ldx);
    if (sizeof(VT) == 8 && epl > 4) epl = 4;
    switch (epl) {
        case 1: return launch_spmm_t_epl<VT, 1>(A, dY, L, ldy, dX, ldx, split, tn, ws, st);
        case 2: return launch_spmm_t_epl<VT, 2>(A, dY, L, ldy, dX, ldx, split, tn, ws, st);
        case 4: return launch_spmm_t_epl<VT, 4>(A, dY, L, ldy, dX, ldx, split, tn, ws, st);
        default:
            if constexpr (sizeof(VT) <= 4) return launch_spmm_t_epl<VT, 8>(A, dY, L, ldy, dX, ldx, split, tn, ws, st);
            return launch_spmm_t_epl<VT, 4>(A, dY, L, ldy, dX, ldx, split, tn, ws, st);
    }
}

}  // namespace spd

using namespace spd;

// The two SpMM entry points: overwrite Y, or add to it.
static spd_status spmm_entry(const spd_csr *A, const void *X, int64_t L, int64_t ldx, int x_type, void *Y, int64_t ldy,
                             int y_type, int split, const spd_tune *tune, void *ws, size_t ws_bytes, void *stream,
                             bool accumulate) {
    spd_status s = check_csr(A, true);
    if (s) return s;
    if (L < 0) return fail(SPD_ERR_SHAPE, "L %lld < 0", (long long)L);
    if (x_type != A->vtype) return fail(SPD_ERR_DTYPE, "X type %d differs from the value type %d", x_type, A->vtype);
    if (y_type != result_type(A->vtype)) return fail(SPD_ERR_DTYPE, "Y type %d; expected %d", y_type, result_type(A->vtype));
    if ((s = check_dense("X", X, A->ncols, L, ldx, x_type))) return s;
    if ((s = check_dense("Y", Y, A->nrows, L, ldy, y_type))) return s;
    if ((uint64_t)ldx * dtype_size(x_type) >= (uint64_t(1) << 32))
        return fail(SPD_ERR_SHAPE, "X row stride of %lld elements exceeds 4 GiB", (long long)ldx);
    Tuning tn;
    if ((s = read_tune(tune, &tn))) return s;
    split = resolve_split(split);
    if (split != SPD_SPLIT_ROW && split != SPD_SPLIT_NNZ) return fail(SPD_ERR_ARG, "unknown split %d", split);
    WsLayout Lw = layout_warp(A->nrows, A->nnz, split, tn.unit_items, L, true);
    if ((s = check_ws(Lw, ws, ws_bytes))) return s;
    cudaStream_t st = as_stream(stream);
    if ((s = checked_csr(A, "A", st))) return s;
    if (A->nrows == 0 || L == 0) return SPD_OK;
    switch (A->vtype) {
        case SPD_F64: s = launch_spmm<double>(A, X, L, ldx, Y, ldy, split, tn, ws, st, accumulate); break;
        case SPD_F32: s = launch_spmm<float>(A, X, L, ldx, Y, ldy, split, tn, ws, st, accumulate); break;
        case SPD_BF16: s = launch_spmm<__nv_bfloat16>(A, X, L, ldx, Y, ldy, split, tn, ws, st, accumulate); break;
        default: return fail(SPD_ERR_DTYPE, "unknown value type %d", A->vtype);
    }
    return checked_finish(s, accumulate ? "spd_spmm_accumulate" : "spd_spmm", st);
}

extern "C" {


spd_status spd_spmm(const spd_csr *A, const void *X, int64_t L, int64_t ldx, int x_type, void *Y, int64_t ldy,
                    int y_type, int split, const spd_tune *tune, void *ws, size_t ws_bytes, void *stream) {
    return spmm_entry(A, X, L, ldx, x_type, Y, ldy, y_type, split, tune, ws, ws_bytes, stream, false);
}

spd_status spd_spmm_accumulate(const spd_csr *A, const void *X, int64_t L, int64_t ldx, int x_type, void *Y,
                               int64_t ldy, int y_type, int split, const spd_tune *tune, void *ws, size_t ws_bytes,
                               void *stream) {
    return spmm_entry(A, X, L, ldx, x_type, Y, ldy, y_type, split, tune, ws, ws_bytes, stream, true);
}

spd_status spd_spmm_t(const spd_csr *A, const void *dY, int64_t L, int64_t ldy, int dy_type, void *dX, int64_t ldx,
                      int dx_type, int split, const spd_tune *tune, void *ws, size_t ws_bytes, void *stream) {
    spd_status s = check_csr(A, true);
    if (s) return s;
    if (L < 0) return fail(SPD_ERR_SHAPE, "L %lld < 0", (long long)L);
    if (dy_type != A->vtype) return fail(SPD_ERR_DTYPE, "dY type %d differs from the value type %d", dy_type, A->vtype);
    if (dx_type != result_type(A->vtype)) return fail(SPD_ERR_DTYPE, "dX type %d; expected %d", dx_type, result_type(A->vtype));
    if ((s = check_dense("dY", dY, A->nrows, L, ldy, dy_type))) return s;
    if ((s = check_dense("dX", dX, A->ncols, L, ldx, dx_type))) return s;
    Tuning tn;
    if ((s = read_tune(tune, &tn))) return s;
    split = resolve_split(split);
    if (split != SPD_SPLIT_ROW && split != SPD_SPLIT_NNZ) return fail(SPD_ERR_ARG, "unknown split %d", split);
    WsLayout Lw = layout_warp(A->nrows, A->nnz, split, tn.unit_items, L, false);
    if ((s = check_ws(Lw, ws, ws_bytes))) return s;
    cudaStream_t st = as_stream(stream);
    if ((s = checked_csr(A, "A", st))) return s;
    if (L == 0) return SPD_OK;
    switch (A->vtype) {
        case SPD_F64: s = launch_spmm_t<double>(A, dY, L, ldy, dX, ldx, split, tn, ws, st); break;
        case SPD_F32: s = launch_spmm_t<float>(A, dY, L, ldy, dX, ldx, split, tn, ws, st); break;
        case SPD_BF16: s = launch_spmm_t<__nv_bfloat16>(A, dY, L, ldy, dX, ldx, split, tn, ws, st); break;
        default: return fail(SPD_ERR_DTYPE, "unknown value type %d", A->vtype);
    }
    return checked_finish(s, "spd_spmm_t", st);
}

}  // extern "C"
