// spd_spmm_piece.cuh -- the per-warp body of SpMM Y(i,l) = A(i,j) * X(j,l)
// (Section VI-A) over one piece of the flattened coordinate tree, shared by the
// single-matrix kernel and the persistent batched kernel.
//
// The 32 lanes span a tile of 32*EPL dense columns, so every nonzero costs one
// coalesced row of X. crd/vals are streamed in windows of 32 through this warp's
// shared-memory slots; U rows of X are loaded back to back per group. A row is written
// once, when its end item is reached; rows longer than 4096 nonzeros accumulate with
// Kahan's compensated summation in the binary32 modes. When the piece ends inside a
// row, that row's partial is returned as a binary64 carry.
#pragma once

#include "spd_internal.cuh"

namespace spd {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int32_t kLongRow = 4096;

// Blocks of 256 threads per SM the SpMM kernels must fit: 4 caps them at 64 registers,
// so 32 warps stay resident to keep enough rows of X in flight.
constexpr int kSpmmMinBlocks = 4;

template <typename T, int N>
__device__ __forceinline__ void zero(T (&a)[N]) {
#pragma unroll
    for (int e = 0; e < N; ++e) a[e] = (T)0;
}

// Window of row ends: lane q holds the end of row rw + q (true_end) while the warp
// walks rows rw .. rw+31. Rows >= r1 are not completed by this piece.
struct RowWindow {
    int32_t rw;        // first row of the window
    int32_t true_end;  // pos[rw + lane + 1] (or INT_MAX past n)
    __device__ __forceinline__ void load(int32_t base, int64_t n, const int32_t *pos, int lane) {
        rw = base;
        int64_t q = (int64_t)base + lane;
        true_end = q < n ? ld_stream(pos + q + 1) : INT_MAX;
    }
    __device__ __forceinline__ int32_t end_of(int32_t r) const { return __shfl_sync(kFullMask, true_end, r - rw); }
};

// One piece [b.r0, b.p0) -> [b.r1, b.p1) of matrix (n, pos, crd, vals) times X into Y.
// s_crd / s_val: this warp's two 32-entry windows in shared memory. carry_row /
// carry_val (nullable): where the partial of row b.r1 goes when the piece ends inside it.
template <typename VT, int EPL, int U, bool FULLTILE>
__device__ __forceinline__ void spmm_piece(int64_t n, const int32_t *__restrict__ pos,
                                           const int32_t *__restrict__ crd, const VT *__restrict__ vals,
                                           const VT *__restrict__ X, uint32_t ldx_bytes,
                                           typename Traits<VT>::out *__restrict__ Y, int64_t ldy, int64_t L,
                                           const PieceBounds b, const int64_t col, const int lane,
                                           int32_t *s_crd, typename Traits<VT>::acc *s_val,
                                           int32_t *carry_row, bool write_carry_row, double *carry_val) {
    using AT = typename Traits<VT>::acc;
    using OT = typename Traits<VT>::out;
    const bool active = FULLTILE || col < L;
    // this lane's columns of row 0 of X; row j starts j * ldx_bytes further (one wide
    // multiply-add per gathered row)
    const char *__restrict__ Xc = reinterpret_cast<const char *>(X + col);
    auto xrow = [&](int32_t j) { return reinterpret_cast<const VT *>(Xc + (uint64_t)(uint32_t)j * ldx_bytes); };

    AT acc[EPL], cmp[EPL];
    zero(acc);
    zero(cmp);
    int32_t r = b.r0;
    RowWindow win;
    win.load(r, n, pos, lane);
    int32_t cur_start = r < n ? __ldg(pos + r) : b.p1;
    int32_t true_end = r < n ? win.end_of(r) : INT_MAX;
    int32_t cur_end = r < b.r1 ? true_end : INT_MAX;
    bool kahan = (sizeof(AT) == 4) && (true_end - cur_start > kLongRow);

    auto emit = [&]() {
        if (active) {
            OT o[EPL];
#pragma unroll
            for (int e = 0; e < EPL; ++e) o[e] = (OT)(acc[e] - cmp[e]);
            st_vec(Y + (int64_t)r * ldy + col, o);
        }
        zero(acc);
        zero(cmp);
        cur_start = cur_end;
        ++r;
        if (r - win.rw == 32) win.load(r, n, pos, lane);
        true_end = r < n ? win.end_of(r) : INT_MAX;
        cur_end = r < b.r1 ? true_end : INT_MAX;
        kahan = (sizeof(AT) == 4) && (true_end - cur_start > kLongRow);
    };

    // The piece's nonzeros are streamed in windows of 32: each lane loads one crd/vals
    // pair of the next window while the current window is consumed from this warp's
    // shared-memory slots, four entries per broadcast read. Entries are consumed in
    // groups of U whose rows of X are loaded back to back. A group inside the current row
    // (the common case) takes the fast path: U broadcast-multiply-adds, no checks. The
    // loops stay rolled so that the kernel fits the instruction cache.
    int32_t pb = b.p0;
    int cnt = (b.p1 - pb) < 32 ? (b.p1 - pb) : 32;
    int buf = 0;
    s_crd[lane] = lane < cnt ? ld_stream(crd + pb + lane) : 0;
    s_val[lane] = lane < cnt ? (AT)ld_stream(vals + pb + lane) : (AT)0;
    __syncwarp();
    while (pb < b.p1) {
        const int32_t pn = pb + 32;
        const int cnt_n = b.p1 - pn <= 0 ? 0 : (b.p1 - pn < 32 ? b.p1 - pn : 32);
        const int32_t c_n = lane < cnt_n ? ld_stream(crd + pn + lane) : 0;
        const AT v_n = lane < cnt_n ? (AT)ld_stream(vals + pn + lane) : (AT)0;
        const int32_t *wc = s_crd + buf * 32;
        const AT *wv = s_val + buf * 32;
#pragma unroll 1
        for (int j0 = 0; j0 < cnt; j0 += U) {
            AT xv[U][EPL];
            int32_t cj[U];
            AT vj[U];
#pragma unroll
            for (int q = 0; q < U / 4; ++q) {
                const int4 c4 = *reinterpret_cast<const int4 *>(wc + j0 + 4 * q);
                cj[4 * q] = c4.x; cj[4 * q + 1] = c4.y; cj[4 * q + 2] = c4.z; cj[4 * q + 3] = c4.w;
            }
            const int gcnt = cnt - j0 < U ? cnt - j0 : U;  // valid entries of this group
            if (active && gcnt == U) {
#pragma unroll
                for (int u = 0; u < U; ++u) ld_vec<EPL>(xrow(cj[u]), xv[u]);
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (active && u < gcnt) ld_vec<EPL>(xrow(cj[u]), xv[u]);
                    else zero(xv[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) vj[u] = wv[j0 + u];
            if (!kahan && gcnt == U && (int64_t)pb + j0 + U <= (int64_t)cur_end) {
                // fast path: the whole group lies inside the current row
#pragma unroll
                for (int u = 0; u < U; ++u) {
#pragma unroll
                    for (int e = 0; e < EPL; ++e) acc[e] = fma(vj[u], xv[u][e], acc[e]);
                }
                continue;
            }
            // general path: consume the group one row segment at a time; rows (empty ones
            // included) that end before the next entry are written at the one emit site
            int lo = 0;
            while (lo < gcnt) {
                while (cur_end <= pb + j0 + lo) emit();
                const int64_t in_row = (int64_t)cur_end - (pb + j0);
                const int hi = in_row < gcnt ? (int)in_row : gcnt;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (u >= lo && u < hi) {
                        if (kahan) {
#pragma unroll
                            for (int e = 0; e < EPL; ++e) kahan_fma(acc[e], cmp[e], vj[u], xv[u][e]);
                        } else {
#pragma unroll
                            for (int e = 0; e < EPL; ++e) acc[e] = fma(vj[u], xv[u][e], acc[e]);
                        }
                    }
                }
                lo = hi;
            }
        }
        buf ^= 1;
        __syncwarp();
        s_crd[buf * 32 + lane] = c_n;
        s_val[buf * 32 + lane] = v_n;
        __syncwarp();
        pb = pn;
        cnt = cnt_n;
    }
    while (r < b.r1) emit();  // rows ending after the last nonzero, empty rows included

    if (carry_row) {
        int32_t start = b.r1 < n ? __ldg(pos + b.r1) : b.p1;
        if (start < b.p0) start = b.p0;
        const bool has = b.p1 > start;
        if (lane == 0 && write_carry_row) *carry_row = has ? b.r1 : -1;
        if (has && active) {
#pragma unroll
            for (int e = 0; e < EPL; ++e) carry_val[col + e] = (double)acc[e] - (double)cmp[e];
        }
    }
}

}  // namespace spd
