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

// Warps per SM the SpMM kernels must fit: 32 caps them at 64 registers, so enough rows
// of X stay in flight. As launch bounds: blocks of up to kWarpBlockMax threads, this
// many of them resident.
constexpr int kSpmmResidentWarps = 32;
constexpr int kSpmmMinBlocks = kSpmmResidentWarps * 32 / kWarpBlockMax;


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

// The U values of a group from this warp's shared window (p aligned to U elements):
// 16-byte reads.
template <int U>
__device__ __forceinline__ void ld_window(const float *p, float (&v)[U]) {
#pragma unroll
    for (int q = 0; q < U / 4; ++q) {
        const float4 t = *reinterpret_cast<const float4 *>(p + 4 * q);
        v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
    }
}
template <int U>
__device__ __forceinline__ void ld_window(const double *p, double (&v)[U]) {
#pragma unroll
    for (int q = 0; q < U / 2; ++q) {
        const double2 t = *reinterpret_cast<const double2 *>(p + 2 * q);
        v[2 * q] = t.x; v[2 * q + 1] = t.y;
    }
}

// One piece [b.r0, b.p0) -> [b.r1, b.p1) of matrix (n, pos, crd, vals) times X into Y.
// s_crd / s_val: this warp's two 32-entry windows in shared memory. carry_row /
// carry_val (nullable): where the partial of row b.r1 goes when the piece ends inside it.
// ACC: add the product to Y (Y += A X) instead of overwriting it; rows of A without
// entries leave Y untouched.
template <typename VT, int EPL, int U, bool FULLTILE, bool ACC = false>
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
        if (active && (!ACC || true_end > cur_start)) {
            OT o[EPL];
#pragma unroll
            for (int e = 0; e < EPL; ++e) o[e] = (OT)(acc[e] - cmp[e]);
            if constexpr (ACC) {
                OT old[EPL];
                ld_vec<EPL>(Y + (int64_t)r * ldy + col, old);
#pragma unroll
                for (int e = 0; e < EPL; ++e) o[e] = old[e] + o[e];
            }
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
            ld_window<U>(wv + j0, vj);
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

// The same piece computed by lane groups: NG = 32/G groups of G lanes, each lane with
// one 16-byte vector (EPL elements) of the G*EPL columns starting at `col` (this lane's
// first column). For narrow L (G*EPL < 32*EPL of spmm_piece) the groups take different
// entries of the same rows side by side, so every gather instruction still moves a full
// vector per lane. Each group keeps its own partial of the current row; the partials
// are summed across the groups (a butterfly over the lane bits above G) when the row is
// written or carried, and group 0 writes. Entry q of a 32-entry window sits in slot
// (q % NG) * G + q / NG so that the U entries a group takes in one step are adjacent.
// s_cmp: this warp's 32*EPL slots for the Kahan compensations of a long row (kept out of
// registers, long rows being rare). Other arguments as for spmm_piece.
template <typename VT, int EPL, int G, int U, bool FULLTILE, bool ACC = false>
__device__ __forceinline__ void spmm_piece_grouped(int64_t n, const int32_t *__restrict__ pos,
                                                   const int32_t *__restrict__ crd, const VT *__restrict__ vals,
                                                   const VT *__restrict__ X, uint32_t ldx_bytes,
                                                   typename Traits<VT>::out *__restrict__ Y, int64_t ldy, int64_t L,
                                                   const PieceBounds b, const int64_t col, const int lane,
                                                   int32_t *s_crd, typename Traits<VT>::acc *s_val,
                                                   typename Traits<VT>::acc *s_cmp, int32_t *carry_row,
                                                   bool write_carry_row, double *carry_val) {
    using AT = typename Traits<VT>::acc;
    using OT = typename Traits<VT>::out;
    constexpr int NG = 32 / G;    // entries consumed side by side
    constexpr int STEP = NG * U;  // entries per step of the warp
    static_assert(G >= 4 && G < 32 && (G & (G - 1)) == 0, "group width");
    static_assert(U % 4 == 0 && U <= G, "a step must fit in one window");
    const int gi = lane / G;
    const bool active = FULLTILE || col < L;
    const bool writer = active && gi == 0;
    const int my_slot = (lane % NG) * G + lane / NG;
    const char *__restrict__ Xc = reinterpret_cast<const char *>(X + col);
    auto xrow = [&](int32_t j) { return reinterpret_cast<const VT *>(Xc + (uint64_t)(uint32_t)j * ldx_bytes); };

    AT acc[EPL];
    zero(acc);
    AT *cmp = s_cmp + lane;  // compensation of element e at cmp[32 * e]
    bool touched = false;    // some group accumulated an entry of row r (warp-uniform)
    int32_t r = b.r0;
    RowWindow win;
    win.load(r, n, pos, lane);
    int32_t cur_start = r < n ? __ldg(pos + r) : b.p1;
    int32_t true_end = r < n ? win.end_of(r) : INT_MAX;
    int32_t cur_end = r < b.r1 ? true_end : INT_MAX;
    bool kahan = (sizeof(AT) == 4) && (true_end - cur_start > kLongRow);
    auto clear_cmp = [&]() {
#pragma unroll
        for (int e = 0; e < EPL; ++e) cmp[32 * e] = (AT)0;
    };
    if (kahan) clear_cmp();

    auto emit = [&]() {
        if (kahan) {
#pragma unroll
            for (int e = 0; e < EPL; ++e) acc[e] -= cmp[32 * e];
        }
        if (touched) {
#pragma unroll
            for (int e = 0; e < EPL; ++e) {
#pragma unroll
                for (int m = G; m < 32; m <<= 1) acc[e] += __shfl_xor_sync(kFullMask, acc[e], m);
            }
        }
        if (writer && (!ACC || true_end > cur_start)) {
            OT o[EPL];
#pragma unroll
            for (int e = 0; e < EPL; ++e) o[e] = (OT)acc[e];
            if constexpr (ACC) {
                OT old[EPL];
                ld_vec<EPL>(Y + (int64_t)r * ldy + col, old);
#pragma unroll
                for (int e = 0; e < EPL; ++e) o[e] = old[e] + o[e];
            }
            st_vec(Y + (int64_t)r * ldy + col, o);
        }
        zero(acc);
        touched = false;
        cur_start = cur_end;
        ++r;
        if (r - win.rw == 32) win.load(r, n, pos, lane);
        true_end = r < n ? win.end_of(r) : INT_MAX;
        cur_end = r < b.r1 ? true_end : INT_MAX;
        kahan = (sizeof(AT) == 4) && (true_end - cur_start > kLongRow);
        if (kahan) clear_cmp();
    };

    int32_t pb = b.p0;
    int cnt = (b.p1 - pb) < 32 ? (b.p1 - pb) : 32;
    int buf = 0;
    s_crd[my_slot] = lane < cnt ? ld_stream(crd + pb + lane) : 0;
    s_val[my_slot] = lane < cnt ? (AT)ld_stream(vals + pb + lane) : (AT)0;
    __syncwarp();
    while (pb < b.p1) {
        const int32_t pn = pb + 32;
        const int cnt_n = b.p1 - pn <= 0 ? 0 : (b.p1 - pn < 32 ? b.p1 - pn : 32);
        const int32_t c_n = lane < cnt_n ? ld_stream(crd + pn + lane) : 0;
        const AT v_n = lane < cnt_n ? (AT)ld_stream(vals + pn + lane) : (AT)0;
        const int32_t *wc = s_crd + buf * 32;
        const AT *wv = s_val + buf * 32;
#pragma unroll 1
        for (int j0 = 0; j0 < cnt; j0 += STEP) {
            XVec<VT, EPL> xv[U];
            int32_t cj[U];
            AT vj[U];
            const int sb = gi * G + j0 / NG;  // slot of this group's first entry of the step
#pragma unroll
            for (int q = 0; q < U / 4; ++q) {
                const int4 c4 = *reinterpret_cast<const int4 *>(wc + sb + 4 * q);
                cj[4 * q] = c4.x; cj[4 * q + 1] = c4.y; cj[4 * q + 2] = c4.z; cj[4 * q + 3] = c4.w;
            }
            const int gcnt = cnt - j0 < STEP ? cnt - j0 : STEP;  // valid entries of this step
            if (active && gcnt == STEP) {
#pragma unroll
                for (int u = 0; u < U; ++u) xv[u].load(xrow(cj[u]));
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (active && u * NG + gi < gcnt) xv[u].load(xrow(cj[u]));
                    else xv[u].clear();
                }
            }
            ld_window<U>(wv + sb, vj);
            if (!kahan && gcnt == STEP && (int64_t)pb + j0 + STEP <= (int64_t)cur_end) {
                // fast path: the whole step lies inside the current row
#pragma unroll
                for (int u = 0; u < U; ++u) {
#pragma unroll
                    for (int e = 0; e < EPL; ++e) acc[e] = fma(vj[u], (AT)xv[u].at(e), acc[e]);
                }
                touched = true;
                continue;
            }
            // general path: one row segment at a time (entry k of the step is u*NG + gi)
            int lo = 0;
            while (lo < gcnt) {
                while (cur_end <= pb + j0 + lo) emit();
                const int64_t in_row = (int64_t)cur_end - (pb + j0);
                const int hi = in_row < gcnt ? (int)in_row : gcnt;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int k = u * NG + gi;
                    if (k >= lo && k < hi) {
                        if (kahan) {
#pragma unroll
                            for (int e = 0; e < EPL; ++e) {
                                AT c = cmp[32 * e];
                                kahan_fma(acc[e], c, vj[u], (AT)xv[u].at(e));
                                cmp[32 * e] = c;
                            }
                        } else {
#pragma unroll
                            for (int e = 0; e < EPL; ++e) acc[e] = fma(vj[u], (AT)xv[u].at(e), acc[e]);
                        }
                    }
                }
                touched = true;
                lo = hi;
            }
        }
        buf ^= 1;
        __syncwarp();
        s_crd[buf * 32 + my_slot] = c_n;
        s_val[buf * 32 + my_slot] = v_n;
        __syncwarp();
        pb = pn;
        cnt = cnt_n;
    }
    while (r < b.r1) emit();

    if (carry_row) {
        int32_t start = b.r1 < n ? __ldg(pos + b.r1) : b.p1;
        if (start < b.p0) start = b.p0;
        const bool has = b.p1 > start;  // warp-uniform
        if (lane == 0 && write_carry_row) *carry_row = has ? b.r1 : -1;
        if (has) {
            double t[EPL];
#pragma unroll
            for (int e = 0; e < EPL; ++e) {
                t[e] = (double)acc[e] - (kahan ? (double)cmp[32 * e] : 0.0);
#pragma unroll
                for (int m = G; m < 32; m <<= 1) t[e] += __shfl_xor_sync(kFullMask, t[e], m);
            }
            if (writer) {
#pragma unroll
                for (int e = 0; e < EPL; ++e) carry_val[col + e] = t[e];
            }
        }
    }
}

// Lane shape of the SpMM kernels: EPL elements per lane and groups of G lanes. G == 32
// runs spmm_piece (one entry per warp step), G < 32 spmm_piece_grouped with 16-byte
// vectors.
template <int E, int G_>
struct LaneShape {
    static constexpr int epl = E;
    static constexpr int group = G_;
};

// Shared memory of one warp of an SpMM kernel: two crd/vals windows, plus the Kahan
// slots of the grouped body.
template <typename VT>
inline size_t spmm_warp_smem(int epl, int group) {
    using AT = typename Traits<VT>::acc;
    return 64 * (sizeof(int32_t) + sizeof(AT)) + (group < 32 ? (size_t)32 * epl * sizeof(AT) : 0);
}

// Calls f(LaneShape<EPL, G>{}) for a lane shape chosen by pick_spmm_shape: grouped
// shapes use the 16-byte vector of VT; G == 32 shapes any EPL in 1..8 (1..4 binary64).
template <typename VT, typename F>
inline auto with_lane_shape(int epl, int group, F &&f) {
    constexpr int V = (int)(16 / sizeof(VT));
    if (group < 32) {
        if (group == 4) return f(LaneShape<V, 4>{});
        if (group == 8) return f(LaneShape<V, 8>{});
        return f(LaneShape<V, 16>{});
    }
    switch (epl) {
        case 1: return f(LaneShape<1, 32>{});
        case 2: return f(LaneShape<2, 32>{});
        case 4: return f(LaneShape<4, 32>{});
        default:
            if constexpr (sizeof(VT) <= 4) return f(LaneShape<8, 32>{});
            return f(LaneShape<4, 32>{});
    }
}

}  // namespace spd
