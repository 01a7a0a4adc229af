// spd_spadd3.cu -- SpAdd3 A(i,j) = B(i,j) + C(i,j) + D(i,j) (Section VI-A) on three CSR
// operands of one shape. A's pattern, the union of the three patterns, is not known in
// advance, so A is assembled in two phases (Section V-B, the two-phase parallel
// assembly): a symbolic pass counts each row's union and a scan turns the counts into
// A's pos; after the caller has sized crd/vals, a numeric pass writes them with no
// synchronisation between writers.
//
// Work: the rows of the three operands are fused into one coordinate tree whose row i
// holds |B_i| + |C_i| + |D_i| items (pos_sum = pos_B + pos_C + pos_D), and that tree is
// split either by rows (universe partition) or into pieces of equal item counts
// (coordinate fusion and non-zero partition, as for the other statements). A piece that
// starts or ends inside a row takes that row's columns from a value boundary derived
// from the item offset (row_boundary). Neighbouring pieces derive the same boundary, so
// each column of A is produced by exactly one piece. One thread merges a piece's three
// sorted lists (at most unit_items entries); values are summed as written, (B + C) + D,
// over the operands that store the coordinate.
#include "spd_internal.cuh"

namespace spd {

constexpr int kSpadd3Threads = 128;
constexpr int64_t kSpadd3UnitDefault = 64;

struct Csr3 {
    const int32_t *pos[3];
    const int32_t *crd[3];
    const void *vals[3];
};

__global__ void pos_sum_kernel(int64_t n, Csr3 m, int32_t *__restrict__ psum) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += stride)
        psum[i] = m.pos[0][i] + m.pos[1][i] + m.pos[2][i];
}

// First index of sorted a[lo, hi) whose value is >= v.
__device__ __forceinline__ int32_t lower_bound(const int32_t *a, int32_t lo, int32_t hi, int32_t v) {
    int32_t b = lo, e = hi;
    while (b < e) {
        const int32_t mid = b + ((e - b) >> 1);  // b + e may pass 2^31 in an operand near the size limit
        if (a[mid] < v) b = mid + 1;
        else e = mid;
    }
    return b;
}

// Boundary column for item offset t (0 < t < len) of row r, whose three lists hold len
// entries together: the entry of the row's longest list (the first of them on a tie) at
// the same fraction of its length. It does not depend on which piece asks and does not
// decrease with t, so neighbouring pieces agree on it and the column ranges they take
// from the row never overlap; with lists of similar spread the pieces stay balanced.
__device__ __forceinline__ int32_t row_boundary(const Csr3 &m, int64_t r, int64_t t, int64_t len) {
    int g = 0;
    int32_t gb = m.pos[0][r], glen = m.pos[0][r + 1] - gb;
#pragma unroll
    for (int q = 1; q < 3; ++q) {
        const int32_t b = m.pos[q][r], l = m.pos[q][r + 1] - b;
        if (l > glen) {
            g = q;
            gb = b;
            glen = l;
        }
    }
    const int32_t *gc = g == 0 ? m.crd[0] : (g == 1 ? m.crd[1] : m.crd[2]);  // no indexing by a variable
    return gc[gb + (int32_t)((t * glen) / len)];
}

template <typename VT>
__device__ __forceinline__ typename Traits<VT>::acc val_at(const void *v, int32_t p) {
    return (typename Traits<VT>::acc)to_acc(static_cast<const VT *>(v)[p]);
}

// Output writer of the numeric phase. A thread's outputs form one contiguous run of A
// (its piece's); writing them one by one leaves 32-byte sectors partly written while
// thousands of other runs compete for L2, so each thread gathers the outputs of one
// aligned group of 8 positions in its own shared-memory slots and writes the group out
// as whole sectors (vector stores) when it is complete, element by element otherwise.
template <typename OT>
struct GroupWriter {
    int32_t *s_c;  // this thread's 8 slots
    OT *s_v;
    int32_t *a_crd;
    OT *a_val;
    int64_t first;  // first position written into the current group
    bool vec;       // a_crd / a_val allow aligned 32-byte (crd) and 8-element (vals) groups

    __device__ __forceinline__ void flush(int64_t last) {  // positions [first, last] of one group
        const int64_t g0 = last & ~int64_t(7);
        if (vec && first == g0 && last == g0 + 7) {
            const int4 *c4 = reinterpret_cast<const int4 *>(s_c);
            int4 *dc = reinterpret_cast<int4 *>(a_crd + g0);
            dc[0] = c4[0];
            dc[1] = c4[1];
            if constexpr (sizeof(OT) == 4) {
                const float4 *v4 = reinterpret_cast<const float4 *>(s_v);
                float4 *dv = reinterpret_cast<float4 *>(a_val + g0);
                dv[0] = v4[0];
                dv[1] = v4[1];
            } else {
                const double2 *v2 = reinterpret_cast<const double2 *>(s_v);
                double2 *dv = reinterpret_cast<double2 *>(a_val + g0);
#pragma unroll
                for (int q = 0; q < 4; ++q) dv[q] = v2[q];
            }
        } else {
            for (int64_t g = first; g <= last; ++g) {
                a_crd[g] = s_c[g & 7];
                a_val[g] = s_v[g & 7];
            }
        }
        first = last + 1;
    }
    __device__ __forceinline__ void put(int64_t g, int32_t j, OT v, int64_t end) {
        s_c[g & 7] = j;
        s_v[g & 7] = v;
        if ((g & 7) == 7 || g == end - 1) flush(g);
    }
};

// Merges the part of piece c that lies in row r, columns [vlo, vhi); returns the number
// of A entries produced. NUMERIC: hands them to the writer from position k0 on.
template <typename VT, bool NUMERIC>
__device__ __forceinline__ int64_t merge_row(const Csr3 &m, int64_t r, int32_t vlo, int32_t vhi,
                             GroupWriter<typename Traits<VT>::out> *wr, int64_t k0, int64_t kend) {
    using AT = typename Traits<VT>::acc;
    int32_t p[3], e[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int32_t b = m.pos[q][r], en = m.pos[q][r + 1];
        p[q] = vlo > INT32_MIN ? lower_bound(m.crd[q], b, en, vlo) : b;
        e[q] = vhi < INT32_MAX ? lower_bound(m.crd[q], p[q], en, vhi) : en;
    }
    int64_t k = 0;
    int32_t c[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) c[q] = p[q] < e[q] ? m.crd[q][p[q]] : INT32_MAX;
    while (true) {
        const int32_t j = min(c[0], min(c[1], c[2]));
        if (j == INT32_MAX) break;
        AT v = 0;
        bool have = false;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            if (c[q] == j) {
                if (NUMERIC) {
                    const AT t = val_at<VT>(m.vals[q], p[q]);
                    v = have ? v + t : t;
                }
                have = true;
                ++p[q];
                c[q] = p[q] < e[q] ? m.crd[q][p[q]] : INT32_MAX;
            }
        }
        if (NUMERIC) wr->put(k0 + k, j, (typename Traits<VT>::out)v, kend);
        ++k;
    }
    return k;
}

// One thread per piece of the fused tree (rows r0 .. r1 with item offsets p0, p1 into
// pos_sum). SYMBOLIC (NUMERIC = false): adds each row's union count to a_pos[r] and
// stores the piece's total in piece_cnt[c]. NUMERIC: writes positions
// [piece_start[c], piece_start[c + 1]).
template <typename VT, bool NUMERIC>
__global__ void __launch_bounds__(kSpadd3Threads) spadd3_kernel(
    int64_t n, Csr3 m, const int32_t *__restrict__ psum, const int32_t *__restrict__ prow,
    const int32_t *__restrict__ ppos, int64_t npieces, int64_t P, int32_t *__restrict__ a_pos,
    int32_t *__restrict__ piece_cnt, const int32_t *__restrict__ piece_start, int32_t *__restrict__ a_crd,
    typename Traits<VT>::out *__restrict__ a_val, bool vec) {
    using OT = typename Traits<VT>::out;
    __shared__ __align__(16) int32_t s_c[NUMERIC ? kSpadd3Threads * 8 : 1];
    __shared__ __align__(16) OT s_v[NUMERIC ? kSpadd3Threads * 8 : 1];
    const int64_t np = prow ? npieces : P;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= np) return;
    const PieceBounds b = prow ? nnz_piece(c, prow, ppos) : row_piece(c, P, n, psum);
    GroupWriter<OT> wr;
    int64_t k = 0, kend = 0;
    if (NUMERIC) {
        wr.s_c = s_c + threadIdx.x * 8;
        wr.s_v = s_v + threadIdx.x * 8;
        wr.a_crd = a_crd;
        wr.a_val = a_val;
        wr.vec = vec;
        k = piece_start[c];
        kend = piece_start[c + 1];
        wr.first = k;
    }
    int64_t total = 0;
    for (int64_t r = b.r0; r <= b.r1 && r < n; ++r) {
        const int64_t base = psum[r], len = (int64_t)psum[r + 1] - base;
        const int64_t ts = r == b.r0 ? (int64_t)b.p0 - base : 0;
        const int64_t te = r == b.r1 ? (int64_t)b.p1 - base : len;
        if (te <= ts) continue;  // nothing of row r in this piece (or an empty row of A)
        const int32_t vlo = ts > 0 ? row_boundary(m, r, ts, len) : INT32_MIN;
        const int32_t vhi = te < len ? row_boundary(m, r, te, len) : INT32_MAX;
        if (vlo >= vhi) continue;  // the range lies inside one column's run: a later piece owns it
        const int64_t cnt = merge_row<VT, NUMERIC>(m, r, vlo, vhi, &wr, k, kend);
        if (!NUMERIC && cnt) atomicAdd(a_pos + r, (int32_t)cnt);
        k += cnt;
        total += cnt;
    }
    if (!NUMERIC) {
        piece_cnt[c] = (int32_t)total;
        if (c == np - 1) piece_cnt[np] = 0;  // the scan then leaves the total at [np]
    }
}

// Workspace: pos_sum, the partition, the per-piece counts/starts and the scan's tile
// sums. The symbolic call fills it; the numeric call reads it unchanged.
struct Spadd3Layout {
    int64_t npieces = 0, P = 0;
    size_t psum = 0, prow = 0, ppos = 0, pcnt = 0, sums = 0, total = 0;
};

static Spadd3Layout spadd3_layout(int64_t n, int64_t items, int split, int64_t unit, int64_t row_pieces) {
    Spadd3Layout L;
    if (split == SPD_SPLIT_ROW) {
        L.P = row_pieces > 0 ? row_pieces : ceil_div(items > 0 ? items : 1, unit);
        if (L.P > n && n > 0) L.P = n;
        if (L.P < 1) L.P = 1;
        L.npieces = L.P;
    } else {
        L.npieces = ceil_div(items, unit);
    }
    const int64_t np1 = L.npieces + 1;
    size_t off = 0;
    L.psum = off;
    off += align_up(sizeof(int32_t) * (size_t)(n + 1));
    L.prow = off;
    off += align_up(sizeof(int32_t) * (size_t)np1);
    L.ppos = off;
    off += align_up(sizeof(int32_t) * (size_t)np1);
    L.pcnt = off;
    off += align_up(sizeof(int32_t) * (size_t)np1);
    const int64_t scan_n = (n + 1) > np1 ? (n + 1) : np1;
    L.sums = off;
    off += align_up(sizeof(int32_t) * (size_t)scan_tile_count(scan_n));
    L.total = off;
    return L;
}

static spd_status check_spadd3(const spd_csr *B, const spd_csr *C, const spd_csr *D) {
    const spd_csr *m[3] = {B, C, D};
    for (int q = 0; q < 3; ++q) {
        spd_status s = check_csr(m[q], true);
        if (s) return s;
    }
    for (int q = 1; q < 3; ++q) {
        if (m[q]->nrows != B->nrows || m[q]->ncols != B->ncols)
            return fail(SPD_ERR_SHAPE, "operand %d is %lld x %lld, B is %lld x %lld", q + 1, (long long)m[q]->nrows,
                        (long long)m[q]->ncols, (long long)B->nrows, (long long)B->ncols);
        if (m[q]->vtype != B->vtype) return fail(SPD_ERR_DTYPE, "operands differ in value type");
    }
    if (B->nnz + C->nnz + D->nnz > SPD_MAX_INDEX)
        return fail(SPD_ERR_SHAPE, "nnz(B) + nnz(C) + nnz(D) exceeds SPD_MAX_INDEX");
    return SPD_OK;
}

static spd_status checked_operands(const spd_csr *B, const spd_csr *C, const spd_csr *D, cudaStream_t st) {
    spd_status s = checked_csr(B, "B", st);
    if (!s) s = checked_csr(C, "C", st);
    if (!s) s = checked_csr(D, "D", st);
    return s;
}

static Csr3 make_csr3(const spd_csr *B, const spd_csr *C, const spd_csr *D) {
    Csr3 m;
    const spd_csr *a[3] = {B, C, D};
    for (int q = 0; q < 3; ++q) {
        m.pos[q] = a[q]->pos;
        m.crd[q] = a[q]->crd;
        m.vals[q] = a[q]->vals;
    }
    return m;
}

template <typename VT, bool NUMERIC>
static spd_status launch_spadd3(const spd_csr *B, const Csr3 &m, const Spadd3Layout &L, bool nnz_split, char *w,
                                int32_t *a_pos, int32_t *a_crd, void *a_val, cudaStream_t st) {
    using OT = typename Traits<VT>::out;
    const int64_t work = L.npieces;
    const unsigned grid = (unsigned)ceil_div(work > 0 ? work : 1, kSpadd3Threads);
    const bool vec = a_crd && a_val && aligned(a_crd, 32) && aligned(a_val, 8 * sizeof(OT));
    spadd3_kernel<VT, NUMERIC><<<grid, kSpadd3Threads, 0, st>>>(
        B->nrows, m, reinterpret_cast<const int32_t *>(w + L.psum),
        nnz_split ? reinterpret_cast<const int32_t *>(w + L.prow) : nullptr,
        nnz_split ? reinterpret_cast<const int32_t *>(w + L.ppos) : nullptr, L.npieces, L.P, a_pos,
        reinterpret_cast<int32_t *>(w + L.pcnt), reinterpret_cast<const int32_t *>(w + L.pcnt), a_crd,
        static_cast<OT *>(a_val), vec);
    return check_launch(NUMERIC ? "spadd3_kernel(numeric)" : "spadd3_kernel(symbolic)");
}

}  // namespace spd

using namespace spd;

extern "C" {

spd_status spd_spadd3_workspace_size(const spd_csr *B, const spd_csr *C, const spd_csr *D, int split,
                                     const spd_tune *tune, size_t *bytes) {
    if (!bytes) return fail(SPD_ERR_NULL, "bytes is NULL");
    spd_status s = check_spadd3(B, C, D);
    if (s) return s;
    Tuning tn;
    if ((s = read_tune(tune, &tn))) return s;
    split = resolve_split(split);
    if (split != SPD_SPLIT_ROW && split != SPD_SPLIT_NNZ) return fail(SPD_ERR_ARG, "unknown split %d", split);
    const int64_t unit = tune && tune->unit_items ? tn.unit_items : kSpadd3UnitDefault;
    *bytes = spadd3_layout(B->nrows, B->nrows + B->nnz + C->nnz + D->nnz, split, unit, tn.row_pieces).total;
    return SPD_OK;
}

spd_status spd_spadd3_symbolic(const spd_csr *B, const spd_csr *C, const spd_csr *D, int split,
                               const spd_tune *tune, int32_t *a_pos, int64_t *nnz_out, void *ws, size_t ws_bytes,
                               void *stream) {
    spd_status s = check_spadd3(B, C, D);
    if (s) return s;
    if (!a_pos || !nnz_out) return fail(SPD_ERR_NULL, "a_pos/nnz_out is NULL");
    if (!aligned(a_pos, 4)) return fail(SPD_ERR_ALIGN, "a_pos not 4-byte aligned");
    Tuning tn;
    if ((s = read_tune(tune, &tn))) return s;
    split = resolve_split(split);
    if (split != SPD_SPLIT_ROW && split != SPD_SPLIT_NNZ) return fail(SPD_ERR_ARG, "unknown split %d", split);
    const int64_t n = B->nrows, items = n + B->nnz + C->nnz + D->nnz;
    const int64_t unit = tune && tune->unit_items ? tn.unit_items : kSpadd3UnitDefault;
    const Spadd3Layout L = spadd3_layout(n, items, split, unit, tn.row_pieces);
    if (!ws) return fail(SPD_ERR_WORKSPACE, "workspace is NULL (%zu bytes needed)", L.total);
    if (ws_bytes < L.total) return fail(SPD_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, L.total);
    if (!aligned(ws, 256)) return fail(SPD_ERR_ALIGN, "workspace not 256-byte aligned");
    cudaStream_t st = as_stream(stream);
    if ((s = checked_operands(B, C, D, st))) return s;
    char *w = static_cast<char *>(ws);
    const Csr3 m = make_csr3(B, C, D);
    int32_t *psum = reinterpret_cast<int32_t *>(w + L.psum);
    int32_t *sums = reinterpret_cast<int32_t *>(w + L.sums);
    cudaError_t e = cudaMemsetAsync(a_pos, 0, sizeof(int32_t) * (size_t)(n + 1), st);
    if (e != cudaSuccess) return fail(SPD_ERR_CUDA, "memset: %s", cudaGetErrorString(e));
    const int64_t psum_blocks = ceil_div(n + 1, 256);
    pos_sum_kernel<<<(unsigned)(psum_blocks < 152 * 32 ? psum_blocks : 152 * 32), 256, 0, st>>>(n, m, psum);
    if ((s = check_launch("pos_sum_kernel"))) return s;
    const bool nnz_split = split == SPD_SPLIT_NNZ;
    if (nnz_split && L.npieces > 0) {
        s = launch_merge_partition(n, items - n, psum, unit, L.npieces, reinterpret_cast<int32_t *>(w + L.prow),
                                   reinterpret_cast<int32_t *>(w + L.ppos), st);
        if (s) return s;
    }
    if (L.npieces > 0) {
        switch (B->vtype) {
            case SPD_F64: s = launch_spadd3<double, false>(B, m, L, nnz_split, w, a_pos, nullptr, nullptr, st); break;
            case SPD_F32: s = launch_spadd3<float, false>(B, m, L, nnz_split, w, a_pos, nullptr, nullptr, st); break;
            default: s = launch_spadd3<__nv_bfloat16, false>(B, m, L, nnz_split, w, a_pos, nullptr, nullptr, st);
        }
        if (s) return s;
        // piece counts -> piece starts; row counts -> A's pos
        if ((s = exclusive_scan_i32(reinterpret_cast<int32_t *>(w + L.pcnt), L.npieces + 1, sums, st))) return s;
    }
    if ((s = exclusive_scan_i32(a_pos, n + 1, sums, st))) return s;
    int32_t total = 0;
    e = cudaMemcpyAsync(&total, a_pos + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(SPD_ERR_CUDA, "symbolic phase: %s", cudaGetErrorString(e));
    *nnz_out = total;
    return SPD_OK;
}

spd_status spd_spadd3_numeric(const spd_csr *B, const spd_csr *C, const spd_csr *D, int split,
                              const spd_tune *tune, const int32_t *a_pos, int64_t a_nnz, int32_t *a_crd,
                              void *a_vals, int a_type, void *ws, size_t ws_bytes, void *stream) {
    spd_status s = check_spadd3(B, C, D);
    if (s) return s;
    if (!a_pos) return fail(SPD_ERR_NULL, "a_pos is NULL");
    if (a_nnz < 0) return fail(SPD_ERR_SHAPE, "a_nnz %lld < 0", (long long)a_nnz);
    if (a_nnz > 0 && (!a_crd || !a_vals)) return fail(SPD_ERR_NULL, "a_crd/a_vals is NULL");
    if (a_type != result_type(B->vtype)) return fail(SPD_ERR_DTYPE, "a_type %d; expected %d", a_type, result_type(B->vtype));
    if ((a_crd && !aligned(a_crd, 4)) || (a_vals && !aligned(a_vals, dtype_size(a_type))))
        return fail(SPD_ERR_ALIGN, "a_crd/a_vals misaligned");
    Tuning tn;
    if ((s = read_tune(tune, &tn))) return s;
    split = resolve_split(split);
    if (split != SPD_SPLIT_ROW && split != SPD_SPLIT_NNZ) return fail(SPD_ERR_ARG, "unknown split %d", split);
    const int64_t n = B->nrows, items = n + B->nnz + C->nnz + D->nnz;
    const int64_t unit = tune && tune->unit_items ? tn.unit_items : kSpadd3UnitDefault;
    const Spadd3Layout L = spadd3_layout(n, items, split, unit, tn.row_pieces);
    if (!ws) return fail(SPD_ERR_WORKSPACE, "workspace is NULL (%zu bytes needed)", L.total);
    if (ws_bytes < L.total) return fail(SPD_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, L.total);
    if (!aligned(ws, 256)) return fail(SPD_ERR_ALIGN, "workspace not 256-byte aligned");
    cudaStream_t st = as_stream(stream);
    if ((s = checked_operands(B, C, D, st))) return s;
    if (L.npieces == 0 || a_nnz == 0) return SPD_OK;
    const Csr3 m = make_csr3(B, C, D);
    char *w = static_cast<char *>(ws);
    const bool nnz_split = split == SPD_SPLIT_NNZ;
    switch (B->vtype) {
        case SPD_F64: s = launch_spadd3<double, true>(B, m, L, nnz_split, w, nullptr, a_crd, a_vals, st); break;
        case SPD_F32: s = launch_spadd3<float, true>(B, m, L, nnz_split, w, nullptr, a_crd, a_vals, st); break;
        default: s = launch_spadd3<__nv_bfloat16, true>(B, m, L, nnz_split, w, nullptr, a_crd, a_vals, st);
    }
    return checked_finish(s, "spd_spadd3_numeric", st);
}

}  // extern "C"
