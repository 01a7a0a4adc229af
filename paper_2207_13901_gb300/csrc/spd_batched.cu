// spd_batched.cu -- many SpMM products Y_m = A_m X_m (Section VI-A) in one persistent
// launch.
//
// A plan lays every matrix's pieces (row split: universe partition of its rows; nnz
// split: fused non-zero partition of its coordinate tree) end to end into one global
// work list. The persistent kernel runs one block group per SM; its warps take global
// pieces g, g + W, g + 2W, ... (pieces are equal in item count, so a static stride
// balances them), read the matrix of each piece from a table the plan writes (one load
// instead of a search over hundreds of matrices), and run the same per-warp SpMM body as
// the single-matrix kernel. A second
// launch adds the binary64 carries of nnz-split matrices. Both launches are stream
// ordered, allocate nothing and do not synchronize, so a run can be captured in a CUDA
// graph and replayed.
#include <vector>

#include "spd_spmm_piece.cuh"

namespace spd {

struct BatchDesc {
    int64_t n;
    const int32_t *pos;
    const int32_t *crd;
    const void *vals;
    const void *X;
    void *Y;
    int64_t ldy;
    uint32_t ldx_bytes;
    int32_t split;      // SPD_SPLIT_ROW or SPD_SPLIT_NNZ
    int64_t P;          // pieces of this matrix
    int64_t piece0;     // global index of its first piece
    int64_t part_off;   // nnz split: first of its P+1 boundaries in prow/ppos
    int64_t carry_off;  // nnz split: first of its P carries
};


template <typename VT, int EPL, int G, bool FULLTILE>
__global__ void __launch_bounds__(kWarpBlockMax, kSpmmMinBlocks) spmm_batched_kernel(const BatchDesc *__restrict__ descs,
                                                           const int32_t *__restrict__ pmat,
                                                           int64_t total, int64_t L, const int32_t *__restrict__ prow,
                                                           const int32_t *__restrict__ ppos, int32_t *carry_row,
                                                           double *carry_val) {
    using AT = typename Traits<VT>::acc;
    using OT = typename Traits<VT>::out;
    extern __shared__ __align__(16) unsigned char batch_smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int64_t wpb = blockDim.x >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * wpb;
    const int64_t col = (int64_t)blockIdx.y * (G * EPL) + (int64_t)(lane % G) * EPL;
    int32_t *s_crd = reinterpret_cast<int32_t *>(batch_smem) + wid * 64;
    AT *s_val = reinterpret_cast<AT *>(batch_smem + wpb * 64 * sizeof(int32_t)) + wid * 64;
    AT *s_cmp = reinterpret_cast<AT *>(batch_smem + wpb * 64 * sizeof(int32_t)) + wpb * 64 + wid * 32 * EPL;
    for (int64_t g = (int64_t)blockIdx.x * wpb + wid; g < total; g += nwarps) {
        const BatchDesc &d = descs[__ldg(pmat + g)];
        const int64_t c = g - d.piece0;
        const bool nnz_split = d.split == SPD_SPLIT_NNZ;
        const PieceBounds b = nnz_split ? nnz_piece(c, prow + d.part_off, ppos + d.part_off)
                                        : row_piece(c, d.P, d.n, d.pos);
        const VT *vals = static_cast<const VT *>(d.vals);
        const VT *X = static_cast<const VT *>(d.X);
        OT *Y = static_cast<OT *>(d.Y);
        int32_t *crow = nnz_split ? carry_row + d.carry_off + c : nullptr;
        double *cval = nnz_split ? carry_val + (d.carry_off + c) * L : nullptr;
        if constexpr (G == 32)
            spmm_piece<VT, EPL, 4, FULLTILE>(d.n, d.pos, d.crd, vals, X, d.ldx_bytes, Y, d.ldy, L, b, col, lane, s_crd,
                                             s_val, crow, blockIdx.y == 0, cval);
        else
            spmm_piece_grouped<VT, EPL, G, 4, FULLTILE>(d.n, d.pos, d.crd, vals, X, d.ldx_bytes, Y, d.ldy, L, b, col,
                                                        lane, s_crd, s_val, s_cmp, crow, blockIdx.y == 0, cval);
    }
}

// Adds the carries of consecutive pieces of one nnz-split matrix that ended inside the
// same row (one warp per global piece, one lane per column).
template <typename OT>
__global__ void spmm_batched_fixup_kernel(const BatchDesc *__restrict__ descs, const int32_t *__restrict__ pmat,
                                          int64_t total, int64_t L,
                                          const int32_t *__restrict__ carry_row,
                                          const double *__restrict__ carry_val) {
    const int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t col = (int64_t)blockIdx.y * 32 + (threadIdx.x & 31);
    if (g >= total || col >= L) return;
    const BatchDesc &d = descs[pmat[g]];
    if (d.split != SPD_SPLIT_NNZ) return;
    const int64_t c = g - d.piece0;
    const int32_t *cr = carry_row + d.carry_off;
    const double *cv = carry_val + d.carry_off * L;
    const int32_t row = cr[c];
    if (row < 0) return;
    if (c > 0 && cr[c - 1] == row) return;
    double s = 0.0;
    for (int64_t e = c; e < d.P && cr[e] == row; ++e) s += cv[e * L + col];
    OT *yp = static_cast<OT *>(d.Y) + (int64_t)row * d.ldy + col;
    *yp = (OT)((double)*yp + s);
}

struct BatchLayout {
    size_t desc = 0, pstart = 0, pmat = 0, prow = 0, ppos = 0, crow = 0, cval = 0, total = 0;
    int64_t pieces = 0, nparts = 0, ncarry = 0;
};

static BatchLayout batch_layout(int64_t count, const spd_batch_item *items, int64_t L, const Tuning &tn) {
    BatchLayout B;
    for (int64_t m = 0; m < count; ++m) {
        const spd_batch_item &it = items[m];
        const int64_t unit = it.unit_items > 0 ? it.unit_items : tn.unit_items;
        const int64_t P = ceil_div(it.A.nrows + it.A.nnz, unit);  // 0 for an empty matrix
        B.pieces += P;
        if (resolve_split(it.split) == SPD_SPLIT_NNZ) {
            B.nparts += P + 1;
            B.ncarry += P;
        }
    }
    size_t off = 0;
    B.desc = off;
    off += align_up(sizeof(BatchDesc) * (size_t)(count > 0 ? count : 1));
    B.pstart = off;
    off += align_up(sizeof(int64_t) * (size_t)(count + 1));
    B.pmat = off;  // matrix of every global piece
    off += align_up(sizeof(int32_t) * (size_t)(B.pieces > 0 ? B.pieces : 1));
    B.prow = off;
    off += align_up(sizeof(int32_t) * (size_t)(B.nparts > 0 ? B.nparts : 1));
    B.ppos = off;
    off += align_up(sizeof(int32_t) * (size_t)(B.nparts > 0 ? B.nparts : 1));
    B.crow = off;
    off += align_up(sizeof(int32_t) * (size_t)(B.ncarry > 0 ? B.ncarry : 1));
    B.cval = off;
    off += align_up(sizeof(double) * (size_t)(B.ncarry > 0 ? B.ncarry : 1) * (size_t)(L > 0 ? L : 1));
    B.total = off;
    return B;
}

static spd_status check_batch(int64_t count, const spd_batch_item *items, int64_t L, int vtype) {
    if (count < 0) return fail(SPD_ERR_SHAPE, "count %lld < 0", (long long)count);
    if (count > 0 && !items) return fail(SPD_ERR_NULL, "items is NULL");
    if (L < 0) return fail(SPD_ERR_SHAPE, "L %lld < 0", (long long)L);
    if (dtype_size(vtype) == 0) return fail(SPD_ERR_DTYPE, "unknown value type %d", vtype);
    for (int64_t m = 0; m < count; ++m) {
        const spd_batch_item &it = items[m];
        spd_status s = check_csr(&it.A, true);
        if (s) {
            char why[256];
            snprintf(why, sizeof(why), "%s", spd_last_error());
            return fail(s, "item %lld: %s", (long long)m, why);
        }
        if (it.A.vtype != vtype) return fail(SPD_ERR_DTYPE, "item %lld: value type %d != %d", (long long)m, it.A.vtype, vtype);
        if ((s = check_dense("X", it.X, it.A.ncols, L, it.ldx, vtype))) return s;
        if ((s = check_dense("Y", it.Y, it.A.nrows, L, it.ldy, result_type(vtype)))) return s;
        if ((uint64_t)it.ldx * dtype_size(vtype) >= (uint64_t(1) << 32))
            return fail(SPD_ERR_SHAPE, "item %lld: X row stride exceeds 4 GiB", (long long)m);
        const int sp = resolve_split(it.split);
        if (sp != SPD_SPLIT_ROW && sp != SPD_SPLIT_NNZ) return fail(SPD_ERR_ARG, "item %lld: unknown split", (long long)m);
        if (it.unit_items && (it.unit_items < 32 || it.unit_items > 65536 || it.unit_items % 32))
            return fail(SPD_ERR_ARG, "item %lld: unit_items %d", (long long)m, it.unit_items);
    }
    return SPD_OK;
}

template <typename VT, int EPL, int G, bool FULLTILE>
static spd_status launch_batched(const spd_batch_plan *pl, cudaStream_t st) {
    using OT = typename Traits<VT>::out;
    char *w = static_cast<char *>(pl->ws);
    const BatchDesc *descs = reinterpret_cast<const BatchDesc *>(w + pl->off_desc);
    const int32_t *pmat = reinterpret_cast<const int32_t *>(w + pl->off_pmat);
    const int32_t *prow = reinterpret_cast<const int32_t *>(w + pl->off_prow);
    const int32_t *ppos = reinterpret_cast<const int32_t *>(w + pl->off_ppos);
    int32_t *crow = reinterpret_cast<int32_t *>(w + pl->off_crow);
    double *cval = reinterpret_cast<double *>(w + pl->off_cval);
    const int64_t ctiles = ceil_div(pl->L, G * EPL);
    const size_t smem = (size_t)(pl->block_threads / 32) * spmm_warp_smem<VT>(EPL, G);
    dim3 grid((unsigned)pl->grid, (unsigned)ctiles);
    spmm_batched_kernel<VT, EPL, G, FULLTILE><<<grid, pl->block_threads, smem, st>>>(
        descs, pmat, pl->total_pieces, pl->L, prow, ppos, crow, cval);
    spd_status s = check_launch("spmm_batched_kernel");
    if (s || !pl->has_nnz) return s;
    dim3 fgrid((unsigned)ceil_div(pl->total_pieces, 8), (unsigned)ceil_div(pl->L, 32));
    spmm_batched_fixup_kernel<OT><<<fgrid, 256, 0, st>>>(descs, pmat, pl->total_pieces, pl->L, crow, cval);
    return check_launch("spmm_batched_fixup_kernel");
}

template <typename VT>
static spd_status dispatch_batched(const spd_batch_plan *pl, cudaStream_t st) {
    const bool full = pl->fulltile != 0;
    return with_lane_shape<VT>(pl->epl, pl->group, [&](auto sh) {
        constexpr int E = decltype(sh)::epl, G = decltype(sh)::group;
        return full ? launch_batched<VT, E, G, true>(pl, st) : launch_batched<VT, E, G, false>(pl, st);
    });
}

template <typename VT>
static int batched_blocks_per_sm(int epl, int group, bool full, int threads) {
    const size_t smem = (size_t)(threads / 32) * spmm_warp_smem<VT>(epl, group);
    int blocks = 0;
    const cudaError_t e = with_lane_shape<VT>(epl, group, [&](auto sh) {
        constexpr int E = decltype(sh)::epl, G = decltype(sh)::group;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &blocks, full ? spmm_batched_kernel<VT, E, G, true> : spmm_batched_kernel<VT, E, G, false>, threads, smem);
    });
    if (e != cudaSuccess || blocks < 1) {
        cudaGetLastError();
        return 1;
    }
    return blocks;
}

}  // namespace spd

using namespace spd;

extern "C" {

spd_status spd_spmm_batched_workspace_size(int64_t count, const spd_batch_item *items, int64_t L, int vtype,
                                           const spd_tune *tune, size_t *bytes) {
    if (!bytes) return fail(SPD_ERR_NULL, "bytes is NULL");
    spd_status s = check_batch(count, items, L, vtype);
    if (s) return s;
    Tuning tn;
    if ((s = read_tune(tune, &tn))) return s;
    *bytes = batch_layout(count, items, L, tn).total;
    return SPD_OK;
}

spd_status spd_spmm_batched_plan(int64_t count, const spd_batch_item *items, int64_t L, int vtype,
                                 const spd_tune *tune, void *ws, size_t ws_bytes, spd_batch_plan *plan,
                                 void *stream) {
    if (!plan) return fail(SPD_ERR_NULL, "plan is NULL");
    spd_status s = check_batch(count, items, L, vtype);
    if (s) return s;
    Tuning tn;
    if ((s = read_tune(tune, &tn))) return s;
    const BatchLayout B = batch_layout(count, items, L, tn);
    if (!ws) return fail(SPD_ERR_WORKSPACE, "workspace is NULL (%zu bytes needed)", B.total);
    if (ws_bytes < B.total) return fail(SPD_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, B.total);
    if (!aligned(ws, 256)) return fail(SPD_ERR_ALIGN, "workspace not 256-byte aligned");
    cudaStream_t st = as_stream(stream);
    for (int64_t m = 0; m < count && checked_mode(); ++m)
        if ((s = checked_csr(&items[m].A, "a batch matrix", st))) return s;

    // one lane shape that suits every matrix: lane groups only when every matrix allows
    // 16-byte vectors (decided by the largest X when the tuning leaves it open)
    const size_t vs = dtype_size(vtype), os = dtype_size(result_type(vtype));
    uint64_t x_max = 0;
    for (int64_t m = 0; m < count; ++m) {
        const uint64_t xb = (uint64_t)items[m].A.ncols * (uint64_t)items[m].ldx * vs;
        if (xb > x_max) x_max = xb;
    }
    SpmmShape shape = pick_spmm_shape(L, vs, os, nullptr, 0, nullptr, 0, tn.lane_groups, x_max);
    for (int64_t m = 0; m < count && shape.group < 32; ++m)
        if (pick_spmm_shape(L, vs, os, items[m].X, items[m].ldx, items[m].Y, items[m].ldy, tn.lane_groups, x_max)
                .group == 32)
            shape.group = 32;
    if (shape.group == 32) {  // 32 lanes at the narrowest width any matrix allows
        int epl = 8;
        for (int64_t m = 0; m < count; ++m) {
            const int e = pick_epl(L, vs, os, items[m].X, items[m].ldx, items[m].Y, items[m].ldy);
            if (e < epl) epl = e;
        }
        if (vs == 8 && epl > 4) epl = 4;
        if (count == 0) epl = 1;
        shape.epl = epl;
    }
    const int epl = shape.epl;

    std::vector<BatchDesc> descs((size_t)count);
    std::vector<int64_t> pstart((size_t)count + 1);
    std::vector<int32_t> pmat((size_t)B.pieces);
    int64_t piece = 0, part = 0, carry = 0;
    bool has_nnz = false;
    for (int64_t m = 0; m < count; ++m) {
        const spd_batch_item &it = items[m];
        const int64_t unit = it.unit_items > 0 ? it.unit_items : tn.unit_items;
        const int64_t items_m = it.A.nrows + it.A.nnz;
        const int64_t P = ceil_div(items_m, unit);  // 0 for an empty matrix
        BatchDesc &d = descs[(size_t)m];
        d.n = it.A.nrows;
        d.pos = it.A.pos;
        d.crd = it.A.crd;
        d.vals = it.A.vals;
        d.X = it.X;
        d.Y = it.Y;
        d.ldy = it.ldy;
        d.ldx_bytes = (uint32_t)(it.ldx * (int64_t)vs);
        d.split = resolve_split(it.split);
        d.P = P;
        d.piece0 = piece;
        d.part_off = d.carry_off = 0;
        if (d.split == SPD_SPLIT_NNZ) {
            d.part_off = part;
            d.carry_off = carry;
            part += P + 1;
            carry += P;
            has_nnz = true;
        }
        pstart[(size_t)m] = piece;
        for (int64_t q = 0; q < P; ++q) pmat[(size_t)(piece + q)] = (int32_t)m;
        piece += P;
    }
    pstart[(size_t)count] = piece;
    char *w = static_cast<char *>(ws);
    cudaError_t e = cudaSuccess;
    if (count > 0) e = cudaMemcpyAsync(w + B.desc, descs.data(), sizeof(BatchDesc) * descs.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w + B.pstart, pstart.data(), sizeof(int64_t) * pstart.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && piece > 0)
        e = cudaMemcpyAsync(w + B.pmat, pmat.data(), sizeof(int32_t) * pmat.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(SPD_ERR_CUDA, "plan copy: %s", cudaGetErrorString(e));
    int32_t *prow = reinterpret_cast<int32_t *>(w + B.prow);
    int32_t *ppos = reinterpret_cast<int32_t *>(w + B.ppos);
    for (int64_t m = 0; m < count; ++m) {
        const BatchDesc &d = descs[(size_t)m];
        if (d.split != SPD_SPLIT_NNZ || d.P == 0) continue;
        const int64_t unit = items[m].unit_items > 0 ? items[m].unit_items : tn.unit_items;
        if ((s = launch_merge_partition(d.n, items[m].A.nnz, d.pos, unit, d.P, prow + d.part_off, ppos + d.part_off, st)))
            return s;
    }
    e = cudaStreamSynchronize(st);  // the host copies of the descriptors end with this call
    if (e != cudaSuccess) return fail(SPD_ERR_CUDA, "plan: %s", cudaGetErrorString(e));

    const bool full = L > 0 && L % (shape.group * epl) == 0;
    int sms = 152;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int threads = tn.block_threads;
    int bps = 1;
    switch (vtype) {
        case SPD_F64: bps = batched_blocks_per_sm<double>(epl, shape.group, full, threads); break;
        case SPD_F32: bps = batched_blocks_per_sm<float>(epl, shape.group, full, threads); break;
        default: bps = batched_blocks_per_sm<__nv_bfloat16>(epl, shape.group, full, threads); break;
    }
    const int64_t need = ceil_div(piece > 0 ? piece : 1, threads / 32);
    int64_t grid = (int64_t)sms * bps;
    if (grid > need) grid = need;

    plan->count = count;
    plan->total_pieces = piece;
    plan->L = L;
    plan->vtype = vtype;
    plan->epl = epl;
    plan->group = shape.group;
    plan->block_threads = threads;
    plan->grid = (int32_t)grid;
    plan->fulltile = full ? 1 : 0;
    plan->has_nnz = has_nnz ? 1 : 0;
    plan->ws = ws;
    plan->off_desc = B.desc;
    plan->off_pstart = B.pstart;
    plan->off_pmat = B.pmat;
    plan->off_prow = B.prow;
    plan->off_ppos = B.ppos;
    plan->off_crow = B.crow;
    plan->off_cval = B.cval;
    return SPD_OK;
}

spd_status spd_spmm_batched_run(const spd_batch_plan *plan, void *stream) {
    if (!plan) return fail(SPD_ERR_NULL, "plan is NULL");
    if (plan->total_pieces == 0 || plan->L == 0) return SPD_OK;
    if (!plan->ws) return fail(SPD_ERR_WORKSPACE, "plan has no workspace");
    cudaStream_t st = as_stream(stream);
    spd_status s;
    switch (plan->vtype) {
        case SPD_F64: s = dispatch_batched<double>(plan, st); break;
        case SPD_F32: s = dispatch_batched<float>(plan, st); break;
        case SPD_BF16: s = dispatch_batched<__nv_bfloat16>(plan, st); break;
        default: return fail(SPD_ERR_DTYPE, "unknown value type %d", plan->vtype);
    }
    return checked_finish(s, "spd_spmm_batched_run", st);
}

}  // extern "C"
