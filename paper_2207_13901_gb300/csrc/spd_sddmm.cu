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
// The contraction over k is one dot product per stored position, on the CUDA cores by
// default. With bfloat16 operands (K a multiple of 32) form 2 runs it on the tensor cores,
// 16 positions at a time (sddmm_mma_kernel below): parity-green, but measured slower on
// the R-MAT workload (the kernel is bound by the gathers and their latency, not by the
// multiply-adds), so the autotuner times both.
#include "spd_internal.cuh"

namespace spd {

constexpr unsigned FULLM = 0xffffffffu;

template <typename VT, int EPL, int G, int KT>
__global__ void __launch_bounds__(kWarpBlockMax) sddmm_warp_kernel(
    int64_t n, const int32_t *__restrict__ pos, const int32_t *__restrict__ crd, const VT *__restrict__ vals,
    const VT *__restrict__ C, int64_t ldc, const VT *__restrict__ Dnk, int64_t ldd, int64_t K, uint32_t ldc_b,
    uint32_t ldd_b, typename Traits<VT>::out *__restrict__ out, const int32_t *__restrict__ prow,
    const int32_t *__restrict__ ppos, int64_t npieces, int64_t P) {
    using AT = typename Traits<VT>::acc;
    using OT = typename Traits<VT>::out;
    constexpr int NPG = 32 / G;                             // positions per warp step
    constexpr int U = 4;                                    // warp steps in flight
    extern __shared__ __align__(16) unsigned char sddmm_smem[];  // one window per warp
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid;
    if (c >= (prow ? npieces : P)) return;
    const PieceBounds b = prow ? nnz_piece(c, prow, ppos) : row_piece(c, P, n, pos);
    int32_t *s_crd = reinterpret_cast<int32_t *>(sddmm_smem) + wid * 64;  // crd [32], row [32]
    int32_t *s_row = s_crd + 32;
    AT *s_val = reinterpret_cast<AT *>(sddmm_smem + (blockDim.x >> 5) * 64 * sizeof(int32_t)) + wid * 32;
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
    // Binary32: crd/vals of the window are loaded one window ahead, the next window's
    // loads in flight while this one is consumed (K=32 and 128 measured 1.5-7% faster).
    // bfloat16, and binary32 with two k tiles of C kept in registers (K=256: 8% slower),
    // load each window as it starts.
    constexpr bool kPrefetch = sizeof(VT) == 4 && KT != 2;
    int32_t nx_crd = 0;
    AT nx_val = (AT)1;
    if (kPrefetch) {
        nx_crd = lane < b.p1 - b.p0 ? ld_stream(crd + b.p0 + lane) : 0;
        nx_val = (lane < b.p1 - b.p0 && vals) ? (AT)ld_stream(vals + b.p0 + lane) : (AT)1;
    }
    for (int32_t pb = b.p0; pb < b.p1; pb += 32) {
        const int cnt = (b.p1 - pb) < 32 ? (b.p1 - pb) : 32;
        const bool valid = lane < cnt;
        int32_t my_crd;
        AT my_val;
        if (kPrefetch) {
            my_crd = nx_crd;
            my_val = nx_val;
            const int32_t pn = pb + 32;
            const bool vn = lane < b.p1 - pn;
            nx_crd = vn ? ld_stream(crd + pn + lane) : 0;
            nx_val = (vn && vals) ? (AT)ld_stream(vals + pn + lane) : (AT)1;
        } else {
            my_crd = valid ? ld_stream(crd + pb + lane) : 0;
            my_val = (valid && vals) ? (AT)ld_stream(vals + pb + lane) : (AT)1;
        }
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

// ------------------------------------------------------------------ tensor-core form
//
// bfloat16 operands with binary32 accumulation, K a multiple of 32: the contraction over
// k of 16 consecutive positions runs on the tensor cores (mma.sync m16n8k16, bf16 inputs,
// fp32 accumulators). A is the 16 positions' rows of Dnk (16 x 16 per k step), B holds
// the rows of C of the distinct rows of those positions (up to 8 columns; a second pass
// takes the 9th to 16th), and the result column of each position's own row is its dot
// product. The order of k inside a dot product is free, so the fragment slots of a lane
// (k slots 2t, 2t+1, 2t+8, 2t+9 of a 16-wide step, t = lane % 4) are mapped to 8
// consecutive k of each row: every operand load is one 16-byte vector, and A and B use the
// same map, so the sum is the dot product. Each product of two bfloat16 values is exact
// in binary32.
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                               uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(kWarpBlockMax) sddmm_mma_kernel(
    int64_t n, const int32_t *__restrict__ pos, const int32_t *__restrict__ crd,
    const __nv_bfloat16 *__restrict__ vals, const __nv_bfloat16 *__restrict__ C, uint32_t ldc_b,
    const __nv_bfloat16 *__restrict__ Dnk, uint32_t ldd_b, int64_t K, float *__restrict__ out,
    const int32_t *__restrict__ prow, const int32_t *__restrict__ ppos, int64_t npieces, int64_t P) {
    const int lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= (prow ? npieces : P)) return;  // whole warp
    const PieceBounds b = prow ? nnz_piece(c, prow, ppos) : row_piece(c, P, n, pos);
    const int g = lane >> 2, t = lane & 3;  // fragment row group and k slot group of this lane
    const int ksteps = (int)(K / 32);       // 32 k per step: two m16n8k16 steps
    const char *Db = reinterpret_cast<const char *>(Dnk) + (size_t)t * 16;
    const char *Cb = reinterpret_cast<const char *>(C) + (size_t)t * 16;
    auto ld16 = [](const char *p) { return __ldg(reinterpret_cast<const uint4 *>(p)); };

    PosRows pr;
    pr.load(b.r0, n, pos, lane);
    for (int32_t pb = b.p0; pb < b.p1; pb += 32) {
        const int cnt = (b.p1 - pb) < 32 ? (b.p1 - pb) : 32;
        const bool valid = lane < cnt;
        const int32_t my_crd = valid ? ld_stream(crd + pb + lane) : 0;
        const float my_val = (valid && vals) ? __bfloat162float(__ldcs(vals + pb + lane)) : 1.f;
        const int32_t my_row = pr.find(pb + lane, valid, n, pos, lane);
        const int32_t next_rw = __shfl_sync(FULLM, my_row, cnt - 1);
        if (next_rw != pr.rw) pr.load(next_rw, n, pos, lane);
        // both halves of the window (positions 0..15 and 16..31) at once, so the gathers
        // of 32 positions are in flight together
        const int m = lane & 15, hb = lane >> 4;  // lane m of half hb describes position 16*hb + m
        const int32_t rm = __shfl_sync(FULLM, my_row, 16 * hb + m);
        const int32_t rp = __shfl_sync(FULLM, my_row, 16 * hb + (m > 0 ? m - 1 : 0));
        const bool vm = 16 * hb + m < cnt;
        const uint32_t st_all = __ballot_sync(FULLM, vm && (m == 0 || rm != rp));
        uint32_t starts[2];
        int nslots[2];
        int32_t jg[2], jh[2], crow[2][2];
        bool vg[2], vh[2], cv[2][2];
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            starts[hh] = (st_all >> (16 * hh)) & 0xffffu;  // bit q: position 16*hh + q starts a row
            nslots[hh] = __popc(starts[hh]);
            // rows of Dnk for positions g and g + 8 of the half
            jg[hh] = __shfl_sync(FULLM, my_crd, 16 * hh + g);
            jh[hh] = __shfl_sync(FULLM, my_crd, 16 * hh + g + 8);
            vg[hh] = 16 * hh + g < cnt;
            vh[hh] = 16 * hh + g + 8 < cnt;
            // row of C for column g of pass 0 and pass 1
#pragma unroll
            for (int ps = 0; ps < 2; ++ps) {
                const unsigned at = __fns(starts[hh], 0, 8 * ps + g + 1);
                cv[hh][ps] = at != 0xffffffffu;
                crow[hh][ps] = __shfl_sync(FULLM, my_row, 16 * hh + (cv[hh][ps] ? (int)at : 0));
            }
        }
        const bool two = nslots[0] > 8 || nslots[1] > 8;  // a second pass (warp-uniform)
        float acc[2][2][4];
#pragma unroll
        for (int hh = 0; hh < 2; ++hh)
#pragma unroll
            for (int ps = 0; ps < 2; ++ps)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[hh][ps][e] = 0.f;
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll 1
        for (int s = 0; s < ksteps; ++s) {
            uint4 a[2], h[2], b0[2];
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                a[hh] = vg[hh] ? ld16(Db + (uint64_t)(uint32_t)jg[hh] * ldd_b + s * 64) : z;
                h[hh] = vh[hh] ? ld16(Db + (uint64_t)(uint32_t)jh[hh] * ldd_b + s * 64) : z;
                b0[hh] = cv[hh][0] ? ld16(Cb + (uint64_t)(uint32_t)crow[hh][0] * ldc_b + s * 64) : z;
            }
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                mma_bf16_16816(acc[hh][0], a[hh].x, h[hh].x, a[hh].y, h[hh].y, b0[hh].x, b0[hh].y);
                mma_bf16_16816(acc[hh][0], a[hh].z, h[hh].z, a[hh].w, h[hh].w, b0[hh].z, b0[hh].w);
            }
            if (two) {
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const uint4 b1 = cv[hh][1] ? ld16(Cb + (uint64_t)(uint32_t)crow[hh][1] * ldc_b + s * 64) : z;
                    mma_bf16_16816(acc[hh][1], a[hh].x, h[hh].x, a[hh].y, h[hh].y, b1.x, b1.y);
                    mma_bf16_16816(acc[hh][1], a[hh].z, h[hh].z, a[hh].w, h[hh].w, b1.z, b1.w);
                }
            }
        }
        // position g's dot sits in column slot(g) of fragment row g: lane 4g + slot/2,
        // element slot % 2 (fragment rows g + 8: elements 2 + slot % 2)
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int sg = __popc(starts[hh] & ((2u << g) - 1u)) - 1;
            const int sh = __popc(starts[hh] & ((2u << (g + 8)) - 1u)) - 1;
            const float bg = __shfl_sync(FULLM, my_val, 16 * hh + g), bh = __shfl_sync(FULLM, my_val, 16 * hh + g + 8);
#pragma unroll
            for (int ps = 0; ps < 2; ++ps) {
                const int lg = sg - 8 * ps, lh = sh - 8 * ps;
                const float dg = (lg & 1) ? acc[hh][ps][1] : acc[hh][ps][0];  // selects: no indexed registers
                const float dh = (lh & 1) ? acc[hh][ps][3] : acc[hh][ps][2];
                if (vg[hh] && lg >= 0 && lg < 8 && (lg >> 1) == t) __stcs(out + pb + 16 * hh + g, bg * dg);
                if (vh[hh] && lh >= 0 && lh < 8 && (lh >> 1) == t) __stcs(out + pb + 16 * hh + g + 8, bh * dh);
            }
        }
    }
}

static spd_status launch_sddmm_mma(const spd_csr *B, const void *C, int64_t K, int64_t ldc, const void *Dnk,
                                   int64_t ldd, void *outv, int split, const Tuning &tn, void *ws, cudaStream_t st) {
    using BT = __nv_bfloat16;
    const uint32_t ldc_b = (uint32_t)(ldc * 2), ldd_b = (uint32_t)(ldd * 2);
    const int threads = tn.block_threads;
    const int wpb = threads / 32;
    const BT *v = static_cast<const BT *>(B->vals);
    const BT *cc = static_cast<const BT *>(C);
    const BT *dd = static_cast<const BT *>(Dnk);
    float *o = static_cast<float *>(outv);
    if (split == SPD_SPLIT_ROW) {
        int64_t P = tn.row_pieces > 0 ? tn.row_pieces : ceil_div(B->nrows + B->nnz, tn.unit_items);
        if (P < 1) P = 1;
        sddmm_mma_kernel<<<(unsigned)ceil_div(P, wpb), threads, 0, st>>>(B->nrows, B->pos, B->crd, v, cc, ldc_b, dd,
                                                                        ldd_b, K, o, nullptr, nullptr, 0, P);
        return check_launch("sddmm_mma_kernel(row)");
    }
    WsLayout Lw = layout_warp(B->nrows, B->nnz, split, tn.unit_items, 0, false);
    char *w = static_cast<char *>(ws);
    int32_t *prow = reinterpret_cast<int32_t *>(w + Lw.part_row);
    int32_t *ppos = reinterpret_cast<int32_t *>(w + Lw.part_pos);
    spd_status s = launch_merge_partition(B->nrows, B->nnz, B->pos, tn.unit_items, Lw.npieces, prow, ppos, st);
    if (s) return s;
    sddmm_mma_kernel<<<(unsigned)ceil_div(Lw.npieces, wpb), threads, 0, st>>>(
        B->nrows, B->pos, B->crd, v, cc, ldc_b, dd, ldd_b, K, o, prow, ppos, Lw.npieces, 0);
    return check_launch("sddmm_mma_kernel(nnz)");
}

template <typename VT, int EPL, int G, int KT>
static spd_status launch_sddmm_g(const spd_csr *B, const void *C, int64_t K, int64_t ldc, const void *Dnk,
                                 int64_t ldd, void *outv, int split, const Tuning &tn, void *ws, cudaStream_t st) {
    using OT = typename Traits<VT>::out;
    const uint32_t ldc_b = (uint32_t)(ldc * (int64_t)sizeof(VT)), ldd_b = (uint32_t)(ldd * (int64_t)sizeof(VT));
    using AT = typename Traits<VT>::acc;
    const int threads = tn.block_threads;
    const int wpb = threads / 32;
    const size_t smem = (size_t)wpb * 32 * (2 * sizeof(int32_t) + sizeof(AT));
    const VT *v = static_cast<const VT *>(B->vals);
    const VT *cc = static_cast<const VT *>(C);
    const VT *dd = static_cast<const VT *>(Dnk);
    OT *o = static_cast<OT *>(outv);
    if (split == SPD_SPLIT_ROW) {
        int64_t P = tn.row_pieces > 0 ? tn.row_pieces : ceil_div(B->nrows + B->nnz, tn.unit_items);
        if (P < 1) P = 1;
        sddmm_warp_kernel<VT, EPL, G, KT><<<(unsigned)ceil_div(P, wpb), threads, smem, st>>>(
            B->nrows, B->pos, B->crd, v, cc, ldc, dd, ldd, K, ldc_b, ldd_b, o, nullptr, nullptr, 0, P);
        return check_launch("sddmm_warp_kernel(row)");
    }
    WsLayout Lw = layout_warp(B->nrows, B->nnz, split, tn.unit_items, 0, false);
    char *w = static_cast<char *>(ws);
    int32_t *prow = reinterpret_cast<int32_t *>(w + Lw.part_row);
    int32_t *ppos = reinterpret_cast<int32_t *>(w + Lw.part_pos);
    spd_status s = launch_merge_partition(B->nrows, B->nnz, B->pos, tn.unit_items, Lw.npieces, prow, ppos, st);
    if (s) return s;
    sddmm_warp_kernel<VT, EPL, G, KT><<<(unsigned)ceil_div(Lw.npieces, wpb), threads, smem, st>>>(
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
    if constexpr (sizeof(VT) == 2) {
        // tensor cores: K a multiple of 32, rows of C and Dnk in 16-byte vectors with pitches below 4 GiB
        const bool mma_ok = K > 0 && K % 32 == 0 && ldc % 8 == 0 && ldd % 8 == 0 && aligned(C, 16) &&
                            aligned(Dnk, 16) && ldc * 2 <= (int64_t)UINT32_MAX && ldd * 2 <= (int64_t)UINT32_MAX;
        if (mma_ok && tn.form == 2) return launch_sddmm_mma(B, C, K, ldc, Dnk, ldd, outv, split, tn, ws, st);
    }
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
