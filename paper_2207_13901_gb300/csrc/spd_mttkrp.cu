// spd_mttkrp.cu -- SpMTTKRP A(i,l) = B(i,j,k) * C(j,l) * D(k,l) (Section VI-A) on a
// CSF tensor B = {Dense, Compressed, Compressed}.
//
// Every entry (i,j,k) contributes (B(i,j,k) * C(j,:)) * D(k,:) to row i of A, formed in
// the order the statement is written. In the binary32 modes a slice with more than 4096
// entries is accumulated with Kahan's compensated summation: each warp step's U entries
// are summed into a short local partial, and that partial is added to the slice's running
// sum with a compensation term (kept in shared memory). One warp consumes one piece of entries; entries
// come in windows of 32 whose fiber (hence j) and slice (i) each lane finds with a
// lane-parallel search over 32-entry windows of pos2 and pos1. Lanes form groups of G
// (G * EPL covers R), so a warp step covers 32/G entries; the groups' partial rows are
// summed across the warp only when the slice changes.
//   Nnz split (the GPU schedule of Section VI-A): coordinate fusion of levels 2 and 3 and
//     a non-zero partition of the fused items (each fiber's entries followed by one
//     "fiber end" item), so pieces balance entries and fibers. Piece c writes the slices
//     [s_c, s_{c+1}) whose last fiber ends inside it, where s_c = #{i : pos1[i+1] <= first
//     fiber of piece c} (s_0 = 0, s_last = I); the partial of the slice a piece ends in
//     is a binary64 carry added by the fix-up kernel.
//   Row split: universe partition of the slices, [floor(c I/P), floor((c+1) I/P)).
// The contraction per entry is a scaled row of D (no dense reuse within a warp), so the
// work stays on the CUDA cores. The kernel is bound by instruction issue (the factor rows
// come from L2), so rows are addressed as a 32-bit index times a 32-bit byte pitch (one
// wide multiply-add) and warp steps that lie wholly inside a slice segment skip the
// per-entry bounds checks.
#include "spd_internal.cuh"

namespace spd {

constexpr int32_t kLongSlice = 4096;  // slices with more entries are accumulated with compensation

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

// 32 resident warps a SM (64 registers): measured faster than 24 with the compensation
// kept spill-free (73 registers).
constexpr int kMttkrpResidentWarps = 32;

// Shared memory of one warp: the values and Kahan compensations of a window (AT), then
// its j, k and slice (int32).
template <typename VT>
inline size_t mttkrp_warp_smem(int epl) {
    return 32 * (1 + (size_t)epl) * sizeof(typename Traits<VT>::acc) + 3 * 32 * sizeof(int32_t);
}

template <typename VT, int EPL, int G>
__global__ void __launch_bounds__(kWarpBlockMax, kMttkrpResidentWarps * 32 / kWarpBlockMax) spmttkrp_warp_kernel(
    int64_t I, int64_t F, const int32_t *__restrict__ pos1, const int32_t *__restrict__ crd1,
    const int32_t *__restrict__ pos2, const int32_t *__restrict__ crd2, const VT *__restrict__ vals,
    const VT *__restrict__ C, uint32_t ldc_b, const VT *__restrict__ D, uint32_t ldd_b, int64_t R,
    typename Traits<VT>::out *__restrict__ A, int64_t lda, const int32_t *__restrict__ pfib,
    const int32_t *__restrict__ ppos, const int32_t *__restrict__ pslice, int64_t npieces, int64_t P,
    int32_t *__restrict__ carry_row, double *__restrict__ carry_val) {
    using AT = typename Traits<VT>::acc;
    using OT = typename Traits<VT>::out;
    constexpr int NPG = 32 / G;         // entries per warp step
    constexpr int U = 4;  // warp steps in flight
    extern __shared__ __align__(16) unsigned char mttkrp_smem[];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid;
    if (c >= (pfib ? npieces : P)) return;
    const int gi = lane / G, gl = lane % G;
    const int64_t col = (int64_t)blockIdx.y * (G * EPL) + (int64_t)gl * EPL;
    const bool active = col < R;
    const char *Cl = reinterpret_cast<const char *>(C) + (size_t)col * sizeof(VT);
    const char *Dl = reinterpret_cast<const char *>(D) + (size_t)col * sizeof(VT);

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
    (void)f1;
    AT *s_v = reinterpret_cast<AT *>(mttkrp_smem) + wid * 32 * (1 + EPL);
    AT *cmp = s_v + 32 + lane;  // Kahan compensation of element e of a long slice at cmp[32 * e]
    int32_t *s_j = reinterpret_cast<int32_t *>(mttkrp_smem + (blockDim.x >> 5) * 32 * (1 + EPL) * sizeof(AT)) + wid * 96;
    int32_t *s_k = s_j + 32, *s_sl = s_j + 64;

    AT acc[EPL];
#pragma unroll
    for (int e = 0; e < EPL; ++e) acc[e] = 0;
    bool dirty = false;  // acc holds contributions
    int32_t cs = s0;     // slice being accumulated (the same in every lane)
    // A window whose last entry lies in slice cs lies wholly in it and needs no slice
    // search. Taken for bfloat16 operands only: with binary32 operands the extra live
    // values spill at the 64-register cap and the kernel measured slower.
    constexpr bool kSkipSearch = sizeof(VT) == 2;
    int32_t cs_end = kSkipSearch && cs < I ? __ldg(pos1 + cs + 1) : INT_MAX;  // its end, in fibers
    // whether slice s holds more than kLongSlice entries (binary32 accumulation only);
    // the same four loads in every lane of the warp
    constexpr bool kComp = sizeof(AT) == 4;  // binary64 sums need no compensation
    auto long_slice = [&](int32_t s) {
        if (!kComp || s >= I) return false;
        return __ldg(pos2 + __ldg(pos1 + s + 1)) - __ldg(pos2 + __ldg(pos1 + s)) > kLongSlice;
    };
    bool ka = long_slice(cs);  // compensated accumulation of slice cs
    auto clear_cmp = [&]() {
#pragma unroll
        for (int e = 0; e < EPL; ++e) cmp[32 * e] = (AT)0;
    };
    if (kComp && ka) clear_cmp();

    // total of acc over the groups of the warp (every lane ends with it)
    auto warp_total = [&](AT (&t)[EPL]) {
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
            t[e] = kComp && ka ? acc[e] - cmp[32 * e] : acc[e];
#pragma unroll
            for (int off = G; off < 32; off <<= 1) t[e] += __shfl_xor_sync(0xffffffffu, t[e], off);
        }
    };
    // slice cs is complete: write it, then zeros for the empty slices before `next`
    auto finish_to = [&](int32_t next) {
        AT t[EPL];
        warp_total(t);
        if (gi == 0 && active) {
            OT o[EPL];
#pragma unroll
            for (int e = 0; e < EPL; ++e) o[e] = (OT)t[e];
            st_vec(A + (int64_t)cs * lda + col, o);
#pragma unroll
            for (int e = 0; e < EPL; ++e) o[e] = (OT)0;
            const int32_t stop = next < s1 ? next : s1;
            for (int32_t i = cs + 1; i < stop; ++i) st_vec(A + (int64_t)i * lda + col, o);
        }
#pragma unroll
        for (int e = 0; e < EPL; ++e) acc[e] = 0;
        dirty = false;
        cs = next;
        if (kSkipSearch) cs_end = cs < I ? __ldg(pos1 + cs + 1) : INT_MAX;
        ka = long_slice(cs);
        if (kComp && ka) clear_cmp();
    };

    PosRows fw, sw;  // fiber ends (in entries) and slice ends (in fibers)
    fw.load(f0, F, pos2, lane);
    sw.load(s0, I, pos1, lane);
    for (int32_t pb = p0; pb < p1; pb += 32) {
        const int cnt = (p1 - pb) < 32 ? (p1 - pb) : 32;
        const bool valid = lane < cnt;
        const int32_t my_k = valid ? ld_stream(crd2 + pb + lane) : 0;
        const AT my_v = valid ? (AT)ld_stream(vals + pb + lane) : (AT)0;
        const int32_t my_f = fw.find(pb + lane, valid, F, pos2, lane);
        const int32_t nf = __shfl_sync(0xffffffffu, my_f, cnt - 1);
        // every entry of the window lies at or after slice cs, so when the last one lies
        // before cs_end they all lie in slice cs
        const int32_t my_sl = kSkipSearch && nf < cs_end ? cs : sw.find(my_f, valid, I, pos1, lane);
        const int32_t my_j = valid ? __ldg(crd1 + my_f) : 0;
        __syncwarp();
        s_j[lane] = my_j;
        s_k[lane] = my_k;
        s_sl[lane] = my_sl;
        s_v[lane] = my_v;
        __syncwarp();
        const int32_t ns = __shfl_sync(0xffffffffu, my_sl, cnt - 1);
        if (nf != fw.rw) fw.load(nf, F, pos2, lane);
        if (ns != sw.rw) sw.load(ns, I, pos1, lane);
        int a = 0;
        while (a < cnt) {  // segments of entries that share a slice
            const int32_t seg = s_sl[a];
            const unsigned other = __ballot_sync(0xffffffffu, valid && lane >= a && my_sl != seg);
            const int bnd = other ? __ffs(other) - 1 : cnt;
            if (seg != cs) finish_to(seg);
#pragma unroll 1
            for (int t0 = a; t0 < bnd; t0 += NPG * U) {
                XVec<VT, EPL> cv[U], dv[U];  // bfloat16 stays packed until the multiply
                AT v[U];
                if (t0 + NPG * U <= bnd) {  // every entry of the step lies in the segment
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int j = t0 + u * NPG + gi;
                        v[u] = s_v[j];
                        if (active) {
                            cv[u].load(reinterpret_cast<const VT *>(Cl + (uint64_t)(uint32_t)s_j[j] * ldc_b));
                            dv[u].load(reinterpret_cast<const VT *>(Dl + (uint64_t)(uint32_t)s_k[j] * ldd_b));
                        } else {
                            cv[u].clear();
                            dv[u].clear();
                        }
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int j = t0 + u * NPG + gi;
                        v[u] = j < bnd ? s_v[j] : (AT)0;
                        if (active && j < bnd) {
                            cv[u].load(reinterpret_cast<const VT *>(Cl + (uint64_t)(uint32_t)s_j[j] * ldc_b));
                            dv[u].load(reinterpret_cast<const VT *>(Dl + (uint64_t)(uint32_t)s_k[j] * ldd_b));
                        } else {
                            cv[u].clear();
                            dv[u].clear();
                        }
                    }
                }
                if (!kComp || !ka) {
#pragma unroll
                    for (int u = 0; u < U; ++u) {
#pragma unroll
                        for (int e = 0; e < EPL; ++e) acc[e] = fma(v[u] * (AT)cv[u].at(e), (AT)dv[u].at(e), acc[e]);
                    }
                } else {
                    // the step's U entries summed locally, then added to the running sum with
                    // Kahan's compensation
#pragma unroll
                    for (int e = 0; e < EPL; ++e) {
                        AT loc = (AT)0;
#pragma unroll
                        for (int u = 0; u < U; ++u) loc = fma(v[u] * (AT)cv[u].at(e), (AT)dv[u].at(e), loc);
                        const AT y = loc - cmp[32 * e];
                        const AT t = acc[e] + y;
                        cmp[32 * e] = (t - acc[e]) - y;
                        acc[e] = t;
                    }
                }
            }
            dirty = true;
            a = bnd;
        }
    }
    // slices cs .. s1-1 have their last fiber inside this piece
    if (cs < s1) finish_to(s1);
    // the piece may end inside slice s1: its partial is a binary64 carry
    if (carry_row) {
        const bool has = dirty && cs == s1 && s1 < I;
        AT t[EPL];
        warp_total(t);
        if (lane == 0 && blockIdx.y == 0) carry_row[c] = has ? s1 : -1;
        if (has && gi == 0 && active) {
#pragma unroll
            for (int e = 0; e < EPL; ++e) carry_val[c * R + col + e] = (double)t[e];
        }
    }
}

template <typename VT, int EPL, int G>
static spd_status launch_mttkrp_g(const spd_csf3 *B, const void *C, int64_t ldc, const void *D, int64_t ldd,
                                  int64_t R, void *A, int64_t lda, int split, const Tuning &tn, void *ws,
                                  cudaStream_t st) {
    using OT = typename Traits<VT>::out;
    const int threads = tn.block_threads;
    const int wpb = threads / 32;
    const size_t smem = (size_t)wpb * mttkrp_warp_smem<VT>(EPL);
    const int64_t ctiles = ceil_div(R, G * EPL);
    const uint32_t ldc_b = (uint32_t)(ldc * (int64_t)sizeof(VT)), ldd_b = (uint32_t)(ldd * (int64_t)sizeof(VT));
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
        spmttkrp_warp_kernel<VT, EPL, G><<<grid, threads, smem, st>>>(
            B->dim0, B->nfib, B->pos1, B->crd1, B->pos2, B->crd2, v, cc, ldc_b, dd, ldd_b, R, aa, lda, nullptr,
            nullptr, nullptr, 0, P, nullptr, nullptr);
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
    spmttkrp_warp_kernel<VT, EPL, G><<<grid, threads, smem, st>>>(
        B->dim0, B->nfib, B->pos1, B->crd1, B->pos2, B->crd2, v, cc, ldc_b, dd, ldd_b, R, aa, lda, pfib, ppos, psl,
        Lw.npieces, 0, crow, cval);
    if ((s = check_launch("spmttkrp_warp_kernel(nnz)"))) return s;
    return launch_carry_fixup<OT>(Lw.npieces, R, crow, cval, reinterpret_cast<int32_t *>(w + Lw.chunk_row),
                                  reinterpret_cast<double *>(w + Lw.chunk_val), aa, lda, st);
}

template <typename VT, int EPL>
static spd_status launch_mttkrp_epl(const spd_csf3 *B, const void *C, int64_t ldc, const void *D, int64_t ldd,
                                    int64_t R, void *A, int64_t lda, int split, const Tuning &tn, void *ws,
                                    cudaStream_t st) {
    const int64_t lanes = ceil_div(R > 0 ? R : 1, EPL);
    if (lanes <= 4) return launch_mttkrp_g<VT, EPL, 4>(B, C, ldc, D, ldd, R, A, lda, split, tn, ws, st);
    if (lanes <= 8) return launch_mttkrp_g<VT, EPL, 8>(B, C, ldc, D, ldd, R, A, lda, split, tn, ws, st);
    if (lanes <= 16) return launch_mttkrp_g<VT, EPL, 16>(B, C, ldc, D, ldd, R, A, lda, split, tn, ws, st);
    return launch_mttkrp_g<VT, EPL, 32>(B, C, ldc, D, ldd, R, A, lda, split, tn, ws, st);
}

template <typename VT>
static spd_status launch_mttkrp(const spd_csf3 *B, const void *C, int64_t ldc, const void *D, int64_t ldd, int64_t R,
                                void *A, int64_t lda, int split, const Tuning &tn, void *ws, cudaStream_t st) {
    using OT = typename Traits<VT>::out;
    constexpr int V = 16 / sizeof(VT) < 16 / sizeof(OT) ? 16 / sizeof(VT) : 16 / sizeof(OT);  // one 16-byte vector
    const bool vec = R % V == 0 && ldc % V == 0 && ldd % V == 0 && lda % V == 0 && aligned(C, 16) && aligned(D, 16) &&
                     aligned(A, 16);
    if (vec) return launch_mttkrp_epl<VT, V>(B, C, ldc, D, ldd, R, A, lda, split, tn, ws, st);
    return launch_mttkrp_epl<VT, 1>(B, C, ldc, D, ldd, R, A, lda, split, tn, ws, st);
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
    if ((uint64_t)ldc * dtype_size(factor_type) > UINT32_MAX || (uint64_t)ldd * dtype_size(factor_type) > UINT32_MAX)
        return fail(SPD_ERR_SHAPE, "C or D row stride exceeds 4 GiB");
    Tuning tn;
    if ((s = read_tune(tune, &tn))) return s;
    split = resolve_split(split);
    if (split != SPD_SPLIT_ROW && split != SPD_SPLIT_NNZ) return fail(SPD_ERR_ARG, "unknown split %d", split);
    WsLayout Lw = layout_mttkrp(B->nfib, B->nnz, split, tn.unit_items, R);
    if ((s = check_ws(Lw, ws, ws_bytes))) return s;
    cudaStream_t st = as_stream(stream);
    if ((s = checked_csf3(B, "B", st))) return s;
    if (B->dim0 == 0 || R == 0) return SPD_OK;
    switch (B->vtype) {
        case SPD_F64: s = launch_mttkrp<double>(B, C, ldc, D, ldd, R, A, lda, split, tn, ws, st); break;
        case SPD_F32: s = launch_mttkrp<float>(B, C, ldc, D, ldd, R, A, lda, split, tn, ws, st); break;
        case SPD_BF16: s = launch_mttkrp<__nv_bfloat16>(B, C, ldc, D, ldd, R, A, lda, split, tn, ws, st); break;
        default: return fail(SPD_ERR_DTYPE, "unknown value type %d", B->vtype);
    }
    return checked_finish(s, "spd_spmttkrp", st);
}
