// spd_spmv.cu -- SpMV y(i) = A(i,j) * x(j) and SpTTV A(i,j) = B(i,j,k) * c(k)
// (Section VI-A). SpTTV is the same computation over B's level 3: every fiber (i,j)
// is one output entry (the output keeps B's (i,j) structure, Section V-B).
//
// One thread block consumes one piece of the flattened coordinate tree, tile by tile:
//   1. each row whose end item falls in the tile sets that item's bit in a shared
//      bitmap of the tile (item index = nonzeros before the row end + earlier row
//      ends); a popcount prefix over the bitmap words gives, for any item, the number
//      of row ends before it, i.e. where the merge path crosses that item. The tile's
//      products vals[p] * x[crd[p]] are computed with coalesced crd/vals loads and x
//      gathers into shared memory;
//   2. every thread takes IPT consecutive items of the tile (its start row is one
//      popcount away), sums products and writes the rows it completes;
//   3. a block-wide segmented scan hands each thread the partial sum of the row it
//      started in, and carries the open row into the next tile (compensated when a
//      row spans tiles, i.e. is longer than one tile).
// Row split: piece c = rows [floor(c n/P), floor((c+1) n/P)) (the universe partition of
// the generated code in Section IV-C). Nnz split: pieces of equal item count from the
// partition array; the partial row at each piece end goes to a binary64 carry that a
// fix-up kernel adds to the row (the reduction into the output of Section II-D).
#include "spd_internal.cuh"

namespace spd {

constexpr int kSpmvWarpIPT = 8;  // items per lane of a warp tile

// Fault word of the kernels in this file (see kFaultBulkWait).
static __device__ unsigned int g_spmv_fault;

spd_status take_device_faults(unsigned int *flags) {
    unsigned int h = 0;
    const unsigned int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&h, g_spmv_fault, sizeof(h));
    if (e == cudaSuccess && h) e = cudaMemcpyToSymbol(g_spmv_fault, &zero, sizeof(zero));
    if (e != cudaSuccess) return fail(SPD_ERR_CUDA, "fault word: %s", cudaGetErrorString(e));
    *flags = h;
    return SPD_OK;
}

// Diagnostic of the bounded wait: one thread arms an mbarrier for 16 bytes of bulk copies
// that are never issued and waits for them with the wait the warp-tile kernels use. The
// wait gives up after kWaitLimitNs and records kFaultBulkWait in the fault word, as a
// stalled copy would; the kernel touches no memory but its own shared memory and ends
// with no copy in flight.
__global__ void bounded_wait_probe_kernel() {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar);
        mbar_fence_init();
        mbar_arrive_expect(&bar, 16);
        mbar_wait(&bar, 0, &g_spmv_fault);
    }
}

// Shared-memory index with one padding word per 32 entries: each thread consumes IPT
// consecutive entries, so without the skew a warp's 32 threads would fall on only
// 32/IPT banks.
__device__ __forceinline__ int skew(int i) { return i + (i >> 5); }

// Resident blocks per SM: 8 for bfloat16 values; 6 otherwise, which leaves the binary32
// and binary64 tiles enough registers not to spill (measured faster on power-law rows).
template <typename VT, int NT, int IPT>
__global__ void __launch_bounds__(NT, sizeof(VT) == 2 ? 8 : 6) spmv_tile_kernel(
    int64_t n, const int32_t *__restrict__ pos, const int32_t *__restrict__ crd, const VT *__restrict__ vals,
    const VT *__restrict__ x, typename Traits<VT>::out *__restrict__ y,
    const int32_t *__restrict__ prow, const int32_t *__restrict__ ppos,  // nnz split
    int64_t P, int64_t nouter, const int32_t *__restrict__ outer,         // row split
    int32_t *__restrict__ carry_row, double *__restrict__ carry_val) {
    using AT = typename Traits<VT>::acc;
    using OT = typename Traits<VT>::out;
    constexpr int TILE = NT * IPT;
    constexpr int NW = NT / 32;
    constexpr int NWORDS = TILE / 32;  // bitmap words of a tile
    constexpr unsigned FULL = 0xffffffffu;
    static_assert(32 % IPT == 0 && NWORDS == 64, "a thread's items share one bitmap word; warp 0 scans 64 words");
    __shared__ uint32_t s_bits[NWORDS];     // bit k of the tile: item k is a row end
    __shared__ int32_t s_wpre[NWORDS + 1];  // row ends before each word; [NWORDS] = all
    __shared__ AT s_prod[TILE + TILE / 32];
    __shared__ AT s_wv[NW];
    __shared__ int s_wf[NW];
    __shared__ AT s_tv;
    __shared__ int s_tf;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t c = blockIdx.x;
    PieceBounds b;
    if (prow) {
        b = nnz_piece(c, prow, ppos);
    } else if (outer) {
        // SpTTV row split: slices [floor(c I/P), floor((c+1) I/P)) and, by image, their fibers
        int64_t i0 = (c * nouter) / P, i1 = ((c + 1) * nouter) / P;
        b.r0 = __ldg(outer + i0);
        b.r1 = __ldg(outer + i1);
        b.p0 = __ldg(pos + b.r0);
        b.p1 = __ldg(pos + b.r1);
    } else {
        b = row_piece(c, P, n, pos);
    }
    int32_t r = b.r0, p = b.p0;
    AT carry_hi = 0, carry_lo = 0;  // partial of row r accumulated over earlier tiles
    for (int w = tid; w < NWORDS; w += NT) s_bits[w] = 0u;  // later tiles clear it at their end
    __syncthreads();

    while (true) {
        const int64_t rem_rows = (int64_t)b.r1 - r, rem_nnz = (int64_t)b.p1 - p;
        if (rem_rows + rem_nnz == 0) break;
        const int nr = (int)(rem_rows < TILE ? rem_rows : TILE);
        const int items = (int)((rem_rows + rem_nnz) < TILE ? (rem_rows + rem_nnz) : TILE);
        // Binary32 values: crd and vals of the tile's nonzeros are loaded before its row
        // ends are known, so that their latency overlaps the row-end phase. The tile holds
        // at most jmax nonzeros; the positions past its actual count (one per row end in
        // the tile) are loaded again by the next tile, and x is gathered only for the
        // actual ones. Measured 2.6-6.4% faster in binary32; the other value types spill
        // with the loads held across the phase, so they load after it.
        constexpr bool kEarly = sizeof(VT) == 4;
        int32_t cc[IPT];
        AT vv[IPT];
        if (kEarly) {
            const int jmax = (int)(rem_nnz < TILE ? rem_nnz : TILE);
#pragma unroll
            for (int k = 0; k < IPT; ++k) {
                const int q = tid + k * NT;
                cc[k] = q < jmax ? ld_stream(crd + p + q) : 0;
                vv[k] = q < jmax ? (AT)ld_stream(vals + p + q) : (AT)0;
            }
        }
        // row ends of the tile, NT rows at a time: a further chunk only while the last row
        // of the previous one still ended inside the tile (a tile of power-law rows holds
        // about a hundred row ends; a run of empty rows can hold up to TILE)
        if (nr == 0) __syncthreads();
        for (int q0 = 0; q0 < nr; q0 += NT) {
            const int q = q0 + tid;
            bool more = false;
            if (q < nr) {
                const int64_t e = (int64_t)ld_stream(pos + r + 1 + q) - p + q;  // item index of row q's end
                if (e < items) {
                    atomicOr(&s_bits[e >> 5], 1u << (e & 31));
                    more = q == q0 + NT - 1;
                }
            }
            if (!__syncthreads_or(more)) break;
        }
        if (wid == 0) {  // exclusive popcount prefix of the 64 words, two per lane
            const int c0 = __popc(s_bits[2 * lane]), c1 = __popc(s_bits[2 * lane + 1]);
            int inc = c0 + c1;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int t = __shfl_up_sync(FULL, inc, off);
                if (lane >= off) inc += t;
            }
            s_wpre[2 * lane] = inc - c0 - c1;
            s_wpre[2 * lane + 1] = inc - c1;
            if (lane == 31) s_wpre[NWORDS] = inc;
        }
        __syncthreads();
        const int ic = s_wpre[NWORDS];  // row ends in the tile
        const int jc = items - ic;
        // products of the tile's nonzeros: coalesced crd/vals (unless loaded early), gathered x
        if (!kEarly) {
#pragma unroll
            for (int k = 0; k < IPT; ++k) {
                const int q = tid + k * NT;
                cc[k] = q < jc ? ld_stream(crd + p + q) : 0;
                vv[k] = q < jc ? (AT)ld_stream(vals + p + q) : (AT)0;
            }
        }
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const int q = tid + k * NT;
            if (q < jc) s_prod[skew(q)] = vv[k] * (AT)ld_gather(x + cc[k]);
        }
        __syncthreads();
        // this thread's IPT items of the tile
        const int k0 = tid * IPT < items ? tid * IPT : items;
        const int k1 = k0 + IPT < items ? k0 + IPT : items;
        const int word = k0 < TILE ? (k0 >> 5) : NWORDS - 1;
        const int sh = k0 & 31;
        const uint32_t wbits = s_bits[word];
        const uint32_t mine = k0 < TILE ? wbits >> sh : 0u;  // bit k: item k0 + k is a row end
        const int i0 = s_wpre[word] + __popc(sh ? (wbits & ((1u << sh) - 1u)) : 0u);
        // the thread's items in order, without branches: a row end writes the row's running
        // sum (the first one of the thread is completed by the scan below)
        const uint32_t valid = (k1 - k0 >= IPT) ? ((1u << IPT) - 1u) : ((1u << (k1 - k0)) - 1u);
        const uint32_t ends = mine & valid, nzs = valid & ~mine;
        AT acc = 0, first_val = 0;
        int i = i0;
        bool first = true;
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const bool isend = (ends >> k) & 1u;
            const AT pv = ((nzs >> k) & 1u) ? s_prod[skew(k0 + k - i)] : (AT)0;
            acc += pv;
            if (isend) {
                if (first) first_val = acc;
                else y[r + i] = (OT)acc;
                first = false;
                acc = 0;
                ++i;
            }
        }
        const int first_row = first ? -1 : i0;
        // block-wide segmented inclusive scan of (ended-a-row, tail partial)
        int f = first_row >= 0;
        AT v = acc;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int pf = __shfl_up_sync(FULL, f, off);
            AT pv = __shfl_up_sync(FULL, v, off);
            if (lane >= off) {
                if (!f) v += pv;
                f |= pf;
            }
        }
        if (lane == 31) {
            s_wf[wid] = f;
            s_wv[wid] = v;
        }
        __syncthreads();
        // segmented exclusive scan of the warps' (flag, partial) with shuffles: lane w of
        // every warp holds warp w's pair, and each warp takes the prefix of the warps before it
        AT wp_v = 0;
        int wp_f = 0;
        {
            int sf = lane < NW ? s_wf[lane] : 0;
            AT sv = lane < NW ? s_wv[lane] : (AT)0;
#pragma unroll
            for (int off = 1; off < NW; off <<= 1) {
                const int pf = __shfl_up_sync(FULL, sf, off);
                const AT pv = __shfl_up_sync(FULL, sv, off);
                if (lane >= off) {
                    if (!sf) sv += pv;
                    sf |= pf;
                }
            }
            const AT iv = __shfl_sync(FULL, sv, (wid + 31) & 31);
            const int iff = __shfl_sync(FULL, sf, (wid + 31) & 31);
            if (wid > 0) {
                wp_v = iv;
                wp_f = iff;
            }
        }
        const AT incl_v = f ? v : wp_v + v;
        const int incl_f = f | wp_f;
        AT ev = __shfl_up_sync(FULL, incl_v, 1);
        int ef = __shfl_up_sync(FULL, incl_f, 1);
        if (lane == 0) {
            ev = wp_v;
            ef = wp_f;
        }
        if (tid == NT - 1) {
            s_tv = incl_v;
            s_tf = incl_f;
        }
        if (first_row >= 0) {
            AT tot = first_val + ev;
            if (!ef) {  // the tile's first completed row is row r: add what earlier tiles carried
                AT hi = carry_hi, lo = carry_lo;
                comp_add(hi, lo, tot);
                tot = hi + lo;
            }
            y[r + first_row] = (OT)tot;
        }
        __syncthreads();
        const AT tv = s_tv;
        const int tf = s_tf;
        if (tf) {
            carry_hi = tv;
            carry_lo = 0;
        } else {
            comp_add(carry_hi, carry_lo, tv);
        }
        for (int w = tid; w < NWORDS; w += NT) s_bits[w] = 0u;  // every read of the bitmap is done
        r += ic;
        p += jc;
        __syncthreads();
    }
    if (carry_row && tid == 0) {
        // the piece ends inside row r1: hand its partial to the fix-up when it is non-empty
        int32_t start = b.r1 < n ? __ldg(pos + b.r1) : b.p1;
        if (start < b.p0) start = b.p0;
        bool has = b.p1 > start;
        carry_row[c] = has ? b.r1 : -1;
        carry_val[c] = has ? (double)carry_hi + (double)carry_lo : 0.0;
    }
}

// ------------------------------------------------------------------ warp-tile form
//
// One warp consumes one piece, tile by tile (T = 32 * IPT items), with no block-wide
// barrier:
//   * the row ends of the tile set bits in a per-warp bitmap (the ends of the next 64
//     rows are fetched one tile ahead, two per lane; a run of more row ends is loaded
//     together); a warp scan of the popcounts of each lane's IPT bits places every lane
//     on its first row;
//   * the tile's window of crd (the next T coordinates) arrives in shared memory by a
//     1-D bulk copy (TMA) issued one tile ahead into a double buffer and completing on an
//     mbarrier per buffer (bounded wait); vals are streamed with plain coalesced loads
//     issued together with the gathers of x, so one latency covers both;
//   * the products vals * x[crd] go to a skewed per-warp array; each lane sums its IPT
//     items in order without branches; a segmented warp scan hands each lane the
//     partial of the row it started in, and the open row is carried into the next tile
//     with compensated addition.
// crd not 16-byte aligned takes plain coalesced loads into the same buffers.
template <typename VT, int IPT>
struct WarpSpmvLayout {
    using AT = typename Traits<VT>::acc;
    static constexpr int T = 32 * IPT;
    static constexpr int BUF = T + 16;  // staged elements: the window plus its 16-byte alignment slack
    static constexpr size_t off_bar = 0;                                    // 2 mbarriers
    static constexpr size_t off_bits = 16;                                  // IPT words
    static constexpr size_t off_crd = (off_bits + 4 * IPT + 15) / 16 * 16;  // [2][BUF] int32
    static constexpr size_t off_val = off_crd + 2 * BUF * 4;                // [2][BUF] VT
    static constexpr size_t off_prod = (off_val + 2 * BUF * sizeof(VT) + 15) / 16 * 16;  // [T + T/32] AT
    static constexpr size_t bytes = (off_prod + (T + T / 32) * sizeof(AT) + 15) / 16 * 16;  // per warp
};

template <typename VT, int IPT, bool BULK>
__global__ void __launch_bounds__(256) spmv_warp_kernel(
    int64_t n, int64_t nnz, const int32_t *__restrict__ pos, const int32_t *__restrict__ crd,
    const VT *__restrict__ vals, const VT *__restrict__ x, typename Traits<VT>::out *__restrict__ y,
    const int32_t *__restrict__ prow, const int32_t *__restrict__ ppos, int64_t npieces,  // nnz split
    int64_t P, int64_t nouter, const int32_t *__restrict__ outer,                         // row split
    int32_t *__restrict__ carry_row, double *__restrict__ carry_val) {
    using AT = typename Traits<VT>::acc;
    using OT = typename Traits<VT>::out;
    using Lay = WarpSpmvLayout<VT, IPT>;
    constexpr int T = Lay::T;
    constexpr int LPW = 32 / IPT;  // lanes per bitmap word
    constexpr unsigned FULL = 0xffffffffu;
    constexpr uint32_t MASK = IPT == 32 ? FULL : ((1u << IPT) - 1u);
    static_assert(32 % IPT == 0 && IPT >= 2, "a lane's items share one bitmap word");
    extern __shared__ __align__(16) unsigned char spmv_smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid;
    if (c >= (prow ? npieces : P)) return;  // whole warp
    unsigned char *ws = spmv_smem + (size_t)wid * Lay::bytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(ws + Lay::off_bar);
    uint32_t *bits = reinterpret_cast<uint32_t *>(ws + Lay::off_bits);
    int32_t *s_crd = reinterpret_cast<int32_t *>(ws + Lay::off_crd);
    VT *s_val = reinterpret_cast<VT *>(ws + Lay::off_val);
    AT *s_prod = reinterpret_cast<AT *>(ws + Lay::off_prod);
    constexpr int EV = (int)(16 / sizeof(VT));  // values per 16 bytes

    PieceBounds b;
    if (prow) {
        b = nnz_piece(c, prow, ppos);
    } else if (outer) {  // SpTTV row split: slices [floor(c I/P), floor((c+1) I/P)) and their fibers
        const int64_t i0 = (c * nouter) / P, i1 = ((c + 1) * nouter) / P;
        b.r0 = __ldg(outer + i0);
        b.r1 = __ldg(outer + i1);
        b.p0 = __ldg(pos + b.r0);
        b.p1 = __ldg(pos + b.r1);
    } else {
        b = row_piece(c, P, n, pos);
    }

    // bulk copies of crd and vals [ps, ps + T) (clamped to nnz) into buffer bi, by lane 0:
    // each starts at the 16-byte boundary below ps and, at the array's end, stops at the
    // last 16-byte boundary; the few elements after it are loaded by the lanes after the wait
    auto span = [&](int32_t ps, int E, int64_t &a, int64_t &e, int64_t &end) {
        end = (int64_t)ps + T < nnz ? (int64_t)ps + T : nnz;
        a = ps & ~(int64_t)(E - 1);
        e = (end + E - 1) & ~(int64_t)(E - 1);
        if (e > nnz) e = end & ~(int64_t)(E - 1);
        if (e < a) e = a;
    };
    auto issue = [&](int bi, int32_t ps) {
        int64_t ac, ec, av, ev, end;
        span(ps, 4, ac, ec, end);
        span(ps, EV, av, ev, end);
        const uint32_t cb = (uint32_t)((ec - ac) * 4), vb = (uint32_t)((ev - av) * sizeof(VT));
        mbar_arrive_expect(&bar[bi], cb + vb);
        if (cb) bulk_g2s(s_crd + bi * Lay::BUF, crd + ac, cb, &bar[bi]);
        if (vb) bulk_g2s(s_val + bi * Lay::BUF, vals + av, vb, &bar[bi]);
    };

    int32_t r = b.r0, p = b.p0;
    AT carry_hi = 0, carry_lo = 0;  // partial of row r accumulated over earlier tiles
    int buf = 0;
    uint32_t phase = 0;     // bit i: parity of the next completion of buffer i
    uint32_t inflight = 0;  // bit i: a bulk copy into buffer i is outstanding
    if (BULK) {
        if (lane == 0) {
            mbar_init(&bar[0]);
            mbar_init(&bar[1]);
            mbar_fence_init();
        }
        __syncwarp();
        if ((int64_t)b.r1 - r + b.p1 - p > 0) {
            if (lane == 0) issue(0, p);
            inflight = 1u;
        }
    }
    // ends of rows r .. r+63, two per lane (the next tile's are fetched one tile ahead)
    int32_t rend0 = (int64_t)r + lane < n ? ld_stream(pos + r + 1 + lane) : INT_MAX;
    int32_t rend1 = (int64_t)r + 32 + lane < n ? ld_stream(pos + r + 33 + lane) : INT_MAX;

    while (true) {
        const int64_t rem_rows = (int64_t)b.r1 - r, rem_nnz = (int64_t)b.p1 - p;
        if (rem_rows + rem_nnz == 0) break;
        const int items = (int)(rem_rows + rem_nnz < T ? rem_rows + rem_nnz : T);
        const int nr = (int)(rem_rows < items ? rem_rows : items);  // rows that may end in the tile
        if (lane < IPT) bits[lane] = 0u;
        __syncwarp();
        {
            // item index of row r + q's end (rows past n read as INT_MAX: saturate)
            auto item_of = [&](int32_t end_pos, int q) {
                const int64_t e = (int64_t)end_pos - p + q;
                return e < items ? (int)e : INT_MAX;
            };
            int e = item_of(rend0, lane);
            if (lane < nr && e < items) atomicOr(&bits[e >> 5], 1u << (e & 31));
            e = item_of(rend1, 32 + lane);
            if (32 + lane < nr && e < items) atomicOr(&bits[e >> 5], 1u << (e & 31));
            if (nr > 64 && __shfl_sync(FULL, e, 31) < items) {
                // more than 64 rows end in the tile (a run of short or empty rows): the
                // remaining row ends, loaded together, 32 at a time per lane group
                for (int q0 = 64; q0 < nr; q0 += 128) {
                    int32_t me[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int q = q0 + 32 * k + lane;
                        me[k] = q < nr ? ld_stream(pos + r + 1 + q) : INT_MAX;
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int q = q0 + 32 * k + lane;
                        e = q < nr ? item_of(me[k], q) : INT_MAX;
                        if (e < items) atomicOr(&bits[e >> 5], 1u << (e & 31));
                    }
                    if (__shfl_sync(FULL, e, 31) >= items) break;
                }
            }
        }
        __syncwarp();
        const uint32_t mine = (bits[lane / LPW] >> ((lane % LPW) * IPT)) & MASK;
        int incl = __popc(mine);
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int t = __shfl_up_sync(FULL, incl, off);
            if (lane >= off) incl += t;
        }
        const int i0 = incl - __popc(mine);          // row ends before this lane's first item
        const int ic = __shfl_sync(FULL, incl, 31);  // row ends in the tile
        const int jc = items - ic;                   // nonzeros in the tile
        const int32_t rn = r + ic, pn = p + jc;
        const bool more = (int64_t)b.r1 - rn + b.p1 - pn > 0;
        rend0 = (int64_t)rn + lane < n ? ld_stream(pos + rn + 1 + lane) : INT_MAX;
        rend1 = (int64_t)rn + 32 + lane < n ? ld_stream(pos + rn + 33 + lane) : INT_MAX;

        // element p + q of the tile sits at wc[oc + q] / wv[ov + q]
        const int32_t *wc = s_crd + buf * Lay::BUF;
        const VT *wv = s_val + buf * Lay::BUF;
        int oc = 0, ov = 0;
        if (BULK) {
            if (more) {  // the other buffer was last read before the previous tile's final __syncwarp
                if (lane == 0) {
                    fence_proxy_async();
                    issue(buf ^ 1, pn);
                }
                inflight |= 1u << (buf ^ 1);
            }
            const bool ok = mbar_wait(&bar[buf], (phase >> buf) & 1u, &g_spmv_fault);
            inflight &= ~(1u << buf);
            phase ^= 1u << buf;
            if (!__all_sync(FULL, ok)) {  // give up (fault word set); wait once more for our copies
                if ((inflight >> (buf ^ 1)) & 1u) mbar_wait(&bar[buf ^ 1], (phase >> (buf ^ 1)) & 1u, &g_spmv_fault);
                return;
            }
            int64_t ac, ec, av, ev, end;
            span(p, 4, ac, ec, end);
            span(p, EV, av, ev, end);
            oc = (int)(p - ac);
            ov = (int)(p - av);
            // the last elements of the arrays that the bulk copies could not cover
            if (lane < end - ec) s_crd[buf * Lay::BUF + (int)(ec - ac) + lane] = ld_stream(crd + ec + lane);
            if (lane < end - ev) s_val[buf * Lay::BUF + (int)(ev - av) + lane] = vals[ev + lane];
        } else {
            int32_t *dc = s_crd + buf * Lay::BUF;
            VT *dv = s_val + buf * Lay::BUF;
#pragma unroll
            for (int k = 0; k < IPT; ++k) {
                const int q = lane + 32 * k;
                if (q < jc) {
                    dc[q] = ld_stream(crd + p + q);
                    dv[q] = vals[p + q];
                }
            }
        }
        __syncwarp();
        // products of the tile's nonzeros (coalesced reads of the window, gathered x,
        // all of a lane's gathers issued before any is used)
        {
            AT xv[IPT];
#pragma unroll
            for (int k = 0; k < IPT; ++k) {
                const int q = lane + 32 * k;
                xv[k] = q < jc ? ld_gather(x + wc[oc + q]) : (AT)0;
            }
#pragma unroll
            for (int k = 0; k < IPT; ++k) {
                const int q = lane + 32 * k;
                if (q < jc) s_prod[skew(q)] = to_acc(wv[ov + q]) * xv[k];
            }
        }
        __syncwarp();
        // this lane's IPT items of the tile, in order, without branches: a row end writes
        // the running sum of the row (the first one of the lane is completed by the scan)
        const int k0 = lane * IPT;
        const uint32_t valid = k0 >= items ? 0u : (items - k0 >= IPT ? MASK : ((1u << (items - k0)) - 1u));
        const uint32_t ends = mine & valid;
        const int nz = __popc(valid & ~ends);  // nonzeros of this lane
        const int j0 = k0 - i0;
        AT acc = 0, first_val = 0;
        int i = i0;
        bool first = true;
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const bool isend = (ends >> k) & 1u;
            const bool isnz = ((valid & ~ends) >> k) & 1u;
            const int jj = j0 + k - (i - i0);  // nonzero index of item k when it is one
            const AT pv = isnz ? s_prod[skew(jj)] : (AT)0;
            acc += pv;
            if (isend) {
                if (first) first_val = acc;
                else y[r + i] = (OT)acc;
                first = false;
                acc = 0;
                ++i;
            }
        }
        (void)nz;
        const int first_row = first ? -1 : i0;
        // segmented inclusive scan of (ended a row, tail partial) over the warp
        int f = first_row >= 0;
        AT v = acc;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int pf = __shfl_up_sync(FULL, f, off);
            const AT pv = __shfl_up_sync(FULL, v, off);
            if (lane >= off) {
                if (!f) v += pv;
                f |= pf;
            }
        }
        AT ev = __shfl_up_sync(FULL, v, 1);
        int ef = __shfl_up_sync(FULL, f, 1);
        if (lane == 0) {
            ev = 0;
            ef = 0;
        }
        if (first_row >= 0) {
            AT tot = first_val + ev;
            if (!ef) {  // the tile's first completed row is row r: add what earlier tiles carried
                AT hi = carry_hi, lo = carry_lo;
                comp_add(hi, lo, tot);
                tot = hi + lo;
            }
            y[r + first_row] = (OT)tot;
        }
        const AT tv = __shfl_sync(FULL, v, 31);
        if (__shfl_sync(FULL, f, 31)) {
            carry_hi = tv;
            carry_lo = 0;
        } else {
            comp_add(carry_hi, carry_lo, tv);
        }
        r = rn;
        p = pn;
        buf ^= 1;
        __syncwarp();  // every lane is done with this tile's buffers before they are refilled
    }
    if (carry_row && lane == 0) {
        // the piece ends inside row r1: hand its partial to the fix-up when it is non-empty
        int32_t start = b.r1 < n ? __ldg(pos + b.r1) : b.p1;
        if (start < b.p0) start = b.p0;
        const bool has = b.p1 > start;
        carry_row[c] = has ? b.r1 : -1;
        carry_val[c] = has ? (double)carry_hi + (double)carry_lo : 0.0;
    }
}

// Adds the binary64 carries of consecutive pieces that ended inside the same row to the
// value the completing piece wrote (one thread per run of pieces).
template <typename OT>
__global__ void carry_fixup_scalar_kernel(int64_t npieces, const int32_t *__restrict__ carry_row,
                                          const double *__restrict__ carry_val, OT *__restrict__ y) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= npieces) return;
    int32_t row = carry_row[c];
    if (row < 0) return;
    if (c > 0 && carry_row[c - 1] == row) return;
    double s = 0.0;  // the run in batches of 8 independent loads, summed in piece order
    for (int64_t d = c; d < npieces; d += 8) {
        int32_t tag[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) tag[k] = d + k < npieces ? carry_row[d + k] : -1;
        double v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = tag[k] == row ? carry_val[d + k] : 0.0;
        bool more = true;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            more = more && tag[k] == row;
            if (more) s += v[k];
        }
        if (!more) break;
    }
    y[row] = (OT)((double)y[row] + s);
}

// Shared host path of SpMV (n rows of `pos`) and SpTTV (n = fibers, pos = pos2; the
// row split then partitions the nouter slices of `outer` = pos1). One warp per piece:
// the nnz split cuts the items into pieces of kSpmvTile, the row split into P row pieces.
template <typename VT, bool BULK>
static spd_status launch_spmv_warp(int64_t n, int64_t nnz, const int32_t *pos, const int32_t *crd, const void *vals,
                                   const void *x, void *y, int split, const Tuning &tn, int64_t nouter,
                                   const int32_t *outer, void *ws, cudaStream_t st) {
    using OT = typename Traits<VT>::out;
    using Lay = WarpSpmvLayout<VT, kSpmvWarpIPT>;
    constexpr int WPB = kSpmvThreads / 32;
    const size_t smem = (size_t)WPB * Lay::bytes;
    auto kern = spmv_warp_kernel<VT, kSpmvWarpIPT, BULK>;
    // The shared memory of binary64 tiles exceeds the 48 KiB default. The limit is an
    // attribute of the function in the current context (a process may use several GPUs
    // or recreate its context), so it is set on every such launch; the call is cheap.
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return fail(SPD_ERR_CUDA, "spmv_warp_kernel attribute: %s", cudaGetErrorString(e));
    }
    const VT *v = static_cast<const VT *>(vals);
    const VT *xx = static_cast<const VT *>(x);
    OT *yy = static_cast<OT *>(y);
    if (split == SPD_SPLIT_ROW) {
        int64_t P = tn.row_pieces;
        if (P <= 0) P = ceil_div(n + nnz, kSpmvTile);
        if (P < 1) P = 1;
        kern<<<(unsigned)ceil_div(P, WPB), kSpmvThreads, smem, st>>>(n, nnz, pos, crd, v, xx, yy, nullptr, nullptr, 0,
                                                                    P, nouter, outer, nullptr, nullptr);
        return check_launch("spmv_warp_kernel(row)");
    }
    WsLayout L = layout_spmv(n, nnz, split);
    char *w = static_cast<char *>(ws);
    int32_t *prow = reinterpret_cast<int32_t *>(w + L.part_row);
    int32_t *ppos = reinterpret_cast<int32_t *>(w + L.part_pos);
    int32_t *crow = reinterpret_cast<int32_t *>(w + L.carry_row);
    double *cval = reinterpret_cast<double *>(w + L.carry_val);
    spd_status s = launch_merge_partition(n, nnz, pos, kSpmvTile, L.npieces, prow, ppos, st);
    if (s) return s;
    kern<<<(unsigned)ceil_div(L.npieces, WPB), kSpmvThreads, smem, st>>>(n, nnz, pos, crd, v, xx, yy, prow, ppos,
                                                                        L.npieces, 0, 0, nullptr, crow, cval);
    s = check_launch("spmv_warp_kernel(nnz)");
    if (s) return s;
    carry_fixup_scalar_kernel<OT><<<(unsigned)ceil_div(L.npieces, 256), 256, 0, st>>>(L.npieces, crow, cval, yy);
    return check_launch("carry_fixup_scalar_kernel");
}

// The block-tile form: one thread block per piece (spmv_tile_kernel).
template <typename VT>
static spd_status launch_spmv_tile(int64_t n, int64_t nnz, const int32_t *pos, const int32_t *crd, const void *vals,
                              const void *x, void *y, int split, const Tuning &tn, int64_t nouter,
                              const int32_t *outer, void *ws, cudaStream_t st) {
    using OT = typename Traits<VT>::out;
    const VT *v = static_cast<const VT *>(vals);
    const VT *xx = static_cast<const VT *>(x);
    OT *yy = static_cast<OT *>(y);
    if (split == SPD_SPLIT_ROW) {
        int64_t P = tn.row_pieces;
        if (P <= 0) P = ceil_div(n + nnz, kSpmvTile);
        if (P < 1) P = 1;
        spmv_tile_kernel<VT, kSpmvThreads, kSpmvIPT><<<(unsigned)P, kSpmvThreads, 0, st>>>(
            n, pos, crd, v, xx, yy, nullptr, nullptr, P, nouter, outer, nullptr, nullptr);
        return check_launch("spmv_tile_kernel(row)");
    }
    WsLayout L = layout_spmv(n, nnz, split);
    char *w = static_cast<char *>(ws);
    int32_t *prow = reinterpret_cast<int32_t *>(w + L.part_row);
    int32_t *ppos = reinterpret_cast<int32_t *>(w + L.part_pos);
    int32_t *crow = reinterpret_cast<int32_t *>(w + L.carry_row);
    double *cval = reinterpret_cast<double *>(w + L.carry_val);
    spd_status s = launch_merge_partition(n, nnz, pos, kSpmvTile, L.npieces, prow, ppos, st);
    if (s) return s;
    spmv_tile_kernel<VT, kSpmvThreads, kSpmvIPT><<<(unsigned)L.npieces, kSpmvThreads, 0, st>>>(
        n, pos, crd, v, xx, yy, prow, ppos, 0, 0, nullptr, crow, cval);
    s = check_launch("spmv_tile_kernel(nnz)");
    if (s) return s;
    carry_fixup_scalar_kernel<OT><<<(unsigned)ceil_div(L.npieces, 256), 256, 0, st>>>(L.npieces, crow, cval, yy);
    return check_launch("carry_fixup_scalar_kernel");
}

template <typename VT>
static spd_status launch_spmv(int64_t n, int64_t nnz, const int32_t *pos, const int32_t *crd, const void *vals,
                              const void *x, void *y, int split, const Tuning &tn, int64_t nouter,
                              const int32_t *outer, void *ws, cudaStream_t st) {
    if (tn.form != 2) return launch_spmv_tile<VT>(n, nnz, pos, crd, vals, x, y, split, tn, nouter, outer, ws, st);
    if (aligned(crd, 16) && aligned(vals, 16))
        return launch_spmv_warp<VT, true>(n, nnz, pos, crd, vals, x, y, split, tn, nouter, outer, ws, st);
    return launch_spmv_warp<VT, false>(n, nnz, pos, crd, vals, x, y, split, tn, nouter, outer, ws, st);
}

static spd_status dispatch_spmv(int vtype, int64_t n, int64_t nnz, const int32_t *pos, const int32_t *crd,
                                const void *vals, const void *x, void *y, int split, const Tuning &tn,
                                int64_t nouter, const int32_t *outer, void *ws, cudaStream_t st) {
    switch (vtype) {
        case SPD_F64: return launch_spmv<double>(n, nnz, pos, crd, vals, x, y, split, tn, nouter, outer, ws, st);
        case SPD_F32: return launch_spmv<float>(n, nnz, pos, crd, vals, x, y, split, tn, nouter, outer, ws, st);
        case SPD_BF16:
            return launch_spmv<__nv_bfloat16>(n, nnz, pos, crd, vals, x, y, split, tn, nouter, outer, ws, st);
        default: return fail(SPD_ERR_DTYPE, "unknown value type %d", vtype);
    }
}

// Nnz-split SpMV with default tuning on a scratch area the caller already owns (laid out
// as layout_spmv describes); used by the entry point that allocates nothing.
spd_status spmv_nnz_on_scratch(const spd_csr *A, const void *x, void *y, void *scratch, cudaStream_t st) {
    Tuning tn;
    read_tune(nullptr, &tn);
    return dispatch_spmv(A->vtype, A->nrows, A->nnz, A->pos, A->crd, A->vals, x, y, SPD_SPLIT_NNZ, tn, 0, nullptr,
                         scratch, st);
}

}  // namespace spd

using namespace spd;

extern "C" {

spd_status spd_spmv(const spd_csr *A, const void *x, int x_type, void *y, int y_type, int split,
                    const spd_tune *tune, void *ws, size_t ws_bytes, void *stream) {
    spd_status s = check_csr(A, true);
    if (s) return s;
    if (x_type != A->vtype) return fail(SPD_ERR_DTYPE, "x type %d differs from the value type %d", x_type, A->vtype);
    if (y_type != result_type(A->vtype)) return fail(SPD_ERR_DTYPE, "y type %d; expected %d", y_type, result_type(A->vtype));
    if (A->ncols > 0 && !x) return fail(SPD_ERR_NULL, "x is NULL");
    if (A->nrows > 0 && !y) return fail(SPD_ERR_NULL, "y is NULL");
    if ((x && !aligned(x, dtype_size(x_type))) || (y && !aligned(y, dtype_size(y_type))))
        return fail(SPD_ERR_ALIGN, "x or y not aligned to its element size");
    Tuning tn;
    if ((s = read_tune(tune, &tn))) return s;
    split = resolve_split(split);
    if (split != SPD_SPLIT_ROW && split != SPD_SPLIT_NNZ) return fail(SPD_ERR_ARG, "unknown split %d", split);
    WsLayout L = layout_spmv(A->nrows, A->nnz, split);
    if ((s = check_ws(L, ws, ws_bytes))) return s;
    cudaStream_t st = as_stream(stream);
    if ((s = checked_csr(A, "A", st))) return s;
    if (A->nrows == 0) return SPD_OK;
    return checked_finish(
        dispatch_spmv(A->vtype, A->nrows, A->nnz, A->pos, A->crd, A->vals, x, y, split, tn, 0, nullptr, ws, st),
        "spd_spmv", st);
}

spd_status spd_fault_status(uint32_t *flags, void *stream) {
    if (!flags) return fail(SPD_ERR_NULL, "flags is NULL");
    cudaError_t e = cudaStreamSynchronize(as_stream(stream));
    if (e != cudaSuccess) return fail(SPD_ERR_CUDA, "spd_fault_status: %s", cudaGetErrorString(e));
    unsigned int f = 0;
    spd_status s = take_device_faults(&f);
    *flags = f;
    if (s) return s;
    return f ? fail(SPD_ERR_TIMEOUT, "a kernel's bounded wait for its bulk copies gave up (flags 0x%x)", f) : SPD_OK;
}

spd_status spd_probe_bounded_wait(void *stream) {
    bounded_wait_probe_kernel<<<1, 32, 0, as_stream(stream)>>>();
    return check_launch("bounded_wait_probe_kernel");
}

spd_status spd_spttv(const spd_csf3 *B, const void *c, int c_type, void *out_vals, int out_type, int split,
                     const spd_tune *tune, void *ws, size_t ws_bytes, void *stream) {
    spd_status s = check_csf3(B);
    if (s) return s;
    if (c_type != B->vtype) return fail(SPD_ERR_DTYPE, "c type %d differs from the value type %d", c_type, B->vtype);
    if (out_type != result_type(B->vtype)) return fail(SPD_ERR_DTYPE, "output type %d; expected %d", out_type, result_type(B->vtype));
    if (B->dim2 > 0 && !c) return fail(SPD_ERR_NULL, "c is NULL");
    if (B->nfib > 0 && !out_vals) return fail(SPD_ERR_NULL, "out_vals is NULL");
    if ((c && !aligned(c, dtype_size(c_type))) || (out_vals && !aligned(out_vals, dtype_size(out_type))))
        return fail(SPD_ERR_ALIGN, "c or out_vals not aligned to its element size");
    Tuning tn;
    if ((s = read_tune(tune, &tn))) return s;
    split = resolve_split(split);
    if (split != SPD_SPLIT_ROW && split != SPD_SPLIT_NNZ) return fail(SPD_ERR_ARG, "unknown split %d", split);
    WsLayout L = layout_spmv(B->nfib, B->nnz, split);
    if ((s = check_ws(L, ws, ws_bytes))) return s;
    cudaStream_t st = as_stream(stream);
    if ((s = checked_csf3(B, "B", st))) return s;
    if (B->nfib == 0) return SPD_OK;
    if (split == SPD_SPLIT_ROW && tn.row_pieces <= 0) {
        int64_t P = ceil_div(B->nfib + B->nnz, kSpmvTile);
        tn.row_pieces = P < B->dim0 ? P : B->dim0;
        if (tn.row_pieces < 1) tn.row_pieces = 1;
    }
    return checked_finish(dispatch_spmv(B->vtype, B->nfib, B->nnz, B->pos2, B->crd2, B->vals, c, out_vals, split, tn,
                                        B->dim0, split == SPD_SPLIT_ROW ? B->pos1 : nullptr, ws, st),
                          "spd_spttv", st);
}

}  // extern "C"
