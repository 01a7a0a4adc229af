// spd_transpose.cu -- the transposed structure of a CSR matrix, i.e. A in the CSC
// encoding: the same {Dense, Compressed} level formats with the dimension order
// reversed (the format language of Section II-B), together with the permutation that
// carries A's values into it. It serves the deterministic SpMM gradient dX = A^T dY:
// with A^T stored, dX is an ordinary SpMM that writes each row of dX once, with no
// atomic scatter (a transposed schedule, cached per sparsity structure).
//
// The permutation is a stable sort of A's positions by column, so the entries of a
// column keep A's row order. It is computed by a least-significant-digit radix sort of
// the column coordinates (8-bit digits) carrying the positions as payload. Every pass is
// a stable counting sort over 256 digits: per-tile digit counts, one exclusive scan of
// the counts in (digit, tile) order, and a scatter in which each warp ranks its items
// among equal digits with a match-any ballot. No step depends on timing, so the result
// is the same on every run.
#include "spd_internal.cuh"

namespace spd {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSortThreads = 256;                    // 8 warps
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortGroups = 16;                      // groups of 32 items per warp
constexpr int kSortTile = kSortThreads * kSortGroups;  // 4096 items per block
constexpr int kDigits = 256;
constexpr int kScanTile = kSortThreads * 16;          // items per block of the scan
static_assert(kSortThreads == kDigits, "the scatter gives each thread one digit");

// Exclusive prefix sum of x over the 256 threads of a block; *total gets the block sum.
// s_warp: 8 ints of shared memory.
__device__ __forceinline__ int32_t block_exclusive_sum(int32_t x, int32_t *s_warp, int32_t *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[w] = inc;
    __syncthreads();
    if (w == 0) {
        int32_t v = lane < kSortWarps ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(kFull, v, o);
            if (lane >= o) v += y;
        }
        if (lane < kSortWarps) s_warp[lane] = v;  // inclusive sums of the warps
    }
    __syncthreads();
    const int32_t before = w > 0 ? s_warp[w - 1] : 0;
    *total = s_warp[kSortWarps - 1];
    __syncthreads();  // s_warp may be reused after the call
    return before + inc - x;
}

// ---------------------------------------------------------------- exclusive scan

// sums[b] = sum of data[b*kScanTile .. (b+1)*kScanTile).
__global__ void __launch_bounds__(kSortThreads) scan_tile_sum_kernel(const int32_t *__restrict__ data, int64_t N,
                                                                    int32_t *__restrict__ sums) {
    __shared__ int32_t s_warp[kSortWarps];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int32_t s = 0;
    for (int k = threadIdx.x; k < kScanTile; k += kSortThreads) {
        const int64_t i = base + k;
        if (i < N) s += data[i];
    }
    int32_t total;
    block_exclusive_sum(s, s_warp, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Thread t of the block owns 16 consecutive items [base + 16t, base + 16t + 16): writes
// their exclusive prefix plus `offset` in place and returns the block total.
__device__ __forceinline__ int32_t scan_block_items(int32_t *data, int64_t N, int64_t base, int32_t offset,
                                                    int32_t *s_warp) {
    int32_t v[16];
    int32_t local = 0;
    const int64_t first = base + (int64_t)threadIdx.x * 16;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        v[k] = first + k < N ? data[first + k] : 0;
        local += v[k];
    }
    int32_t total;
    int32_t run = block_exclusive_sum(local, s_warp, &total) + offset;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        if (first + k < N) data[first + k] = run;
        run += v[k];
    }
    return total;
}

// One block: exclusive scan of the tile sums, in chunks of kScanTile.
__global__ void __launch_bounds__(kSortThreads) scan_sums_kernel(int32_t *__restrict__ sums, int64_t nsums) {
    __shared__ int32_t s_warp[kSortWarps];
    int32_t carry = 0;
    for (int64_t base = 0; base < nsums; base += kScanTile) carry += scan_block_items(sums, nsums, base, carry, s_warp);
}

__global__ void __launch_bounds__(kSortThreads) scan_apply_kernel(int32_t *__restrict__ data, int64_t N,
                                                                 const int32_t *__restrict__ sums) {
    __shared__ int32_t s_warp[kSortWarps];
    scan_block_items(data, N, (int64_t)blockIdx.x * kScanTile, sums[blockIdx.x], s_warp);
}

// In-place exclusive prefix sum of N int32 values (the total must fit in int32); sums
// holds scan_tile_count(N) ints.
int64_t scan_tile_count(int64_t N) { return ceil_div(N, kScanTile) + 1; }

spd_status exclusive_scan_i32(int32_t *data, int64_t N, int32_t *sums, cudaStream_t st) {
    if (N == 0) return SPD_OK;
    const int64_t nt = ceil_div(N, kScanTile);
    scan_tile_sum_kernel<<<(unsigned)nt, kSortThreads, 0, st>>>(data, N, sums);
    scan_sums_kernel<<<1, kSortThreads, 0, st>>>(sums, nt);
    scan_apply_kernel<<<(unsigned)nt, kSortThreads, 0, st>>>(data, N, sums);
    return check_launch("exclusive_scan");
}

// ---------------------------------------------------------------- radix sort passes

// hist[d * ntiles + b] = number of items of tile b whose digit is d.
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(int64_t N, const int32_t *__restrict__ keys,
                                                                 int shift, int32_t *__restrict__ hist,
                                                                 int64_t ntiles) {
    __shared__ int32_t h[kDigits];
    for (int d = threadIdx.x; d < kDigits; d += kSortThreads) h[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int k = threadIdx.x; k < kSortTile; k += kSortThreads) {
        const int64_t i = base + k;
        if (i < N) atomicAdd(&h[((uint32_t)keys[i] >> shift) & (kDigits - 1)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kDigits; d += kSortThreads) hist[(int64_t)d * ntiles + blockIdx.x] = h[d];
}

// Stable scatter of tile b: warp w owns the items [b*T + 512w, b*T + 512w + 512) in 16
// groups of 32. An item's rank among the tile's items of its digit is the count of that
// digit in earlier warps of the tile, plus in earlier groups of its warp, plus in lower
// lanes of its group. The items are first placed in shared memory in tile order sorted
// by digit (a stable local sort), then written out so that consecutive threads write
// consecutive destinations inside each digit's run: destination = the scanned count of
// (digit, tile) + the rank. vals_in == NULL means the identity payload (the item's own
// index).
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(
    int64_t N, const int32_t *__restrict__ keys_in, const int32_t *__restrict__ vals_in, int shift,
    const int32_t *__restrict__ offs, int64_t ntiles, int32_t *__restrict__ keys_out,
    int32_t *__restrict__ vals_out) {
    __shared__ int32_t cnt[kSortWarps][kDigits];
    __shared__ int32_t s_local[kDigits];   // first tile-local slot of each digit
    __shared__ int32_t s_global[kDigits];  // first destination of each digit's run of this tile
    __shared__ int32_t s_warp[kSortWarps];
    __shared__ int32_t s_key[kSortTile], s_val[kSortTile];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = lane; d < kDigits; d += 32) cnt[w][d] = 0;
    __syncwarp();
    const int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
    const int64_t base = tile0 + (int64_t)w * (32 * kSortGroups);
    const int items = (int)(N - tile0 < kSortTile ? N - tile0 : kSortTile);
    int32_t key[kSortGroups], val[kSortGroups];
#pragma unroll
    for (int g = 0; g < kSortGroups; ++g) {
        const int64_t i = base + g * 32 + lane;
        const bool valid = i < N;
        key[g] = valid ? keys_in[i] : 0;
        val[g] = valid ? (vals_in ? vals_in[i] : (int32_t)i) : 0;
        const int d = valid ? (int)(((uint32_t)key[g] >> shift) & (kDigits - 1)) : kDigits;  // kDigits: no item
        const unsigned peers = __match_any_sync(kFull, d);
        if (valid && lane == __ffs(peers) - 1) cnt[w][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit (one thread each): the tile's total, then each warp's first local slot
    {
        const int d = threadIdx.x;  // kSortThreads == kDigits
        int32_t tot = 0;
#pragma unroll
        for (int ww = 0; ww < kSortWarps; ++ww) tot += cnt[ww][d];
        int32_t all;
        const int32_t start = block_exclusive_sum(tot, s_warp, &all);
        s_local[d] = start;
        s_global[d] = offs[(int64_t)d * ntiles + blockIdx.x];
        int32_t run = start;
#pragma unroll
        for (int ww = 0; ww < kSortWarps; ++ww) {
            const int32_t c = cnt[ww][d];
            cnt[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
    const unsigned below = (1u << lane) - 1u;
#pragma unroll
    for (int g = 0; g < kSortGroups; ++g) {
        const int64_t i = base + g * 32 + lane;
        const bool valid = i < N;
        const int d = valid ? (int)(((uint32_t)key[g] >> shift) & (kDigits - 1)) : kDigits;
        const unsigned peers = __match_any_sync(kFull, d);
        if (valid) {
            const int32_t slot = cnt[w][d] + __popc(peers & below);
            s_key[slot] = key[g];
            s_val[slot] = val[g];
        }
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) cnt[w][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    for (int t = threadIdx.x; t < items; t += kSortThreads) {
        const int32_t k = s_key[t];
        const int d = (int)(((uint32_t)k >> shift) & (kDigits - 1));
        const int32_t dest = s_global[d] + (t - s_local[d]);
        keys_out[dest] = k;
        vals_out[dest] = s_val[t];
    }
}

// ---------------------------------------------------------------- structure of A^T

// t_pos[j] = first sorted position whose column is >= j, for j in [0, m]: position q
// writes the columns in (key[q-1], key[q]] (key[-1] = -1, key[N] = m).
__global__ void col_bounds_kernel(int64_t N, int64_t m, const int32_t *__restrict__ skeys,
                                  int32_t *__restrict__ t_pos) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q <= N; q += stride) {
        int64_t lo = (q > 0 ? (int64_t)skeys[q - 1] : -1) + 1;
        int64_t hi = q < N ? (int64_t)skeys[q] : m;
        if (lo < 0) lo = 0;  // coordinates outside [0, m) (an unvalidated structure) write nothing outside t_pos
        if (hi > m) hi = m;
        for (int64_t j = lo; j <= hi; ++j) t_pos[j] = (int32_t)q;
    }
}

// rowid[p] = the row of position p (one warp per row; positions outside [0, nnz) of an
// unvalidated structure are skipped).
__global__ void row_ids_kernel(int64_t n, int64_t nnz, const int32_t *__restrict__ pos, int32_t *__restrict__ rowid) {
    const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int lane = threadIdx.x & 31;
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += wstride) {
        const int64_t b = pos[i] > 0 ? pos[i] : 0;
        const int64_t e = pos[i + 1] < nnz ? pos[i + 1] : nnz;
        for (int64_t p = b + lane; p < e; p += 32) rowid[p] = (int32_t)i;
    }
}

// t_crd[q] = rowid[perm[q]].
__global__ void gather_rows_kernel(int64_t N, const int32_t *__restrict__ perm, const int32_t *__restrict__ rowid,
                                   int32_t *__restrict__ t_crd) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += stride) t_crd[q] = rowid[perm[q]];
}

template <typename W>
__global__ void gather_vals_kernel(int64_t N, const int32_t *__restrict__ perm, const W *__restrict__ in,
                                   W *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += stride) out[q] = in[perm[q]];
}

// Workspace: two key buffers and one payload buffer of N ints, the (digit, tile)
// counts and the scan's tile sums.
struct TransposeLayout {
    size_t keys0 = 0, keys1 = 0, pay = 0, hist = 0, sums = 0, total = 0;
    int64_t ntiles = 0, nhist = 0;
};

static TransposeLayout transpose_layout(int64_t N) {
    TransposeLayout T;
    T.ntiles = ceil_div(N, kSortTile);
    T.nhist = T.ntiles * kDigits;
    const size_t nb = align_up(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    size_t off = 0;
    T.keys0 = off;
    off += nb;
    T.keys1 = off;
    off += nb;
    T.pay = off;
    off += nb;
    T.hist = off;
    off += align_up(sizeof(int32_t) * (size_t)(T.nhist > 0 ? T.nhist : 1));
    T.sums = off;
    off += align_up(sizeof(int32_t) * (size_t)scan_tile_count(T.nhist));
    T.total = off;
    return T;
}

// Radix passes needed for column coordinates below m: 8 bits each, at least one.
static int radix_passes(int64_t m) {
    int bits = 0;
    while (bits < 31 && (int64_t(1) << bits) < m) ++bits;
    const int p = (bits + 7) / 8;
    return p > 0 ? p : 1;
}

static unsigned grid_for(int64_t work, int threads) {
    int64_t g = ceil_div(work > 0 ? work : 1, threads);
    if (g > 152 * 64) g = 152 * 64;
    return (unsigned)g;
}

}  // namespace spd

using namespace spd;

extern "C" {

spd_status spd_csr_transpose_workspace_size(const spd_csr *A, size_t *bytes) {
    if (!bytes) return fail(SPD_ERR_NULL, "bytes is NULL");
    spd_status s = check_csr(A, false);
    if (s) return s;
    *bytes = transpose_layout(A->nnz).total;
    return SPD_OK;
}

spd_status spd_csr_transpose(const spd_csr *A, int32_t *t_pos, int32_t *t_crd, int32_t *perm, void *ws,
                             size_t ws_bytes, void *stream) {
    spd_status s = check_csr(A, false);
    if (s) return s;
    const int64_t N = A->nnz, m = A->ncols;
    if (!t_pos) return fail(SPD_ERR_NULL, "t_pos is NULL");
    if (N > 0 && (!t_crd || !perm)) return fail(SPD_ERR_NULL, "t_crd/perm is NULL");
    if (!aligned(t_pos, 4) || (t_crd && !aligned(t_crd, 4)) || (perm && !aligned(perm, 4)))
        return fail(SPD_ERR_ALIGN, "t_pos/t_crd/perm not 4-byte aligned");
    const TransposeLayout T = transpose_layout(N);
    if (!ws) return fail(SPD_ERR_WORKSPACE, "workspace is NULL (%zu bytes needed)", T.total);
    if (ws_bytes < T.total) return fail(SPD_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, T.total);
    if (!aligned(ws, 256)) return fail(SPD_ERR_ALIGN, "workspace not 256-byte aligned");
    cudaStream_t st = as_stream(stream);
    if ((s = checked_csr(A, "A", st))) return s;
    char *w = static_cast<char *>(ws);
    int32_t *keys[2] = {reinterpret_cast<int32_t *>(w + T.keys0), reinterpret_cast<int32_t *>(w + T.keys1)};
    int32_t *pay = reinterpret_cast<int32_t *>(w + T.pay);
    int32_t *hist = reinterpret_cast<int32_t *>(w + T.hist);
    int32_t *sums = reinterpret_cast<int32_t *>(w + T.sums);

    const int32_t *skeys = keys[0];
    if (N > 0) {
        // pass i sorts by bits [8i, 8i+8); the last pass writes its payload into perm
        const int P = radix_passes(m);
        const int32_t *kin = A->crd;
        const int32_t *vin = nullptr;  // identity payload
        for (int i = 0; i < P; ++i) {
            int32_t *kout = keys[i & 1];
            int32_t *vout = ((P - 1 - i) % 2 == 0) ? perm : pay;
            radix_hist_kernel<<<(unsigned)T.ntiles, kSortThreads, 0, st>>>(N, kin, 8 * i, hist, T.ntiles);
            if ((s = check_launch("radix_hist_kernel"))) return s;
            if ((s = exclusive_scan_i32(hist, T.nhist, sums, st))) return s;
            radix_scatter_kernel<<<(unsigned)T.ntiles, kSortThreads, 0, st>>>(N, kin, vin, 8 * i, hist, T.ntiles,
                                                                              kout, vout);
            if ((s = check_launch("radix_scatter_kernel"))) return s;
            kin = kout;
            vin = vout;
            skeys = kout;
        }
        // the payload buffer is free now: row of every position, then the rows in
        // sorted order
        row_ids_kernel<<<grid_for(A->nrows * 32, 256), 256, 0, st>>>(A->nrows, N, A->pos, pay);
        gather_rows_kernel<<<grid_for(N, 256), 256, 0, st>>>(N, perm, pay, t_crd);
        if ((s = check_launch("gather_rows_kernel"))) return s;
    }
    col_bounds_kernel<<<grid_for(N + 1, 256), 256, 0, st>>>(N, m, skeys, t_pos);
    return checked_finish(check_launch("col_bounds_kernel"), "spd_csr_transpose", st);
}

spd_status spd_gather_vals(int64_t n, const int32_t *perm, const void *in, void *out, int vtype, void *stream) {
    if (n < 0) return fail(SPD_ERR_SHAPE, "n %lld < 0", (long long)n);
    const size_t es = dtype_size(vtype);
    if (es == 0) return fail(SPD_ERR_DTYPE, "unknown value type %d", vtype);
    if (n == 0) return SPD_OK;
    if (!perm || !in || !out) return fail(SPD_ERR_NULL, "perm/in/out is NULL");
    if (!aligned(perm, 4) || !aligned(in, es) || !aligned(out, es)) return fail(SPD_ERR_ALIGN, "perm/in/out misaligned");
    cudaStream_t st = as_stream(stream);
    const unsigned g = grid_for(n, 256);
    switch (es) {
        case 8:
            gather_vals_kernel<uint64_t><<<g, 256, 0, st>>>(n, perm, static_cast<const uint64_t *>(in),
                                                             static_cast<uint64_t *>(out));
            break;
        case 4:
            gather_vals_kernel<uint32_t><<<g, 256, 0, st>>>(n, perm, static_cast<const uint32_t *>(in),
                                                             static_cast<uint32_t *>(out));
            break;
        default:
            gather_vals_kernel<uint16_t><<<g, 256, 0, st>>>(n, perm, static_cast<const uint16_t *>(in),
                                                             static_cast<uint16_t *>(out));
    }
    return checked_finish(check_launch("gather_vals_kernel"), "spd_gather_vals", st);
}

}  // extern "C"
