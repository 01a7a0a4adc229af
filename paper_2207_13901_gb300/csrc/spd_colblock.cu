// spd_colblock.cu -- universe partition of a CSR matrix's Compressed level by coordinate
// value ranges (the Compressed row of the partitioning table in Section IV-B:
// partitionByValueRanges on crd, then its preimage in pos). Block b keeps the entries
// whose column lies in [bounds[b], bounds[b+1]); each block is written out as its own
// CSR in the same {Dense, Compressed} format, with a permutation into A's positions so
// that values can be carried over (spd_gather_vals).
//
// With the blocks, Y = A X becomes a sequence of products Y += A_b X, each of which reads
// only the rows bounds[b] .. bounds[b+1]-1 of X: when that slab fits in L2, every gather
// of the product is an L2 hit, at the price of one more pass over Y per block (the
// single-GPU counterpart of partitioning the dense operand across GPUs).
//
// Three steps: a count kernel (thread per row; the split points of a row are found by
// binary search, which the sortedness of a row's columns allows), one exclusive scan per
// block (the blocks' pos), and a gather kernel (warp per row) that writes the blocks'
// crd and the permutation.
#include <vector>

#include "spd_internal.cuh"

namespace spd {

// First index of sorted a[lo, hi) whose value is >= v.
__device__ __forceinline__ int32_t first_at_least(const int32_t *a, int32_t lo, int32_t hi, int32_t v) {
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// blk_pos[b*(n+1) + i] = entries of row i in block b; blk_pos[b*(n+1) + n] = 0.
__global__ void colblock_count_kernel(int64_t n, const int32_t *__restrict__ pos, const int32_t *__restrict__ crd,
                                      int64_t nblk, const int32_t *__restrict__ bounds, int32_t *__restrict__ blk_pos) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += stride) {
        if (i == n) {
            for (int64_t b = 0; b < nblk; ++b) blk_pos[b * (n + 1) + n] = 0;
            continue;
        }
        const int32_t e = pos[i + 1];
        int32_t lo = pos[i];
        for (int64_t b = 0; b < nblk; ++b) {
            const int32_t hi = b == nblk - 1 ? e : first_at_least(crd, lo, e, bounds[b + 1]);
            blk_pos[b * (n + 1) + i] = hi - lo;
            lo = hi;
        }
    }
}

__global__ void colblock_totals_kernel(int64_t n, int64_t nblk, const int32_t *__restrict__ blk_pos,
                                       int32_t *__restrict__ totals) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nblk) totals[b] = blk_pos[b * (n + 1) + n];
}

// Warp per row: the entries of row i in block b go to blk_crd[off[b] + blk_pos_b[i] ...].
__global__ void colblock_gather_kernel(int64_t n, const int32_t *__restrict__ pos, const int32_t *__restrict__ crd,
                                       int64_t nblk, const int32_t *__restrict__ blk_pos,
                                       const int64_t *__restrict__ off, int32_t *__restrict__ blk_crd,
                                       int32_t *__restrict__ perm) {
    const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int lane = threadIdx.x & 31;
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += wstride) {
        int32_t lo = pos[i];
        for (int64_t b = 0; b < nblk; ++b) {
            const int32_t cnt = blk_pos[b * (n + 1) + i + 1] - blk_pos[b * (n + 1) + i];
            const int64_t dst = off[b] + blk_pos[b * (n + 1) + i];
            for (int32_t k = lane; k < cnt; k += 32) {
                blk_crd[dst + k] = crd[lo + k];
                perm[dst + k] = lo + k;
            }
            lo += cnt;
        }
    }
}

struct ColblockLayout {
    size_t bounds = 0, totals = 0, off = 0, sums = 0, total = 0;
};

static ColblockLayout colblock_layout(int64_t n, int64_t nblk) {
    ColblockLayout L;
    size_t o = 0;
    L.bounds = o;
    o += align_up(sizeof(int32_t) * (size_t)(nblk + 1));
    L.totals = o;
    o += align_up(sizeof(int32_t) * (size_t)nblk);
    L.off = o;
    o += align_up(sizeof(int64_t) * (size_t)(nblk + 1));
    L.sums = o;
    o += align_up(sizeof(int32_t) * (size_t)scan_tile_count(n + 1));
    L.total = o;
    return L;
}

static unsigned grid_of(int64_t work, int threads) {
    int64_t g = ceil_div(work > 0 ? work : 1, threads);
    return (unsigned)(g < 152 * 64 ? g : 152 * 64);
}

}  // namespace spd

using namespace spd;

extern "C" {

spd_status spd_csr_column_blocks_workspace_size(const spd_csr *A, int64_t nblk, size_t *bytes) {
    if (!bytes) return fail(SPD_ERR_NULL, "bytes is NULL");
    spd_status s = check_csr(A, false);
    if (s) return s;
    if (nblk < 1 || nblk > 65536) return fail(SPD_ERR_ARG, "nblk %lld not in [1, 65536]", (long long)nblk);
    *bytes = colblock_layout(A->nrows, nblk).total;
    return SPD_OK;
}

spd_status spd_csr_column_blocks(const spd_csr *A, int64_t nblk, const int32_t *bounds, int32_t *blk_pos,
                                 int32_t *blk_crd, int32_t *perm, int64_t *blk_nnz, void *ws, size_t ws_bytes,
                                 void *stream) {
    spd_status s = check_csr(A, false);
    if (s) return s;
    if (nblk < 1 || nblk > 65536) return fail(SPD_ERR_ARG, "nblk %lld not in [1, 65536]", (long long)nblk);
    if (!bounds || !blk_pos || !blk_nnz) return fail(SPD_ERR_NULL, "bounds/blk_pos/blk_nnz is NULL");
    if (A->nnz > 0 && (!blk_crd || !perm)) return fail(SPD_ERR_NULL, "blk_crd/perm is NULL");
    if (bounds[0] != 0 || bounds[nblk] != A->ncols)
        return fail(SPD_ERR_ARG, "bounds must start at 0 and end at ncols (%lld)", (long long)A->ncols);
    for (int64_t b = 0; b < nblk; ++b)
        if (bounds[b + 1] < bounds[b]) return fail(SPD_ERR_ARG, "bounds decrease at %lld", (long long)b);
    if (!aligned(blk_pos, 4) || (blk_crd && !aligned(blk_crd, 4)) || (perm && !aligned(perm, 4)))
        return fail(SPD_ERR_ALIGN, "blk_pos/blk_crd/perm not 4-byte aligned");
    const ColblockLayout L = colblock_layout(A->nrows, nblk);
    if (!ws) return fail(SPD_ERR_WORKSPACE, "workspace is NULL (%zu bytes needed)", L.total);
    if (ws_bytes < L.total) return fail(SPD_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, L.total);
    if (!aligned(ws, 256)) return fail(SPD_ERR_ALIGN, "workspace not 256-byte aligned");
    cudaStream_t st = as_stream(stream);
    if ((s = checked_csr(A, "A", st))) return s;
    char *w = static_cast<char *>(ws);
    int32_t *d_bounds = reinterpret_cast<int32_t *>(w + L.bounds);
    int32_t *d_totals = reinterpret_cast<int32_t *>(w + L.totals);
    int64_t *d_off = reinterpret_cast<int64_t *>(w + L.off);
    int32_t *sums = reinterpret_cast<int32_t *>(w + L.sums);
    const int64_t n = A->nrows;
    cudaError_t e = cudaMemcpyAsync(d_bounds, bounds, sizeof(int32_t) * (size_t)(nblk + 1), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(SPD_ERR_CUDA, "bounds copy: %s", cudaGetErrorString(e));
    colblock_count_kernel<<<grid_of(n + 1, 256), 256, 0, st>>>(n, A->pos, A->crd, nblk, d_bounds, blk_pos);
    if ((s = check_launch("colblock_count_kernel"))) return s;
    for (int64_t b = 0; b < nblk; ++b)
        if ((s = exclusive_scan_i32(blk_pos + b * (n + 1), n + 1, sums, st))) return s;
    colblock_totals_kernel<<<(unsigned)ceil_div(nblk, 256), 256, 0, st>>>(n, nblk, blk_pos, d_totals);
    if ((s = check_launch("colblock_totals_kernel"))) return s;
    std::vector<int32_t> tot((size_t)nblk);
    e = cudaMemcpyAsync(tot.data(), d_totals, sizeof(int32_t) * (size_t)nblk, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(SPD_ERR_CUDA, "block totals: %s", cudaGetErrorString(e));
    std::vector<int64_t> off((size_t)nblk + 1, 0);
    for (int64_t b = 0; b < nblk; ++b) {
        blk_nnz[b] = tot[(size_t)b];
        off[(size_t)b + 1] = off[(size_t)b] + tot[(size_t)b];
    }
    if (A->nnz == 0) return SPD_OK;
    e = cudaMemcpyAsync(d_off, off.data(), sizeof(int64_t) * (size_t)(nblk + 1), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(SPD_ERR_CUDA, "offsets copy: %s", cudaGetErrorString(e));
    colblock_gather_kernel<<<grid_of(n * 32, 256), 256, 0, st>>>(n, A->pos, A->crd, nblk, blk_pos, d_off, blk_crd,
                                                                  perm);
    if ((s = check_launch("colblock_gather_kernel"))) return s;
    // the host vectors above must outlive the copies: wait for them before returning
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(SPD_ERR_CUDA, "column blocks: %s", cudaGetErrorString(e));
    return SPD_OK;
}

}  // extern "C"
