// spd_core.cu -- status handling, argument checks, workspace layouts, the work
// partitions (Sections II-B, III-A, IV-B/C) and structure validation (Section III-B).
#include <atomic>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "spd_internal.cuh"

namespace spd {

static thread_local char g_last_error[512] = "";

spd_status fail(spd_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return s;
}

spd_status check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(SPD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return SPD_OK;
}

spd_status check_csr(const spd_csr *A, bool need_vals) {
    if (!A) return fail(SPD_ERR_NULL, "matrix descriptor is NULL");
    if (A->nrows < 0 || A->ncols < 0 || A->nnz < 0)
        return fail(SPD_ERR_SHAPE, "negative size (nrows=%lld ncols=%lld nnz=%lld)", (long long)A->nrows,
                    (long long)A->ncols, (long long)A->nnz);
    if (A->nrows > SPD_MAX_INDEX || A->ncols > SPD_MAX_INDEX || A->nnz > SPD_MAX_INDEX)
        return fail(SPD_ERR_SHAPE, "sizes exceed SPD_MAX_INDEX (nrows=%lld ncols=%lld nnz=%lld)",
                    (long long)A->nrows, (long long)A->ncols, (long long)A->nnz);
    if (A->nrows == 0 && A->nnz != 0) return fail(SPD_ERR_SHAPE, "a matrix without rows has no entries");
    if (A->ncols == 0 && A->nnz != 0) return fail(SPD_ERR_SHAPE, "a matrix without columns has no entries");
    if (!A->pos) return fail(SPD_ERR_NULL, "pos is NULL");
    if (A->nnz > 0 && !A->crd) return fail(SPD_ERR_NULL, "crd is NULL");
    if (dtype_size(A->vtype) == 0) return fail(SPD_ERR_DTYPE, "unknown value type %d", A->vtype);
    if (need_vals && A->nnz > 0 && !A->vals) return fail(SPD_ERR_NULL, "vals is NULL");
    if (!aligned(A->pos, 4) || (A->crd && !aligned(A->crd, 4))) return fail(SPD_ERR_ALIGN, "pos/crd not 4-byte aligned");
    if (A->vals && !aligned(A->vals, dtype_size(A->vtype))) return fail(SPD_ERR_ALIGN, "vals not aligned to its element size");
    return SPD_OK;
}

spd_status check_csf3(const spd_csf3 *B) {
    if (!B) return fail(SPD_ERR_NULL, "tensor descriptor is NULL");
    if (B->dim0 < 0 || B->dim1 < 0 || B->dim2 < 0 || B->nfib < 0 || B->nnz < 0)
        return fail(SPD_ERR_SHAPE, "negative size");
    if (B->dim0 > SPD_MAX_INDEX || B->dim1 > SPD_MAX_INDEX || B->dim2 > SPD_MAX_INDEX ||
        B->nfib > SPD_MAX_INDEX || B->nnz > SPD_MAX_INDEX)
        return fail(SPD_ERR_SHAPE, "sizes exceed SPD_MAX_INDEX");
    if ((B->dim0 == 0 || B->dim1 == 0) && B->nfib != 0) return fail(SPD_ERR_SHAPE, "fibers in an empty tensor");
    if ((B->nfib == 0 || B->dim2 == 0) && B->nnz != 0) return fail(SPD_ERR_SHAPE, "entries without fibers");
    if (!B->pos1 || !B->pos2) return fail(SPD_ERR_NULL, "pos1/pos2 is NULL");
    if (B->nfib > 0 && !B->crd1) return fail(SPD_ERR_NULL, "crd1 is NULL");
    if (B->nnz > 0 && (!B->crd2 || !B->vals)) return fail(SPD_ERR_NULL, "crd2/vals is NULL");
    if (dtype_size(B->vtype) == 0) return fail(SPD_ERR_DTYPE, "unknown value type %d", B->vtype);
    if (!aligned(B->pos1, 4) || !aligned(B->pos2, 4) || (B->crd1 && !aligned(B->crd1, 4)) ||
        (B->crd2 && !aligned(B->crd2, 4)))
        return fail(SPD_ERR_ALIGN, "pos/crd not 4-byte aligned");
    if (B->vals && !aligned(B->vals, dtype_size(B->vtype))) return fail(SPD_ERR_ALIGN, "vals misaligned");
    return SPD_OK;
}

spd_status read_tune(const spd_tune *t, Tuning *out) {
    out->unit_items = kWarpUnitDefault;
    out->row_pieces = 0;
    out->block_threads = kWarpBlockDefault;
    out->inflight = 8;
    out->lane_groups = 0;
    out->form = 0;
    if (!t) return SPD_OK;
    if (t->unit_items) {
        if (t->unit_items < 32 || t->unit_items > 65536 || t->unit_items % 32)
            return fail(SPD_ERR_ARG, "unit_items %d not a multiple of 32 in [32, 65536]", t->unit_items);
        out->unit_items = t->unit_items;
    }
    if (t->row_pieces) {
        if (t->row_pieces < 0) return fail(SPD_ERR_ARG, "row_pieces %d < 1", t->row_pieces);
        out->row_pieces = t->row_pieces;
    }
    if (t->block_threads) {
        // the warp kernels are compiled for blocks of at most 256 threads
        if (t->block_threads < 64 || t->block_threads > kWarpBlockMax || t->block_threads % 32)
            return fail(SPD_ERR_ARG, "block_threads %d not a multiple of 32 in [64, %d]", t->block_threads,
                        kWarpBlockMax);
        out->block_threads = t->block_threads;
    }
    if (t->inflight) {
        if (t->inflight != 4 && t->inflight != 8) return fail(SPD_ERR_ARG, "inflight %d is not 4 or 8", t->inflight);
        out->inflight = t->inflight;
    }
    if (t->lane_groups < 0 || t->lane_groups > 2) return fail(SPD_ERR_ARG, "lane_groups %d not in 0..2", t->lane_groups);
    out->lane_groups = t->lane_groups;
    if (t->form < 0 || t->form > 2) return fail(SPD_ERR_ARG, "form %d not in 0..2", t->form);
    out->form = t->form;
    return SPD_OK;
}

int resolve_split(int split) {
    if (split == SPD_SPLIT_AUTO) return SPD_SPLIT_NNZ;
    return split;
}

WsLayout make_layout(int64_t npieces, int64_t width, bool need_partition, bool need_carry, bool aux, bool chunks) {
    WsLayout L;
    L.npieces = npieces;
    size_t off = 0;
    if (need_partition && npieces > 0) {
        L.part_row = off;
        off += align_up(sizeof(int32_t) * (size_t)(npieces + 1));
        L.part_pos = off;
        off += align_up(sizeof(int32_t) * (size_t)(npieces + 1));
        if (aux) {
            L.part_aux = off;
            off += align_up(sizeof(int32_t) * (size_t)(npieces + 1));
        }
    }
    if (need_carry && npieces > 0) {
        L.carry_row = off;
        off += align_up(sizeof(int32_t) * (size_t)npieces);
        L.carry_val = off;
        off += align_up(sizeof(double) * (size_t)npieces * (size_t)(width > 0 ? width : 1));
        if (chunks) {
            const int64_t nch = ceil_div(npieces, kCarryChunk);
            L.chunk_row = off;
            off += align_up(sizeof(int32_t) * (size_t)nch);
            L.chunk_val = off;
            off += align_up(sizeof(double) * (size_t)nch * (size_t)(width > 0 ? width : 1));
        }
    }
    L.total = off;
    return L;
}

spd_status check_ws(const WsLayout &L, void *ws, size_t ws_bytes) {
    if (L.total == 0) return SPD_OK;
    if (!ws) return fail(SPD_ERR_WORKSPACE, "workspace is NULL (%zu bytes needed)", L.total);
    if (ws_bytes < L.total) return fail(SPD_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, L.total);
    if (!aligned(ws, 256)) return fail(SPD_ERR_ALIGN, "workspace not 256-byte aligned");
    return SPD_OK;
}

spd_status check_dense(const char *name, const void *p, int64_t rows, int64_t L, int64_t ld, int t) {
    if (ld < L) return fail(SPD_ERR_SHAPE, "%s: leading dimension %lld < %lld", name, (long long)ld, (long long)L);
    if (rows > 0 && L > 0 && !p) return fail(SPD_ERR_NULL, "%s is NULL", name);
    if (p && !aligned(p, dtype_size(t))) return fail(SPD_ERR_ALIGN, "%s not aligned to its element size", name);
    return SPD_OK;
}

int pick_epl(int64_t L, size_t in_size, size_t out_size, const void *in, int64_t ld_in, const void *out,
             int64_t ld_out) {
    int max_epl = (int)(32 / in_size);
    if (max_epl > 8) max_epl = 8;
    int epl = 1;
    while (epl < max_epl && 32 * epl < L) epl *= 2;
    while (epl > 1) {
        size_t vin = (size_t)epl * in_size, vout = (size_t)epl * out_size;
        size_t ain = vin > 16 ? 16 : vin, aout = vout > 16 ? 16 : vout;
        bool ok = (L % epl == 0) && (ld_in % epl == 0) && (ld_out % epl == 0) && aligned(in, ain) &&
                  (out == nullptr || aligned(out, aout));
        if (ok) break;
        epl /= 2;
    }
    return epl;
}

SpmmShape pick_spmm_shape(int64_t L, size_t in_size, size_t out_size, const void *in, int64_t ld_in,
                          const void *out, int64_t ld_out, int lane_groups, uint64_t x_bytes) {
    const int vec = (int)(16 / in_size);
    const size_t vout = (size_t)vec * out_size;
    const bool vec_ok = L > 0 && L % vec == 0 && ld_in % vec == 0 && ld_out % vec == 0 && aligned(in, 16) &&
                        (out == nullptr || aligned(out, vout > 16 ? 16 : vout));
    const bool want = lane_groups == 1 || (lane_groups == 0 && x_bytes <= (uint64_t(64) << 20));
    if (vec_ok && want) {
        const int64_t lanes = L / vec;
        int g = 4;
        while (g < lanes) g *= 2;
        if (g < 32) return SpmmShape{vec, g};
    }
    int epl = pick_epl(L, in_size, out_size, in, ld_in, out, ld_out);
    if (in_size == 8 && epl > 4) epl = 4;
    return SpmmShape{epl, 32};
}

WsLayout layout_spmv(int64_t n, int64_t nnz, int split) {
    if (split == SPD_SPLIT_ROW || n + nnz == 0) return make_layout(0, 0, false, false, false);
    return make_layout(ceil_div(n + nnz, kSpmvTile), 1, true, true, false);
}

WsLayout layout_warp(int64_t n, int64_t nnz, int split, int64_t unit, int64_t width, bool carries) {
    if (split == SPD_SPLIT_ROW || n + nnz == 0) return make_layout(0, 0, false, false, false);
    return make_layout(ceil_div(n + nnz, unit), width, true, carries, false, carries);
}

WsLayout layout_mttkrp(int64_t F, int64_t nnz, int split, int64_t unit, int64_t R) {
    if (split == SPD_SPLIT_ROW || F + nnz == 0) return make_layout(0, 0, false, false, false);
    return make_layout(ceil_div(F + nnz, unit), R, true, true, true, true);
}

// ------------------------------------------------------------------ partition kernels

// Fused non-zero partition as a preimage (Section III-A): every row r colors the piece
// boundaries d = t*unit that fall on its items (e_{r-1}, e_r], where e_r = pos[r+1] + r
// is the index of row r's end item. One pass over pos, fully parallel, no search.
__global__ void merge_partition_kernel(int64_t n, int64_t nnz, const int32_t *__restrict__ pos, int64_t unit,
                                       int64_t npieces, int32_t *__restrict__ prow, int32_t *__restrict__ ppos) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r > n) return;
    if (r == n) {
        prow[npieces] = (int32_t)n;
        ppos[npieces] = (int32_t)nnz;
        return;
    }
    // item indices stay below nrows + nnz < 2^32, so the divisions run in 32 bits
    const uint32_t u = (uint32_t)unit;
    const uint32_t e = (uint32_t)__ldg(pos + r + 1) + (uint32_t)r;
    int64_t t_lo = 0;
    if (r > 0) {
        const uint32_t e_prev = (uint32_t)__ldg(pos + r) + (uint32_t)r - 1u;
        t_lo = (int64_t)(e_prev / u) + 1;
    }
    int64_t t_hi = (int64_t)(e / u);
    if (t_hi > npieces - 1) t_hi = npieces - 1;
    for (int64_t t = t_lo; t <= t_hi; ++t) {
        prow[t] = (int32_t)r;
        ppos[t] = (int32_t)(t * unit - r);
    }
}

// Universe partition into P pieces: bounds floor(c n / P) and their image in crd.
__global__ void row_partition_kernel(int64_t n, const int32_t *__restrict__ pos, int64_t P, int32_t *__restrict__ prow,
                                     int32_t *__restrict__ ppos) {
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c > P) return;
    int64_t r = (c * n) / P;
    prow[c] = (int32_t)r;
    ppos[c] = __ldg(pos + r);
}

spd_status launch_merge_partition(int64_t n, int64_t nnz, const int32_t *pos, int64_t unit, int64_t npieces,
                                  int32_t *prow, int32_t *ppos, cudaStream_t st) {
    int64_t threads = n + 1;
    int block = 256;
    int64_t grid = ceil_div(threads, block);
    merge_partition_kernel<<<(unsigned)grid, block, 0, st>>>(n, nnz, pos, unit, npieces, prow, ppos);
    return check_launch("merge_partition_kernel");
}

// ------------------------------------------------------------------ validation

struct ValidateOut {
    unsigned long long count;
    long long first;
};

__global__ void validate_init_kernel(ValidateOut *o) {
    o->count = 0;
    o->first = LLONG_MAX;
}

__device__ __forceinline__ void report_bad(ValidateOut *o, long long idx) {
    atomicAdd(&o->count, 1ull);
    atomicMin(&o->first, idx);
}

// One Compressed level (Section III-B): pos[0] == 0, pos non-decreasing,
// pos[nparent] == nchild, 0 <= crd < dim. `base` offsets the reported index.
__global__ void validate_level_kernel(int64_t nparent, int64_t dim, int64_t nchild, const int32_t *__restrict__ pos,
                                      const int32_t *__restrict__ crd, long long base, ValidateOut *o) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t total = (nparent + 1) > nchild ? (nparent + 1) : nchild;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        if (t <= nparent) {
            int32_t v = __ldg(pos + t);
            bool bad = false;
            if (t == 0 && v != 0) bad = true;
            if (t > 0 && v < __ldg(pos + t - 1)) bad = true;
            if (t == nparent && (int64_t)v != nchild) bad = true;
            if (bad) report_bad(o, base + t);
        }
        if (t < nchild) {
            int32_t c = __ldcs(crd + t);
            if (c < 0 || (int64_t)c >= dim) report_bad(o, base + nparent + 1 + t);
        }
    }
}

static spd_status run_validate(int nlevels, const int64_t *nparent, const int64_t *dim, const int64_t *nchild,
                               const int32_t *const *pos, const int32_t *const *crd, void *ws, size_t ws_bytes,
                               int64_t *violations, int64_t *first_bad, cudaStream_t st) {
    if (!ws) return fail(SPD_ERR_WORKSPACE, "validate needs a workspace of 64 bytes");
    if (ws_bytes < 64) return fail(SPD_ERR_WORKSPACE, "validate workspace %zu < 64 bytes", ws_bytes);
    if (!aligned(ws, 16)) return fail(SPD_ERR_ALIGN, "workspace not 16-byte aligned");
    if (!violations || !first_bad) return fail(SPD_ERR_NULL, "output pointers are NULL");
    ValidateOut *o = reinterpret_cast<ValidateOut *>(ws);
    validate_init_kernel<<<1, 1, 0, st>>>(o);
    long long base = 0;
    for (int l = 0; l < nlevels; ++l) {
        int64_t total = (nparent[l] + 1) > nchild[l] ? (nparent[l] + 1) : nchild[l];
        int64_t grid = ceil_div(total, 256);
        if (grid > 152 * 16) grid = 152 * 16;
        if (grid < 1) grid = 1;
        validate_level_kernel<<<(unsigned)grid, 256, 0, st>>>(nparent[l], dim[l], nchild[l], pos[l], crd[l], base, o);
        base += nparent[l] + 1 + nchild[l];
    }
    spd_status s = check_launch("validate_level_kernel");
    if (s) return s;
    ValidateOut h;
    cudaError_t e = cudaMemcpyAsync(&h, o, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(SPD_ERR_CUDA, "validate: %s", cudaGetErrorString(e));
    *violations = (int64_t)h.count;
    *first_bad = h.count ? (int64_t)h.first : -1;
    if (h.count) return fail(SPD_ERR_STRUCTURE, "%llu violations, first at index %lld", h.count, h.first);
    return SPD_OK;
}

// ------------------------------------------------------------------ checked mode

// -1 until the first query reads SPD_DEBUG from the environment; then 0 or 1.
static std::atomic<int> g_checked{-1};
// The device status word of checked mode (a ValidateOut, padded to the 64 bytes that
// run_validate asks of a workspace); one per process, its users serialized by the mutex.
static __device__ __align__(16) unsigned char g_checked_word[64];
static std::mutex g_checked_mutex;

bool checked_mode() {
    int c = g_checked.load();
    if (c < 0) {
        const char *e = getenv("SPD_DEBUG");
        c = (e && *e && strcmp(e, "0") != 0) ? 1 : 0;
        int expected = -1;
        if (!g_checked.compare_exchange_strong(expected, c)) c = expected;
    }
    return c == 1;
}

static spd_status not_capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return fail(SPD_ERR_CUDA, "checked mode: %s", cudaGetErrorString(e));
    if (cs != cudaStreamCaptureStatusNone)
        return fail(SPD_ERR_ARG, "checked mode synchronizes the stream and cannot run inside a graph capture");
    return SPD_OK;
}

static spd_status checked_levels(int nlevels, const int64_t *np, const int64_t *dm, const int64_t *nc,
                                 const int32_t *const *ps, const int32_t *const *cs, const char *name,
                                 cudaStream_t st) {
    spd_status s = not_capturing(st);
    if (s) return s;
    std::lock_guard<std::mutex> lock(g_checked_mutex);
    void *word = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&word, g_checked_word);
    if (e != cudaSuccess) return fail(SPD_ERR_CUDA, "checked mode: %s", cudaGetErrorString(e));
    int64_t violations = 0, first_bad = -1;
    s = run_validate(nlevels, np, dm, nc, ps, cs, word, sizeof(g_checked_word), &violations, &first_bad, st);
    if (s == SPD_ERR_STRUCTURE)
        return fail(s, "checked mode: %s breaks the level format (%lld violations, first at index %lld)", name,
                    (long long)violations, (long long)first_bad);
    return s;
}

spd_status checked_csr(const spd_csr *A, const char *name, cudaStream_t st) {
    if (!checked_mode()) return SPD_OK;
    int64_t np[1] = {A->nrows}, dm[1] = {A->ncols}, nc[1] = {A->nnz};
    const int32_t *ps[1] = {A->pos}, *cs[1] = {A->crd};
    return checked_levels(1, np, dm, nc, ps, cs, name, st);
}

spd_status checked_csf3(const spd_csf3 *B, const char *name, cudaStream_t st) {
    if (!checked_mode()) return SPD_OK;
    int64_t np[2] = {B->dim0, B->nfib}, dm[2] = {B->dim1, B->dim2}, nc[2] = {B->nfib, B->nnz};
    const int32_t *ps[2] = {B->pos1, B->pos2}, *cs[2] = {B->crd1, B->crd2};
    return checked_levels(2, np, dm, nc, ps, cs, name, st);
}

spd_status checked_finish(spd_status s, const char *call, cudaStream_t st) {
    if (s != SPD_OK || !checked_mode()) return s;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e == cudaSuccess && cs != cudaStreamCaptureStatusNone) return SPD_OK;  // captured work runs later
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return fail(SPD_ERR_CUDA, "%s: %s", call, cudaGetErrorString(e));
    unsigned int faults = 0;
    spd_status f = take_device_faults(&faults);
    if (f) return f;
    if (faults) return fail(SPD_ERR_TIMEOUT, "%s: a bounded device wait gave up (flags 0x%x)", call, faults);
    return SPD_OK;
}

}  // namespace spd

using namespace spd;

extern "C" {

int spd_abi_version(void) { return SPD_ABI_VERSION; }

const char *spd_status_str(int s) {
    switch (s) {
        case SPD_OK: return "ok";
        case SPD_ERR_NULL: return "null pointer";
        case SPD_ERR_SHAPE: return "invalid or inconsistent sizes";
        case SPD_ERR_DTYPE: return "unsupported element type";
        case SPD_ERR_ALIGN: return "misaligned pointer or leading dimension";
        case SPD_ERR_STRUCTURE: return "pos/crd break the level format";
        case SPD_ERR_WORKSPACE: return "workspace missing or too small";
        case SPD_ERR_CUDA: return "CUDA error";
        case SPD_ERR_OOM: return "out of memory";
        case SPD_ERR_TIMEOUT: return "device wait timed out";
        case SPD_ERR_ARG: return "argument out of range";
        default: return "unknown status";
    }
}

const char *spd_last_error(void) { return g_last_error; }

spd_status spd_set_checked(int on) {
    if (on != 0 && on != 1) return fail(SPD_ERR_ARG, "spd_set_checked takes 0 or 1, not %d", on);
    g_checked.store(on);
    return SPD_OK;
}

int spd_checked(void) { return checked_mode() ? 1 : 0; }

spd_status spd_csr_validate(const spd_csr *A, void *ws, size_t ws_bytes, int64_t *violations, int64_t *first_bad,
                            void *stream) {
    g_last_error[0] = 0;
    spd_status s = check_csr(A, false);
    if (s) return s;
    int64_t np[1] = {A->nrows}, dm[1] = {A->ncols}, nc[1] = {A->nnz};
    const int32_t *ps[1] = {A->pos}, *cs[1] = {A->crd};
    return run_validate(1, np, dm, nc, ps, cs, ws, ws_bytes, violations, first_bad, as_stream(stream));
}

spd_status spd_csf3_validate(const spd_csf3 *B, void *ws, size_t ws_bytes, int64_t *violations, int64_t *first_bad,
                             void *stream) {
    g_last_error[0] = 0;
    spd_status s = check_csf3(B);
    if (s) return s;
    int64_t np[2] = {B->dim0, B->nfib}, dm[2] = {B->dim1, B->dim2}, nc[2] = {B->nfib, B->nnz};
    const int32_t *ps[2] = {B->pos1, B->pos2}, *cs[2] = {B->crd1, B->crd2};
    return run_validate(2, np, dm, nc, ps, cs, ws, ws_bytes, violations, first_bad, as_stream(stream));
}

spd_status spd_csr_workspace_size(int op, const spd_csr *A, int split, int64_t width, const spd_tune *tune,
                                  size_t *bytes) {
    g_last_error[0] = 0;
    if (!bytes) return fail(SPD_ERR_NULL, "bytes is NULL");
    spd_status s = check_csr(A, false);
    if (s) return s;
    Tuning tn;
    if ((s = read_tune(tune, &tn))) return s;
    split = resolve_split(split);
    if (split != SPD_SPLIT_ROW && split != SPD_SPLIT_NNZ) return fail(SPD_ERR_ARG, "unknown split %d", split);
    if (width < 0) return fail(SPD_ERR_SHAPE, "width %lld < 0", (long long)width);
    WsLayout L;
    switch (op) {
        case SPD_OP_SPMV: L = layout_spmv(A->nrows, A->nnz, split); break;
        case SPD_OP_SPMM: L = layout_warp(A->nrows, A->nnz, split, tn.unit_items, width, true); break;
        case SPD_OP_SPMM_T: L = layout_warp(A->nrows, A->nnz, split, tn.unit_items, width, false); break;
        case SPD_OP_SDDMM: L = layout_warp(A->nrows, A->nnz, split, tn.unit_items, 0, false); break;
        default: return fail(SPD_ERR_ARG, "op %d is not a CSR operation", op);
    }
    *bytes = L.total;
    return SPD_OK;
}

spd_status spd_csf3_workspace_size(int op, const spd_csf3 *B, int split, int64_t width, const spd_tune *tune,
                                   size_t *bytes) {
    g_last_error[0] = 0;
    if (!bytes) return fail(SPD_ERR_NULL, "bytes is NULL");
    spd_status s = check_csf3(B);
    if (s) return s;
    Tuning tn;
    if ((s = read_tune(tune, &tn))) return s;
    split = resolve_split(split);
    if (split != SPD_SPLIT_ROW && split != SPD_SPLIT_NNZ) return fail(SPD_ERR_ARG, "unknown split %d", split);
    if (width < 0) return fail(SPD_ERR_SHAPE, "width %lld < 0", (long long)width);
    WsLayout L;
    switch (op) {
        case SPD_OP_SPTTV: L = layout_spmv(B->nfib, B->nnz, split); break;
        case SPD_OP_SPMTTKRP: L = layout_mttkrp(B->nfib, B->nnz, split, tn.unit_items, width); break;
        default: return fail(SPD_ERR_ARG, "op %d is not a CSF operation", op);
    }
    *bytes = L.total;
    return SPD_OK;
}

spd_status spd_csr_partition(const spd_csr *A, int split, int64_t npieces, int64_t unit_items, int32_t *rows_out,
                             int32_t *pos_out, void *stream) {
    g_last_error[0] = 0;
    spd_status s = check_csr(A, false);
    if (s) return s;
    if (!rows_out || !pos_out) return fail(SPD_ERR_NULL, "output arrays are NULL");
    cudaStream_t st = as_stream(stream);
    split = resolve_split(split);
    if (split == SPD_SPLIT_ROW) {
        if (npieces < 1 || npieces > INT32_MAX) return fail(SPD_ERR_ARG, "npieces %lld out of range", (long long)npieces);
        if ((s = checked_csr(A, "A", st))) return s;
        int64_t grid = ceil_div(npieces + 1, 256);
        row_partition_kernel<<<(unsigned)grid, 256, 0, st>>>(A->nrows, A->pos, npieces, rows_out, pos_out);
        return checked_finish(check_launch("row_partition_kernel"), "spd_csr_partition", st);
    }
    if (split != SPD_SPLIT_NNZ) return fail(SPD_ERR_ARG, "unknown split %d", split);
    if (unit_items < 1) return fail(SPD_ERR_ARG, "unit_items %lld < 1", (long long)unit_items);
    int64_t want = ceil_div(A->nrows + A->nnz, unit_items);
    if (npieces != want)
        return fail(SPD_ERR_SHAPE, "npieces %lld != ceil((nrows+nnz)/unit_items) = %lld", (long long)npieces,
                    (long long)want);
    if ((s = checked_csr(A, "A", st))) return s;
    return checked_finish(launch_merge_partition(A->nrows, A->nnz, A->pos, unit_items, npieces, rows_out, pos_out, st),
                          "spd_csr_partition", st);
}

}  // extern "C"
