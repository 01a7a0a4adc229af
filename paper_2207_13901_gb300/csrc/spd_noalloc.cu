// spd_noalloc.cu -- SpMV for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocator) at all: code running inside a
// host application or plugin framework that owns every device allocation, or a
// latency-critical path that may not pay for an allocator call and the device
// synchronisation it can imply. The regular spd_spmv asks such a caller for a
// workspace it cannot provide, so spd_spmv_noalloc runs the same nnz-split SpMV on a
// fixed scratch area that lives inside this library instead.
//
// The scratch is one file-scope __device__ array of kNoAllocScratchBytes (1 MiB). Every
// GPU that loads the library holds that megabyte until the process exits; it is
// created with the module, so no call allocates anything.
#include <mutex>

#include "spd_internal.cuh"

namespace spd {

spd_status spmv_nnz_on_scratch(const spd_csr *A, const void *x, void *y, void *scratch, cudaStream_t st);

constexpr size_t kNoAllocScratchBytes = size_t(1) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// In host code g_noalloc_scratch names a host-side shadow, not device memory, so the
// kernels get the device address that cudaGetSymbolAddress reports, looked up once per
// device (with that device current) and cached.
static std::mutex g_scratch_mutex;
static void *g_scratch_addr[128];

static spd_status noalloc_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(SPD_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= 128) return fail(SPD_ERR_ARG, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(SPD_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return SPD_OK;
}

}  // namespace spd

using namespace spd;

extern "C" spd_status spd_spmv_noalloc(const spd_csr *A, const void *x, int x_type, void *y, int y_type,
                                       void *stream) {
    spd_status s = check_csr(A, true);
    if (s) return s;
    if (x_type != A->vtype) return fail(SPD_ERR_DTYPE, "x type %d differs from the value type %d", x_type, A->vtype);
    if (y_type != result_type(A->vtype)) return fail(SPD_ERR_DTYPE, "y type %d; expected %d", y_type, result_type(A->vtype));
    if (A->ncols > 0 && !x) return fail(SPD_ERR_NULL, "x is NULL");
    if (A->nrows > 0 && !y) return fail(SPD_ERR_NULL, "y is NULL");
    if ((x && !aligned(x, dtype_size(x_type))) || (y && !aligned(y, dtype_size(y_type))))
        return fail(SPD_ERR_ALIGN, "x or y not aligned to its element size");
    const WsLayout L = layout_spmv(A->nrows, A->nnz, SPD_SPLIT_NNZ);
    if (L.total > kNoAllocScratchBytes)
        return fail(SPD_ERR_SHAPE,
                    "nrows + nnz = %lld needs %zu bytes of scratch; spd_spmv_noalloc has %zu (use spd_spmv with a "
                    "workspace)",
                    (long long)(A->nrows + A->nnz), L.total, kNoAllocScratchBytes);
    cudaStream_t st = as_stream(stream);
    if ((s = checked_csr(A, "A", st))) return s;
    if (A->nrows == 0) return SPD_OK;
    void *scratch = nullptr;
    if ((s = noalloc_scratch(&scratch))) return s;
    // Every scratch byte the kernels read is written earlier in the same call (partition
    // boundaries, then one carry per piece), so nothing has to be cleared between calls.
    return checked_finish(spmv_nnz_on_scratch(A, x, y, scratch, st), "spd_spmv_noalloc", st);
}
