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
#include <cuda.h>

#include <mutex>

#include "spd_internal.cuh"

namespace spd {

spd_status spmv_nnz_on_scratch(const spd_csr *A, const void *x, void *y, void *scratch, cudaStream_t st);

constexpr size_t kNoAllocScratchBytes = size_t(1) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// In host code g_noalloc_scratch names a host-side shadow, not device memory, so the
// kernels get the device address that cudaGetSymbolAddress reports. The array exists
// once per CUDA context that loads this library's module (not once per device: a caller
// may make its own driver-API context current, and cudaDeviceReset ends a context whose
// successor loads the module again), so the address is cached per context, keyed by the
// driver's unique context id, and looked up again for a context not seen before.
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

struct ScratchSlot {
    unsigned long long ctx_id;
    void *addr;
};
constexpr int kScratchSlots = 64;
static std::mutex g_scratch_mutex;
static ScratchSlot g_slots[kScratchSlots];
static int g_slot_count = 0, g_slot_next = 0;

// Unique id of the calling thread's current context (0 when none is current). The two
// driver functions are reached through the runtime, so the library needs no link
// against the driver library.
static spd_status current_context_id(unsigned long long *id) {
    static std::once_flag once;
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
            get_id = reinterpret_cast<CtxGetIdFn>(f2);
        }
    });
    if (!get_current || !get_id) return fail(SPD_ERR_CUDA, "cuCtxGetCurrent / cuCtxGetId are not available");
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS) return fail(SPD_ERR_CUDA, "cuCtxGetCurrent failed");
    *id = 0;
    if (ctx && get_id(ctx, id) != CUDA_SUCCESS) return fail(SPD_ERR_CUDA, "cuCtxGetId failed");
    return SPD_OK;
}

// Device address of the scratch array in the current context. A context's first call
// does the lookup; it is refused while `st` is being captured into a graph.
static spd_status noalloc_scratch(cudaStream_t st, void **out) {
    unsigned long long id = 0;
    spd_status s = current_context_id(&id);
    if (s) return s;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (id) {
        for (int k = 0; k < g_slot_count; ++k)
            if (g_slots[k].ctx_id == id) {
                *out = g_slots[k].addr;
                return SPD_OK;
            }
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        cudaError_t e = cudaStreamIsCapturing(st, &cap);
        if (e != cudaSuccess) return fail(SPD_ERR_CUDA, "cudaStreamIsCapturing: %s", cudaGetErrorString(e));
        if (cap != cudaStreamCaptureStatusNone)
            return fail(SPD_ERR_ARG, "the first spd_spmv_noalloc call in a CUDA context must come before stream capture");
    }
    // With no context current yet, this runtime call makes the device's primary
    // context current; its id is read afterwards.
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return fail(SPD_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    if (!id && (s = current_context_id(&id))) return s;
    if (id) {
        const int k = g_slot_count < kScratchSlots ? g_slot_count++ : g_slot_next;
        if (g_slot_count == kScratchSlots) g_slot_next = (k + 1) % kScratchSlots;
        g_slots[k] = {id, p};
    }
    *out = p;
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
    if ((s = noalloc_scratch(st, &scratch))) return s;
    // Every scratch byte the kernels read is written earlier in the same call (partition
    // boundaries, then one carry per piece), so nothing has to be cleared between calls.
    return checked_finish(spmv_nnz_on_scratch(A, x, y, scratch, st), "spd_spmv_noalloc", st);
}
