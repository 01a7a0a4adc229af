// spd_internal.cuh -- shared device helpers and host-side argument plumbing of libspd.
//
// Layout and vocabulary follow the level formats of Sections II-B and III-B of
// SpDISTAL (arXiv 2207.13901): a Compressed level is (pos, crd) with the children of
// parent entry i at positions [pos[i], pos[i+1]).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>
#include <cstdio>
#include <cstring>

#include "../../include/spd.h"

namespace spd {

// ------------------------------------------------------------------ element types

template <typename VT> struct Traits;
template <> struct Traits<double> {
    using acc = double;  // accumulation type
    using out = double;  // result type
    static constexpr int code = SPD_F64;
};
template <> struct Traits<float> {
    using acc = float;
    using out = float;
    static constexpr int code = SPD_F32;
};
template <> struct Traits<__nv_bfloat16> {
    using acc = float;
    using out = float;
    static constexpr int code = SPD_BF16;
};

__device__ __forceinline__ float to_acc(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ double to_acc(double v) { return v; }

// Streaming (evict-first) loads for data read exactly once: crd, vals, pos windows.
__device__ __forceinline__ int32_t ld_stream(const int32_t *p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float *p) { return __ldcs(p); }
__device__ __forceinline__ double ld_stream(const double *p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const __nv_bfloat16 *p) { return __bfloat162float(__ldcs(p)); }

// Cached loads for gathered dense operands (reused through L1/L2).
__device__ __forceinline__ float ld_gather(const float *p) { return __ldg(p); }
__device__ __forceinline__ double ld_gather(const double *p) { return __ldg(p); }
__device__ __forceinline__ float ld_gather(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }

// Loads N consecutive elements starting at p (p aligned to N elements when N > 1)
// and converts them to the accumulation type.
template <int N>
__device__ __forceinline__ void ld_vec(const float *p, float (&o)[N]) {
    if constexpr (N == 1) {
        o[0] = __ldg(p);
    } else if constexpr (N == 2) {
        float2 v = __ldg(reinterpret_cast<const float2 *>(p));
        o[0] = v.x; o[1] = v.y;
    } else {
#pragma unroll
        for (int q = 0; q < N / 4; ++q) {
            float4 v = __ldg(reinterpret_cast<const float4 *>(p) + q);
            o[4 * q + 0] = v.x; o[4 * q + 1] = v.y; o[4 * q + 2] = v.z; o[4 * q + 3] = v.w;
        }
    }
}
template <int N>
__device__ __forceinline__ void ld_vec(const double *p, double (&o)[N]) {
    if constexpr (N == 1) {
        o[0] = __ldg(p);
    } else {
#pragma unroll
        for (int q = 0; q < N / 2; ++q) {
            double2 v = __ldg(reinterpret_cast<const double2 *>(p) + q);
            o[2 * q + 0] = v.x; o[2 * q + 1] = v.y;
        }
    }
}
template <int N>
__device__ __forceinline__ void ld_vec(const __nv_bfloat16 *p, float (&o)[N]) {
    if constexpr (N == 1) {
        o[0] = __bfloat162float(__ldg(p));
    } else if constexpr (N == 2) {
        float2 f = __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162 *>(p)));
        o[0] = f.x; o[1] = f.y;
    } else if constexpr (N == 4) {
        uint2 raw = __ldg(reinterpret_cast<const uint2 *>(p));
        __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162 *>(&raw.x);
        __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162 *>(&raw.y);
        float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
        o[0] = fa.x; o[1] = fa.y; o[2] = fb.x; o[3] = fb.y;
    } else {
#pragma unroll
        for (int q = 0; q < N / 8; ++q) {
            uint4 raw = __ldg(reinterpret_cast<const uint4 *>(p) + q);
            uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                float2 f = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162 *>(&w[h]));
                o[8 * q + 2 * h] = f.x;
                o[8 * q + 2 * h + 1] = f.y;
            }
        }
    }
}

// Stores N consecutive results (p aligned to N elements when N > 1), streaming.
template <int N>
__device__ __forceinline__ void st_vec(float *p, const float (&v)[N]) {
    if constexpr (N == 1) {
        __stcs(p, v[0]);
    } else if constexpr (N == 2) {
        __stcs(reinterpret_cast<float2 *>(p), make_float2(v[0], v[1]));
    } else {
#pragma unroll
        for (int q = 0; q < N / 4; ++q)
            __stcs(reinterpret_cast<float4 *>(p) + q, make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]));
    }
}
template <int N>
__device__ __forceinline__ void st_vec(double *p, const double (&v)[N]) {
    if constexpr (N == 1) {
        __stcs(p, v[0]);
    } else {
#pragma unroll
        for (int q = 0; q < N / 2; ++q)
            __stcs(reinterpret_cast<double2 *>(p) + q, make_double2(v[2 * q], v[2 * q + 1]));
    }
}

template <typename T, int N>
__device__ __forceinline__ void zero(T (&a)[N]) {
#pragma unroll
    for (int e = 0; e < N; ++e) a[e] = (T)0;
}

// One lane's EPL elements of a dense row, as loaded by one vector access. bfloat16
// elements stay packed two per register and are widened only when multiplied (exactly:
// a bfloat16 is the upper half of the binary32 of the same value).
template <typename VT, int EPL>
struct XVec {
    VT v[EPL];
    __device__ __forceinline__ void load(const VT *p) { ld_vec<EPL>(p, v); }
    __device__ __forceinline__ void clear() { zero(v); }
    __device__ __forceinline__ VT at(int e) const { return v[e]; }
};
template <int EPL>
struct XVec<__nv_bfloat16, EPL> {
    static constexpr int W = EPL >= 2 ? EPL / 2 : 1;
    uint32_t w[W];
    __device__ __forceinline__ void load(const __nv_bfloat16 *p) {
        if constexpr (EPL == 1) {
            w[0] = (uint32_t)__bfloat16_as_ushort(__ldg(p));
        } else if constexpr (EPL == 2) {
            w[0] = __ldg(reinterpret_cast<const unsigned int *>(p));
        } else if constexpr (EPL == 4) {
            const uint2 r = __ldg(reinterpret_cast<const uint2 *>(p));
            w[0] = r.x; w[1] = r.y;
        } else {
#pragma unroll
            for (int q = 0; q < EPL / 8; ++q) {
                const uint4 r = __ldg(reinterpret_cast<const uint4 *>(p) + q);
                w[4 * q] = r.x; w[4 * q + 1] = r.y; w[4 * q + 2] = r.z; w[4 * q + 3] = r.w;
            }
        }
    }
    __device__ __forceinline__ void clear() { zero(w); }
    __device__ __forceinline__ float at(int e) const {
        const uint32_t x = w[e >> 1];
        return __uint_as_float((e & 1) ? (x & 0xffff0000u) : (x << 16));
    }
};

// Kahan's compensated accumulation of a product a*b: s carries the running sum and c the
// negated rounding error of the additions so far (s - c approximates the exact sum).
template <typename T>
__device__ __forceinline__ void kahan_fma(T &s, T &c, T a, T b) {
    const T y = fma(a, b, -c);
    const T t = s + y;
    c = (t - s) - y;
    s = t;
}

// Compensated accumulation (Neumaier's variant of Kahan summation): hi + lo carries
// the running sum; lo collects the rounding error of every addition.
template <typename T>
__device__ __forceinline__ void comp_add(T &hi, T &lo, T b) {
    T s = hi + b;
    if (fabs(hi) >= fabs(b)) lo += (hi - s) + b;
    else lo += (b - s) + hi;
    hi = s;
}

// ------------------------------------------------------------------ bulk copies (TMA)

// A kernel whose bounded wait gives up ORs a kFault* bit into the device fault word of its
// translation unit and returns early (its results are then unspecified); spd_fault_status
// reads and clears the words.
constexpr unsigned kFaultBulkWait = 1u;  // a bulk copy did not complete within kWaitLimitNs
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // 1 s

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// One-arrival mbarrier for the completion of bulk copies (PTX ISA, "mbarrier").
__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
// Makes initialized mbarriers visible to the asynchronous (bulk copy) proxy.
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// The single arrival of a phase, announcing `bytes` of bulk copies that complete it.
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits until the phase of `bar` with the given parity has completed, for at most
// kWaitLimitNs; false (and kFaultBulkWait set in *fault) when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned int *fault) {
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_test(bar, parity)) {
        if (global_ns() - t0 > kWaitLimitNs) {
            atomicOr(fault, kFaultBulkWait);
            return false;
        }
    }
    return true;
}
// Orders this thread's earlier generic-proxy accesses of shared memory before later
// bulk copies into it.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// 1-D bulk copy (TMA) of `bytes` from global to shared memory, completing on `bar`.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// ------------------------------------------------------------------ partitions

// Merge-path state of the flattened coordinate tree: after d items, `rows` rows have
// ended and `pos` children have been consumed (rows + pos == d). Row r's end item
// sits at index pos[r+1] + r of the sequence (its children come first).
struct PieceBounds {
    int32_t r0, p0, r1, p1;
};

// Bounds of piece c of the universe (row) partition into P pieces:
// rows [floor(c n / P), floor((c+1) n / P)) and, by image, positions [pos[r0], pos[r1]).
__device__ __forceinline__ PieceBounds row_piece(int64_t c, int64_t P, int64_t n, const int32_t *pos) {
    PieceBounds b;
    b.r0 = (int32_t)((c * n) / P);
    b.r1 = (int32_t)(((c + 1) * n) / P);
    b.p0 = __ldg(pos + b.r0);
    b.p1 = __ldg(pos + b.r1);
    return b;
}

// Bounds of piece c of the fused non-zero partition, read from a partition array.
__device__ __forceinline__ PieceBounds nnz_piece(int64_t c, const int32_t *prow, const int32_t *ppos) {
    PieceBounds b;
    b.r0 = __ldg(prow + c);
    b.p0 = __ldg(ppos + c);
    b.r1 = __ldg(prow + c + 1);
    b.p1 = __ldg(ppos + c + 1);
    return b;
}

// Lane-parallel lookup of the parent of 32 children at once. Lane q of the window holds
// the end (in children) of parent rw + q; find() returns, for each lane, the parent
// whose child range holds the lane's child P, advancing the window as needed (parents
// must be >= rw).
struct PosRows {
    int32_t rw;
    int32_t wend;
    __device__ __forceinline__ void load(int32_t base, int64_t n, const int32_t *pos, int lane) {
        rw = base;
        wend = ((int64_t)base + lane < n) ? ld_stream(pos + base + lane + 1) : INT_MAX;
    }
    // Row of position P for every lane with `valid` (the rows must be >= rw).
    __device__ __forceinline__ int32_t find(int32_t P, bool valid, int64_t n, const int32_t *pos, int lane) {
        int32_t row = 0;
        bool done = !valid;
        while (true) {
            // number of window rows that end at or before P (0..32); every lane takes part
            // in every shuffle (the full mask requires it), the lane's own test follows
            int lo = __shfl_sync(0xffffffffu, wend, 31) <= P ? 32 : 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int32_t w = __shfl_sync(0xffffffffu, wend, (lo + step - 1) & 31);
                if (lo < 32 && w <= P) lo += step;
            }
            if (!done && lo < 32) {
                row = rw + lo;
                done = true;
            }
            if (!__any_sync(0xffffffffu, !done)) break;
            load(rw + 32, n, pos, lane);
        }
        return row;
    }
};

// Sums each of the U values of every lane over its group of G lanes. Returns, in each
// lane, the total of value u_of(lane) (see below); all values are summed exactly once.
template <int G, int U, typename T>
__device__ __forceinline__ T group_reduce(T (&v)[U], int lane) {
    int count = U;
#pragma unroll
    for (int off = G / 2; off >= 1; off >>= 1) {
        if (count > 1) {
            const int half = count / 2;
            const bool upper = (lane & off) != 0;
#pragma unroll
            for (int i = 0; i < U / 2; ++i) {
                if (i < half) {
                    const T send = upper ? v[i] : v[half + i];
                    const T keep = upper ? v[half + i] : v[i];
                    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
                }
            }
            count = half;
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], off);
        }
    }
    return v[0];
}

// Which of the U values a lane holds after group_reduce, and whether it writes it.
template <int G, int U>
__device__ __forceinline__ int reduced_index(int lane, bool &writer) {
    int u = 0, count = U, last = G;
#pragma unroll
    for (int off = G / 2; off >= 1; off >>= 1) {
        if (count > 1) {
            const int half = count / 2;
            if (lane & off) u += half;
            count = half;
            last = off;
        }
    }
    // after the halving steps the remaining butterfly makes every lane of a block of
    // `last` lanes hold the same total; the first lane of each block writes it
    writer = U == 1 ? (lane % G) == 0 : (lane & (last - 1)) == 0;
    return u;
}

// ------------------------------------------------------------------ host plumbing

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Records an error detail for spd_last_error() and returns the status.
spd_status fail(spd_status s, const char *fmt, ...);
spd_status check_launch(const char *what);
inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

inline bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
inline size_t dtype_size(int t) { return t == SPD_F64 ? 8 : t == SPD_F32 ? 4 : t == SPD_BF16 ? 2 : 0; }
inline int result_type(int t) { return t == SPD_F64 ? SPD_F64 : SPD_F32; }
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

spd_status check_csr(const spd_csr *A, bool need_vals);
spd_status check_csf3(const spd_csf3 *B);

// Checked mode (spd_set_checked / SPD_DEBUG=1 in the environment). When it is on, the
// compute calls validate their sparse operands through a device status word before they
// launch anything (returning SPD_ERR_STRUCTURE with the first bad index), and wait for
// their own work afterwards so that a launch or execution error is reported by the call
// that caused it. Both helpers return SPD_OK at once when checked mode is off.
bool checked_mode();
spd_status checked_csr(const spd_csr *A, const char *name, cudaStream_t st);
spd_status checked_csf3(const spd_csf3 *B, const char *name, cudaStream_t st);
spd_status checked_finish(spd_status s, const char *call, cudaStream_t st);
// Reads and clears the device fault words of the kernels with bounded waits (OR of the
// kFault* bits); synchronous, not for use during a graph capture.
spd_status take_device_faults(unsigned int *flags);

// Defaults shared by the size queries and the compute calls.
constexpr int kSpmvThreads = 256;   // threads of the tile-per-block SpMV / SpTTV kernel
constexpr int kSpmvIPT = 8;         // items per thread of one tile
constexpr int kSpmvTile = kSpmvThreads * kSpmvIPT;
constexpr int kWarpUnitDefault = 2048;  // items per warp unit (warp-per-unit kernels)
constexpr int kWarpBlockDefault = 256;
constexpr int kWarpBlockMax = 512;      // largest block of the warp-per-unit kernels

struct Tuning {
    int64_t unit_items;   // warp-unit size of SPD_SPLIT_NNZ (warp kernels)
    int64_t row_pieces;   // P of SPD_SPLIT_ROW (0 = per-kernel default)
    int block_threads;    // threads per block (warp kernels)
    int inflight;         // dense rows in flight per group (SpMM)
    int lane_groups;      // SpMM lane shape: 0 = by the size of X, 1 = groups, 2 = 32 lanes
    int form;             // kernel form (0 = library's choice): SpMV/SpTTV 1 = block tiles, 2 = warp tiles;
                          // SDDMM 1 = CUDA cores, 2 = tensor cores
};
spd_status read_tune(const spd_tune *t, Tuning *out);
int resolve_split(int split);

// Workspace of one partitioned call: the partition arrays (nnz split only) and the
// binary64 carries of outer entries cut by piece boundaries.
struct WsLayout {
    int64_t npieces = 0;
    size_t part_row = 0, part_pos = 0, part_aux = 0, carry_row = 0, carry_val = 0;
    size_t chunk_row = 0, chunk_val = 0;  // sums of the carries of kCarryChunk pieces
    size_t total = 0;
};
// Pieces per chunk of the two-level carry fix-up.
constexpr int kCarryChunk = 32;
// npieces pieces, `width` carried values per piece, `aux` = extra int32 per boundary,
// `chunks` = room for the chunk sums of the row fix-up.
WsLayout make_layout(int64_t npieces, int64_t width, bool need_partition, bool need_carry, bool aux,
                     bool chunks = false);

// Launches the fused non-zero partition of a level (pos, n parents, nnz children) into
// the boundary arrays prow/ppos (npieces + 1 entries each).
spd_status launch_merge_partition(int64_t n, int64_t nnz, const int32_t *pos, int64_t unit,
                                  int64_t npieces, int32_t *prow, int32_t *ppos, cudaStream_t st);

// Workspace layouts of the calls (shared by the size queries and the compute calls).
WsLayout layout_spmv(int64_t n, int64_t nnz, int split);
WsLayout layout_warp(int64_t n, int64_t nnz, int split, int64_t unit, int64_t width, bool carries);
WsLayout layout_mttkrp(int64_t F, int64_t nnz, int split, int64_t unit, int64_t R);

spd_status check_ws(const WsLayout &L, void *ws, size_t ws_bytes);
spd_status check_dense(const char *name, const void *p, int64_t rows, int64_t L, int64_t ld, int t);

// Elements per lane for the warp kernels: the smallest power of two that lets 32 lanes
// cover L, capped by a 32-byte vector, lowered until the pointers and leading
// dimensions allow vector accesses of that width.
int pick_epl(int64_t L, size_t in_size, size_t out_size, const void *in, int64_t ld_in, const void *out,
             int64_t ld_out);

// Lane shape of the SpMM kernels. group == 32: one entry per warp step, epl from
// pick_epl. group in {4, 8, 16}: lane groups with one 16-byte vector per lane, used
// when L needs fewer than 32 such lanes, the operands allow 16-byte vectors and
// lane_groups asks for it (1) or leaves it to the size of X (0: x_bytes <= 64 MiB).
struct SpmmShape {
    int epl;
    int group;
};
SpmmShape pick_spmm_shape(int64_t L, size_t in_size, size_t out_size, const void *in, int64_t ld_in,
                          const void *out, int64_t ld_out, int lane_groups, uint64_t x_bytes);

// Device-wide exclusive prefix sum of N int32 values in place (three launches on
// `st`); `sums` holds scan_tile_count(N) ints of scratch.
int64_t scan_tile_count(int64_t N);
spd_status exclusive_scan_i32(int32_t *data, int64_t N, int32_t *sums, cudaStream_t st);

// Zero rows x L of a row-major matrix with leading dimension lda (one warp per row).
template <typename OT>
__global__ void zero_rows_kernel(int64_t rows, int64_t L, OT *__restrict__ A, int64_t lda) {
    const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < rows; i += wstride)
        for (int64_t l = threadIdx.x & 31; l < L; l += 32) A[i * lda + l] = (OT)0;
}

template <typename OT>
inline spd_status launch_zero_rows(int64_t rows, int64_t L, OT *A, int64_t lda, cudaStream_t st) {
    if (rows <= 0 || L <= 0) return SPD_OK;
    int64_t grid = ceil_div(rows, 8);
    if (grid > 152 * 64) grid = 152 * 64;
    zero_rows_kernel<OT><<<(unsigned)grid, 256, 0, st>>>(rows, L, A, lda);
    return check_launch("zero_rows_kernel");
}

// Adds the binary64 carries of consecutive pieces that ended inside the same outer entry
// (row or slice) to the value the completing piece wrote. One warp per piece, one lane
// per column; only the first piece of each run does the work.
// First level of the row fix-up: for every chunk of kCarryChunk consecutive pieces that
// all ended inside the same row, the sum of their carries (in piece order) and that row;
// other chunks get row -1. One warp per chunk, each lane EPL columns.
template <int EPL>
__global__ void carry_chunk_kernel(int64_t npieces, int64_t L, const int32_t *__restrict__ carry_row,
                                   const double *__restrict__ carry_val, int32_t *__restrict__ chunk_row,
                                   double *__restrict__ chunk_val) {
    const int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const int64_t nch = (npieces + kCarryChunk - 1) / kCarryChunk;
    if (k >= nch) return;  // whole warp
    const int64_t c0 = k * kCarryChunk;
    const int32_t mine = c0 + lane < npieces ? carry_row[c0 + lane] : -2;
    const int32_t row = __shfl_sync(0xffffffffu, mine, 0);
    const bool whole = row >= 0 && __all_sync(0xffffffffu, mine == row);
    if (blockIdx.y == 0 && lane == 0) chunk_row[k] = whole ? row : -1;
    const int64_t col = ((int64_t)blockIdx.y * 32 + lane) * EPL;
    if (!whole || col >= L) return;
    double s[EPL];
#pragma unroll
    for (int e = 0; e < EPL; ++e) s[e] = 0.0;
#pragma unroll 4
    for (int d = 0; d < kCarryChunk; ++d) {
        double v[EPL];
        ld_vec<EPL>(carry_val + (c0 + d) * L + col, v);
#pragma unroll
        for (int e = 0; e < EPL; ++e) s[e] += v[e];
    }
    double *o = chunk_val + k * L + col;
#pragma unroll
    for (int e = 0; e < EPL; ++e) o[e] = s[e];
}

// Adds the binary64 carries of consecutive pieces that ended inside the same row to the
// row the completing piece wrote: one warp per piece (only the first piece of a run
// works), each lane EPL consecutive columns (vector loads of the carries and of Y). A run
// is walked piece by piece up to a chunk boundary, then a chunk at a time while whole
// chunks lie inside it, then piece by piece again: a row spanning thousands of pieces
// costs about a hundred dependent loads instead of thousands. The order of the sums is
// fixed by the chunking, so results do not change from run to run.
template <typename OT, int EPL>
__global__ void carry_fixup_rows_kernel(int64_t npieces, int64_t L, const int32_t *__restrict__ carry_row,
                                        const double *__restrict__ carry_val, const int32_t *__restrict__ chunk_row,
                                        const double *__restrict__ chunk_val, OT *__restrict__ Y, int64_t ldy) {
    const int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t col = ((int64_t)blockIdx.y * 32 + (threadIdx.x & 31)) * EPL;
    if (c >= npieces || col >= L) return;
    const int32_t row = carry_row[c];
    if (row < 0) return;
    if (c > 0 && carry_row[c - 1] == row) return;
    double s[EPL];
    ld_vec<EPL>(carry_val + c * L + col, s);
    int64_t d = c + 1;
    while (d < npieces) {
        if (d % kCarryChunk == 0 && chunk_row[d / kCarryChunk] == row) {
            double v[EPL];
            ld_vec<EPL>(chunk_val + (d / kCarryChunk) * L + col, v);
#pragma unroll
            for (int e = 0; e < EPL; ++e) s[e] += v[e];
            d += kCarryChunk;
            continue;
        }
        if (carry_row[d] != row) break;
        double v[EPL];
        ld_vec<EPL>(carry_val + d * L + col, v);
#pragma unroll
        for (int e = 0; e < EPL; ++e) s[e] += v[e];
        ++d;
    }
    OT *yp = Y + (int64_t)row * ldy + col;
    OT o[EPL];
    ld_vec<EPL>(yp, o);
#pragma unroll
    for (int e = 0; e < EPL; ++e) o[e] = (OT)((double)o[e] + s[e]);
    st_vec(yp, o);
}

// Both levels of the row fix-up; chunk_row / chunk_val: the workspace's chunk area.
template <typename OT>
inline spd_status launch_carry_fixup(int64_t npieces, int64_t L, const int32_t *crow, const double *cval,
                                     int32_t *chunk_row, double *chunk_val, OT *Y, int64_t ldy, cudaStream_t st) {
    if (npieces <= 0 || L <= 0) return SPD_OK;
    const int64_t nch = (npieces + kCarryChunk - 1) / kCarryChunk;
    const bool vec4 = L % 4 == 0 && ldy % 4 == 0 && aligned(Y, 4 * sizeof(OT)) && aligned(cval, 32) &&
                      aligned(chunk_val, 32);
    if (vec4) {
        carry_chunk_kernel<4><<<dim3((unsigned)ceil_div(nch, 8), (unsigned)ceil_div(L, 128)), 256, 0, st>>>(
            npieces, L, crow, cval, chunk_row, chunk_val);
        dim3 grid((unsigned)ceil_div(npieces, 8), (unsigned)ceil_div(L, 128));
        carry_fixup_rows_kernel<OT, 4><<<grid, 256, 0, st>>>(npieces, L, crow, cval, chunk_row, chunk_val, Y, ldy);
    } else {
        carry_chunk_kernel<1><<<dim3((unsigned)ceil_div(nch, 8), (unsigned)ceil_div(L, 32)), 256, 0, st>>>(
            npieces, L, crow, cval, chunk_row, chunk_val);
        dim3 grid((unsigned)ceil_div(npieces, 8), (unsigned)ceil_div(L, 32));
        carry_fixup_rows_kernel<OT, 1><<<grid, 256, 0, st>>>(npieces, L, crow, cval, chunk_row, chunk_val, Y, ldy);
    }
    return check_launch("carry_fixup_rows_kernel");
}

}  // namespace spd
