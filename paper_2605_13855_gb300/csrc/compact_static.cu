// compact_static.cu -- allocation-free variant of the active-set compaction.
//
// The paper has no counterpart to this entry point.  It exists for callers
// that cannot allocate device memory: code that must never trigger the
// implicit device-wide synchronisation of cudaMalloc / cudaFree (a training
// loop overlapping several streams), plug-ins that run inside another
// runtime which owns the whole device memory budget and hands out no
// allocator, and embedded or real-time users that forbid allocation after
// start-up.  They get the ascending index list of a mask without a context
// and without any allocation: the block-count scratch lives in a file-scope
// __device__ array of fixed size, so every GPU that loads the library holds
// it (about 16 KiB) until the process exits.
//
// Properties the caller has to respect:
//   * n <= kStaticMaxSplats (16,777,216); larger masks are rejected.
//   * All calls share the one scratch array and it keeps the contents of the
//     last call; every slot a call reads is written earlier by the same call,
//     so nothing needs clearing.  Calls that overlap on the GPU (different
//     streams, or different host threads on one device) race on it and give
//     wrong results: serialise them.
//   * The first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (with that device current) and caches it; make that
//     first call before any stream capture on that device.  The cached address
//     is kept for the process: a device reset (cudaDeviceReset) or a new
//     primary context between calls would leave it stale.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/sparseoit.h"
#include "common.cuh"

namespace soit {
namespace {

constexpr int kThreads = 256;
constexpr int kPer = 16;
constexpr int kBlockElems = kThreads * kPer;                  // 4096
constexpr int64_t kStaticMaxSplats = SPARSEOIT_STATIC_MAX_SPLATS;
constexpr int kStaticBlocks = (int)(kStaticMaxSplats / kBlockElems);  // 4096

// Block counts, then (in place) block offsets.  Only host code needs the
// address through cudaGetSymbolAddress; these kernels receive it as a pointer.
static __device__ __align__(256) int g_compact_scratch[kStaticBlocks];

__device__ __forceinline__ int block_exclusive_scan(int v, int *warp_tot, int *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int w = 0; w < kThreads / 32; ++w) {
            const int t = warp_tot[w];
            warp_tot[w] = run;
            run += t;
        }
        *total = run;
    }
    __syncthreads();
    return warp_tot[warp] + incl - v;
}

// Bit k set iff mask[i0 + k] != 0 (k < kPer, i0 + k < n): one 16-byte load when the run is aligned
// and whole, else byte loads.  Per 32-bit word x, ((x & 0x7f7f7f7f) + 0x7f7f7f7f) | x has the top
// bit of each byte set iff that byte is non-zero (no carry crosses a byte), and multiplying the
// four top bits by 1 + 2^7 + 2^14 + 2^21 gathers them into bits 28..31 in byte order.
__device__ __forceinline__ unsigned mask_bits16(const uint8_t *__restrict__ mask, int64_t i0, int64_t n) {
    static_assert(kPer == 16, "one uint4 a thread");
    const uint8_t *p = mask + i0;
    if (i0 + kPer <= n && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
        unsigned bits = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t t = (((w[k] & 0x7f7f7f7fu) + 0x7f7f7f7fu) | w[k]) & 0x80808080u;
            bits |= ((t * 0x00204081u) >> 28) << (4 * k);
        }
        return bits;
    }
    unsigned bits = 0;
    for (int k = 0; k < kPer; ++k)
        if (i0 + k < n && p[k] != 0) bits |= 1u << k;
    return bits;
}

__global__ void __launch_bounds__(kThreads) static_count_kernel(const uint8_t *__restrict__ mask, int64_t n,
                                                                int *__restrict__ scratch) {
    __shared__ int wt[kThreads / 32];
    __shared__ int tot;
    const int64_t i0 = (int64_t)blockIdx.x * kBlockElems + (int64_t)threadIdx.x * kPer;
    const int c = __popc(mask_bits16(mask, i0, n));
    block_exclusive_scan(c, wt, &tot);
    if (threadIdx.x == 0) scratch[blockIdx.x] = tot;
}

// One block of 1024 threads: exclusive scan of nblk block counts in place;
// the total goes to *count.
__global__ void __launch_bounds__(1024) static_scan_kernel(int *__restrict__ scratch, int nblk,
                                                           int64_t *__restrict__ count) {
    __shared__ int ws[32];
    __shared__ int carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nblk; base += 1024) {
        const int i = base + tid;
        const int v = i < nblk ? scratch[i] : 0;
        int incl = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane == 31) ws[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int s = ws[lane], si = s;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, si, off);
                if (lane >= off) si += y;
            }
            ws[lane] = si - s;
        }
        __syncthreads();
        const int ex = carry + ws[warp] + incl - v;
        if (i < nblk) scratch[i] = ex;
        __syncthreads();
        if (tid == 1023) carry = ex + v;
        __syncthreads();
    }
    if (tid == 0) *count = carry;
}

__global__ void __launch_bounds__(kThreads) static_write_kernel(const uint8_t *__restrict__ mask, int64_t n,
                                                                const int *__restrict__ scratch,
                                                                int32_t *__restrict__ idx) {
    __shared__ int wt[kThreads / 32];
    __shared__ int tot;
    const int64_t i0 = (int64_t)blockIdx.x * kBlockElems + (int64_t)threadIdx.x * kPer;
    const unsigned bits = mask_bits16(mask, i0, n);
    int pos = scratch[blockIdx.x] + block_exclusive_scan(__popc(bits), wt, &tot);
    for (int k = 0; k < kPer; ++k)
        if (bits & (1u << k)) idx[pos++] = (int32_t)(i0 + k);
}

std::mutex g_setup_mutex;
int *g_scratch_ptr[64] = {nullptr};  // device address of g_compact_scratch, per device id

}  // namespace
}  // namespace soit

extern "C" int sparseoit_compact_active_static(const uint8_t *d_mask, int64_t n, int32_t *d_idx, int64_t *d_count,
                                               void *stream) {
    using namespace soit;
    if (n < 0 || n > kStaticMaxSplats) return SPARSEOIT_ERR_INVALID_ARG;  // beyond the static scratch
    if (!d_count || (n > 0 && (!d_mask || !d_idx))) return SPARSEOIT_ERR_INVALID_ARG;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) return SPARSEOIT_ERR_CUDA;
    int *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_compact_scratch);
            if (e != cudaSuccess || !p) return SPARSEOIT_ERR_CUDA;
            g_scratch_ptr[dev] = static_cast<int *>(p);
        }
        scratch = g_scratch_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int nblk = (int)((n + kBlockElems - 1) / kBlockElems);
    if (nblk == 0) {
        e = cudaMemsetAsync(d_count, 0, sizeof(int64_t), st);
    } else {
        static_count_kernel<<<nblk, kThreads, 0, st>>>(d_mask, n, scratch);
        static_scan_kernel<<<1, 1024, 0, st>>>(scratch, nblk, d_count);
        static_write_kernel<<<nblk, kThreads, 0, st>>>(d_mask, n, scratch, d_idx);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? SPARSEOIT_OK : SPARSEOIT_ERR_CUDA;
}
