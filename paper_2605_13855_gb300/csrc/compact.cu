// compact.cu -- active-set stream compaction (Sec. 4.1, "marks each gaussian
// by two categories of labels").  From the new mask and the previous one,
// four ascending index lists are produced in one ordered compaction:
//   active A = {i : new_i},  complement = {i : !new_i},
//   D+ = {i : prev_i && !new_i} (newly frozen),  D- = {i : new_i && !prev_i}.
// Three passes: per-block counts of the four predicates, a one-block scan
// of the block counts, then per-block ordered writes.  The four counts of a
// thread (<= 16 each) and of a block (<= 4096) are packed into 16-bit lanes
// of one 64-bit integer so that a single block scan serves all four lists.
#include "common.cuh"
#include "launch.h"

namespace soit {

constexpr int kCompactThreads = 256;
constexpr int kPerThread = 16;
constexpr int kPerBlock = kCompactThreads * kPerThread;  // 4096

__device__ __forceinline__ unsigned long long pred_bits(uint8_t nw, uint8_t pv) {
    const unsigned a = nw != 0, p = pv != 0;
    return (unsigned long long)a | ((unsigned long long)(1u - a) << 16) | ((unsigned long long)(p & (1u - a)) << 32) |
           ((unsigned long long)(a & (1u - p)) << 48);
}

__device__ __forceinline__ unsigned long long block_exclusive_scan_u64(unsigned long long v,
                                                                        unsigned long long *warp_tot,
                                                                        unsigned long long *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long run = 0;
        for (int w = 0; w < kCompactThreads / 32; ++w) {
            const unsigned long long t = warp_tot[w];
            warp_tot[w] = run;
            run += t;
        }
        *total = run;
    }
    __syncthreads();
    return warp_tot[warp] + incl - v;
}

__global__ void __launch_bounds__(kCompactThreads) compact_count_kernel(const uint8_t *__restrict__ nw,
                                                                        const uint8_t *__restrict__ pv, int64_t n,
                                                                        int *__restrict__ blk_counts, int nblk) {
    __shared__ unsigned long long wt[kCompactThreads / 32];
    __shared__ unsigned long long tot;
    const int64_t i0 = (int64_t)blockIdx.x * kPerBlock + (int64_t)threadIdx.x * kPerThread;
    unsigned long long c = 0;
    for (int k = 0; k < kPerThread; ++k) {
        const int64_t i = i0 + k;
        if (i < n) c += pred_bits(nw[i], pv ? pv[i] : (uint8_t)0);
    }
    block_exclusive_scan_u64(c, wt, &tot);
    if (threadIdx.x == 0) {
        for (int p = 0; p < 4; ++p) blk_counts[p * nblk + blockIdx.x] = (int)((tot >> (16 * p)) & 0xffffull);
    }
}

// One block: exclusive scan of the 4 x nblk block counts, totals to totals[4].
__global__ void __launch_bounds__(1024) compact_scan_kernel(int *__restrict__ blk_counts, int nblk,
                                                            int64_t *__restrict__ totals) {
    __shared__ int64_t carry[4];
    __shared__ int64_t wsum[4][32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 4) carry[tid] = 0;
    __syncthreads();
    for (int base = 0; base < nblk; base += 1024) {
        const int i = base + tid;
        for (int p = 0; p < 4; ++p) {
            const int64_t v = i < nblk ? blk_counts[p * nblk + i] : 0;
            int64_t incl = v;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                int64_t y = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += y;
            }
            if (lane == 31) wsum[p][warp] = incl;
            __syncthreads();
            if (warp == 0) {
                int64_t ws = wsum[p][lane], wi = ws;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    int64_t y = __shfl_up_sync(0xffffffffu, wi, off);
                    if (lane >= off) wi += y;
                }
                wsum[p][lane] = wi - ws;
            }
            __syncthreads();
            const int64_t ex = carry[p] + wsum[p][warp] + incl - v;
            if (i < nblk) blk_counts[p * nblk + i] = (int)ex;
            __syncthreads();
            if (tid == 1023) carry[p] = ex + v;
            __syncthreads();
        }
    }
    if (tid < 4) totals[tid] = carry[tid];
}

__global__ void __launch_bounds__(kCompactThreads) compact_write_kernel(
    const uint8_t *__restrict__ nw, const uint8_t *__restrict__ pv, int64_t n, const int *__restrict__ blk_offsets,
    int nblk, int *__restrict__ out_a, int *__restrict__ out_c, int *__restrict__ out_p, int *__restrict__ out_m,
    uint8_t *__restrict__ mask_store) {
    __shared__ unsigned long long wt[kCompactThreads / 32];
    __shared__ unsigned long long tot;
    const int64_t i0 = (int64_t)blockIdx.x * kPerBlock + (int64_t)threadIdx.x * kPerThread;
    unsigned long long bits[kPerThread];
    unsigned long long c = 0;
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const int64_t i = i0 + k;
        bits[k] = i < n ? pred_bits(nw[i], pv ? pv[i] : (uint8_t)0) : 0ull;
        c += bits[k];
    }
    unsigned long long ex = block_exclusive_scan_u64(c, wt, &tot);
    int pos[4];
    for (int p = 0; p < 4; ++p) pos[p] = blk_offsets[p * nblk + blockIdx.x] + (int)((ex >> (16 * p)) & 0xffffull);
    int *outs[4] = {out_a, out_c, out_p, out_m};
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const int64_t i = i0 + k;
        if (i >= n) break;
        for (int p = 0; p < 4; ++p)
            if ((bits[k] >> (16 * p)) & 1ull) outs[p][pos[p]++] = (int)i;
        mask_store[i] = (uint8_t)(bits[k] & 1ull);
    }
}

int64_t compact_scratch_ints(int64_t n) { return 4 * ((n + kPerBlock - 1) / kPerBlock) + 4; }

int launch_compact(const uint8_t *mask_new, const uint8_t *mask_prev, int64_t n, int *blk_counts, int64_t *totals,
                   int *idx_active, int *idx_comp, int *idx_plus, int *idx_minus, uint8_t *mask_store,
                   cudaStream_t st) {
    const int nblk = (int)((n + kPerBlock - 1) / kPerBlock);
    if (nblk == 0) {
        cudaMemsetAsync(totals, 0, 4 * sizeof(int64_t), st);
        return 0;
    }
    compact_count_kernel<<<nblk, kCompactThreads, 0, st>>>(mask_new, mask_prev, n, blk_counts, nblk);
    compact_scan_kernel<<<1, 1024, 0, st>>>(blk_counts, nblk, totals);
    compact_write_kernel<<<nblk, kCompactThreads, 0, st>>>(mask_new, mask_prev, n, blk_counts, nblk, idx_active,
                                                           idx_comp, idx_plus, idx_minus, mask_store);
    return 0;
}

}  // namespace soit
