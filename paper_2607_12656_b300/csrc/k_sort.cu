// Device sorting and scanning shared by the renderer and the encoder: an exclusive u32 scan
// (three launches: per-block sums, one block scanning the sums, per-block apply) and a stable
// LSD radix sort of (u32 key, u32 value) pairs, 8-bit digits, one pass = per-block digit
// counts, a digit-major scan of the counts, a stable scatter.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sgs_device.cuh"
#include "sgs_internal.h"

namespace sgs {

// ------------------------------------------------------------------ scan (exclusive, u32)

__device__ __forceinline__ uint32_t block_scan_1024(uint32_t v, uint32_t *sm /*[32]*/, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) sm[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = sm[lane], wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        sm[lane] = wi - w;
        if (lane == 31) sm[32] = wi;
    }
    __syncthreads();
    const uint32_t ex = sm[warp] + incl - v;
    *total = sm[32];
    __syncthreads();
    return ex;
}

// sums[b] = sum of in[b * 1024 .. +1024)
__global__ void __launch_bounds__(kScanBlock) k_scan_sums(const uint32_t *in, uint64_t n, uint32_t *sums) {
    __shared__ uint32_t sm[33];
    const uint64_t i = (uint64_t)blockIdx.x * kScanBlock + threadIdx.x;
    uint32_t tot;
    block_scan_1024(i < n ? in[i] : 0u, sm, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// exclusive scan of sums[0 .. m) in place by one block; sums[m] = total
__global__ void __launch_bounds__(kScanBlock) k_scan_top(uint32_t *sums, uint32_t m) {
    __shared__ uint32_t sm[33];
    uint32_t carry = 0;
    for (uint32_t base = 0; base < m; base += kScanBlock) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < m ? sums[i] : 0u;
        uint32_t tot;
        const uint32_t ex = block_scan_1024(v, sm, &tot);
        if (i < m) sums[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) sums[m] = carry;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_apply(const uint32_t *in, uint64_t n, const uint32_t *sums,
                                                            uint32_t *out) {
    __shared__ uint32_t sm[33];
    const uint64_t i = (uint64_t)blockIdx.x * kScanBlock + threadIdx.x;
    uint32_t tot;
    const uint32_t ex = block_scan_1024(i < n ? in[i] : 0u, sm, &tot);
    if (i < n) out[i] = sums[blockIdx.x] + ex;
}


__device__ __forceinline__ uint32_t digit_of(uint32_t key, int shift) { return (key >> shift) & 255u; }

// counts[d * nb + b] = items of block b with digit d
__global__ void __launch_bounds__(kSortThreads) k_sort_count(const uint32_t *keys, uint32_t n, int shift, uint32_t nb,
                                                              uint32_t *counts) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * kSortChunk;
    uint32_t d[kSortRounds];  // the keys are loaded before any count is added: all in flight
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const uint64_t i = base + (uint64_t)r * kSortThreads + threadIdx.x;
        d[r] = i < n ? digit_of(keys[i], shift) : 256u;
    }
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r)
        if (d[r] < 256u) atomicAdd(&h[d[r]], 1u);
    __syncthreads();
    counts[(size_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: item order within a block is round-major, lanes in order; ranks among equal
// digits come from match_any inside a warp and a per-digit prefix over the warps.  The block
// first places its items in shared memory in block-sorted order, then writes each digit's
// run to its global place, so consecutive threads store to consecutive addresses.
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(const uint32_t *keys, const uint32_t *vals, uint32_t n,
                                                                int shift, uint32_t nb, const uint32_t *offs,
                                                                uint32_t *keys_out, uint32_t *vals_out) {
    __shared__ uint32_t cnt[kSortThreads / 32][256];
    __shared__ uint32_t run[256], lbase[256], goff[256], scan_sm[8];
    __shared__ uint32_t sk[kSortChunk];
    __shared__ uint32_t sv[kSortChunk];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    run[threadIdx.x] = 0;
    goff[threadIdx.x] = offs[(size_t)threadIdx.x * nb + blockIdx.x];
    const uint64_t base = (uint64_t)blockIdx.x * kSortChunk;
    uint32_t key[kSortRounds];
    uint32_t val[kSortRounds], dig[kSortRounds], lrank[kSortRounds];
    // every round's items are loaded before the first barrier: all of a thread's loads in flight
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        const uint64_t i = base + (uint64_t)r * kSortThreads + threadIdx.x;
        const bool live = i < n;
        key[r] = live ? keys[i] : 0u;
        val[r] = live ? vals[i] : 0u;
        dig[r] = live ? digit_of(key[r], shift) : 256u;  // no digit: matches no real one
    }
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r) {
        for (int w = 0; w < kSortThreads / 32; ++w) cnt[w][threadIdx.x] = 0;
        __syncthreads();
        const bool live = dig[r] < 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, dig[r]);
        const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        if (live && rank == 0) cnt[warp][dig[r]] = __popc(peers);
        __syncthreads();
        {   // thread t: prefix of digit t over the warps, continuing the block's running count
            uint32_t acc = run[threadIdx.x];
            for (int w = 0; w < kSortThreads / 32; ++w) {
                const uint32_t c = cnt[w][threadIdx.x];
                cnt[w][threadIdx.x] = acc;
                acc += c;
            }
            run[threadIdx.x] = acc;
        }
        __syncthreads();
        lrank[r] = live ? cnt[warp][dig[r]] + rank : 0u;
        __syncthreads();
    }
    uint32_t total;
    lbase[threadIdx.x] = block_excl_scan_256(run[threadIdx.x], &total, scan_sm);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortRounds; ++r)
        if (dig[r] < 256u) {
            const uint32_t p = lbase[dig[r]] + lrank[r];
            sk[p] = key[r];
            sv[p] = val[r];
        }
    __syncthreads();
    const uint32_t m = (uint32_t)min((uint64_t)kSortChunk, (uint64_t)n - base);
    for (uint32_t k = threadIdx.x; k < m; k += kSortThreads) {
        const uint32_t kk = sk[k];
        const uint32_t d = digit_of(kk, shift);
        const uint32_t g = goff[d] + (k - lbase[d]);
        keys_out[g] = kk;
        vals_out[g] = sv[k];
    }
}


cudaError_t scan_u32(const uint32_t *in, uint64_t n, uint32_t *sums, uint32_t *out, cudaStream_t st) {
    const uint32_t nb = (uint32_t)((n + kScanBlock - 1) / kScanBlock);
    if (nb == 0) return cudaSuccess;
    k_scan_sums<<<nb, kScanBlock, 0, st>>>(in, n, sums);
    k_scan_top<<<1, kScanBlock, 0, st>>>(sums, nb);
    k_scan_apply<<<nb, kScanBlock, 0, st>>>(in, n, sums, out);
    return cudaGetLastError();
}

cudaError_t radix_pass(const uint32_t *keys, const uint32_t *vals, uint32_t n, int shift, uint32_t *cnt,
                       uint32_t *cnt_off, uint32_t *csums, uint32_t *keys_out, uint32_t *vals_out, cudaStream_t st) {
    const uint32_t nb = (n + kSortChunk - 1) / kSortChunk;
    if (nb == 0) return cudaSuccess;
    k_sort_count<<<nb, kSortThreads, 0, st>>>(keys, n, shift, nb, cnt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = scan_u32(cnt, 256ull * nb, csums, cnt_off, st)) != cudaSuccess) return e;
    k_sort_scatter<<<nb, kSortThreads, 0, st>>>(keys, vals, n, shift, nb, cnt_off, keys_out, vals_out);
    return cudaGetLastError();
}

}  // namespace sgs
