// Device helpers shared by the sgs kernels (rANS group streams, tables, scans, dequant).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sgs_internal.h"

namespace sgs {

__device__ __forceinline__ uint32_t ld_u16(const uint8_t *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8);
}

__device__ __forceinline__ float ld_f32(const uint8_t *p) {  // p 4-byte aligned
    return *reinterpret_cast<const float *>(p);
}

// Dequantization (fp32): v = fl(fl(q * step) + offset), two roundings, never fused.
__device__ __forceinline__ float dequant(uint32_t q, float step, float offset) {
    return __fadd_rn(__fmul_rn((float)q, step), offset);
}

__device__ __forceinline__ uint64_t warp_max_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        uint64_t n = __shfl_xor_sync(0xffffffffu, v, o);
        v = n > v ? n : v;
    }
    return v;
}

// Block-wide exclusive scan of one u32 per thread (blockDim.x == 256); *total = sum.
__device__ __forceinline__ uint32_t block_excl_scan_256(uint32_t v, uint32_t *total,
                                                        uint32_t *sm /*[8]*/) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t n = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += n;
    }
    if (lane == 31) sm[warp] = incl;
    __syncthreads();
    uint32_t wbase = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        uint32_t s = sm[w];
        if (w < warp) wbase += s;
        tot += s;
    }
    __syncthreads();
    *total = tot;
    return wbase + incl - v;
}

// Copies n expanded tables (cdf[257] + bucket[256] each) into shared memory.
__device__ __forceinline__ void load_tables_smem(const uint8_t *tables, int n, uint32_t *s_cdf,
                                                 uint8_t *s_bucket) {
    for (int i = threadIdx.x; i < n * kTabCdfWords; i += blockDim.x) {
        int t = i / kTabCdfWords, k = i - t * kTabCdfWords;
        s_cdf[i] = reinterpret_cast<const uint32_t *>(tables + (size_t)t * kTabBytes)[k];
    }
    for (int i = threadIdx.x; i < n * 256; i += blockDim.x) {
        int t = i >> 8, k = i & 255;
        s_bucket[i] = tables[(size_t)t * kTabBytes + kTabCdfWords * 4 + k];
    }
}

// One rANS decode step (M = 2^16) against a cdf[257] + bucket[256] table.
__device__ __forceinline__ uint32_t rans_sym(uint32_t &x, const uint32_t *cdf,
                                             const uint8_t *bucket) {
    const uint32_t slot = x & 0xFFFFu;
    uint32_t s = bucket[slot >> 8];
    while (s < 255 && cdf[s + 1] <= slot) ++s;
    const uint32_t lo = cdf[s];
    const uint32_t f = cdf[s + 1] - lo;
    x = f * (x >> 16) + slot - lo;
    return s;
}

// Word stream of one group of up to 32 lanes, read through a shared-memory window of
// kWinWords words that the warp refills with coalesced 16-byte loads.
constexpr uint32_t kWinWords = 1024;

struct GroupStream {
    const uint8_t *w;   // group stream (16-byte aligned)
    uint32_t n_words;
    uint32_t ptr;       // next word to read
    uint32_t wbase;     // first word held in the window
    uint32_t wlimit;    // refill once ptr passes this (wbase + kWinWords - 32)
    uint16_t *win;      // this warp's window
    bool bad;
};

// Loads words [base, base + kWinWords) of the stream into the window (zero past the end).
__device__ __forceinline__ void window_fill(GroupStream &gs, uint32_t base) {
    const int lane = threadIdx.x & 31;
    gs.wbase = base;
    gs.wlimit = base + kWinWords - 32;
    const uint4 *src = reinterpret_cast<const uint4 *>(gs.w) + (base >> 3);
    uint4 *dst = reinterpret_cast<uint4 *>(gs.win);
    const uint32_t n16 = (gs.n_words + 7) >> 3;  // 16-byte units holding stream words
#pragma unroll
    for (uint32_t i = lane; i < kWinWords / 8; i += 32) {
        uint4 v = make_uint4(0, 0, 0, 0);
        if ((base >> 3) + i < n16) v = src[i];
        dst[i] = v;
    }
    __syncwarp();
}

// Opens group g's stream (bounds-checked against the payload), fills the window and reads
// this lane's initial state (hi word, lo word).  Returns false if the group table is bad.
__device__ __forceinline__ bool group_open(const uint8_t *bits, uint64_t grp_sec,
                                           uint64_t pay_off, uint64_t pay_len, uint32_t G,
                                           uint32_t g, int nl, int lane, GroupStream &gs,
                                           uint32_t &x, uint16_t *win) {
    const uint64_t *goff = reinterpret_cast<const uint64_t *>(bits + grp_sec);
    const uint32_t *gw = reinterpret_cast<const uint32_t *>(bits + grp_sec + 8ull * (G + 1));
    const uint64_t o = goff[g];
    const uint32_t nw = gw[g];
    // the window reads whole 16-byte units: the padded stream must hold them
    const bool ok = (o <= pay_len) && (((2ull * nw + 15) & ~15ull) <= pay_len - o) &&
                    (nw >= 2u * (uint32_t)nl) && (o % 16 == 0);
    gs.w = bits + pay_off + (ok ? o : 0);
    gs.n_words = ok ? nw : 0;
    gs.ptr = 2u * (uint32_t)nl;
    gs.win = win;
    gs.bad = !ok;
    window_fill(gs, 0);
    x = 0x10000u;
    if (ok && lane < nl) {
        x = ((uint32_t)win[2 * lane] << 16) | win[2 * lane + 1];
        if (x < 0x10000u) gs.bad = true;
    }
    return ok;
}

// Renormalisation shared by the group: lanes whose state fell below 2^16 read the next
// words in ascending lane order.  Reads past the group's words mark the stream bad.
__device__ __forceinline__ void group_refill(GroupStream &gs, uint32_t &x, bool active) {
    const bool need = active && x < 0x10000u;
    const uint32_t mask = __ballot_sync(0xffffffffu, need);
    if (mask == 0) return;
    if (gs.ptr > gs.wlimit) window_fill(gs, gs.ptr & ~7u);
    if (need) {
        const uint32_t idx = gs.ptr + __popc(mask & ((1u << (threadIdx.x & 31)) - 1u));
        uint32_t w = 0;
        if (idx < gs.n_words) w = gs.win[idx - gs.wbase]; else gs.bad = true;
        x = (x << 16) | w;
    }
    gs.ptr += __popc(mask);
}

// ------------------------------------------------------------------ batched stages

// Persistent loop: each CTA claims items in increasing order with an atomic counter, finds
// the owning scene by binary search, copies its parameters to shared memory and runs
// body(params, item within the scene, items of the scene, same), where `same` says that this
// CTA's previous item belonged to the same scene (shared-memory state the body derived from
// the scene's parameters is still there).
template <typename P, typename Body>
__device__ __forceinline__ void run_items(const MultiArgs &m, Body body) {
    __shared__ uint32_t s_item;
    __shared__ int s_scene;
    __shared__ __align__(16) uint8_t s_par[(sizeof(P) + 15) & ~size_t(15)];
    int prev = -1;
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t item = atomicAdd(m.counter, 1u);
            int lo = 0, hi = m.n - 1;  // last scene whose first item <= item
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (m.prefix[mid] <= item) lo = mid; else hi = mid - 1;
            }
            s_item = item;
            s_scene = lo;
        }
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= m.total) break;
        const int sc = s_scene;
        const bool same = sc == prev;
        prev = sc;
        const uint4 *src = reinterpret_cast<const uint4 *>(m.params + (size_t)sc * m.stride);
        uint4 *dst = reinterpret_cast<uint4 *>(s_par);
        if (!same)
            for (uint32_t i = threadIdx.x; i < sizeof(s_par) / 16; i += blockDim.x) dst[i] = src[i];
        __syncthreads();
        body(*reinterpret_cast<const P *>(s_par), item - m.prefix[sc], m.prefix[sc + 1] - m.prefix[sc], same);
        __syncthreads();
    }
}

}  // namespace sgs
