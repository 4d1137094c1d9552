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

// The same for q < 2^23 without an integer conversion: 2^23 + q is exact in fp32 (its bits
// are 0x4B000000 | q), so subtracting 2^23 leaves (float)q exactly.
__device__ __forceinline__ float dequant_small(uint32_t q, float step, float offset) {
    const float qf = __fsub_rn(__uint_as_float(0x4B000000u | q), 8388608.0f);
    return __fadd_rn(__fmul_rn(qf, step), offset);
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

// Copies n expanded tables into shared memory: each table's cdf[257] (padded to
// kTabCdfStride words, s_cdf [n][kTabCdfStride]) and, if s_lut is not NULL, its slot lookup
// (s_lut [n][kLutBuckets]); both 16-byte aligned.  A table is its padded cdf followed by its
// lookup, so the copy is 16-byte units throughout, all of a thread's loads in flight together.
__device__ __forceinline__ void load_cdf_smem(const uint8_t *tables, int n, uint32_t *s_cdf, uint8_t *s_lut = nullptr) {
    constexpr int kC = kTabCdfBytes / 16, kT = kTabBytes / 16;  // uint4 of a cdf row, of a table
    static_assert(kTabBytes == kTabCdfBytes + kLutBuckets && kTabBytes % 16 == 0, "table layout");
    const int per = s_lut ? kT : kC;
    const uint4 *src = reinterpret_cast<const uint4 *>(tables);
#pragma unroll 4
    for (int i = threadIdx.x; i < n * per; i += blockDim.x) {
        const int t = i / per, k = i - t * per;
        const uint4 v = src[t * kT + k];
        if (k < kC) reinterpret_cast<uint4 *>(s_cdf)[t * kC + k] = v;
        else reinterpret_cast<uint4 *>(s_lut)[t * (kLutBuckets / 16) + (k - kC)] = v;
    }
}

// The symbol s with cdf[s] <= slot < cdf[s+1] (cdf[0] = 0, cdf[256] = 2^16 > slot): the
// largest index whose cdf is at most slot, by eight branch-free halvings -- the same cost
// for every lane of a warp, whatever the distribution's shape.
__device__ __forceinline__ uint32_t cdf_search(const uint32_t *cdf, uint32_t slot) {
    uint32_t s = 0;
#pragma unroll
    for (uint32_t st = 128; st > 0; st >>= 1) s += (cdf[s + st] <= slot) ? st : 0u;
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

// One static-table symbol from state x (tables: cdf[257] and the 1,024-bucket slot lookup):
// the symbol s with cdf[s] <= slot < cdf[s + 1] lies between the symbols holding the bucket's
// first slot (lut[b]) and the next bucket's first slot (lut[b + 1]).  One advance from lut[b] is
// predicated; lanes that need more (a slot among many rare symbols crowded into one bucket)
// binary-search the rest of that range, so a warp never walks a crowded bucket linearly.
// Then the state update.
__device__ __forceinline__ uint32_t rans_symbol(const uint32_t *cdf, const uint8_t *lut, uint32_t &x) {
    const uint32_t slot = x & 0xFFFFu, b = slot >> kLutShift;
    uint32_t s = lut[b];
    uint32_t lo = cdf[s], hi = cdf[s + 1];
    if (hi <= slot) {
        lo = hi;
        hi = cdf[++s + 1];
    }
    if (hi <= slot) {
        // cdf[s + 1] <= slot: the answer is in [s + 1, e], e = the symbol holding the next
        // bucket's first slot (255 for the last bucket; cdf[256] = 2^16 > slot)
        uint32_t a = s + 1, e = b + 1 < (uint32_t)kLutBuckets ? lut[b + 1] : 255u;
        while (a < e) {  // largest m in [a, e] with cdf[m] <= slot
            const uint32_t m = (a + e + 1) >> 1;
            if (cdf[m] <= slot) a = m; else e = m - 1;
        }
        s = a;
        lo = cdf[s];
        hi = cdf[s + 1];
    }
    x = (hi - lo) * (x >> 16) + slot - lo;
    return s;
}

// group_refill with the window position kept relative (wrel = next word's index in the window)
// and no per-word bound: words past the group's stream read as zero from the window (never
// from memory past the payload), and the caller's final check wbase + wrel == n_words turns
// any over-read into a corrupt-stream status.  lt = the lanes below this one.
// Refills the window unless `room` more words can be read from it.
__device__ __forceinline__ void window_ensure(GroupStream &gs, uint32_t &wrel, uint32_t room) {
    if (wrel > kWinWords - room) {
        const uint32_t ptr = gs.wbase + wrel;
        window_fill(gs, ptr & ~7u);
        wrel = ptr - gs.wbase;
    }
}

// CHECK: the window is checked here (room for this step's 32 words); otherwise the caller
// made room for several steps with window_ensure.
template <bool CHECK = true>
__device__ __forceinline__ void group_renorm(GroupStream &gs, uint32_t &x, uint32_t &wrel, uint32_t lt, bool can) {
    const bool need = can && x < 0x10000u;
    const uint32_t mask = __ballot_sync(0xffffffffu, need);
    if (CHECK) window_ensure(gs, wrel, 32);
    if (need) x = __byte_perm(x, gs.win[wrel + __popc(mask & lt)], 0x1054);  // x << 16 | word
    wrel += __popc(mask);
}

// ------------------------------------------------------------------ fixed-length items

// Channel-wise fixed-length decoding (Sec. 3.4.1): one warp item = one channel x 1,024 rows.
constexpr int kFixWarps = 8;          // warps of a k_fixed CTA
constexpr int kFixRows = 1024;        // rows per warp item
constexpr int kFixMaxBits = 16;
constexpr int kFixStage = 32 * kFixMaxBits + 2;  // staged words per warp (an item's + 2)

struct FixedParams {
    const uint8_t *bits;
    uint64_t chan_off, tab_off, pay_off, pay_len;
    uint32_t n_rows;
    uint32_t n_items_per_chan;
    float *out;
    const uint32_t *out_index;
    int *status;
};

// A whole item of B-bit values, VEC layout: lane j's rows 128 k + 4 j .. + 3 start at bit
// 128 B k + 4 B j, i.e. word 4 B k + (4 B j >> 5) at the lane's fixed shift (4 B j) & 31, so
// two funnel shifts of three staged words give the 64-bit window holding all four values
// (4 B <= 64) and every further offset is a constant.
template <int B>
__device__ __forceinline__ void fixed_full_vec(const uint32_t *sw, float *outc, float step, float offset,
                                               uint32_t lane) {
    constexpr uint32_t mask = (1u << B) - 1u;
    const uint32_t bl = 4u * B * lane;
    const uint32_t *q0 = sw + (bl >> 5);
    const uint32_t s = bl & 31u;
#pragma unroll
    for (int k = 0; k < kFixRows / 128; ++k) {
        const uint32_t *q = q0 + 4 * B * k;
        const uint32_t t0 = __funnelshift_r(q[0], q[1], s), t1 = __funnelshift_r(q[1], q[2], s);
        float v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int o = i * B;
            const uint32_t x = o == 0 ? t0 : (o < 32 ? __funnelshift_r(t0, t1, o & 31) : t1 >> ((o - 32) & 31));
            v[i] = dequant_small(x & mask, step, offset);
        }
        __stcs(reinterpret_cast<float4 *>(outc + 128 * k + 4 * lane), make_float4(v[0], v[1], v[2], v[3]));
    }
}

// Warp item `item` (channel item / n_items_per_chan); sw = this warp's kFixStage staging
// words in shared memory.  VEC: every channel's output base is 16-byte aligned and there is
// no out_index, so lane j writes rows 4j..4j+3 (+128 k) with one 16-byte store; otherwise one
// 4-byte store per row.
template <bool VEC>
__device__ __forceinline__ void fixed_warp_item(const FixedParams &p, uint64_t item, uint32_t *sw) {
    const int lane = threadIdx.x & 31;
    if (item >= (uint64_t)kNChan * p.n_items_per_chan) return;  // n_items_per_chan < 2^22
    const uint32_t c = (uint32_t)item / p.n_items_per_chan;
    const uint32_t blk = (uint32_t)item - c * p.n_items_per_chan;
    const uint32_t b = *reinterpret_cast<const uint32_t *>(p.bits + p.chan_off + 4 * (2 * kNChan + c));
    const float step = ld_f32(p.bits + p.chan_off + 4 * c);
    const float offset = ld_f32(p.bits + p.chan_off + 4 * (kNChan + c));
    const uint64_t *coff = reinterpret_cast<const uint64_t *>(p.bits + p.tab_off);
    const uint64_t cbeg = coff[c], cend = coff[c + 1];
    const uint64_t nwords_chan = ((uint64_t)p.n_rows * b + 31) / 32;
    if (b < 1 || b > kFixMaxBits || cbeg > cend || cend > p.pay_len || cbeg % 16 != 0 ||
        (cend - cbeg) < 4 * nwords_chan) {
        if (lane == 0) set_status(p.status, SGS_E_CORRUPT);
        return;
    }
    const uint32_t *w = reinterpret_cast<const uint32_t *>(p.bits + p.pay_off + cbeg);
    const uint64_t w0 = (uint64_t)blk * 32 * b;   // first word of this item
    const uint32_t nw = 32 * b;
    __syncwarp();  // the previous item's reads of sw are done
    // packed words and outputs are touched once: streaming (evict-first) accesses keep them
    // from displacing the octree's working set in L2 while the two halves run together
    for (uint32_t i = lane; i < nw + 2; i += 32)
        sw[i] = (w0 + i < nwords_chan) ? __ldcs(w + w0 + i) : 0u;
    __syncwarp();
    const uint32_t mask = (1u << b) - 1u;  // b <= 16
    const uint32_t r0 = blk * kFixRows;
    const uint32_t rows = p.n_rows - r0 < (uint32_t)kFixRows ? p.n_rows - r0 : (uint32_t)kFixRows;
    float *outc = p.out + (size_t)c * p.n_rows + r0;
    if (VEC && rows == (uint32_t)kFixRows) {
        switch (b) {
#define SGS_FIX_CASE(B) \
    case B: fixed_full_vec<B>(sw, outc, step, offset, (uint32_t)lane); break;
            SGS_FIX_CASE(1) SGS_FIX_CASE(2) SGS_FIX_CASE(3) SGS_FIX_CASE(4) SGS_FIX_CASE(5) SGS_FIX_CASE(6)
            SGS_FIX_CASE(7) SGS_FIX_CASE(8) SGS_FIX_CASE(9) SGS_FIX_CASE(10) SGS_FIX_CASE(11) SGS_FIX_CASE(12)
            SGS_FIX_CASE(13) SGS_FIX_CASE(14) SGS_FIX_CASE(15) SGS_FIX_CASE(16)
#undef SGS_FIX_CASE
        }
    } else if (VEC) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t rl = (uint32_t)k * 128 + 4 * lane;
            uint32_t bit = rl * b;
            float v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t wi = bit >> 5;
                v[q] = dequant(__funnelshift_r(sw[wi], sw[wi + 1], bit & 31) & mask, step, offset);
                bit += b;
            }
            if (rl + 4 <= rows) {
                __stcs(reinterpret_cast<float4 *>(outc + rl), make_float4(v[0], v[1], v[2], v[3]));
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (rl + q < rows) __stcs(outc + rl + q, v[q]);
            }
        }
    } else {
#pragma unroll 4
        for (int k = 0; k < 32; ++k) {
            const uint32_t rl = (uint32_t)k * 32 + lane;
            if (rl >= rows) break;
            const uint32_t bit = rl * b;
            const uint32_t wi = bit >> 5;
            const float v = dequant(__funnelshift_r(sw[wi], sw[wi + 1], bit & 31) & mask, step, offset);
            if (p.out_index) __stcs(p.out + (size_t)c * p.n_rows + p.out_index[r0 + rl], v);
            else __stcs(outc + rl, v);
        }
    }
}

// ------------------------------------------------------------------ batched stages

// The device's global nanosecond timer (PTX special register %globaltimer).
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

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
        if (m.done && threadIdx.x == 0) {
            // the CTA's writes for this item precede the count: the last item of the scene
            // to finish is the one whose increment reaches need
            __threadfence();
            const uint32_t g = m.scene_id[sc];
            if (atomicAdd(m.done + g, 1u) + 1u == m.need[g]) m.t_done[g] = globaltimer_ns();
        }
    }
}

}  // namespace sgs
