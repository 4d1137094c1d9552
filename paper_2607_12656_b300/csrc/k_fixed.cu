// Channel-wise fixed-length decoding on sm_103a (Sec. 3.4.1, the "UltraFast" coder: each
// channel's quantized values stored at a fixed bit width).  Channel c's n values sit
// LSB-first at bits [i b_c, (i+1) b_c) of its own little-endian u32 stream.
//
// One warp per (channel, 1024 rows): 1024 values of b bits are exactly 32 b words, so the
// warp stages its words in shared memory with coalesced loads, then lane j extracts rows
// j, j+32, ... through a 64-bit funnel of two words and writes the dequantized fp32 values
// v = fl(fl(q * step) + offset) with coalesced 128-byte stores.  HBM-bound: per Gaussian it
// reads sum(b_c)/8 bytes and writes 224.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "sgs_device.cuh"
#include "sgs_internal.h"

namespace sgs {

constexpr int kFixWarps = 8;
constexpr int kFixRows = 1024;       // rows per warp item
constexpr int kFixMaxBits = 16;

struct FixedParams {
    const uint8_t *bits;
    uint64_t chan_off, tab_off, pay_off, pay_len;
    uint32_t n_rows;
    uint32_t n_items_per_chan;
    float *out;
    const uint32_t *out_index;
    int *status;
};

// VEC: every channel's output base is 16-byte aligned and there is no out_index, so lane j
// writes rows 4j..4j+3 (+128 k) with one 16-byte store; otherwise one 4-byte store per row.
template <bool VEC>
__device__ __forceinline__ void fixed_body(const FixedParams &p, uint32_t vb) {
    __shared__ uint32_t s_words[kFixWarps][32 * kFixMaxBits + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t item = (uint64_t)vb * kFixWarps + warp;
    const uint32_t c = (uint32_t)(item / p.n_items_per_chan);
    if (c >= (uint32_t)kNChan) return;
    const uint32_t blk = (uint32_t)(item - (uint64_t)c * p.n_items_per_chan);
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
    uint32_t *sw = s_words[warp];
    for (uint32_t i = lane; i <= nw; i += 32)
        sw[i] = (w0 + i < nwords_chan) ? w[w0 + i] : 0u;
    __syncwarp();
    const uint32_t mask = (1u << b) - 1u;  // b <= 16
    const uint32_t r0 = blk * kFixRows;
    const uint32_t rows = p.n_rows - r0 < (uint32_t)kFixRows ? p.n_rows - r0 : (uint32_t)kFixRows;
    float *outc = p.out + (size_t)c * p.n_rows + r0;
    if (VEC) {
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
                *reinterpret_cast<float4 *>(outc + rl) = make_float4(v[0], v[1], v[2], v[3]);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (rl + q < rows) outc[rl + q] = v[q];
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
            if (p.out_index) p.out[(size_t)c * p.n_rows + p.out_index[r0 + rl]] = v;
            else outc[rl] = v;
        }
    }
}

template <bool VEC>
__global__ void __launch_bounds__(32 * kFixWarps) k_fixed(FixedParams p) { fixed_body<VEC>(p, blockIdx.x); }

template <bool VEC>
__global__ void __launch_bounds__(32 * kFixWarps) k_fixed_multi(MultiArgs m) {
    run_items<FixedParams>(m, [](const FixedParams &p, uint32_t vb, uint32_t, bool) { fixed_body<VEC>(p, vb); });
}

// Parameters of one scene; returns its CTAs (0: nothing to do) and whether it takes the
// vector-store variant.
uint32_t make_fixed(const uint8_t *bits, const sgs_scene_info &info, const sgs_scene_out &out,
                    int *status, FixedParams *pp, bool *vec) {
    FixedParams &p = *pp;
    memset(&p, 0, sizeof(p));
    p.bits = bits;
    p.chan_off = info.off[S_CHAN];
    p.tab_off = info.off[S_ATTR_TAB];
    p.pay_off = info.off[S_ATTR_PAY];
    p.pay_len = info.total_len - info.off[S_ATTR_PAY];
    p.n_rows = info.n_rows;
    p.n_items_per_chan = (info.n_rows + kFixRows - 1) / kFixRows;
    p.out = out.attr;
    p.out_index = out.out_index;
    p.status = status;
    *vec = !out.out_index && (info.n_rows % 4 == 0) && (((uintptr_t)out.attr & 15) == 0);
    if (info.n_rows == 0) return 0;
    const uint64_t items = (uint64_t)p.n_items_per_chan * kNChan;
    return (uint32_t)((items + kFixWarps - 1) / kFixWarps);
}

cudaError_t launch_fixed(const uint8_t *bits, const sgs_scene_info &info,
                         const sgs_scene_out &out, int *status, cudaStream_t st) {
    FixedParams p;
    bool vec;
    const uint32_t grid = make_fixed(bits, info, out, status, &p, &vec);
    if (grid == 0) return cudaSuccess;
    if (vec) k_fixed<true><<<grid, 32 * kFixWarps, 0, st>>>(p);
    else k_fixed<false><<<grid, 32 * kFixWarps, 0, st>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ batched stage

uint32_t stage_fixed(const SceneRef &r, bool vec_variant, void *par) {
    FixedParams p;
    bool vec;
    const uint32_t n = make_fixed(r.bits, *r.info, *r.out, r.status, &p, &vec);
    if (vec != vec_variant) return 0;
    memcpy(par, &p, sizeof(p));
    return n;
}

size_t stage_fixed_bytes() { return sizeof(FixedParams); }

cudaError_t launch_fixed_multi(bool vec, const MultiArgs &m, cudaStream_t st) {
    if (vec) return launch_persistent(k_fixed_multi<true>, 32 * kFixWarps, 0, m, st);
    return launch_persistent(k_fixed_multi<false>, 32 * kFixWarps, 0, m, st);
}

}  // namespace sgs
