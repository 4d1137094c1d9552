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

static_assert(kFixWarps == (int)kFixWarpsMax, "the launch shape's cap is the staging array's size");

// A CTA of blockDim.x / 32 warps (at most kFixWarps) takes that many consecutive items.
template <bool VEC>
__device__ __forceinline__ void fixed_body(const FixedParams &p, uint32_t vb) {
    __shared__ uint32_t s_words[kFixWarps][kFixStage];
    const int warp = threadIdx.x >> 5;
    fixed_warp_item<VEC>(p, (uint64_t)vb * (blockDim.x >> 5) + warp, s_words[warp]);
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
                         const sgs_scene_out &out, int *status, cudaStream_t st, uint32_t warps) {
    FixedParams p;
    bool vec;
    if (make_fixed(bits, info, out, status, &p, &vec) == 0) return cudaSuccess;
    const uint32_t w = (warps >= 1 && warps <= (uint32_t)kFixWarps) ? warps : (uint32_t)kFixWarps;
    const uint64_t items = (uint64_t)p.n_items_per_chan * kNChan;
    const uint32_t grid = (uint32_t)((items + w - 1) / w);
    if (vec) k_fixed<true><<<grid, 32 * w, 0, st>>>(p);
    else k_fixed<false><<<grid, 32 * w, 0, st>>>(p);
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
