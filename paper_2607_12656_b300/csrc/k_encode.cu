// Interleaved rANS encoding of the attribute streams on the device (the encoder side of
// Sec. 3.4's entropy coding; rANS with 32-bit state, 16-bit words, 16-bit probabilities).
//
// The group stream of 32 lanes is defined by the decoder's order: initial states, then for
// each step the renormalisation words of the lanes in ascending lane order.  The encoder runs
// the same schedule backwards -- steps descending and, within a step, lanes descending -- so a
// warp encodes one group: at each step the lanes that must emit a word get its position from
// the ballot of emitting lanes above them; then the final states are appended (lanes
// descending, low half first) and the group's words are reversed into the payload.  Symbols
// come in lane-major order with their frequency f (>= 1) and cumulative frequency.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "sgs_internal.h"

namespace sgs {

namespace {

constexpr int kEncWarps = 8;

// Group g -> words [0, n) of its stream in emission order at temp + temp_off[g]; *n to words[g].
__global__ void __launch_bounds__(32 * kEncWarps) k_rans_encode(const uint32_t *f, const uint32_t *cum,
                                                                const uint64_t *lane_start, uint32_t L,
                                                                uint32_t G, uint16_t *temp,
                                                                const uint64_t *temp_off, uint32_t *words) {
    const int lane = threadIdx.x & 31;
    const uint32_t g = blockIdx.x * kEncWarps + (threadIdx.x >> 5);
    if (g >= G) return;
    const uint32_t j0 = 32 * g;
    const int nl = (int)min(32u, L - j0);
    uint64_t s0 = 0, n = 0;
    if (lane < nl) {
        s0 = lane_start[j0 + lane];
        n = lane_start[j0 + lane + 1] - s0;
    }
    uint64_t maxn = n;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t v = __shfl_xor_sync(0xffffffffu, maxn, o);
        maxn = v > maxn ? v : maxn;
    }
    uint16_t *out = temp + temp_off[g];
    uint32_t x = 1u << 16, cur = 0;
    for (uint64_t tt = maxn; tt-- > 0;) {
        const bool active = tt < n;
        uint32_t fv = 1, cv = 0;
        if (active) {
            fv = f[s0 + tt];
            cv = cum[s0 + tt];
        }
        const bool emit = active && (uint64_t)x >= ((uint64_t)fv << 16);
        const uint32_t mask = __ballot_sync(0xffffffffu, emit);
        if (emit) {
            out[cur + __popc(lane < 31 ? mask >> (lane + 1) : 0u)] = (uint16_t)(x & 0xFFFFu);
            x >>= 16;
        }
        cur += __popc(mask);
        if (active) x = ((x / fv) << 16) + (x % fv) + cv;
    }
    if (lane < nl) {
        const uint32_t i = cur + 2u * (uint32_t)(nl - 1 - lane);
        out[i] = (uint16_t)(x & 0xFFFFu);
        out[i + 1] = (uint16_t)(x >> 16);
    }
    if (lane == 0) words[g] = cur + 2u * (uint32_t)nl;
}

// One CTA per group: its words reversed (the decoder reads the stream forwards), as little-
// endian u16 at byte offset goff[g] of the payload (the padding after them stays zero).
__global__ void __launch_bounds__(256) k_rans_reverse(const uint16_t *temp, const uint64_t *temp_off,
                                                      const uint32_t *words, const uint64_t *goff,
                                                      uint8_t *pay) {
    const uint32_t g = blockIdx.x;
    const uint32_t W = words[g];
    const uint16_t *src = temp + temp_off[g];
    uint16_t *dst = reinterpret_cast<uint16_t *>(pay + goff[g]);
    for (uint32_t k = threadIdx.x; k < W; k += blockDim.x) dst[W - 1 - k] = src[k];
}

// f and cum of static-table symbols: symbol p of the lane-major stream is channel p % 56 (every
// lane starts at a row boundary), with table c's f at ftab[c][token], cumulative at ctab[c][token].
__global__ void k_static_fc(const uint8_t *tok, uint64_t n, const uint32_t *ftab, const uint32_t *ctab,
                            uint32_t *f, uint32_t *cum) {
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < n; p += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t c = (uint32_t)(p % kNChan), s = tok[p];
        f[p] = ftab[c * kNSym + s];
        cum[p] = ctab[c * kNSym + s];
    }
}

template <typename T>
struct Dev {
    T *p = nullptr;
    ~Dev() {
        if (p) cudaFree(p);
    }
    bool alloc(size_t count) { return cudaMalloc(&p, (count ? count : 1) * sizeof(T)) == cudaSuccess; }
};

}  // namespace

// Encodes the groups of lane_start (host; L + 1 symbol offsets) from device arrays f, cum into
// the group table and payload sections (host), byte for byte as the host encoder does.
int rans_encode_device(const uint32_t *f, const uint32_t *cum, const std::vector<uint64_t> &lane_start,
                       std::vector<uint8_t> &grp, std::vector<uint8_t> &pay) {
    const uint64_t L = lane_start.size() - 1;
    const uint64_t G = (L + 31) / 32;
    std::vector<uint64_t> temp_off(G + 1, 0);
    for (uint64_t g = 0; g < G; ++g) {
        const uint64_t j0 = 32 * g, j1 = j0 + 32 < L ? j0 + 32 : L;
        // capacity: at most one word per symbol, plus two per lane for the final states
        temp_off[g + 1] = temp_off[g] + (lane_start[j1] - lane_start[j0]) + 2 * (j1 - j0);
    }
    Dev<uint64_t> d_start, d_toff, d_goff;
    Dev<uint16_t> d_temp;
    Dev<uint32_t> d_words;
    if (!d_start.alloc(L + 1) || !d_toff.alloc(G + 1) || !d_goff.alloc(G + 1) || !d_temp.alloc(temp_off[G]) ||
        !d_words.alloc(G))
        return SGS_E_NOMEM;
    if (cudaMemcpy(d_start.p, lane_start.data(), 8 * (L + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_toff.p, temp_off.data(), 8 * (G + 1), cudaMemcpyHostToDevice) != cudaSuccess)
        return SGS_E_CUDA;
    if (G) {
        k_rans_encode<<<(unsigned)((G + kEncWarps - 1) / kEncWarps), 32 * kEncWarps>>>(f, cum, d_start.p, (uint32_t)L,
                                                                                   (uint32_t)G, d_temp.p, d_toff.p,
                                                                                   d_words.p);
        if (cudaGetLastError() != cudaSuccess) return SGS_E_CUDA;
    }
    std::vector<uint32_t> gw(G);
    if (G && cudaMemcpy(gw.data(), d_words.p, 4 * G, cudaMemcpyDeviceToHost) != cudaSuccess) return SGS_E_CUDA;
    std::vector<uint64_t> goff(G + 1, 0);
    for (uint64_t g = 0; g < G; ++g) goff[g + 1] = goff[g] + ((2ull * gw[g] + 15) & ~15ull);
    Dev<uint8_t> d_pay;
    if (!d_pay.alloc(goff[G])) return SGS_E_NOMEM;
    if (cudaMemset(d_pay.p, 0, goff[G] ? goff[G] : 1) != cudaSuccess ||
        cudaMemcpy(d_goff.p, goff.data(), 8 * (G + 1), cudaMemcpyHostToDevice) != cudaSuccess)
        return SGS_E_CUDA;
    if (G) {
        k_rans_reverse<<<(unsigned)G, 256>>>(d_temp.p, d_toff.p, d_words.p, d_goff.p, d_pay.p);
        if (cudaGetLastError() != cudaSuccess) return SGS_E_CUDA;
    }
    const size_t base = pay.size();
    pay.resize(base + goff[G]);
    if (goff[G] && cudaMemcpy(pay.data() + base, d_pay.p, goff[G], cudaMemcpyDeviceToHost) != cudaSuccess)
        return SGS_E_CUDA;
    for (uint64_t g = 0; g <= G; ++g) goff[g] += base;
    grp.resize(8 * (G + 1) + 4 * G);
    memcpy(grp.data(), goff.data(), 8 * (G + 1));
    if (G) memcpy(grp.data() + 8 * (G + 1), gw.data(), 4 * G);
    while (grp.size() % 16) grp.push_back(0);
    return SGS_OK;
}

// Static attribute coding on the device: tokens in lane-major order (host), 56 frequency
// tables (host, [56][256]); f and cum are gathered on the device, then encoded.
int rans_encode_static_device(const uint8_t *tok_lane_major, uint64_t nsym, const uint32_t *ftab,
                              const std::vector<uint64_t> &lane_start, std::vector<uint8_t> &grp,
                              std::vector<uint8_t> &pay) {
    std::vector<uint32_t> ctab((size_t)kNChan * kNSym);
    for (int c = 0; c < kNChan; ++c) {
        uint32_t acc = 0;
        for (int s = 0; s < kNSym; ++s) {
            ctab[(size_t)c * kNSym + s] = acc;
            acc += ftab[(size_t)c * kNSym + s];
        }
    }
    Dev<uint8_t> d_tok;
    Dev<uint32_t> d_ftab, d_ctab, d_f, d_c;
    if (!d_tok.alloc(nsym) || !d_ftab.alloc((size_t)kNChan * kNSym) || !d_ctab.alloc((size_t)kNChan * kNSym) ||
        !d_f.alloc(nsym) || !d_c.alloc(nsym))
        return SGS_E_NOMEM;
    if (cudaMemcpy(d_tok.p, tok_lane_major, nsym, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_ftab.p, ftab, 4ull * kNChan * kNSym, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d_ctab.p, ctab.data(), 4ull * kNChan * kNSym, cudaMemcpyHostToDevice) != cudaSuccess)
        return SGS_E_CUDA;
    if (nsym) {
        const uint64_t blocks = (nsym + 255) / 256;
        k_static_fc<<<(unsigned)(blocks < 148 * 32 ? blocks : 148 * 32), 256>>>(d_tok.p, nsym, d_ftab.p, d_ctab.p,
                                                                              d_f.p, d_c.p);
        if (cudaGetLastError() != cudaSuccess) return SGS_E_CUDA;
    }
    return rans_encode_device(d_f.p, d_c.p, lane_start, grp, pay);
}

}  // namespace sgs
