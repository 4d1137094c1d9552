// Device decoder of the learned geometry coder (SGS_GEO_LEARNED; Sec. 3.4, "Geometry Occupancy
// Coding", Eq. 8: each octree level is coded conditioned on the level above it).
//
// A node of level l is the k-th child (k its child index) of a node of level l - 1 with
// occupancy byte b, and its token is coded with the frequency table the frozen integer context
// model gives the context 8 b + k: inputs u = (b - 128, 32 k - 112, 16 popc(b) - 64,
// 32 rank - 112) (rank = set bits of b below k), channel = l.  The tables depend only on
// (level, context), so one launch computes every valid context's table of every coded level
// first; then level by level, in order, a popcount scan of level l - 1 gives every level-l
// node its context, and the level's rANS lanes (contiguous chunks, about 128 tokens each,
// groups of 32 sharing a word stream) are decoded with per-token tables.  The decoded tokens
// land in the scratch copy of the occupancy bytes, where the octree expansion reads them.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "exp2q_table.h"
#include "sgs_device.cuh"
#include "sgs_internal.h"

namespace sgs {

__constant__ uint32_t kGeoExp2Q[256] = {SGS_EXP2Q_VALUES};

// Frozen model blob (SGS_MODEL_BYTES): i32 m1, sh1, m2, sh2, ms, ss, then (from byte 32)
// i32 B1[56][64], i32 b2[64], i32 b3[256], i8 W1[64][4], i8 W2[64][64], i8 W3[256][64].
constexpr int kGM_B1 = 32, kGM_B2 = 14368, kGM_B3 = 14624, kGM_W1 = 15648, kGM_W2 = 15904, kGM_W3 = 20000;
constexpr int kGCtx = 2048;                 // context ids 8 b + k
constexpr int kGTabU16 = kNSym + 16;        // cdf[0 .. 255] (cdf[256] = 2^16), then cdf[16 j], j < 16
constexpr size_t kGTabBytes = kGTabU16 * 2; // 544, a multiple of 16
constexpr int kGCtxTile = 4096;             // level nodes per context-scan tile (256 threads x 16)

__device__ __forceinline__ int32_t geo_requant(int32_t acc, int32_t m, int32_t sh) {
    int64_t v = ((int64_t)acc * (int64_t)m + ((int64_t)1 << (sh - 1))) >> sh;
    v = v < 0 ? 0 : v;
    return (int32_t)(v > 127 ? 127 : v);
}

// ------------------------------------------------------------------ tables

struct GeoTabParams {
    const uint8_t *model;
    uint16_t *tables;   // [n_levels][kGCtx][kGTabU16]
    int n_levels;
    int level[SGS_MAX_DEPTH];
    int *status;
};

// One warp per (coded level, context id): layer 1 and 2 (two units per lane), the 256 logits
// (eight per lane, symbols 8 lane .. 8 lane + 7), then the integer softmax of the model --
// d_k = zmax - z_k, t_k = min((d_k ms) >> ss, 6144), e_k = EXP2Q[t_k & 255] >> (t_k >> 8),
// R = floor(65280 2^32 / sum e), f_k = 1 + floor(e_k R / 2^32), the remainder 2^16 - sum f
// to the lowest argmax -- and the cumulative table, stored as u16 (every f_k >= 1, so
// cdf[255] < 2^16).  Ids 8 b + k whose bit k of b is clear are not contexts and are skipped.
constexpr int kTabWarps = 8;
__global__ void __launch_bounds__(32 * kTabWarps) k_geo_tables(GeoTabParams p) {
    __shared__ __align__(16) int8_t w3[256 * 64];
    __shared__ __align__(16) int8_t w2[64 * 64];
    __shared__ int8_t w1[256];
    __shared__ int32_t b2[64], b3[256];
    __shared__ uint32_t ex[256];
    __shared__ int32_t h1s[kTabWarps][64], h2s[kTabWarps][64];
    __shared__ int bad;
    const uint8_t *m = p.model;
    const int32_t *hdr = reinterpret_cast<const int32_t *>(m);
    const int32_t m1 = hdr[0], sh1 = hdr[1], m2 = hdr[2], sh2 = hdr[3];
    const uint32_t ms = (uint32_t)hdr[4], ss = (uint32_t)hdr[5];
    if (threadIdx.x == 0)
        bad = !(sh1 >= 1 && sh1 <= 47 && sh2 >= 1 && sh2 <= 47 && m1 >= 0 && m2 >= 0 && ms >= 1 && ms < (1u << 24) &&
                ss <= 24);
    for (int i = threadIdx.x; i < 256 * 64; i += blockDim.x) w3[i] = (int8_t)m[kGM_W3 + i];
    for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) w2[i] = (int8_t)m[kGM_W2 + i];
    bool badb = false;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        w1[i] = (int8_t)m[kGM_W1 + i];
        b3[i] = reinterpret_cast<const int32_t *>(m + kGM_B3)[i];
        badb |= b3[i] >= (1 << 24) || b3[i] <= -(1 << 24);
        ex[i] = kGeoExp2Q[i];
    }
    for (int i = threadIdx.x; i < 64; i += blockDim.x) {
        b2[i] = reinterpret_cast<const int32_t *>(m + kGM_B2)[i];
        badb |= b2[i] >= (1 << 24) || b2[i] <= -(1 << 24);
    }
    __syncthreads();
    if (badb) atomicOr(&bad, 1);
    __syncthreads();
    if (bad) {
        if (threadIdx.x == 0 && blockIdx.x == 0) set_status(p.status, SGS_E_CORRUPT);
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t id = blockIdx.x * kTabWarps + warp;
    const uint32_t li = id / kGCtx, ctx = id % kGCtx;
    if (li >= (uint32_t)p.n_levels) return;
    const uint32_t b = ctx >> 3, k = ctx & 7;
    if (!((b >> k) & 1u)) return;  // not a context
    const int level = p.level[li];
    const int32_t u0 = (int32_t)b - 128, u1 = 32 * (int32_t)k - 112, u2 = 16 * __popc(b) - 64,
                  u3 = 32 * __popc(b & ((1u << k) - 1u)) - 112;
    const int32_t *B1 = reinterpret_cast<const int32_t *>(m + kGM_B1) + 64 * level;
    bool wbad = false;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int o = lane + 32 * h;
        const int32_t bias = B1[o];
        wbad |= bias >= (1 << 24) || bias <= -(1 << 24);
        const int32_t acc = bias + w1[4 * o] * u0 + w1[4 * o + 1] * u1 + w1[4 * o + 2] * u2 + w1[4 * o + 3] * u3;
        h1s[warp][o] = geo_requant(acc, m1, sh1);
    }
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int o = lane + 32 * h;
        int32_t acc = b2[o];
        for (int q = 0; q < 64; ++q) acc += (int32_t)w2[64 * o + q] * h1s[warp][q];
        h2s[warp][o] = geo_requant(acc, m2, sh2);
    }
    __syncwarp();
    int32_t z[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int s = 8 * lane + j;
        int32_t acc = b3[s];
        for (int q = 0; q < 64; ++q) acc += (int32_t)w3[64 * s + q] * h2s[warp][q];
        z[j] = acc;
    }
    // the largest logit, the lowest symbol on ties
    int32_t zmax = z[0];
    int amax = 8 * lane;
#pragma unroll
    for (int j = 1; j < 8; ++j)
        if (z[j] > zmax) { zmax = z[j]; amax = 8 * lane + j; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int32_t oz = __shfl_xor_sync(0xffffffffu, zmax, o);
        const int oa = __shfl_xor_sync(0xffffffffu, amax, o);
        if (oz > zmax || (oz == zmax && oa < amax)) { zmax = oz; amax = oa; }
    }
    uint32_t e[8];
    uint64_t E = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint64_t tt = ((uint64_t)(uint32_t)(zmax - z[j]) * ms) >> ss;
        const uint32_t t = tt > 6144 ? 6144u : (uint32_t)tt;
        e[j] = ex[t & 255] >> (t >> 8);
        E += e[j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) E += __shfl_xor_sync(0xffffffffu, E, o);
    const uint32_t R = (uint32_t)((65280ull << 32) / E);
    uint32_t f[8], S = 0, mine = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint32_t fl = __umulhi(e[j], R);
        f[j] = 1u + fl;
        S += fl;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
    const uint32_t rem = 65536u - 256u - S;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (8 * lane + j == amax) f[j] += rem;
        mine += f[j];
    }
    // cumulative: exclusive scan of the lanes' sums, then inside each lane's eight symbols
    uint32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    uint32_t run = incl - mine;
    uint16_t *T = p.tables + ((size_t)li * kGCtx + ctx) * kGTabU16;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        T[8 * lane + j] = (uint16_t)run;
        if (j == 0 && (lane & 1) == 0) T[kNSym + lane / 2] = (uint16_t)run;  // cdf[16 (lane / 2)]
        run += f[j];
    }
    if (wbad) set_status(p.status, SGS_E_CORRUPT);
}

// ------------------------------------------------------------------ contexts

// Context ids of the nodes of a coded level from the occupancy bytes of the level above:
// k_gctx_reduce writes the popcount sum of each tile of kGCtxTile parents, k_gctx_scan gives
// each tile the sum of the tiles before it and scans inside the tile; the j-th child (child
// index k = the j-th set bit of b) of a parent with byte b takes context 8 b + k.
struct GeoCtxParams {
    const uint8_t *par;   // the level above, n_par bytes
    uint32_t n_par, n_child;
    uint16_t *ctx;        // [n_child]
    uint32_t *tile_sums;
    int *status;
};

__global__ void __launch_bounds__(256) k_gctx_reduce(GeoCtxParams p) {
    __shared__ uint32_t sm[8];
    const uint32_t base = blockIdx.x * kGCtxTile + 16 * threadIdx.x;
    uint32_t c = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) c += base + j < p.n_par ? __popc((uint32_t)p.par[base + j]) : 0u;
    uint32_t tot;
    block_excl_scan_256(c, &tot, sm);
    if (threadIdx.x == 0) p.tile_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(256) k_gctx_scan(GeoCtxParams p) {
    __shared__ uint32_t sm[8];
    const uint32_t tile = blockIdx.x;
    uint32_t before = 0;
    for (uint32_t t = threadIdx.x; t < tile; t += 256) before += p.tile_sums[t];
    uint32_t prefix;
    block_excl_scan_256(before, &prefix, sm);
    const uint32_t base = tile * kGCtxTile + 16 * threadIdx.x;
    uint32_t b[16], c = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        b[j] = base + j < p.n_par ? (uint32_t)p.par[base + j] : 0u;
        c += __popc(b[j]);
    }
    uint32_t tot;
    uint32_t q = prefix + block_excl_scan_256(c, &tot, sm);
    bool bad = false;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        uint32_t bb = b[j];
        while (bb) {
            const uint32_t k = __ffs(bb) - 1;
            bb &= bb - 1;
            if (q < p.n_child) p.ctx[q] = (uint16_t)(8u * b[j] + k); else bad = true;
            ++q;
        }
    }
    if (tile == gridDim.x - 1 && threadIdx.x == 255 && q != p.n_child) bad = true;
    if (bad) set_status(p.status, SGS_E_CORRUPT);
}

// ------------------------------------------------------------------ level decode

struct GeoLDecParams {
    const uint8_t *bits;
    uint64_t grp_sec, pay_off, pay_len;  // the level's group table; the geometry payload
    uint32_t L, G, n;                    // lanes, groups and tokens of the level
    const uint16_t *ctx;
    const uint16_t *tab;                 // the level's [kGCtx][kGTabU16]
    uint8_t *out;                        // the level's occupancy bytes
    int *status;
};

// Symbol of `slot` in a table: the 16-entry block from the coarse row cdf[16 j] (c0, c1: loaded
// one token ahead by the caller), then the symbol inside it; (lo, hi) = (cdf[s], cdf[s + 1]).
// cdf is increasing, so the count of entries at or below slot locates it, the largest of them
// is lo and the smallest above it hi.  Whatever the table holds (one the model check left
// unwritten), every read stays inside it.
__device__ __forceinline__ uint32_t geo_sym(const uint16_t *T, uint4 c0, uint4 c1, uint32_t slot, uint32_t &lo,
                                            uint32_t &hi) {
    const uint32_t cw[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
    uint32_t jb = 0, nxt = 65536u;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t a = cw[i] & 0xFFFFu, b = cw[i] >> 16;
        if (a <= slot) ++jb; else nxt = min(nxt, a);
        if (b <= slot) ++jb; else nxt = min(nxt, b);
    }
    jb = jb ? jb - 1 : 0;  // cdf[0] = 0 <= slot in a valid table; any table stays in bounds
    const uint4 *fq = reinterpret_cast<const uint4 *>(T + 16 * jb);
    const uint4 f0 = __ldg(fq), f1 = __ldg(fq + 1);
    const uint32_t fw[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
    uint32_t r = 0;
    lo = 0;
    hi = nxt;  // the next block's first entry (2^16 after the last block)
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t a = fw[i] & 0xFFFFu, b = fw[i] >> 16;
        if (a <= slot) { ++r; lo = a; } else hi = min(hi, a);
        if (b <= slot) { ++r; lo = b; } else hi = min(hi, b);
    }
    return 16 * jb + r - 1;
}

constexpr int kLDecWarps = 8;

__global__ void __launch_bounds__(32 * kLDecWarps) k_geo_learned_decode(GeoLDecParams p) {
    __shared__ __align__(16) uint16_t win[kLDecWarps][kWinWords];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t g = blockIdx.x * kLDecWarps + warp;
    if (g >= p.G) return;
    const int nl = (int)min(32u, p.L - g * 32);
    const uint64_t j = (uint64_t)g * 32 + lane;
    const uint32_t s0 = lane < nl ? (uint32_t)(j * p.n / p.L) : 0u;
    const uint32_t s1 = lane < nl ? (uint32_t)((j + 1) * p.n / p.L) : 0u;
    const uint32_t n = s1 - s0;
    GroupStream gs;
    uint32_t x;
    group_open(p.bits, p.grp_sec, p.pay_off, p.pay_len, p.G, g, nl, lane, gs, x, win[warp]);
    uint32_t maxn = n;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxn = max(maxn, __shfl_xor_sync(0xffffffffu, maxn, o));
    // the table's coarse row goes on the critical path one token ahead, the context two ahead
    auto coarse = [&](uint32_t c, uint4 &a, uint4 &b) {
        const uint4 *cq = reinterpret_cast<const uint4 *>(p.tab + (size_t)(c & (kGCtx - 1)) * kGTabU16 + kNSym);
        a = __ldg(cq);
        b = __ldg(cq + 1);
    };
    uint32_t c_cur = n ? __ldg(p.ctx + s0) : 0u, c_nxt = n > 1 ? __ldg(p.ctx + s0 + 1) : 0u;
    uint4 q0 = make_uint4(0u, 0u, 0u, 0u), q1 = q0;
    if (n) coarse(c_cur, q0, q1);
    for (uint32_t t = 0; t < maxn; ++t) {
        const bool active = t < n;
        if (active) {
            const uint32_t i = s0 + t;
            const uint16_t *T = p.tab + (size_t)(c_cur & (kGCtx - 1)) * kGTabU16;
            uint4 n0 = q0, n1 = q1;
            if (t + 1 < n) coarse(c_nxt, n0, n1);
            const uint32_t c_nn = t + 2 < n ? __ldg(p.ctx + i + 2) : 0u;
            const uint32_t slot = x & 0xFFFFu;
            uint32_t lo, hi;
            const uint32_t s = geo_sym(T, q0, q1, slot, lo, hi);
            x = (hi - lo) * (x >> 16) + slot - lo;
            p.out[i] = (uint8_t)s;
            q0 = n0;
            q1 = n1;
            c_cur = c_nxt;
            c_nxt = c_nn;
        }
        group_refill(gs, x, active);
    }
    const bool bad = gs.bad || (lane < nl && x != 0x10000u) || (gs.ptr != gs.n_words);
    if (bad) set_status(p.status, SGS_E_CORRUPT);
}

// ------------------------------------------------------------------ host side

// Lanes of a coded level: about 128 tokens each, in whole groups of 32 (the encoder's rule).
uint32_t geo_learned_lanes(uint64_t n) {
    const uint64_t per = 128ull * 32;
    const uint64_t l = (n + per - 1) / per * 32;
    return (uint32_t)(l < 32 ? 32 : l);
}

uint64_t geo_learned_group_bytes(uint64_t n) {
    const uint64_t G = (geo_learned_lanes(n) + 31) / 32;
    return (8 * (G + 1) + 4 * G + 15) & ~15ull;
}

// Scratch of the learned geometry decode beyond the occupancy bytes: the tables of every coded
// level, one level's contexts and the context scan's tile sums.
uint64_t geo_learned_scratch(const sgs_scene_info &info, uint64_t *tab_bytes, uint64_t *ctx_bytes) {
    uint64_t levels = 0, max_child = 0, max_par = 0;
    for (uint32_t l = 1; l < info.depth; ++l)
        if (info.n_level[l] >= kGeoRansMinLevel) {
            ++levels;
            max_child = info.n_level[l] > max_child ? info.n_level[l] : max_child;
            max_par = info.n_level[l - 1] > max_par ? info.n_level[l - 1] : max_par;
        }
    const uint64_t tb = levels * kGCtx * kGTabBytes;
    const uint64_t cb = (2 * max_child + 255) & ~255ull;
    const uint64_t sb = 4 * (max_par / kGCtxTile + 2);
    if (tab_bytes) *tab_bytes = tb;
    if (ctx_bytes) *ctx_bytes = cb;
    return tb + cb + sb;
}

cudaError_t launch_geo_learned(const uint8_t *bits, const sgs_scene_info &info, const GeoPlan &plan,
                               uint8_t *geo_bytes, uint8_t *work, int *status, cudaStream_t st, int *launches) {
    if (plan.n_coded_levels == 0) return cudaSuccess;
    uint64_t tb = 0, cb = 0;
    geo_learned_scratch(info, &tb, &cb);
    uint16_t *tables = reinterpret_cast<uint16_t *>(work);
    uint16_t *ctx = reinterpret_cast<uint16_t *>(work + tb);
    uint32_t *tile_sums = reinterpret_cast<uint32_t *>(work + tb + cb);
    cudaError_t e;
    GeoTabParams tp;
    memset(&tp, 0, sizeof(tp));
    tp.model = bits + info.off[S_GEO_TAB];
    tp.tables = tables;
    tp.n_levels = plan.n_coded_levels;
    for (int k = 0; k < plan.n_coded_levels; ++k) tp.level[k] = plan.coded_level[k];
    tp.status = status;
    k_geo_tables<<<(unsigned)((uint64_t)plan.n_coded_levels * kGCtx / kTabWarps), 32 * kTabWarps, 0, st>>>(tp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int count = 1;
    uint64_t grp = info.off[S_GEO_GRP];
    for (int k = 0; k < plan.n_coded_levels; ++k) {
        const int l = plan.coded_level[k];
        const uint32_t n = plan.n_level[l], np = plan.n_level[l - 1];
        GeoCtxParams cp;
        cp.par = geo_bytes + plan.level_off[l - 1];
        cp.n_par = np;
        cp.n_child = n;
        cp.ctx = ctx;
        cp.tile_sums = tile_sums;
        cp.status = status;
        const uint32_t tiles = (np + kGCtxTile - 1) / kGCtxTile;
        k_gctx_reduce<<<tiles, 256, 0, st>>>(cp);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_gctx_scan<<<tiles, 256, 0, st>>>(cp);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        GeoLDecParams dp;
        dp.bits = bits;
        dp.grp_sec = grp;
        dp.pay_off = info.off[S_GEO_PAY];
        dp.pay_len = info.off[S_ATTR_TAB] - info.off[S_GEO_PAY];
        dp.L = geo_learned_lanes(n);
        dp.G = (dp.L + 31) / 32;
        dp.n = n;
        dp.ctx = ctx;
        dp.tab = tables + (size_t)k * kGCtx * kGTabU16;
        dp.out = geo_bytes + plan.level_off[l];
        dp.status = status;
        k_geo_learned_decode<<<(dp.G + kLDecWarps - 1) / kLDecWarps, 32 * kLDecWarps, 0, st>>>(dp);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        grp += geo_learned_group_bytes(n);
        count += 3;
    }
    if (launches) *launches += count;
    return cudaSuccess;
}

}  // namespace sgs
