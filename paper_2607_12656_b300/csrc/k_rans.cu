// Static-table rANS decoding on sm_103a: channel-wise attribute coding and per-level
// octree-token coding (the entropy coder standing in for the paper's arithmetic coder,
// Sec. 3.4 and Tab. decoding_complexity; rANS with 32-bit state, 16-bit renormalisation,
// 16-bit probabilities).
//
// Parallel structure: one warp per group of 32 lanes (the paper's groups of W Gaussians,
// Sec. 3.4.2, decoded in parallel).  The 32 lanes of a group share one word stream; at each
// step every lane decodes one symbol and the lanes whose state dropped below 2^16 take the
// next words in lane order -- their word index is the popcount of the ballot below them.
// Tables live in shared memory as cdf[257] with a slot lookup of 1,024 buckets; a symbol is
// the bucket's first symbol or one of the few that start after it inside the bucket.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "sgs_internal.h"
#include "sgs_device.cuh"

namespace sgs {

// Expands static tables (32-byte presence mask, then (f-1) as u16 per present symbol; each
// table's offset and size were validated by scene_query) into cdf[257]; one CTA per table.  A
// table whose frequencies do not sum to 2^16 marks the stream corrupt (an all-zero attribute
// table is allowed for an empty scene).
struct TableOffsets {
    uint32_t off[kMaxTables];
};

struct TableParams {
    const uint8_t *bits;
    TableOffsets to;
    uint8_t *tables;
    int n_geo_tables, allow_empty_attr;
    int *status;
};

__device__ __forceinline__ void tables_body(const TableParams &p, uint32_t t) {
    __shared__ uint32_t sm[8];
    __shared__ uint32_t s_cdf[kTabCdfWords];
    const int s = threadIdx.x;
    const uint8_t *bits = p.bits;
    const uint64_t off = p.to.off[t];
    const uint32_t present = (bits[off + (s >> 3)] >> (s & 7)) & 1u;
    uint32_t K;
    const uint32_t rank = block_excl_scan_256(present, &K, sm);
    const uint32_t f = present ? ld_u16(bits + off + 32 + 2ull * rank) + 1u : 0u;
    uint32_t tot;
    const uint32_t c = block_excl_scan_256(f, &tot, sm);
    uint32_t *out_cdf = reinterpret_cast<uint32_t *>(p.tables + (size_t)t * kTabBytes);
    out_cdf[s] = c;
    s_cdf[s] = c;
    if (s == 0) {
        const bool empty_ok = p.allow_empty_attr && (int)t >= p.n_geo_tables && tot == 0;
        if (!(tot == 65536u || empty_ok)) set_status(p.status, SGS_E_CORRUPT);
        // cdf[256] = 2^16 always (a corrupt table was flagged above): every slot < 2^16 then
        // finds its symbol at or below 255 without a bound check in the decoders
        out_cdf[256] = 65536u;
        s_cdf[256] = 65536u;
    }
    __syncthreads();
    // slot lookup: the symbol holding the first slot of each bucket
    uint8_t *lut = p.tables + (size_t)t * kTabBytes + kTabCdfBytes;
    for (int b = s; b < kLutBuckets; b += 256) lut[b] = (uint8_t)cdf_search(s_cdf, (uint32_t)b << kLutShift);
}

__global__ void __launch_bounds__(256) k_tables(TableParams p) { tables_body(p, blockIdx.x); }

__global__ void __launch_bounds__(256) k_tables_multi(MultiArgs m) {
    run_items<TableParams>(m, [](const TableParams &p, uint32_t vb, uint32_t, bool) { tables_body(p, vb); });
}

static uint32_t make_tables(const uint8_t *bits, const sgs_scene_info &info, int n_geo_tables,
                            uint8_t *tables, int *status, TableParams *pp) {
    TableParams &p = *pp;
    memset(&p, 0, sizeof(p));
    p.bits = bits;
    for (uint32_t i = 0; i < info.n_tables; ++i) p.to.off[i] = info.table_off[i];
    p.tables = tables;
    p.n_geo_tables = n_geo_tables;
    p.allow_empty_attr = info.n_rows == 0;
    p.status = status;
    return info.n_tables;
}

cudaError_t launch_tables(const uint8_t *bits, const sgs_scene_info &info, int n_geo_tables,
                          uint8_t *tables, int *status, cudaStream_t st) {
    TableParams p;
    const uint32_t grid = make_tables(bits, info, n_geo_tables, tables, status, &p);
    if (grid == 0) return cudaSuccess;
    k_tables<<<grid, 256, 0, st>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ attributes

struct AttrParams {
    const uint8_t *bits;
    const uint8_t *tables;   // 56 expanded tables
    uint64_t chan_off;       // step[56], offset[56]
    uint64_t grp_sec, pay_off, pay_len;
    uint32_t L, G, n_rows;
    float *out;
    const uint32_t *out_index;
    int *status;
};

constexpr int kAttrWarps = 32;  // one CTA per SM shares one copy of the 56 tables
static_assert(kAttrWarps == (int)kAttrWarpsMax, "the launch shape's cap is the kernel's launch bound");
static_assert(kNChan % 8 == 0, "channels are decoded 8 at a time");
constexpr size_t kAttrCdfSmem = kNChan * kTabCdfBytes + 2 * kNChan * 4;  // cdf, step, offset
constexpr size_t kAttrTabSmem = kAttrCdfSmem + kNChan * kLutBuckets;
constexpr size_t attr_smem(int warps) { return kAttrTabSmem + (size_t)warps * kWinWords * 2; }
constexpr size_t kAttrSmem = attr_smem(kAttrWarps);
static_assert(kAttrCdfSmem % 16 == 0 && kAttrTabSmem % 16 == 0, "lookup and windows must be 16-byte aligned");
static_assert(kAttrSmem <= 227 * 1024, "attribute decoder shared memory");

// One symbol of a channel (tables tc / lut, dequantization so) for every lane of the group,
// then the group's renormalisation.  PRED: some lanes hold no row at this step (`active`);
// otherwise every lane decodes and no lane predicate is evaluated.
template <bool PRED>
__device__ __forceinline__ void attr_symbol(const uint32_t *tc, const uint8_t *lut, float2 so, float *dst, uint32_t &x,
                                            GroupStream &gs, uint32_t &wrel, uint32_t lt, bool active) {
    if (!PRED || active) __stcs(dst, dequant_small(rans_symbol(tc, lut, x), so.x, so.y));
    group_renorm<false>(gs, x, wrel, lt, !PRED || active);
}

template <bool IDX>
__device__ __forceinline__ void rans_attr_body(const AttrParams &p, uint32_t vb, bool reload) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *s_cdf = (uint32_t *)smem;                          // [56][kTabCdfStride]
    float2 *s_so = (float2 *)(smem + kNChan * kTabCdfBytes);  // [56] (step, offset)
    uint8_t *s_lut = smem + kAttrCdfSmem;                         // [56][1024]
    uint16_t *s_win = reinterpret_cast<uint16_t *>(smem + kAttrTabSmem) + (threadIdx.x >> 5) * kWinWords;
    if (reload) {  // (a CTA's next item of the same scene finds the tables in place)
        load_cdf_smem(p.tables, kNChan, s_cdf, s_lut);
        for (int c = threadIdx.x; c < kNChan; c += blockDim.x)  // (a CTA may be a single warp)
            s_so[c] = make_float2(ld_f32(p.bits + p.chan_off + 4 * c), ld_f32(p.bits + p.chan_off + 4 * (kNChan + c)));
        __syncthreads();
    }
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t g = vb * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (g >= p.G) return;
    // the group's rows, dealt round robin to its lanes: lane j holds rows R0 + j + k nl
    const uint32_t nl = min(32u, p.L - g * 32);
    const uint32_t R0 = (uint32_t)((uint64_t)g * 32 * p.n_rows / p.L);
    const uint32_t R1 = (uint32_t)((uint64_t)(g * 32 + nl) * p.n_rows / p.L);
    const uint32_t my_rows = (lane < nl && R0 + lane < R1) ? (R1 - R0 - lane + nl - 1) / nl : 0;
    GroupStream gs;
    uint32_t x;
    group_open(p.bits, p.grp_sec, p.pay_off, p.pay_len, p.G, g, (int)nl, (int)lane, gs, x, s_win);
    // rows [0, minr) every lane holds (none when the group has fewer than 32 lanes), then the
    // rows only some lanes hold
    uint32_t minr = lane < nl ? my_rows : 0u, maxr = my_rows;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        minr = min(minr, __shfl_xor_sync(0xffffffffu, minr, o));
        maxr = max(maxr, __shfl_xor_sync(0xffffffffu, maxr, o));
    }
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t wrel = gs.ptr - gs.wbase;
    const size_t nr = p.n_rows;
    uint32_t row = R0 + lane, rr = 0;
    // row by row, the 56 channels of a row in order (the coding order); channels unrolled by
    // 8 so table and constant offsets are immediates
    for (; rr < minr; ++rr, row += nl) {
        float *o = p.out + (IDX ? p.out_index[row] : row);
        const uint32_t *cdf = s_cdf;
        const uint8_t *lut = s_lut;
        for (int c0 = 0; c0 < kNChan; c0 += 8, cdf += 8 * kTabCdfStride, lut += 8 * kLutBuckets, o += 8 * nr) {
            window_ensure(gs, wrel, 8 * 32);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                attr_symbol<false>(cdf + k * kTabCdfStride, lut + k * kLutBuckets, s_so[c0 + k], o + k * nr, x, gs, wrel,
                                   lt, true);
        }
    }
    for (; rr < maxr; ++rr, row += nl) {
        const bool active = rr < my_rows;
        float *o = p.out + (IDX ? (active ? p.out_index[row] : 0u) : row);
        const uint32_t *cdf = s_cdf;
        const uint8_t *lut = s_lut;
        for (int c0 = 0; c0 < kNChan; c0 += 8, cdf += 8 * kTabCdfStride, lut += 8 * kLutBuckets, o += 8 * nr) {
            window_ensure(gs, wrel, 8 * 32);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                attr_symbol<true>(cdf + k * kTabCdfStride, lut + k * kLutBuckets, s_so[c0 + k], o + k * nr, x, gs, wrel,
                                  lt, active);
        }
    }
    const bool bad = gs.bad || (lane < nl && x != 0x10000u) || (gs.wbase + wrel != gs.n_words);
    if (bad) set_status(p.status, SGS_E_CORRUPT);
}

template <bool IDX>
__global__ void __launch_bounds__(32 * kAttrWarps) k_rans_attr(AttrParams p) { rans_attr_body<IDX>(p, blockIdx.x, true); }

template <bool IDX>
__global__ void __launch_bounds__(32 * kAttrWarps) k_rans_attr_multi(MultiArgs m) {
    run_items<AttrParams>(m, [](const AttrParams &p, uint32_t vb, uint32_t, bool same) {
        rans_attr_body<IDX>(p, vb, !same);
    });
}

static uint32_t make_rans_attr(const uint8_t *bits, const sgs_scene_info &info, const uint8_t *tables,
                               const sgs_scene_out &out, int *status, AttrParams *pp) {
    AttrParams &p = *pp;
    memset(&p, 0, sizeof(p));
    p.bits = bits;
    p.tables = tables;
    p.chan_off = info.off[S_CHAN];
    p.grp_sec = info.off[S_ATTR_GRP];
    p.pay_off = info.off[S_ATTR_PAY];
    p.pay_len = info.total_len - info.off[S_ATTR_PAY];
    p.L = info.lanes;
    p.G = (info.lanes + 31) / 32;
    p.n_rows = info.n_rows;
    p.out = out.attr;
    p.out_index = out.out_index;
    p.status = status;
    if (info.n_rows == 0) return 0;
    return p.G;  // groups (warps); the launcher packs them into CTAs
}

// Warps per CTA of a single-scene static decode: as many as share one copy of the tables
// (kAttrWarps) when there are groups enough for every SM, fewer so that few groups still
// spread over the SMs (each decodes its lanes' long chains alone).
static int attr_warps(uint32_t groups) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 148;
    }
    const uint32_t w = (groups + (uint32_t)sms - 1) / (uint32_t)sms;
    return (int)(w < 1 ? 1 : (w > (uint32_t)kAttrWarps ? (uint32_t)kAttrWarps : w));
}

// Raises the dynamic shared memory limit of `kernel` once.
template <typename K>
static cudaError_t allow_smem(K kernel, size_t bytes, bool *done) {
    if (*done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) *done = true;
    return e;
}

cudaError_t launch_rans_static_attr(const uint8_t *bits, const sgs_scene_info &info,
                                    const uint8_t *tables, const sgs_scene_out &out, int *status,
                                    cudaStream_t st, uint32_t max_warps) {
    AttrParams p;
    const uint32_t groups = make_rans_attr(bits, info, tables, out, status, &p);
    if (groups == 0) return cudaSuccess;
    static bool set0 = false, set1 = false;
    cudaError_t e = allow_smem(k_rans_attr<false>, kAttrSmem, &set0);
    if (e == cudaSuccess) e = allow_smem(k_rans_attr<true>, kAttrSmem, &set1);
    if (e != cudaSuccess) return e;
    int w = attr_warps(groups);
    if (max_warps >= 1 && max_warps < (uint32_t)w) w = (int)max_warps;
    const uint32_t grid = (groups + w - 1) / w;
    if (p.out_index) k_rans_attr<true><<<grid, 32 * w, attr_smem(w), st>>>(p);
    else k_rans_attr<false><<<grid, 32 * w, attr_smem(w), st>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ geometry tokens

struct GeoParams {
    const uint8_t *bits;
    const uint8_t *tables;   // one expanded table per coded level
    uint64_t grp_sec, pay_off, pay_len;
    uint32_t L, G;
    uint64_t n_coded;
    GeoPlan plan;
    uint8_t *geo_bytes;
    int *status;
};

constexpr int kGeoWarps = 8;
// Shared memory of the geometry decoder for nt coded levels: cdf [nt][kTabCdfStride], lookup
// [nt][1024], then one word-stream window per warp.
__host__ __device__ constexpr size_t geo_cdf_smem(int nt) { return (size_t)nt * kTabCdfBytes; }
__host__ __device__ constexpr size_t geo_tab_smem(int nt) { return geo_cdf_smem(nt) + (size_t)nt * kLutBuckets; }
constexpr size_t kGeoTabSmem = geo_tab_smem(SGS_MAX_DEPTH);

__device__ __forceinline__ void rans_geo_body(const GeoParams &p, uint32_t vb) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int nt = p.plan.n_coded_levels;
    uint32_t *s_cdf = (uint32_t *)smem;
    uint8_t *s_lut = smem + geo_cdf_smem(nt);
    uint16_t *s_win = reinterpret_cast<uint16_t *>(smem + geo_tab_smem(nt)) + (threadIdx.x >> 5) * kWinWords;
    __shared__ uint32_t s_start[SGS_MAX_DEPTH + 1];  // first coded token of each coded level
    __shared__ uint32_t s_dbase[SGS_MAX_DEPTH];      // BFS offset of its tokens minus that
    load_cdf_smem(p.tables, nt, s_cdf, s_lut);
    if (threadIdx.x <= (unsigned)nt) s_start[threadIdx.x] = (uint32_t)p.plan.coded_start[threadIdx.x];
    if (threadIdx.x < (unsigned)nt)
        s_dbase[threadIdx.x] = (uint32_t)(p.plan.level_off[p.plan.coded_level[threadIdx.x]] -
                                          p.plan.coded_start[threadIdx.x]);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t g = vb * kGeoWarps + (threadIdx.x >> 5);
    if (g >= p.G) return;
    // the group's tokens, dealt round robin to its lanes: lane j holds tokens I0 + j + k nl
    const int nl = (int)min(32u, p.L - g * 32);
    const uint32_t I0 = (uint32_t)((uint64_t)g * 32 * p.n_coded / p.L);
    const uint32_t I1 = (uint32_t)((uint64_t)(g * 32 + nl) * p.n_coded / p.L);
    const uint32_t n = (lane < nl && I0 + lane < I1) ? (I1 - I0 - lane + nl - 1) / nl : 0;
    GroupStream gs;
    uint32_t x;
    group_open(p.bits, p.grp_sec, p.pay_off, p.pay_len, p.G, g, nl, lane, gs, x, s_win);
    uint32_t maxn = n;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxn = max(maxn, __shfl_xor_sync(0xffffffffu, maxn, o));
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t wrel = gs.ptr - gs.wbase;
    uint32_t i = I0 + lane;
    // coded level k of token i: its table, the token's offset into the level, and where the
    // next coded level starts
    int k = 0;
    while (k + 1 < nt && s_start[k + 1] <= i) ++k;
    const uint32_t *cdf = s_cdf + k * kTabCdfStride;
    const uint8_t *lut = s_lut + k * kLutBuckets;
    uint32_t next = s_start[k + 1];
    uint32_t dbase = s_dbase[k];
    // a lane crosses into the next coded level every few thousand tokens
    auto level_of = [&]() {
        if (i >= next) {
            while (i >= next && k + 1 < nt) {
                ++k;
                cdf += kTabCdfStride;
                lut += kLutBuckets;
                next = s_start[k + 1];
                dbase = s_dbase[k];
            }
        }
    };
    // steps every lane of the group takes (none when the group has fewer than 32 lanes), eight
    // at a time with one window check, then the steps only some lanes take
    uint32_t minn = lane < nl ? n : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) minn = min(minn, __shfl_xor_sync(0xffffffffu, minn, o));
    uint32_t t = 0;
    for (; t + 8 <= minn; t += 8) {
        window_ensure(gs, wrel, 8 * 32);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            level_of();
            p.geo_bytes[dbase + i] = (uint8_t)rans_symbol(cdf, lut, x);
            i += nl;
            group_renorm<false>(gs, x, wrel, lt, true);
        }
    }
    for (; t < maxn; ++t) {
        const bool active = t < n;
        if (active) {
            level_of();
            p.geo_bytes[dbase + i] = (uint8_t)rans_symbol(cdf, lut, x);
            i += nl;
        }
        group_renorm(gs, x, wrel, lt, active);
    }
    const bool bad = gs.bad || (lane < nl && x != 0x10000u) || (gs.wbase + wrel != gs.n_words);
    if (bad) set_status(p.status, SGS_E_CORRUPT);
}

constexpr size_t kGeoSmem = kGeoTabSmem + kGeoWarps * kWinWords * 2;

__global__ void __launch_bounds__(32 * kGeoWarps) k_rans_geo(GeoParams p) { rans_geo_body(p, blockIdx.x); }

__global__ void __launch_bounds__(32 * kGeoWarps) k_rans_geo_multi(MultiArgs m) {
    run_items<GeoParams>(m, [](const GeoParams &p, uint32_t vb, uint32_t, bool) { rans_geo_body(p, vb); });
}

static uint32_t make_rans_geo(const uint8_t *bits, const sgs_scene_info &info, const GeoPlan &plan,
                              const uint8_t *tables, uint8_t *geo_bytes, int *status, GeoParams *pp) {
    GeoParams &p = *pp;
    memset(&p, 0, sizeof(p));
    p.bits = bits;
    p.tables = tables;
    p.grp_sec = info.off[S_GEO_GRP];
    p.pay_off = info.off[S_GEO_PAY];
    p.pay_len = info.off[S_ATTR_TAB] - info.off[S_GEO_PAY];
    p.L = info.geo_lanes;
    p.G = (info.geo_lanes + 31) / 32;
    p.n_coded = info.n_geo_coded;
    p.plan = plan;
    p.geo_bytes = geo_bytes;
    p.status = status;
    if (info.n_geo_coded == 0) return 0;
    return (p.G + kGeoWarps - 1) / kGeoWarps;
}

cudaError_t launch_rans_static_geo(const uint8_t *bits, const sgs_scene_info &info,
                                   const GeoPlan &plan, const uint8_t *tables, uint8_t *geo_bytes,
                                   int *status, cudaStream_t st) {
    GeoParams p;
    const uint32_t grid = make_rans_geo(bits, info, plan, tables, geo_bytes, status, &p);
    if (grid == 0) return cudaSuccess;
    static bool set = false;
    cudaError_t e = allow_smem(k_rans_geo, kGeoSmem, &set);
    if (e != cudaSuccess) return e;
    const size_t smem = geo_tab_smem(plan.n_coded_levels) + kGeoWarps * kWinWords * 2;
    k_rans_geo<<<grid, 32 * kGeoWarps, smem, st>>>(p);
    return cudaGetLastError();
}

// Copies the uncoded levels' bytes (back to back in level order in geo_raw) to their
// breadth-first positions in geo_bytes.
struct RawCopy {
    int n;
    uint64_t src[SGS_MAX_DEPTH + 1];  // prefix offsets within geo_raw
    uint64_t dst[SGS_MAX_DEPTH];
};

struct CopyParams {
    const uint8_t *raw;
    RawCopy rc;
    uint8_t *geo_bytes;
};

constexpr uint32_t kCopyBytes = 256 * 16;  // bytes one CTA copies

__device__ __forceinline__ void geo_copy_body(const CopyParams &p, uint32_t vb) {
    const uint64_t total = p.rc.src[p.rc.n];
    const uint64_t end = min(total, (uint64_t)(vb + 1) * kCopyBytes);
    for (uint64_t i = (uint64_t)vb * kCopyBytes + threadIdx.x; i < end; i += 256) {
        int k = 0;
        while (k + 1 < p.rc.n && p.rc.src[k + 1] <= i) ++k;
        p.geo_bytes[p.rc.dst[k] + (i - p.rc.src[k])] = p.raw[i];
    }
}

__global__ void __launch_bounds__(256) k_geo_copy_raw(CopyParams p) { geo_copy_body(p, blockIdx.x); }

__global__ void __launch_bounds__(256) k_geo_copy_multi(MultiArgs m) {
    run_items<CopyParams>(m, [](const CopyParams &p, uint32_t vb, uint32_t, bool) { geo_copy_body(p, vb); });
}

static uint32_t make_geo_copy(const uint8_t *bits, const sgs_scene_info &info, const GeoPlan &plan,
                              uint8_t *geo_bytes, CopyParams *pp) {
    CopyParams &p = *pp;
    memset(&p, 0, sizeof(p));
    RawCopy &rc = p.rc;
    rc.n = 0;
    rc.src[0] = 0;
    for (int l = 0; l < plan.depth; ++l) {
        bool coded = false;
        for (int k = 0; k < plan.n_coded_levels; ++k) coded |= plan.coded_level[k] == l;
        if (coded) continue;
        rc.dst[rc.n] = plan.level_off[l];
        rc.src[rc.n + 1] = rc.src[rc.n] + plan.n_level[l];
        ++rc.n;
    }
    p.raw = bits + info.off[S_GEO_RAW];
    p.geo_bytes = geo_bytes;
    if (info.geo_mode == SGS_GEO_RAW || info.n_geo == 0 || rc.n == 0 || rc.src[rc.n] == 0) return 0;
    return (uint32_t)((rc.src[rc.n] + kCopyBytes - 1) / kCopyBytes);
}

cudaError_t launch_geo_copy_raw(const uint8_t *bits, const sgs_scene_info &info,
                                const GeoPlan &plan, uint8_t *geo_bytes, cudaStream_t st) {
    CopyParams p;
    const uint32_t grid = make_geo_copy(bits, info, plan, geo_bytes, &p);
    if (grid == 0) return cudaSuccess;
    k_geo_copy_raw<<<grid, 256, 0, st>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ batched stages

uint32_t stage_tables(const SceneRef &r, void *par) {
    TableParams p;
    const uint32_t n = make_tables(r.bits, *r.info, r.plan->n_geo_tables, r.s->tables, r.status, &p);
    memcpy(par, &p, sizeof(p));
    return n;
}
size_t stage_tables_bytes() { return sizeof(TableParams); }
cudaError_t launch_tables_multi(const MultiArgs &m, cudaStream_t st) {
    return launch_persistent(k_tables_multi, 256, 0, m, st);
}

uint32_t stage_rans_attr(const SceneRef &r, bool idx_variant, void *par) {
    if (r.info->mode != SGS_MODE_STATIC || (r.out->out_index != nullptr) != idx_variant) return 0;
    AttrParams p;
    const uint8_t *attr_tables = r.s->tables + (size_t)r.plan->n_geo_tables * kTabBytes;
    const uint32_t groups = make_rans_attr(r.bits, *r.info, attr_tables, *r.out, r.status, &p);
    memcpy(par, &p, sizeof(p));
    return (groups + kAttrWarps - 1) / kAttrWarps;
}
size_t stage_rans_attr_bytes() { return sizeof(AttrParams); }
cudaError_t launch_rans_attr_multi(bool idx, const MultiArgs &m, cudaStream_t st) {
    static bool set0 = false, set1 = false;
    if (idx) {
        cudaError_t e = allow_smem(k_rans_attr_multi<true>, kAttrSmem, &set1);
        if (e != cudaSuccess) return e;
        return launch_persistent(k_rans_attr_multi<true>, 32 * kAttrWarps, kAttrSmem, m, st);
    }
    cudaError_t e = allow_smem(k_rans_attr_multi<false>, kAttrSmem, &set0);
    if (e != cudaSuccess) return e;
    return launch_persistent(k_rans_attr_multi<false>, 32 * kAttrWarps, kAttrSmem, m, st);
}

uint32_t stage_rans_geo(const SceneRef &r, void *par) {
    GeoParams p;
    const uint32_t n = make_rans_geo(r.bits, *r.info, *r.plan, r.s->tables, r.s->geo_bytes, r.status, &p);
    memcpy(par, &p, sizeof(p));
    return n;
}
size_t stage_rans_geo_bytes() { return sizeof(GeoParams); }
cudaError_t launch_rans_geo_multi(const MultiArgs &m, cudaStream_t st) {
    static bool set = false;
    cudaError_t e = allow_smem(k_rans_geo_multi, kGeoSmem, &set);
    if (e != cudaSuccess) return e;
    return launch_persistent(k_rans_geo_multi, 32 * kGeoWarps, kGeoSmem, m, st);
}

uint32_t stage_geo_copy(const SceneRef &r, void *par) {
    CopyParams p;
    const uint32_t n = make_geo_copy(r.bits, *r.info, *r.plan, r.s->geo_bytes, &p);
    memcpy(par, &p, sizeof(p));
    return n;
}
size_t stage_geo_copy_bytes() { return sizeof(CopyParams); }
cudaError_t launch_geo_copy_multi(const MultiArgs &m, cudaStream_t st) {
    return launch_persistent(k_geo_copy_multi, 256, 0, m, st);
}

}  // namespace sgs
