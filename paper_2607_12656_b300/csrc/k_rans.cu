// Static-table rANS decoding on sm_103a: channel-wise attribute coding and per-level
// octree-token coding (the entropy coder standing in for the paper's arithmetic coder,
// Sec. 3.4 and Tab. decoding_complexity; rANS with 32-bit state, 16-bit renormalisation,
// 16-bit probabilities).
//
// Parallel structure: one warp per group of 32 lanes (the paper's groups of W Gaussians,
// Sec. 3.4.2, decoded in parallel).  The 32 lanes of a group share one word stream; at each
// step every lane decodes one symbol and the lanes whose state dropped below 2^16 take the
// next words in lane order -- their word index is the popcount of the ballot below them.
// Tables live in shared memory as cdf[257] plus a 256-bucket index on the top 8 slot bits.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sgs_internal.h"
#include "sgs_device.cuh"

namespace sgs {

// Expands static tables (32-byte presence mask, then (f-1) as u16 per present symbol; each
// table's offset and size were validated by scene_query) into cdf[257] + bucket[256]; one
// CTA per table.  A table whose frequencies do not sum to 2^16 marks the stream corrupt (an
// all-zero attribute table is allowed for an empty scene).
struct TableOffsets {
    uint32_t off[kMaxTables];
};

__global__ void __launch_bounds__(256) k_tables(const uint8_t *bits, TableOffsets to,
                                                uint8_t *tables, int n_geo_tables,
                                                int allow_empty_attr, int *status) {
    __shared__ uint32_t sm[8];
    __shared__ uint32_t cdf[kTabCdfWords];
    const int s = threadIdx.x, t = blockIdx.x;
    const uint64_t off = to.off[t];
    const uint32_t present = (bits[off + (s >> 3)] >> (s & 7)) & 1u;
    uint32_t K;
    const uint32_t rank = block_excl_scan_256(present, &K, sm);
    const uint32_t f = present ? ld_u16(bits + off + 32 + 2ull * rank) + 1u : 0u;
    uint32_t tot;
    const uint32_t c = block_excl_scan_256(f, &tot, sm);
    cdf[s] = c;
    if (s == 0) {
        cdf[256] = tot;
        const bool empty_ok = allow_empty_attr && t >= n_geo_tables && tot == 0;
        if (!(tot == 65536u || empty_ok)) set_status(status, SGS_E_CORRUPT);
    }
    __syncthreads();
    uint32_t *out_cdf = reinterpret_cast<uint32_t *>(tables + (size_t)t * kTabBytes);
    uint8_t *out_bucket = tables + (size_t)t * kTabBytes + kTabCdfWords * 4;
    out_cdf[s] = cdf[s];
    if (s == 0) out_cdf[256] = cdf[256];
    // bucket[b]: largest symbol whose cdf <= b * 256 (a lower bound for any slot >= b*256)
    const uint32_t key = (uint32_t)s << 8;
    int lo = 0, hi = 255;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cdf[mid] <= key) lo = mid; else hi = mid - 1;
    }
    out_bucket[s] = (uint8_t)lo;
}

cudaError_t launch_tables(const uint8_t *bits, const sgs_scene_info &info, int n_geo_tables,
                          uint8_t *tables, int *status, cudaStream_t st) {
    if (info.n_tables == 0) return cudaSuccess;
    TableOffsets to;
    for (uint32_t i = 0; i < info.n_tables; ++i) to.off[i] = info.table_off[i];
    k_tables<<<info.n_tables, 256, 0, st>>>(bits, to, tables, n_geo_tables, info.n_rows == 0, status);
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
constexpr size_t kAttrTabSmem = kNChan * kTabCdfWords * 4 + kNChan * 256 + 2 * kNChan * 4;
constexpr size_t kAttrSmem = kAttrTabSmem + kAttrWarps * kWinWords * 2;
static_assert(kAttrTabSmem % 16 == 0, "window must be 16-byte aligned");

__global__ void __launch_bounds__(32 * kAttrWarps) k_rans_attr(AttrParams p) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *s_cdf = (uint32_t *)smem;                          // [56][257]
    uint8_t *s_bucket = smem + kNChan * kTabCdfWords * 4;         // [56][256]
    float *s_step = (float *)(s_bucket + kNChan * 256);           // [56]
    float *s_off = s_step + kNChan;                               // [56]
    uint16_t *s_win = reinterpret_cast<uint16_t *>(smem + kAttrTabSmem) + (threadIdx.x >> 5) * kWinWords;
    load_tables_smem(p.tables, kNChan, s_cdf, s_bucket);
    if (threadIdx.x < kNChan) {
        s_step[threadIdx.x] = ld_f32(p.bits + p.chan_off + 4 * threadIdx.x);
        s_off[threadIdx.x] = ld_f32(p.bits + p.chan_off + 4 * (kNChan + threadIdx.x));
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t g = blockIdx.x * kAttrWarps + (threadIdx.x >> 5);
    if (g >= p.G) return;
    // the group's rows, dealt round robin to its lanes: lane j holds rows R0 + j + k nl
    const int nl = (int)min(32u, p.L - g * 32);
    const uint64_t R0 = (uint64_t)g * 32 * p.n_rows / p.L;
    const uint64_t R1 = (uint64_t)(g * 32 + nl) * p.n_rows / p.L;
    const uint64_t my_rows = (lane < nl && R0 + lane < R1) ? (R1 - R0 - lane + nl - 1) / nl : 0;
    const uint64_t n = my_rows * kNChan;
    GroupStream gs;
    uint32_t x;
    group_open(p.bits, p.grp_sec, p.pay_off, p.pay_len, p.G, g, nl, lane, gs, x, s_win);
    const uint64_t maxn = warp_max_u64(n);
    uint64_t row = R0 + lane;
    int c = 0;
    for (uint64_t t = 0; t < maxn; ++t) {
        const bool active = t < n;
        if (active) {
            const uint32_t s = rans_sym(x, s_cdf + c * kTabCdfWords, s_bucket + c * 256);
            const uint64_t col = p.out_index ? (uint64_t)p.out_index[row] : row;
            p.out[(uint64_t)c * p.n_rows + col] = dequant(s, s_step[c], s_off[c]);
            if (++c == kNChan) { c = 0; row += nl; }
        }
        group_refill(gs, x, active);
    }
    const bool bad = gs.bad || (lane < nl && x != 0x10000u) || (gs.ptr != gs.n_words);
    if (bad) set_status(p.status, SGS_E_CORRUPT);
}

cudaError_t launch_rans_static_attr(const uint8_t *bits, const sgs_scene_info &info,
                                    const uint8_t *tables, const sgs_scene_out &out, int *status,
                                    cudaStream_t st) {
    if (info.n_rows == 0) return cudaSuccess;
    AttrParams p;
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
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_rans_attr, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kAttrSmem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const unsigned grid = (p.G + kAttrWarps - 1) / kAttrWarps;
    k_rans_attr<<<grid, 32 * kAttrWarps, kAttrSmem, st>>>(p);
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
constexpr size_t kGeoTabSmem = (SGS_MAX_DEPTH * (kTabCdfWords * 4 + 256) + 15) & ~size_t(15);
static_assert(kGeoTabSmem % 16 == 0, "window must be 16-byte aligned");

__global__ void __launch_bounds__(32 * kGeoWarps) k_rans_geo(GeoParams p) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int nt = p.plan.n_coded_levels;
    uint32_t *s_cdf = (uint32_t *)smem;
    uint8_t *s_bucket = smem + (size_t)nt * kTabCdfWords * 4;
    uint16_t *s_win = reinterpret_cast<uint16_t *>(smem + kGeoTabSmem) + (threadIdx.x >> 5) * kWinWords;
    load_tables_smem(p.tables, nt, s_cdf, s_bucket);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t g = blockIdx.x * kGeoWarps + (threadIdx.x >> 5);
    if (g >= p.G) return;
    // the group's tokens, dealt round robin to its lanes: lane j holds tokens I0 + j + k nl
    const int nl = (int)min(32u, p.L - g * 32);
    const uint64_t I0 = (uint64_t)g * 32 * p.n_coded / p.L;
    const uint64_t I1 = (uint64_t)(g * 32 + nl) * p.n_coded / p.L;
    const uint64_t n = (lane < nl && I0 + lane < I1) ? (I1 - I0 - lane + nl - 1) / nl : 0;
    GroupStream gs;
    uint32_t x;
    group_open(p.bits, p.grp_sec, p.pay_off, p.pay_len, p.G, g, nl, lane, gs, x, s_win);
    const uint64_t maxn = warp_max_u64(n);
    uint64_t i = I0 + lane;
    int k = 0;  // coded level of token i
    while (k + 1 < nt && p.plan.coded_start[k + 1] <= i) ++k;
    for (uint64_t t = 0; t < maxn; ++t) {
        const bool active = t < n;
        if (active) {
            while (k + 1 < nt && p.plan.coded_start[k + 1] <= i) ++k;
            const uint32_t s = rans_sym(x, s_cdf + k * kTabCdfWords, s_bucket + k * 256);
            const uint64_t dst = p.plan.level_off[p.plan.coded_level[k]] + (i - p.plan.coded_start[k]);
            p.geo_bytes[dst] = (uint8_t)s;
            i += nl;
        }
        group_refill(gs, x, active);
    }
    const bool bad = gs.bad || (lane < nl && x != 0x10000u) || (gs.ptr != gs.n_words);
    if (bad) set_status(p.status, SGS_E_CORRUPT);
}

cudaError_t launch_rans_static_geo(const uint8_t *bits, const sgs_scene_info &info,
                                   const GeoPlan &plan, const uint8_t *tables, uint8_t *geo_bytes,
                                   int *status, cudaStream_t st) {
    if (info.n_geo_coded == 0) return cudaSuccess;
    GeoParams p;
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
    const size_t smem = kGeoTabSmem + kGeoWarps * kWinWords * 2;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_rans_geo, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const unsigned grid = (p.G + kGeoWarps - 1) / kGeoWarps;
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

__global__ void k_geo_copy_raw(const uint8_t *raw, RawCopy rc, uint8_t *geo_bytes) {
    const uint64_t total = rc.src[rc.n];
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        int k = 0;
        while (k + 1 < rc.n && rc.src[k + 1] <= i) ++k;
        geo_bytes[rc.dst[k] + (i - rc.src[k])] = raw[i];
    }
}

cudaError_t launch_geo_copy_raw(const uint8_t *bits, const sgs_scene_info &info,
                                const GeoPlan &plan, uint8_t *geo_bytes, cudaStream_t st) {
    RawCopy rc;
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
    if (rc.n == 0 || rc.src[rc.n] == 0) return cudaSuccess;
    const uint64_t total = rc.src[rc.n];
    const uint64_t want = (total + 255) / 256;
    const unsigned grid = (unsigned)(want < 4096 ? want : 4096);
    k_geo_copy_raw<<<grid, 256, 0, st>>>(bits + info.off[S_GEO_RAW], rc, geo_bytes);
    return cudaGetLastError();
}

}  // namespace sgs
