// Internal declarations of the sgs library (kernels, launchers, bitstream layout).
// The bitstream layout (all little endian, every section 16-byte aligned):
//   header (256 bytes): u32 magic "SGS1", version, mode, geo_mode, n_in, n_rows, depth,
//     n_leaves, n_dup, n_chan, lanes, geo_lanes; u64 n_geo, n_geo_coded; u64 offsets of the
//     ten sections below and the total length.
//   levels   u32 n_level[D]                     nodes per octree level 0..D-1
//   dup      {u32 rank, u32 extra}[n_dup]       leaf ranks holding extra Gaussians, ascending
//   chan     f32 step[56], f32 offset[56], u32 bits[56]
//   geo_raw  occupancy bytes of the uncoded levels, level order
//   geo_tab  per coded level: 32-byte presence mask + (f-1) as u16 for present symbols,
//            padded to 16 bytes (a level is coded iff geo_mode = RANS and n_level >= 4096)
//   geo_grp  u64 group_off[G+1] (bytes from geo_pay), u32 group_words[G]   (G = ceil(Lg/32))
//   geo_pay  rANS group streams
//   attr_tab fixed: u64 chan_off[57] (bytes from attr_pay); static: 56 tables as geo_tab;
//            learned: the frozen model (SGS_MODEL_BYTES); position-aware learned: the
//            frozen model (SGS_MODEL_PE_BYTES)
//   attr_grp as geo_grp with G = ceil(L/32)
//   attr_pay payload
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sgs.h"

namespace sgs {

constexpr uint32_t kMagic = 0x31534753u;
constexpr uint32_t kVersion = 1;
constexpr int kNChan = 56;
constexpr int kNSym = 256;
constexpr uint32_t kGeoRansMinLevel = 4096;
constexpr int kHeaderBytes = 256;
constexpr int kMaxTables = kNChan + SGS_MAX_DEPTH;
enum Sec { S_LEVELS = 0, S_DUP, S_CHAN, S_GEO_RAW, S_GEO_TAB, S_GEO_GRP, S_GEO_PAY, S_ATTR_TAB,
           S_ATTR_GRP, S_ATTR_PAY, S_TOTAL };

// Expanded static table in device memory: cdf[257] (u32), padded to 16 bytes, then a slot
// lookup lut[1024] (u8): lut[b] = the symbol whose range holds slot 64 b.  A slot's symbol is
// lut[slot >> 6] or one of the symbols that start in the same 64-slot bucket after it.
constexpr int kTabCdfWords = 257;
constexpr int kTabCdfBytes = (kTabCdfWords * 4 + 15) & ~15;  // 1040
constexpr int kTabCdfStride = kTabCdfBytes / 4;               // 260: a table's cdf row in shared memory
constexpr int kLutShift = 6;
constexpr int kLutBuckets = 65536 >> kLutShift;              // 1024
constexpr int kTabBytes = kTabCdfBytes + kLutBuckets;         // 2064

// Per-level facts of one scene's octree, by value in kernel parameters.
struct GeoPlan {
    int depth;
    int n_coded_levels;
    int n_geo_tables;                        // static geometry tables (n_coded_levels for rANS, else 0)
    uint32_t n_level[SGS_MAX_DEPTH + 1];     // [D] = leaves
    uint64_t level_off[SGS_MAX_DEPTH + 1];   // global BFS index of each level's first node
    int coded_level[SGS_MAX_DEPTH];          // coded level ids, ascending
    uint64_t coded_start[SGS_MAX_DEPTH + 1]; // prefix of coded symbols per coded level
};

// Scratch carve-out of one scene decode (device pointers).
struct Scratch {
    uint8_t *geo_bytes;     // n_geo (rANS geometry only)
    uint32_t *p4;           // popcount prefix at every 4-byte word of the tokens (+ total)
    uint32_t *tile_sums;    // popcount sum of each scan tile
    uint32_t *par;          // parent entry (x << 3 | child index) of every node but the root
    uint8_t *tables;        // expanded static tables
    uint32_t *dup_prefix;   // n_dup + 1
    uint8_t *learned;       // learned-mode per-scene work area
    uint32_t *coord;        // position-aware mode: voxel coordinates [3][n_rows] when the
                            // caller asks for none (the attribute model reads them)
    uint8_t *geo_work;      // learned geometry: context tables, contexts, scan tile sums
};

size_t scratch_need(const sgs_scene_info &info, Scratch *layout, uint8_t *base);
size_t octree_scan_tiles(uint64_t n_geo);

// Device status: kernels record the most severe error with atomicMin (codes are negative).
__device__ __forceinline__ void set_status(int *status, int code) {
    atomicMin(status, code);
}

// Launchers (return cudaError_t of the launch).
cudaError_t launch_tables(const uint8_t *bits, const sgs_scene_info &info, int n_geo_tables,
                          uint8_t *tables, int *status, cudaStream_t st);
// Device sort and scan (k_sort.cu).  scan_u32: out[i] = in[0] + .. + in[i-1] for i < n,
// sums[] needs ceil(n / kScanBlock) + 1 words (sums[last] = the total).  radix_pass: one
// stable 8-bit digit pass of an LSD radix sort of n (key, value) pairs on key bits
// [shift, shift + 8); cnt and cnt_off need 256 ceil(n / kSortChunk) words each, csums the
// scan's sums for that many items.
constexpr int kScanBlock = 1024;
constexpr int kSortThreads = 256;
constexpr int kSortRounds = 8;
constexpr int kSortChunk = kSortThreads * kSortRounds;
cudaError_t scan_u32(const uint32_t *in, uint64_t n, uint32_t *sums, uint32_t *out, cudaStream_t st);
cudaError_t radix_pass(const uint32_t *keys, const uint32_t *vals, uint32_t n, int shift, uint32_t *cnt,
                       uint32_t *cnt_off, uint32_t *csums, uint32_t *keys_out, uint32_t *vals_out, cudaStream_t st);

// Launch shapes the attribute decoders accept (sgs_set_launch_shape): warps per CTA.
constexpr uint32_t kAttrWarpsMax = 32;  // static rANS: groups sharing one copy of the tables
constexpr uint32_t kFixWarpsMax = 8;    // fixed-length: (channel, 1,024-row) items per CTA
// max_warps = 0: the built-in shape
cudaError_t launch_rans_static_attr(const uint8_t *bits, const sgs_scene_info &info,
                                    const uint8_t *tables, const sgs_scene_out &out, int *status,
                                    cudaStream_t st, uint32_t max_warps = 0);
cudaError_t launch_rans_static_geo(const uint8_t *bits, const sgs_scene_info &info,
                                   const GeoPlan &plan, const uint8_t *tables, uint8_t *geo_bytes,
                                   int *status, cudaStream_t st);
cudaError_t launch_geo_copy_raw(const uint8_t *bits, const sgs_scene_info &info,
                                const GeoPlan &plan, uint8_t *geo_bytes, cudaStream_t st);
// Learned geometry (SGS_GEO_LEARNED): the coded levels' tokens into geo_bytes, level by level
// (the raw levels copied there first); work = Scratch::geo_work.  *launches += kernels.
cudaError_t launch_geo_learned(const uint8_t *bits, const sgs_scene_info &info, const GeoPlan &plan,
                               uint8_t *geo_bytes, uint8_t *work, int *status, cudaStream_t st, int *launches);
uint64_t geo_learned_scratch(const sgs_scene_info &info, uint64_t *tab_bytes, uint64_t *ctx_bytes);
uint32_t geo_learned_lanes(uint64_t n);
uint64_t geo_learned_group_bytes(uint64_t n);
// The octree reads the raw token section, or the scratch copy of the geometry decoder when
// levels are rANS-coded.  Scan with parent scatter, then the leaf walk, on st.
cudaError_t launch_octree(const sgs_scene_info &info, const GeoPlan &plan, const uint8_t *bits,
                          const Scratch &s, const sgs_scene_out &out, int *status, cudaStream_t st);
cudaError_t launch_fixed(const uint8_t *bits, const sgs_scene_info &info,
                         const sgs_scene_out &out, int *status, cudaStream_t st, uint32_t warps = 0);
// Polls of a bounded device wait before it gives up (the default of sgs_set_wait_limit).
constexpr uint32_t kDefaultWaitPolls = 1u << 24;
cudaError_t launch_learned_decode(const uint8_t *bits, const sgs_scene_info &info,
                                  const sgs_scene_out &out, uint8_t *work, int *status,
                                  cudaStream_t st, uint32_t wait_limit = kDefaultWaitPolls);
size_t learned_work_bytes(const sgs_scene_info &info);
// Position-aware learned decode: reads the rows' voxel coordinates coord [3][n_rows]
// (written by the octree walk before it, in stream order).
cudaError_t launch_learned_pe_decode(const uint8_t *bits, const sgs_scene_info &info,
                                     const sgs_scene_out &out, const uint32_t *coord, int *status,
                                     cudaStream_t st);
// Encoder helper: f and cum of every token under a frozen position-aware model (device).
cudaError_t launch_pe_fc(const uint8_t *model_dev, const uint8_t *tok_dev, const uint32_t *coord_dev,
                         int depth, uint32_t n_rows, uint32_t lanes, uint32_t *f_dev,
                         uint32_t *cum_dev, int *status, cudaStream_t st);
// The outputs a decode works with: the caller's, with the coordinates redirected to
// scratch when the position-aware model needs them and the caller passed none.
sgs_scene_out effective_out(const sgs_scene_info &info, const sgs_scene_out &out, const Scratch &s);

// Encoder helper: f and cum of every token under a frozen model (device arrays).
cudaError_t launch_learned_fc(const uint8_t *model_dev, const uint8_t *tokens_dev,
                              uint32_t n_rows, uint32_t lanes, uint32_t *f_dev,
                              uint32_t *cum_dev, cudaStream_t st);

void make_geo_plan(const sgs_scene_info &info, GeoPlan *plan);

// ------------------------------------------------------------------ batched stages
// A batched decode runs each pipeline stage of many scenes as one persistent launch: CTAs
// claim work items (the single-scene kernel's CTAs, "virtual blocks") in increasing order
// from an atomic counter and look up the owning scene.  Scene s of a stage owns items
// [prefix[s], prefix[s+1]) and the parameter block at params + s * stride.
struct MultiArgs {
    const uint8_t *params;
    uint32_t stride;          // multiple of 16
    const uint32_t *prefix;   // n + 1 entries, strictly increasing
    int n;
    uint32_t total;           // prefix[n]
    uint32_t *counter;        // zero before the launch
    // Completion flags (all NULL when unused): list entry s is scene scene_id[s] of the
    // batch; done[g] counts the finished items of scene g over all launches of a run
    // (zero before the run), need[g] is their number, and the CTA that finishes the last
    // one stamps the device global timer (ns) into t_done[g].
    const uint32_t *scene_id;
    uint32_t *done;
    const uint32_t *need;
    unsigned long long *t_done;
};

// One scene as the stage builders see it (device pointers; the scratch already carved).
struct SceneRef {
    const uint8_t *bits;
    const sgs_scene_info *info;
    const sgs_scene_out *out;
    const Scratch *s;
    const GeoPlan *plan;
    int *status;
};

// CTAs of `kernel` resident on the whole current device (cached per kernel and device).
int resident_ctas(const void *kernel, int threads, size_t smem);

// Launches a persistent grid (at most one wave of resident CTAs).  With m.total = 0 it only
// fills the occupancy cache.
template <typename K>
cudaError_t launch_persistent(K kernel, int threads, size_t smem, const MultiArgs &m, cudaStream_t st) {
    const int r = resident_ctas(reinterpret_cast<const void *>(kernel), threads, smem);
    if (r <= 0) return cudaErrorInvalidConfiguration;
    if (m.total == 0) return cudaSuccess;
    const unsigned grid = m.total < (uint32_t)r ? m.total : (unsigned)r;
    kernel<<<grid, threads, smem, st>>>(m);
    return cudaGetLastError();
}

// Stage builders: write one scene's parameter block to `par` (at most the stage's
// *_bytes()) and return its items, 0 when the scene has no work in the stage.
uint32_t stage_fixed(const SceneRef &r, bool vec_variant, void *par);
size_t stage_fixed_bytes();
cudaError_t launch_fixed_multi(bool vec, const MultiArgs &m, cudaStream_t st);
uint32_t stage_tables(const SceneRef &r, void *par);
size_t stage_tables_bytes();
cudaError_t launch_tables_multi(const MultiArgs &m, cudaStream_t st);
uint32_t stage_rans_attr(const SceneRef &r, bool idx_variant, void *par);
size_t stage_rans_attr_bytes();
cudaError_t launch_rans_attr_multi(bool idx, const MultiArgs &m, cudaStream_t st);
uint32_t stage_rans_geo(const SceneRef &r, void *par);
size_t stage_rans_geo_bytes();
cudaError_t launch_rans_geo_multi(const MultiArgs &m, cudaStream_t st);
uint32_t stage_geo_copy(const SceneRef &r, void *par);
size_t stage_geo_copy_bytes();
cudaError_t launch_geo_copy_multi(const MultiArgs &m, cudaStream_t st);
uint32_t stage_learned(const SceneRef &r, void *par);
size_t stage_learned_bytes();
cudaError_t launch_learned_multi(const MultiArgs &m, cudaStream_t st);
uint32_t stage_learned_pe(const SceneRef &r, void *par);
size_t stage_learned_pe_bytes();
cudaError_t launch_learned_pe_multi(const MultiArgs &m, cudaStream_t st);
// octree: duplicates, popcount scan with parent scatter, leaf walk
uint32_t stage_dup(const SceneRef &r, void *par);
size_t stage_dup_bytes();
cudaError_t launch_dup_multi(const MultiArgs &m, cudaStream_t st);
uint32_t stage_scan(const SceneRef &r, int variant, void *par);  // 0 scan, 1 reduce, 2 scatter
size_t stage_scan_bytes();
cudaError_t launch_scan_multi(int variant, const MultiArgs &m, cudaStream_t st);
uint32_t stage_walk(const SceneRef &r, void *par);
size_t stage_walk_bytes();
cudaError_t launch_walk_multi(const MultiArgs &m, cudaStream_t st);

}  // namespace sgs
