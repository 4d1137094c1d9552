// Sparse-octree decoding on sm_103a (Sec. 3.4, "Geometry Occupancy Coding": occupancy
// tokens, one per internal node, level by level; one position per voxel plus duplicate
// counts as metadata).
//
// The tokens of all levels form one breadth-first array B.  With P(x) = sum of popc(B[h])
// for h < x, the children of node x are the nodes 1 + P(x) + j (j < popc(B[x])), the j-th
// taking child index k = the j-th set bit of B[x]; leaves are numbered after the internal
// nodes.  Two launches decode the tree without any level-by-level synchronisation:
//   1. a device-wide scan of popcounts (reduce, then scan), then a map over the nodes that
//      writes every child's parent entry par[1 + P(x) + j] = x << 3 | k;
//   2. a walk from every leaf up to the root (D dependent loads of par), assembling the
//      leaf's coordinates one bit per level, then writing its position rows.
// The level counts in the header are checked against P (the children of each level are
// exactly the next level), so every parent entry is written once per decode.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "sgs_device.cuh"
#include "sgs_internal.h"

namespace sgs {

constexpr int kScanThreads = 256;
constexpr int kWalkThreads = 256;
constexpr int kWalkIlp = 4;                        // leaves a thread walks together
constexpr uint32_t kWalkLeaves = kWalkThreads * kWalkIlp;  // leaves per CTA

struct LeafOut {
    float *pos;
    uint32_t *coord;
    const uint32_t *out_index;
    uint32_t n_rows, n_leaves, n_dup, depth;
    const uint32_t *dup;        // {rank, extra} pairs
    const uint32_t *dup_prefix; // exclusive prefix of extra
    float scale, half;          // 2^-D, 2^-(D+1)
};

// Every third bit of v, from bit 0 (the inverse of spreading a coordinate over a Morton code).
__device__ __forceinline__ uint32_t compact3(uint64_t v) {
    v &= 0x1249249249249249ull;
    v = (v | (v >> 2)) & 0x10C30C30C30C30C3ull;
    v = (v | (v >> 4)) & 0x100F00F00F00F00Full;
    v = (v | (v >> 8)) & 0x001F0000FF0000FFull;
    v = (v | (v >> 16)) & 0x001F00000000FFFFull;
    v = (v | (v >> 32)) & 0x00000000001FFFFFull;
    return (uint32_t)v;
}

// Writes the rows of leaf u (Morton rank) with Morton code mc (x the high bit of each triple).
__device__ __forceinline__ void write_leaf(const LeafOut &o, uint32_t u, uint64_t mc, int *status) {
    uint32_t row = u, mult = 1;
    if (o.n_dup) {
        uint32_t lo = 0, hi = o.n_dup;  // first dup entry with rank >= u
        while (lo < hi) {
            uint32_t mid = (lo + hi) >> 1;
            if (o.dup[2 * mid] < u) lo = mid + 1; else hi = mid;
        }
        row = u + o.dup_prefix[lo];
        if (lo < o.n_dup && o.dup[2 * lo] == u) mult += o.dup[2 * lo + 1];
    }
    if ((uint64_t)row + mult > o.n_rows) { set_status(status, SGS_E_CORRUPT); return; }
    const uint32_t x = compact3(mc >> 2), y = compact3(mc >> 1), z = compact3(mc);
    // voxel centre coord * 2^-D + 2^-(D+1): exact in fp32 (both operations are exact)
    const float px = __fadd_rn(__fmul_rn((float)x, o.scale), o.half);
    const float py = __fadd_rn(__fmul_rn((float)y, o.scale), o.half);
    const float pz = __fadd_rn(__fmul_rn((float)z, o.scale), o.half);
    const uint64_t n = o.n_rows;
    for (uint32_t r = row; r < row + mult; ++r) {
        const uint64_t col = o.out_index ? (uint64_t)o.out_index[r] : r;
        o.pos[col] = px;
        o.pos[n + col] = py;
        o.pos[2 * n + col] = pz;
        if (o.coord) {
            o.coord[col] = x;
            o.coord[n + col] = y;
            o.coord[2 * n + col] = z;
        }
    }
}

// ------------------------------------------------------------------ popcount scan


// Word k of B with the bytes at or past n cleared.
__device__ __forceinline__ uint32_t word_at(const uint8_t *B, uint64_t n, uint64_t k) {
    if (4 * k + 4 <= n) return reinterpret_cast<const uint32_t *>(B)[k];
    uint32_t w = 0;
    for (uint64_t i = 4 * k; i < n; ++i) w |= (uint32_t)B[i] << (8 * (i - 4 * k));
    return w;
}

// P4[k] = popcount of B[0, 4k) for k = 0 .. ceil(n/4), as a reduce-then-scan over tiles of
// 256 threads x 64 bytes: k_octree_reduce writes each tile's popcount sum, then
// k_octree_scan gives each tile the sum of the tiles before it (a block-wide sum of their
// sums) and scans inside the tile to write P4.  No tile ever waits on another.
struct ScanParams {
    const uint8_t *B;
    uint64_t n, n_words;
    uint32_t *P4;
    uint32_t *par;             // parent entries x << 3 | k of nodes 1 .. total-1
    uint32_t *tile_sums;       // one popcount sum per tile
    int *status;
    int depth;
    uint32_t level_off[SGS_MAX_DEPTH + 2];  // [D + 1] = total node count
};

// The tile's 16 words per thread (bytes at or past n cleared).
__device__ __forceinline__ void tile_words(const uint8_t *B, uint64_t n, uint64_t k, uint32_t (&wd)[16]) {
    const uint64_t w0 = 16 * k;
    if (64 * k + 64 <= n) {
        const uint4 *p = reinterpret_cast<const uint4 *>(B + 64 * k);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint4 v = p[i];
            wd[4 * i] = v.x;
            wd[4 * i + 1] = v.y;
            wd[4 * i + 2] = v.z;
            wd[4 * i + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) wd[i] = (w0 + i) * 4 < n ? word_at(B, n, w0 + i) : 0u;
    }
}

__device__ __forceinline__ void reduce_body(const ScanParams &sp, uint32_t tile) {
    __shared__ uint32_t sm[8];
    uint32_t wd[16];
    tile_words(sp.B, sp.n, (uint64_t)tile * kScanThreads + threadIdx.x, wd);
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) sum += __popc(wd[i]);
    uint32_t tot;
    block_excl_scan_256(sum, &tot, sm);
    if (threadIdx.x == 0) sp.tile_sums[tile] = tot;
}

__device__ __forceinline__ void scan_body(const ScanParams &sp, uint32_t tile) {
    __shared__ uint32_t sm[8];
    __shared__ uint32_t sm_p4[kScanThreads * 17];
    const uint64_t n = sp.n, n_words = sp.n_words;
    const uint64_t k = (uint64_t)tile * kScanThreads + threadIdx.x;  // 64-byte chunk
    uint32_t wd[16];
    tile_words(sp.B, n, k, wd);
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) sum += __popc(wd[i]);
    // tiles before this one
    uint32_t before = 0;
    for (uint32_t t = threadIdx.x; t < tile; t += kScanThreads) before += sp.tile_sums[t];
    uint32_t prefix;
    block_excl_scan_256(before, &prefix, sm);
    uint32_t agg;
    const uint32_t local = block_excl_scan_256(sum, &agg, sm);
    const uint32_t base = prefix + local;  // P at this thread's first word
    // P4 of the tile's 4096 words through shared memory (word w at w + w / 16: conflict-free),
    // then written out contiguously
    uint32_t run = base;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        sm_p4[17 * threadIdx.x + i] = run;
        run += __popc(wd[i]);
    }
    __syncthreads();
    const uint64_t tw = (uint64_t)tile * kScanThreads * 16;  // the tile's first word
#pragma unroll 4
    for (uint32_t j = threadIdx.x; j < kScanThreads * 16; j += kScanThreads)
        if (tw + j <= n_words) sp.P4[tw + j] = sm_p4[j + (j >> 4)];  // P4[n_words] = total
}

// The single-scene chain reduce -> scan -> scatter -> walk may be launched with programmatic
// dependent launch (launch_after): each kernel lets its successor be scheduled as soon as it
// starts, and the successor waits for the predecessor grid's completion (and its writes)
// before reading them, so the launch latency of the next kernel overlaps the tail of this
// one.  Launched normally, the wait returns at once.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__global__ void __launch_bounds__(kScanThreads) k_octree_reduce(ScanParams p) {
    pdl_trigger();
    reduce_body(p, blockIdx.x);
}

__global__ void __launch_bounds__(kScanThreads) k_octree_scan(ScanParams p) {
    pdl_trigger();
    pdl_wait();
    scan_body(p, blockIdx.x);
}

__global__ void __launch_bounds__(kScanThreads) k_octree_reduce_multi(MultiArgs m) {
    run_items<ScanParams>(m, [](const ScanParams &p, uint32_t vb, uint32_t, bool) { reduce_body(p, vb); });
}

__global__ void __launch_bounds__(kScanThreads) k_octree_scan_multi(MultiArgs m) {
    run_items<ScanParams>(m, [](const ScanParams &p, uint32_t vb, uint32_t, bool) { scan_body(p, vb); });
}

// Node x of B: its token and P(x) from the word prefix.
__device__ __forceinline__ void node_at(const uint8_t *B, uint64_t n, const uint32_t *P4,
                                        uint32_t x, uint32_t &byte, uint32_t &p) {
    const uint32_t w = word_at(B, n, x >> 2);
    const uint32_t sh = 8u * (uint32_t)(x & 3);
    byte = (w >> sh) & 0xFFu;
    p = P4[x >> 2] + __popc(w & ((1u << sh) - 1u));
}

// Parent entries: node x's j-th child (child index k = the j-th set bit of B[x]) is node
// 1 + P(x) + j, and gets par = x << 3 | k.  A map over the nodes, kScatterIlp per thread with
// their loads issued first; consecutive threads take consecutive nodes, whose children are
// consecutive, so the stores coalesce.  A child index past the last node marks the stream
// corrupt; that each level's children are exactly the next level is checked by the walk.
constexpr int kScatterIlp = 4;
constexpr uint32_t kScatterNodes = kScanThreads * kScatterIlp;

__device__ __forceinline__ void scatter_body(const ScanParams &sp, uint32_t vb) {
    const uint32_t total = sp.level_off[sp.depth + 1];
    const uint32_t n = (uint32_t)sp.n;  // at most 2^29 internal nodes
    const uint32_t x0 = vb * kScatterNodes + threadIdx.x;
    const uint32_t *B32 = reinterpret_cast<const uint32_t *>(sp.B);
    uint32_t byte[kScatterIlp], y[kScatterIlp];
#pragma unroll
    for (int q = 0; q < kScatterIlp; ++q) {
        const uint32_t x = x0 + q * kScanThreads, k = x >> 2, sh = 8u * (x & 3u);
        byte[q] = 0;
        y[q] = 0;
        if (x < n) {
            // whole words load directly; only the stream's last word is assembled byte by byte
            const uint32_t w = 4 * k + 4 <= n ? __ldg(B32 + k) : word_at(sp.B, n, k);
            byte[q] = (w >> sh) & 0xFFu;
            y[q] = 1u + __ldg(sp.P4 + k) + __popc(w & ((1u << sh) - 1u));
        }
    }
#pragma unroll
    for (int q = 0; q < kScatterIlp; ++q) {
        const uint32_t x = x0 + q * kScanThreads;
        uint32_t b = byte[q], yy = y[q];
        if (yy + __popc(b) > total) {
            set_status(sp.status, SGS_E_CORRUPT);
            continue;
        }
        const uint32_t xe = x << 3;
        while (b) {
            sp.par[yy++] = xe | (uint32_t)(__ffs(b) - 1);
            b &= b - 1;
        }
    }
}

__global__ void __launch_bounds__(kScanThreads) k_octree_scatter(ScanParams p) {
    pdl_trigger();
    pdl_wait();
    scatter_body(p, blockIdx.x);
}

__global__ void __launch_bounds__(kScanThreads) k_octree_scatter_multi(MultiArgs m) {
    run_items<ScanParams>(m, [](const ScanParams &p, uint32_t vb, uint32_t, bool) { scatter_body(p, vb); });
}

// ------------------------------------------------------------------ duplicates

struct DupParams {
    const uint32_t *dup;
    uint32_t n_dup, n_leaves, n_rows;
    uint32_t *dup_prefix;
    int *status;
};

__device__ __forceinline__ void dup_body(const DupParams &p) {
    __shared__ uint32_t sm[8];
    const uint32_t *dup = p.dup;
    const uint32_t n_dup = p.n_dup, n_leaves = p.n_leaves, n_rows = p.n_rows;
    uint32_t *dup_prefix = p.dup_prefix;
    uint32_t carry = 0;
    bool bad = false;
    for (uint32_t base = 0; base < n_dup; base += 256) {
        const uint32_t i = base + threadIdx.x;
        uint32_t e = 0;
        if (i < n_dup) {
            e = dup[2 * i + 1];
            const uint32_t r = dup[2 * i];
            if (r >= n_leaves || e == 0 || e > n_rows || (i > 0 && dup[2 * (i - 1)] >= r)) bad = true;
        }
        uint32_t tot;
        const uint32_t ex = block_excl_scan_256(e, &tot, sm);
        if (i < n_dup) dup_prefix[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) {
        dup_prefix[n_dup] = carry;
        if ((uint64_t)carry + n_leaves != n_rows) bad = true;
    }
    if (bad) set_status(p.status, SGS_E_CORRUPT);
}

__global__ void __launch_bounds__(256) k_dup_prefix(DupParams p) { dup_body(p); }

__global__ void __launch_bounds__(256) k_dup_multi(MultiArgs m) {
    run_items<DupParams>(m, [](const DupParams &p, uint32_t, uint32_t, bool) { dup_body(p); });
}

// ------------------------------------------------------------------ leaf walk

// Level-count check: the popcounts of level l sum to the node count of level l+1, and level
// l's first node has level l+1's first node as its first child.
__device__ __forceinline__ void check_levels(const uint8_t *B, uint64_t n_geo, const uint32_t *P4,
                                             const uint32_t *off, int depth, int *status) {
    const int l = threadIdx.x;
    if (l >= depth) return;
    uint32_t b0, p0, b1, p1;
    node_at(B, n_geo, P4, off[l], b0, p0);
    node_at(B, n_geo, P4, off[l + 1], b1, p1);
    if (1u + p0 != off[l + 1] || p1 - p0 != off[l + 2] - off[l + 1]) set_status(status, SGS_E_CORRUPT);
}

struct WalkParams {
    const uint8_t *B;
    uint64_t n_geo;
    const uint32_t *P4;
    const uint32_t *par;
    uint32_t leaf_lo, n_leaves;  // first leaf's node index, leaf count
    int depth, check;            // CTA 0 of the walk verifies the level counts
    LeafOut leaf;
    uint32_t level_off[SGS_MAX_DEPTH + 2];
    int *status;
};

// Leaves vb * kWalkLeaves + j * kWalkThreads + threadIdx.x, j < kWalkIlp: the D steps of
// the kWalkIlp walks are interleaved so their loads are in flight together.  Step s reads
// the parent entry of the current node: its child index k gives bit s of the coordinates
// (x, y, z) = (bit 2, bit 1, bit 0 of k), its parent index the next node.  Each step must go
// to a smaller index and the walk must end at the root after exactly D steps (D <= 21, so
// bit s stays inside its 21-bit field).
__device__ __forceinline__ void walk_body(const WalkParams &p, uint32_t vb) {
    if (p.check && vb == 0) check_levels(p.B, p.n_geo, p.P4, p.level_off, p.depth, p.status);
    uint32_t y[kWalkIlp], lo[kWalkIlp], hi[kWalkIlp];  // node; Morton code so far (top 3 st bits)
    bool on[kWalkIlp];
    const uint32_t u0 = vb * kWalkLeaves + threadIdx.x;
#pragma unroll
    for (int j = 0; j < kWalkIlp; ++j) {
        const uint32_t u = u0 + j * kWalkThreads;
        on[j] = u < p.n_leaves;
        y[j] = on[j] ? p.leaf_lo + u : 0u;
        lo[j] = hi[j] = 0u;
    }
    bool bad = false;
    for (int st = 0; st < p.depth; ++st) {
        uint32_t e[kWalkIlp];
#pragma unroll
        for (int j = 0; j < kWalkIlp; ++j) e[j] = on[j] ? __ldg(p.par + y[j]) : 0u;
#pragma unroll
        for (int j = 0; j < kWalkIlp; ++j) {
            const uint32_t up = e[j] >> 3;
            const bool ok = up < y[j];
            bad |= on[j] & !ok;
            on[j] &= ok;
            y[j] = up;
            // the 64-bit code shifts right by 3 and takes k = e & 7 into its top bits 61..63
            lo[j] = __funnelshift_r(lo[j], hi[j], 3);
            hi[j] = __funnelshift_r(hi[j], e[j], 3);
        }
    }
    const uint32_t sh = 64u - 3u * (uint32_t)p.depth;
#pragma unroll
    for (int j = 0; j < kWalkIlp; ++j) {
        if (!on[j]) continue;
        if (y[j] != 0) {
            bad = true;
            continue;
        }
        // triple st of the code is the child index taken at step st: (x, y, z) bits st
        const uint64_t code = (((uint64_t)hi[j] << 32) | lo[j]) >> sh;
        write_leaf(p.leaf, u0 + j * kWalkThreads, code, p.status);
    }
    if (bad) set_status(p.status, SGS_E_CORRUPT);
}

__global__ void __launch_bounds__(kWalkThreads) k_octree_walk(WalkParams p) {
    pdl_wait();
    walk_body(p, blockIdx.x);
}

__global__ void __launch_bounds__(kWalkThreads) k_octree_walk_multi(MultiArgs m) {
    run_items<WalkParams>(m, [](const WalkParams &p, uint32_t vb, uint32_t, bool) { walk_body(p, vb); });
}

// ------------------------------------------------------------------ parameters

// The token array the octree kernels read: the stream's raw section, or the scratch copy
// the geometry decoder filled when levels are coded (static or learned).
static const uint8_t *geo_tokens(const uint8_t *bits, const sgs_scene_info &info, const Scratch &s) {
    return (info.geo_mode != SGS_GEO_RAW && info.n_geo) ? s.geo_bytes : bits + info.off[S_GEO_RAW];
}

static LeafOut make_leaf(const uint8_t *bits, const sgs_scene_info &info, const Scratch &s,
                         const sgs_scene_out &out) {
    LeafOut lo;
    memset(&lo, 0, sizeof(lo));
    lo.pos = out.pos;
    lo.coord = out.coord;
    lo.out_index = out.out_index;
    lo.n_rows = info.n_rows;
    lo.n_leaves = info.n_leaves;
    lo.n_dup = info.n_dup;
    lo.depth = info.depth;
    lo.dup = reinterpret_cast<const uint32_t *>(bits + info.off[S_DUP]);
    lo.dup_prefix = s.dup_prefix;
    lo.scale = ldexpf(1.0f, -(int)info.depth);
    lo.half = ldexpf(1.0f, -(int)info.depth - 1);
    return lo;
}

static bool octree_work(const sgs_scene_info &info) { return info.n_rows != 0 && info.n_leaves != 0; }

static uint32_t make_dup(const uint8_t *bits, const sgs_scene_info &info, const Scratch &s, int *status,
                         DupParams *pp) {
    DupParams &p = *pp;
    memset(&p, 0, sizeof(p));
    p.dup = reinterpret_cast<const uint32_t *>(bits + info.off[S_DUP]);
    p.n_dup = info.n_dup;
    p.n_leaves = info.n_leaves;
    p.n_rows = info.n_rows;
    p.dup_prefix = s.dup_prefix;
    p.status = status;
    return (octree_work(info) && info.n_dup) ? 1 : 0;
}

static void level_offsets(const sgs_scene_info &info, const GeoPlan &plan, uint32_t *off) {
    for (int k = 0; k <= plan.depth; ++k) off[k] = (uint32_t)plan.level_off[k];
    off[plan.depth + 1] = (uint32_t)(info.n_geo + info.n_leaves);
}

static uint32_t make_scan(const uint8_t *bits, const sgs_scene_info &info, const GeoPlan &plan,
                          const Scratch &s, int *status, ScanParams *pp) {
    ScanParams &p = *pp;
    memset(&p, 0, sizeof(p));
    p.B = geo_tokens(bits, info, s);
    p.n = info.n_geo;
    p.n_words = (info.n_geo + 3) / 4;
    p.P4 = s.p4;
    p.par = s.par;
    p.tile_sums = s.tile_sums;
    p.status = status;
    p.depth = plan.depth;
    level_offsets(info, plan, p.level_off);
    return octree_work(info) ? (uint32_t)octree_scan_tiles(info.n_geo) : 0;
}

static uint32_t scatter_blocks(const sgs_scene_info &info) {
    return (uint32_t)((info.n_geo + kScatterNodes - 1) / kScatterNodes);
}

static uint32_t make_walk(const uint8_t *bits, const sgs_scene_info &info, const GeoPlan &plan,
                          const Scratch &s, const sgs_scene_out &out, int *status, WalkParams *pp) {
    WalkParams &p = *pp;
    memset(&p, 0, sizeof(p));
    p.B = geo_tokens(bits, info, s);
    p.n_geo = info.n_geo;
    p.P4 = s.p4;
    p.par = s.par;
    p.leaf_lo = (uint32_t)info.n_geo;
    p.n_leaves = info.n_leaves;
    p.depth = plan.depth;
    p.check = 1;
    p.leaf = make_leaf(bits, info, s, out);
    level_offsets(info, plan, p.level_off);
    p.status = status;
    return octree_work(info) ? (info.n_leaves + kWalkLeaves - 1) / kWalkLeaves : 0;
}

// ------------------------------------------------------------------ launcher

// Launches `kernel` after the stream's previous kernel, with programmatic dependent launch when
// `pdl` (the kernel waits for its predecessor's completion itself).  Only beside the static
// attribute decoder, which holds every SM with one CTA: beside the fixed-length unpack the
// early-scheduled CTAs, waiting, take the SM slots the unpack needs (0.087 against 0.077 ms).
template <typename P>
static cudaError_t launch_after(bool pdl, void (*kernel)(P), uint32_t grid, uint32_t block, cudaStream_t st,
                                const P &p) {
    if (!pdl) {
        kernel<<<grid, block, 0, st>>>(p);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, p);
}

cudaError_t launch_octree(const sgs_scene_info &info, const GeoPlan &plan, const uint8_t *bits,
                          const Scratch &s, const sgs_scene_out &out, int *status, cudaStream_t st) {
    if (!octree_work(info)) return cudaSuccess;
    cudaError_t e;
    DupParams dp;
    if (make_dup(bits, info, s, status, &dp)) {
        k_dup_prefix<<<1, 256, 0, st>>>(dp);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    ScanParams sp;
    const uint32_t tiles = make_scan(bits, info, plan, s, status, &sp);
    k_octree_reduce<<<tiles, kScanThreads, 0, st>>>(sp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const bool pdl = info.mode == SGS_MODE_STATIC;
    if ((e = launch_after(pdl, k_octree_scan, tiles, kScanThreads, st, sp)) != cudaSuccess) return e;
    if ((e = launch_after(pdl, k_octree_scatter, scatter_blocks(info), kScanThreads, st, sp)) != cudaSuccess) return e;
    WalkParams wp;
    const uint32_t blocks = make_walk(bits, info, plan, s, out, status, &wp);
    return launch_after(pdl, k_octree_walk, blocks, kWalkThreads, st, wp);
}

// ------------------------------------------------------------------ batched stages

uint32_t stage_dup(const SceneRef &r, void *par) {
    DupParams p;
    const uint32_t n = make_dup(r.bits, *r.info, *r.s, r.status, &p);
    memcpy(par, &p, sizeof(p));
    return n;
}
size_t stage_dup_bytes() { return sizeof(DupParams); }
cudaError_t launch_dup_multi(const MultiArgs &m, cudaStream_t st) {
    return launch_persistent(k_dup_multi, 256, 0, m, st);
}

uint32_t stage_scan(const SceneRef &r, int variant, void *par) {
    ScanParams p;
    const uint32_t n = make_scan(r.bits, *r.info, *r.plan, *r.s, r.status, &p);
    memcpy(par, &p, sizeof(p));
    return (variant == 2 && n) ? scatter_blocks(*r.info) : n;
}
size_t stage_scan_bytes() { return sizeof(ScanParams); }
cudaError_t launch_scan_multi(int variant, const MultiArgs &m, cudaStream_t st) {
    if (variant == 1) return launch_persistent(k_octree_reduce_multi, kScanThreads, 0, m, st);
    if (variant == 2) return launch_persistent(k_octree_scatter_multi, kScanThreads, 0, m, st);
    return launch_persistent(k_octree_scan_multi, kScanThreads, 0, m, st);
}

uint32_t stage_walk(const SceneRef &r, void *par) {
    WalkParams p;
    const uint32_t n = make_walk(r.bits, *r.info, *r.plan, *r.s, *r.out, r.status, &p);
    memcpy(par, &p, sizeof(p));
    return n;
}
size_t stage_walk_bytes() { return sizeof(WalkParams); }
cudaError_t launch_walk_multi(const MultiArgs &m, cudaStream_t st) {
    return launch_persistent(k_octree_walk_multi, kWalkThreads, 0, m, st);
}

// Kernels launch_octree enqueues for a non-empty scene.
int octree_launches(const sgs_scene_info &info, const GeoPlan &) { return (info.n_dup ? 1 : 0) + 4; }

// Scan tiles: every 64-byte chunk up to the one holding word n_words (whose P4 entry is the
// total), 256 chunks per tile.
size_t octree_scan_tiles(uint64_t n_geo) { return (((n_geo + 3) / 4) / 16 + 1 + 255) / 256; }
size_t octree_words(uint64_t n_geo) { return (n_geo + 3) / 4; }

}  // namespace sgs
