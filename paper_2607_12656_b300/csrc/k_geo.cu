// Sparse-octree expansion on sm_103a (Sec. 3.4, "Geometry Occupancy Coding": occupancy
// tokens, one per internal node, level by level; one position per voxel plus duplicate
// counts as metadata).
//
// The tokens of all levels form one breadth-first array B.  With P(x) = sum of popc(B[h])
// for h < x, the children of node x are the nodes 1 + P(x) + j (j < popc(B[x])), leaves
// numbered after the internal nodes.  One device-wide scan (decoupled look-back) writes P at
// every 4-byte word of B, so any node's children follow from two loads: P4[x / 4] plus the
// popcount of the bytes of its word below x.  Expansion is then a map with no block-wide
// synchronisation: a thread takes one node and walks its subtree depth first through up to
// kMaxFuse chain-like levels (a small stack of child iterators in shared memory), writing the
// packed coordinates (x:21 | y:21 | z:21) of the nodes at the end of its levels or, at the
// last level, the voxel-centre positions of the leaf rows.  The few small top levels are
// expanded by one CTA, concurrently with the scan.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "sgs_device.cuh"
#include "sgs_internal.h"

namespace sgs {

constexpr int kScanThreads = 256;
constexpr uint32_t kSpinLimit = 1u << 22;          // bounded look-back wait
constexpr int kTopThreads = 1024;
constexpr uint32_t kTopCap = 2048;                 // levels the top kernel keeps in smem
constexpr int kExpThreads = 128;
constexpr int kMaxFuse = 8;                        // levels one expansion thread walks
constexpr uint64_t kM21 = (1ull << 21) - 1;

struct LeafOut {
    float *pos;
    uint32_t *coord;
    const uint32_t *out_index;
    uint32_t n_rows, n_leaves, n_dup, depth;
    const uint32_t *dup;        // {rank, extra} pairs
    const uint32_t *dup_prefix; // exclusive prefix of extra
    float scale, half;          // 2^-D, 2^-(D+1)
};

__device__ __forceinline__ uint64_t child_code(uint64_t pc, uint32_t k) {
    return (pc << 1) | ((uint64_t)((k >> 2) & 1u) << 42) | ((uint64_t)((k >> 1) & 1u) << 21) |
           (uint64_t)(k & 1u);
}

// Writes the rows of leaf u (Morton rank) with packed coordinates pc.
__device__ __forceinline__ void write_leaf(const LeafOut &o, uint32_t u, uint64_t pc, int *status) {
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
    const uint32_t x = (uint32_t)(pc >> 42), y = (uint32_t)((pc >> 21) & kM21),
                   z = (uint32_t)(pc & kM21);
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

// P4[k] = popcount of B[0, 4k) for k = 0 .. ceil(n/4).  Tile = 256 threads x 64 bytes.
// Tiles must start in increasing order: a tile's look-back waits only on tiles that started
// before it (the single-scene kernel draws tiles from a ticket, the batched one claims items
// in order).
struct ScanParams {
    const uint8_t *B;
    uint64_t n, n_words;
    uint32_t *P4;
    uint64_t *flags;
    uint32_t *ticket;
    int *status;
};

__device__ __forceinline__ void scan_body(const ScanParams &sp, uint32_t tile) {
    __shared__ uint32_t sm[8];
    __shared__ uint32_t s_prefix;
    const uint8_t *B = sp.B;
    const uint64_t n = sp.n, n_words = sp.n_words;
    uint32_t *P4 = sp.P4;
    uint64_t *flags = sp.flags;
    int *status = sp.status;
    const uint64_t k = (uint64_t)tile * kScanThreads + threadIdx.x;  // 64-byte chunk
    const uint64_t w0 = 16 * k;                                      // its first word
    uint32_t cnt[16];
    uint32_t sum = 0;
    if (64 * k + 64 <= n) {
        const uint4 *p = reinterpret_cast<const uint4 *>(B + 64 * k);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint4 v = p[i];
            cnt[4 * i] = __popc(v.x);
            cnt[4 * i + 1] = __popc(v.y);
            cnt[4 * i + 2] = __popc(v.z);
            cnt[4 * i + 3] = __popc(v.w);
        }
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) cnt[i] = (w0 + i) * 4 < n ? __popc(word_at(B, n, w0 + i)) : 0u;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) sum += cnt[i];
    uint32_t agg;
    const uint32_t local = block_excl_scan_256(sum, &agg, sm);
    // decoupled look-back, 32 predecessors per step (flag 1 = aggregate, 2 = inclusive prefix)
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        volatile unsigned long long *vf = reinterpret_cast<volatile unsigned long long *>(flags);
        if (lane == 0) {
            vf[tile] = ((tile == 0 ? 2ull : 1ull) << 32) | agg;
            __threadfence();
        }
        uint32_t prefix = 0;
        int64_t hi = (int64_t)tile - 1;  // newest predecessor not yet summed
        uint32_t spins = 0;
        while (hi >= 0) {
            const int64_t idx = hi - lane;
            unsigned long long v = idx >= 0 ? vf[idx] : (2ull << 32);
            while (__any_sync(0xffffffffu, (v >> 32) == 0)) {
                if (++spins > kSpinLimit) break;
                __nanosleep(32);
                if ((v >> 32) == 0) v = vf[idx];
            }
            if (spins > kSpinLimit) {
                if (lane == 0) set_status(status, SGS_E_TIMEOUT);
                break;
            }
            const uint32_t incl = __ballot_sync(0xffffffffu, (v >> 32) == 2);
            const int stop = incl ? __ffs(incl) - 1 : 31;  // lanes 0..stop contribute
            uint32_t val = (lane <= stop) ? (uint32_t)v : 0u;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
            prefix += val;
            if (incl) break;
            hi -= 32;
        }
        if (lane == 0) {
            if (tile != 0) {
                __threadfence();
                vf[tile] = (2ull << 32) | (uint64_t)(prefix + agg);
            }
            s_prefix = prefix;
        }
    }
    __syncthreads();
    uint32_t run = s_prefix + local;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        if (w0 + i <= n_words) P4[w0 + i] = run;  // P4[n_words] = total
        run += cnt[i];
    }
}

__global__ void __launch_bounds__(kScanThreads) k_octree_scan(ScanParams p) {
    __shared__ uint32_t s_tile;
    if (threadIdx.x == 0) s_tile = atomicAdd(p.ticket, 1u);
    __syncthreads();
    scan_body(p, s_tile);
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

// ------------------------------------------------------------------ top levels (one CTA)

struct TopParams {
    const uint8_t *B;
    GeoPlan plan;
    int l1;               // first level not held in shared memory (or D)
    uint64_t *codes_out;  // codes of level l1 (if l1 < D)
    LeafOut leaf;
    int *status;
};

constexpr uint32_t kTopStage = 8192;  // top-level tokens staged in shared memory

__device__ __forceinline__ void top_body(const TopParams &p) {
    __shared__ uint64_t codes[2][kTopCap];
    __shared__ uint8_t stage[kTopStage];
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) codes[0][0] = 0;
    // all top-level tokens in one coalesced pass (they are contiguous from BFS index 0)
    const uint64_t n_top = p.plan.level_off[p.l1];
    const bool staged = n_top <= kTopStage;
    if (staged)
        for (uint32_t i = threadIdx.x; i < n_top; i += kTopThreads) stage[i] = p.B[i];
    __syncthreads();
    int cur = 0;
    for (int l = 0; l < p.l1; ++l) {
        const uint32_t n = p.plan.n_level[l];
        const uint32_t n_next = p.plan.n_level[l + 1];
        const bool to_leaves = (l + 1 == p.plan.depth);
        const bool to_global = (l + 1 == p.l1) && !to_leaves;
        const uint8_t *Bl = (staged ? stage : p.B) + p.plan.level_off[l];
        if (threadIdx.x == 0) s_carry = 0;
        __syncthreads();
        for (uint32_t base = 0; base < n; base += kTopThreads) {
            const uint32_t i = base + threadIdx.x;
            const uint32_t byte = i < n ? Bl[i] : 0u;
            const uint32_t cnt = __popc(byte);
            uint32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (lane == 31) wsum[warp] = incl;
            __syncthreads();
            if (warp == 0) {
                uint32_t v = wsum[lane], iv = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t t = __shfl_up_sync(0xffffffffu, iv, o);
                    if (lane >= o) iv += t;
                }
                wsum[lane] = iv - v;  // exclusive warp offsets
            }
            __syncthreads();
            uint32_t idx = s_carry + wsum[warp] + incl - cnt;
            if (i < n) {
                const uint64_t pc = codes[cur][i];
                uint32_t b = byte;
                while (b) {
                    const uint32_t k = __ffs(b) - 1;
                    b &= b - 1;
                    const uint64_t cc = child_code(pc, k);
                    if (idx >= n_next) { set_status(p.status, SGS_E_CORRUPT); break; }
                    if (to_leaves) write_leaf(p.leaf, idx, cc, p.status);
                    else if (to_global) p.codes_out[idx] = cc;
                    else codes[cur ^ 1][idx] = cc;
                    ++idx;
                }
            }
            __syncthreads();
            if (threadIdx.x == kTopThreads - 1) s_carry += wsum[31] + incl;
            __syncthreads();
        }
        if (threadIdx.x == 0 && s_carry != n_next) set_status(p.status, SGS_E_CORRUPT);
        cur ^= 1;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kTopThreads) k_octree_top(TopParams p) { top_body(p); }

__global__ void __launch_bounds__(kTopThreads) k_octree_top_multi(MultiArgs m) {
    run_items<TopParams>(m, [](const TopParams &p, uint32_t, uint32_t, bool) { top_body(p); });
}

// ------------------------------------------------------------------ fused levels

// Thread per node x of level ls: depth-first through levels ls .. le-1, emitting the nodes of
// level le (codes) or, when le = D, the leaf rows.  The stack holds one child iterator per
// level (P of the node, remaining child mask, children taken, packed coordinates).
struct ExpandParams {
    const uint8_t *B;
    uint64_t n_geo;
    const uint32_t *P4;
    int ls, le, depth;
    uint64_t level_off[SGS_MAX_DEPTH + 2];  // BFS offset of each level, [D+1] = end of leaves
    const uint64_t *codes_in;               // level ls, indexed by x - level_off[ls]
    uint64_t *codes_out;                    // level le (NULL when le = D)
    LeafOut leaf;
    int check;                              // CTA 0 verifies the level counts
    int *status;
};

__device__ __forceinline__ void expand_body(const ExpandParams &p, uint32_t vb) {
    __shared__ uint32_t s_p[kMaxFuse][kExpThreads];
    __shared__ uint32_t s_it[kMaxFuse][kExpThreads];  // remaining mask | taken << 8
    __shared__ uint64_t s_code[kMaxFuse][kExpThreads];
    __shared__ uint32_t s_off[SGS_MAX_DEPTH + 2];      // level offsets (node indices < 2^32)
    const int tid = threadIdx.x;
    if (tid <= p.depth + 1) s_off[tid] = (uint32_t)p.level_off[tid];
    __syncthreads();
    if (p.check && vb == 0 && tid < p.depth) {
        // sum of the popcounts of level l = nodes of level l+1, and the first child of the
        // level's first node is the next level's first node
        const int l = tid;
        uint32_t b0, p0, b1, p1;
        node_at(p.B, p.n_geo, p.P4, s_off[l], b0, p0);
        node_at(p.B, p.n_geo, p.P4, s_off[l + 1], b1, p1);
        if (1u + p0 != s_off[l + 1] || p1 - p0 != s_off[l + 2] - s_off[l + 1])
            set_status(p.status, SGS_E_CORRUPT);
    }
    const uint32_t lo = s_off[p.ls];
    const uint32_t x = lo + vb * kExpThreads + tid;
    if (x >= s_off[p.ls + 1]) return;
    uint32_t byte, px;
    node_at(p.B, p.n_geo, p.P4, x, byte, px);
    uint64_t code = p.codes_in[x - lo];
    const uint32_t leaf_base = s_off[p.depth];
    int lvl = p.ls;  // level of the current node
    // chains: follow single children without the stack
    while (lvl + 1 < p.le && __popc(byte) == 1) {
        const uint32_t child = 1u + px;
        ++lvl;
        if (child < s_off[lvl] || child >= s_off[lvl + 1]) {
            set_status(p.status, SGS_E_CORRUPT);
            return;
        }
        code = child_code(code, __ffs(byte) - 1);
        node_at(p.B, p.n_geo, p.P4, child, byte, px);
    }
    // depth first through the remaining levels lvl .. le-1
    s_p[0][tid] = px;
    s_it[0][tid] = byte;
    s_code[0][tid] = code;
    const int K = p.le - lvl;
    int d = 0;
    while (d >= 0) {
        const uint32_t it = s_it[d][tid];
        const uint32_t mask = it & 0xFFu;
        if (!mask) { --d; continue; }
        const uint32_t k = __ffs(mask) - 1;
        const uint32_t taken = it >> 8;
        s_it[d][tid] = (mask & (mask - 1)) | ((taken + 1) << 8);
        const uint32_t child = 1u + s_p[d][tid] + taken;
        const int lc = lvl + d + 1;  // level of the child
        if (child < s_off[lc] || child >= s_off[lc + 1]) {
            set_status(p.status, SGS_E_CORRUPT);
            return;
        }
        const uint64_t cc = child_code(s_code[d][tid], k);
        if (d + 1 == K) {
            if (lc == p.depth) write_leaf(p.leaf, child - leaf_base, cc, p.status);
            else p.codes_out[child - s_off[lc]] = cc;
        } else {
            uint32_t cb, cp;
            node_at(p.B, p.n_geo, p.P4, child, cb, cp);
            ++d;
            s_p[d][tid] = cp;
            s_it[d][tid] = cb;
            s_code[d][tid] = cc;
        }
    }
}

__global__ void __launch_bounds__(kExpThreads) k_octree_expand(ExpandParams p) { expand_body(p, blockIdx.x); }

__global__ void __launch_bounds__(kExpThreads) k_octree_expand_multi(MultiArgs m) {
    run_items<ExpandParams>(m, [](const ExpandParams &p, uint32_t vb, uint32_t, bool) { expand_body(p, vb); });
}

int octree_top_level(const GeoPlan &plan) {
    int l1 = 1;
    while (l1 < plan.depth && plan.n_level[l1] <= kTopCap) ++l1;
    return l1;
}

// Level groups [ls, le) of the fused expansion.  A thread's levels run one after another, so
// only chain-like levels are fused: extend while the frontier grows by at most 1/10 over the
// group (branching subtrees would leave a warp waiting for its widest lane), and the group
// holds at most kMaxFuse levels.
int octree_groups(const GeoPlan &plan, int *starts) {
    const int D = plan.depth;
    int n = 0;
    int ls = octree_top_level(plan);
    while (ls < D) {
        int le = ls + 1;
        while (le < D && le - ls < kMaxFuse && (uint64_t)plan.n_level[le] * 10 <= 11ull * plan.n_level[ls]) ++le;
        starts[n++] = ls;
        ls = le;
    }
    starts[n] = D;
    return n;
}

// ------------------------------------------------------------------ parameters

// The token array the octree kernels read: the stream's raw section, or the scratch copy
// the geometry decoder filled when levels are rANS-coded.
static const uint8_t *geo_tokens(const uint8_t *bits, const sgs_scene_info &info, const Scratch &s) {
    return (info.geo_mode == SGS_GEO_RANS && info.n_geo) ? s.geo_bytes : bits + info.off[S_GEO_RAW];
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

static uint32_t make_scan(const uint8_t *bits, const sgs_scene_info &info, const Scratch &s, int *status,
                          ScanParams *pp) {
    ScanParams &p = *pp;
    memset(&p, 0, sizeof(p));
    p.B = geo_tokens(bits, info, s);
    p.n = info.n_geo;
    p.n_words = (info.n_geo + 3) / 4;
    p.P4 = s.p4;
    p.flags = s.scan_flags;
    p.ticket = s.ticket;
    p.status = status;
    return octree_work(info) ? (uint32_t)octree_scan_tiles(info.n_geo) : 0;
}

static uint32_t make_top(const uint8_t *bits, const sgs_scene_info &info, const GeoPlan &plan,
                         const Scratch &s, const sgs_scene_out &out, int *status, TopParams *pp) {
    TopParams &p = *pp;
    memset(&p, 0, sizeof(p));
    const int l1 = octree_top_level(plan);
    p.B = geo_tokens(bits, info, s);
    p.plan = plan;
    p.l1 = l1;
    p.codes_out = (l1 < plan.depth) ? s.codes[0] : nullptr;
    p.leaf = make_leaf(bits, info, s, out);
    p.status = status;
    return octree_work(info) ? 1 : 0;
}

// Expansion group gi (levels starts[gi] .. starts[gi+1]).
static uint32_t make_expand(const uint8_t *bits, const sgs_scene_info &info, const GeoPlan &plan,
                            const Scratch &s, const sgs_scene_out &out, int *status, int gi,
                            ExpandParams *pp) {
    ExpandParams &ep = *pp;
    memset(&ep, 0, sizeof(ep));
    int starts[SGS_MAX_DEPTH + 2];
    const int n_groups = octree_groups(plan, starts);
    if (!octree_work(info) || gi >= n_groups) return 0;
    const int D = plan.depth;
    ep.B = geo_tokens(bits, info, s);
    ep.n_geo = info.n_geo;
    ep.P4 = s.p4;
    ep.depth = D;
    for (int l = 0; l <= D; ++l) ep.level_off[l] = plan.level_off[l];
    ep.level_off[D + 1] = plan.level_off[D] + plan.n_level[D];
    ep.leaf = make_leaf(bits, info, s, out);
    ep.status = status;
    ep.ls = starts[gi];
    ep.le = starts[gi + 1];
    ep.codes_in = s.codes[gi & 1];
    ep.codes_out = ep.le < D ? s.codes[(gi + 1) & 1] : nullptr;
    ep.check = gi == 0;
    return (uint32_t)((plan.n_level[ep.ls] + kExpThreads - 1) / kExpThreads);
}

// ------------------------------------------------------------------ launcher

cudaError_t launch_octree(const sgs_scene_info &info, const GeoPlan &plan,
                          const uint8_t *bits, const Scratch &s, const sgs_scene_out &out,
                          int *status, cudaStream_t st, cudaStream_t st2, cudaEvent_t ev_a,
                          cudaEvent_t ev_b) {
    if (!octree_work(info)) return cudaSuccess;
    cudaError_t e;
    DupParams dp;
    if (make_dup(bits, info, s, status, &dp)) {
        k_dup_prefix<<<1, 256, 0, st>>>(dp);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // the top levels need no prefix: they run on st2 while the scan runs on st
    if (st2 != st) {
        if (cudaEventRecord(ev_a, st) != cudaSuccess || cudaStreamWaitEvent(st2, ev_a, 0) != cudaSuccess)
            return cudaErrorUnknown;
    }
    TopParams tp;
    make_top(bits, info, plan, s, out, status, &tp);
    k_octree_top<<<1, kTopThreads, 0, st2>>>(tp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (st2 != st && cudaEventRecord(ev_b, st2) != cudaSuccess) return cudaErrorUnknown;
    ScanParams sp;
    const uint32_t tiles = make_scan(bits, info, s, status, &sp);
    k_octree_scan<<<tiles, kScanThreads, 0, st>>>(sp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (st2 != st && cudaStreamWaitEvent(st, ev_b, 0) != cudaSuccess) return cudaErrorUnknown;
    ExpandParams ep;
    for (int gi = 0;; ++gi) {
        const uint32_t grid = make_expand(bits, info, plan, s, out, status, gi, &ep);
        if (grid == 0) break;
        k_octree_expand<<<grid, kExpThreads, 0, st>>>(ep);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
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

uint32_t stage_scan(const SceneRef &r, void *par) {
    ScanParams p;
    const uint32_t n = make_scan(r.bits, *r.info, *r.s, r.status, &p);
    memcpy(par, &p, sizeof(p));
    return n;
}
size_t stage_scan_bytes() { return sizeof(ScanParams); }
cudaError_t launch_scan_multi(const MultiArgs &m, cudaStream_t st) {
    return launch_persistent(k_octree_scan_multi, kScanThreads, 0, m, st);
}

uint32_t stage_top(const SceneRef &r, void *par) {
    TopParams p;
    const uint32_t n = make_top(r.bits, *r.info, *r.plan, *r.s, *r.out, r.status, &p);
    memcpy(par, &p, sizeof(p));
    return n;
}
size_t stage_top_bytes() { return sizeof(TopParams); }
cudaError_t launch_top_multi(const MultiArgs &m, cudaStream_t st) {
    return launch_persistent(k_octree_top_multi, kTopThreads, 0, m, st);
}

uint32_t stage_expand(const SceneRef &r, int group, void *par) {
    ExpandParams p;
    const uint32_t n = make_expand(r.bits, *r.info, *r.plan, *r.s, *r.out, r.status, group, &p);
    memcpy(par, &p, sizeof(p));
    return n;
}
size_t stage_expand_bytes() { return sizeof(ExpandParams); }
cudaError_t launch_expand_multi(const MultiArgs &m, cudaStream_t st) {
    return launch_persistent(k_octree_expand_multi, kExpThreads, 0, m, st);
}

int octree_group_count(const sgs_scene_info &info, const GeoPlan &plan) {
    int starts[SGS_MAX_DEPTH + 2];
    return octree_work(info) ? octree_groups(plan, starts) : 0;
}

// Scratch of the octree stage: bytes of each ping-pong code buffer (the widest level that
// starts a fused group, or level l1 written by the top kernel).
void octree_code_buffers(const sgs_scene_info &info, const GeoPlan &plan, uint64_t *pingpong) {
    int starts[SGS_MAX_DEPTH + 2];
    const int n = octree_groups(plan, starts);
    uint64_t m = 1;
    for (int i = 0; i < n; ++i) m = m > plan.n_level[starts[i]] ? m : plan.n_level[starts[i]];
    if (info.n_rows == 0) m = 1;
    *pingpong = 8 * m;
}

// Kernels launch_octree enqueues for a non-empty scene.
int octree_launches(const sgs_scene_info &info, const GeoPlan &plan) {
    int starts[SGS_MAX_DEPTH + 2];
    return (info.n_dup ? 1 : 0) + 2 + octree_groups(plan, starts);
}

// Scan tiles: every 64-byte chunk up to the one holding word n_words (whose P4 entry is the
// total), 256 chunks per tile.
size_t octree_scan_tiles(uint64_t n_geo) { return (((n_geo + 3) / 4) / 16 + 1 + 255) / 256; }
size_t octree_words(uint64_t n_geo) { return (n_geo + 3) / 4; }

}  // namespace sgs
