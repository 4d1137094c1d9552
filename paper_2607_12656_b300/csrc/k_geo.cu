// Sparse-octree expansion on sm_103a (Sec. 3.4, "Geometry Occupancy Coding": occupancy
// tokens, one per internal node, level by level; one position per voxel plus duplicate
// counts as metadata).
//
// The tokens of all levels form one breadth-first array B.  With P(g) = sum of popc(B[h])
// for h < g, the children of node g are the nodes 1 + P(g) + j (j < popc(B[g])), leaves
// numbered after the internal nodes.  So one device-wide scan of popcounts (decoupled
// look-back, one pass over B) fixes every parent -> child index; expansion is then a map per
// level: each node writes its children's packed coordinates (x:21 | y:21 | z:21 bits).
// The few small top levels are expanded by one CTA in shared memory; each deeper level is
// one launch over tiles of 2048 nodes.  Leaves write the fp32 voxel-centre positions of
// their rows (a leaf with duplicates owns several consecutive rows).
#include <cuda_runtime.h>
#include <stdint.h>

#include "sgs_device.cuh"
#include "sgs_internal.h"

namespace sgs {

constexpr int kScanThreads = 256;
constexpr int kChunk = 64;                         // bytes per scan chunk
constexpr int kScanTile = kScanThreads * kChunk;   // 16 KiB of tokens per tile
constexpr uint32_t kSpinLimit = 1u << 22;          // bounded look-back wait
constexpr int kTopThreads = 1024;
constexpr uint32_t kTopCap = 2048;                 // levels the top kernel keeps in smem
constexpr int kLvlThreads = 256;
constexpr int kLvlPer = 8;                         // nodes per thread
constexpr int kLvlTile = kLvlThreads * kLvlPer;
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

__device__ __forceinline__ uint32_t popc_bytes(const uint8_t *B, uint64_t a, uint64_t b) {
    uint32_t s = 0;
    for (uint64_t i = a; i < b; ++i) s += __popc((uint32_t)B[i]);
    return s;
}

__global__ void __launch_bounds__(kScanThreads) k_octree_scan(const uint8_t *B, uint64_t n,
                                                              uint32_t *chunk_prefix,
                                                              uint64_t n_chunks, uint64_t *flags,
                                                              uint32_t *ticket, int *status) {
    __shared__ uint32_t sm[8];
    __shared__ uint32_t s_tile, s_prefix;
    if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint64_t k = (uint64_t)tile * kScanThreads + threadIdx.x;
    const uint64_t a = k * kChunk;
    uint32_t sum = 0;
    if (a + kChunk <= n) {
        const uint4 *p = reinterpret_cast<const uint4 *>(B + a);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint4 v = p[i];
            sum += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
        }
    } else if (a < n) {
        sum = popc_bytes(B, a, n);
    }
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
    if (k < n_chunks) chunk_prefix[k] = s_prefix + local;
    if (k + 1 == n_chunks) chunk_prefix[n_chunks] = s_prefix + local + sum;
}

// P(g): popcount of B[0, g).
__device__ __forceinline__ uint32_t prefix_at(const uint8_t *B, const uint32_t *chunk_prefix,
                                              uint64_t g) {
    const uint64_t c = g / kChunk;
    return chunk_prefix[c] + popc_bytes(B, c * kChunk, g);
}

// Warp-cooperative P(g) (all 32 lanes call; result in every lane).
__device__ __forceinline__ uint32_t prefix_at_warp(const uint8_t *B, const uint32_t *chunk_prefix,
                                                   uint64_t g) {
    const int lane = threadIdx.x & 31;
    const uint64_t c = g / kChunk, base = c * kChunk;
    uint32_t s = 0;
    for (uint64_t i = base + lane; i < g; i += 32) s += __popc((uint32_t)B[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return chunk_prefix[c] + s;
}

// ------------------------------------------------------------------ duplicates

__global__ void __launch_bounds__(256) k_dup_prefix(const uint32_t *dup, uint32_t n_dup,
                                                    uint32_t n_leaves, uint32_t n_rows,
                                                    uint32_t *dup_prefix, int *status) {
    __shared__ uint32_t sm[8];
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
    if (bad) set_status(status, SGS_E_CORRUPT);
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

__global__ void __launch_bounds__(kTopThreads) k_octree_top(TopParams p) {
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

// ------------------------------------------------------------------ deep levels

// Expands one chunk of up to kLvlTile consecutive nodes [x0, x1) of level l.  Thread tid
// handles nodes x0 + 256 q + tid (q < 8, coalesced); all 8 rounds are loaded first, then one
// two-level block scan (warp scans per round, warp totals through shared memory) orders the
// children.  p_x0 = P(x0).  Children go to codes_out[global child index - out_base], or to the
// leaves.  Returns the number of children (block-uniform).  sm: 64 words of shared memory.
__device__ __forceinline__ uint32_t expand_chunk(const uint8_t *B, uint64_t x0, uint64_t x1,
                                                 uint32_t p_x0, const uint64_t *codes_in,
                                                 uint64_t in_base, uint64_t *codes_out,
                                                 uint64_t out_base, uint64_t out_hi,
                                                 const LeafOut *leaf, uint64_t leaf_base,
                                                 uint32_t *sm, int *status) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int Q = kLvlTile / kLvlThreads;
    constexpr int NW = kLvlThreads / 32;
    uint32_t byte[Q];
    uint64_t pc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const uint64_t x = x0 + (uint64_t)q * kLvlThreads + threadIdx.x;
        byte[q] = x < x1 ? B[x] : 0u;
        pc[q] = x < x1 ? codes_in[x - in_base] : 0ull;
    }
    uint32_t ex[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const uint32_t v = __popc(byte[q]);
        uint32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t n = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += n;
        }
        ex[q] = incl - v;
        if (lane == 31) sm[q * NW + warp] = incl;
    }
    __syncthreads();
    uint32_t total = 0;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        uint32_t before = 0, round = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            const uint32_t t = sm[q * NW + w];
            before += w < warp ? t : 0u;
            round += t;
        }
        ex[q] += total + before;
        total += round;
    }
    __syncthreads();  // sm is reused by the next chunk
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        uint64_t child = 1ull + p_x0 + ex[q];  // global BFS index of the first child
        uint32_t b = byte[q];
        while (b) {
            const uint32_t k = __ffs(b) - 1;
            b &= b - 1;
            if (child >= out_hi) { set_status(status, SGS_E_CORRUPT); break; }
            const uint64_t cc = child_code(pc[q], k);
            if (leaf) write_leaf(*leaf, (uint32_t)(child - leaf_base), cc, status);
            else codes_out[child - out_base] = cc;
            ++child;
        }
    }
    return total;
}

struct LevelParams {
    const uint8_t *B;
    const uint32_t *chunk_prefix;
    uint64_t lo, n;          // level's BFS offset and node count
    uint64_t next_lo, n_next;
    const uint64_t *codes_in;   // indexed by x - in_base
    uint64_t in_base;
    uint64_t *codes_out;        // indexed by child - out_base; NULL when the next level is the leaves
    uint64_t out_base;
    LeafOut leaf;
    int *status;
};

__global__ void __launch_bounds__(kLvlThreads) k_octree_level(LevelParams p) {
    __shared__ uint32_t sm[64];
    __shared__ uint32_t s_p;
    const uint64_t x0 = p.lo + (uint64_t)blockIdx.x * kLvlTile;
    const uint64_t x1 = x0 + kLvlTile < p.lo + p.n ? x0 + kLvlTile : p.lo + p.n;
    if (threadIdx.x < 32) {
        const uint32_t pg = prefix_at_warp(p.B, p.chunk_prefix, x0);
        if (threadIdx.x == 0) s_p = pg;
        if (blockIdx.x == 0) {  // sum of popcounts of the level = nodes of the next level
            const uint32_t p_lo = prefix_at_warp(p.B, p.chunk_prefix, p.lo);
            const uint32_t p_hi = prefix_at_warp(p.B, p.chunk_prefix, p.lo + p.n);
            if (threadIdx.x == 0 && (p_hi - p_lo != p.n_next || 1ull + p_lo != p.next_lo))
                set_status(p.status, SGS_E_CORRUPT);
        }
    }
    __syncthreads();
    expand_chunk(p.B, x0, x1, s_p, p.codes_in, p.in_base, p.codes_out, p.out_base,
                 p.next_lo + p.n_next, p.codes_out ? nullptr : &p.leaf, p.next_lo, sm, p.status);
}

// Subtree walk: CTA t owns nodes [lo + t*kLvlTile, ...) of level lc and expands all their
// descendants down to the leaves.  Below lc the tree is nearly a set of chains, so the
// descendants of a tile stay about one tile wide per level; ranges are contiguous in
// breadth-first order, the child range of [a, b) being [1 + P(a), 1 + P(b)).
struct SubtreeParams {
    const uint8_t *B;
    const uint32_t *chunk_prefix;
    int lc, depth;
    uint64_t level_off[SGS_MAX_DEPTH + 2];
    uint64_t *codes_all;  // levels lc..D-1, indexed by BFS index - level_off[lc]
    LeafOut leaf;
    int *status;
};

__global__ void __launch_bounds__(kLvlThreads) k_octree_subtree(SubtreeParams p) {
    __shared__ uint32_t sm[64];
    __shared__ uint32_t s_p;
    const uint64_t base = p.level_off[p.lc];
    uint64_t a = base + (uint64_t)blockIdx.x * kLvlTile;
    uint64_t b = a + kLvlTile < p.level_off[p.lc + 1] ? a + kLvlTile : p.level_off[p.lc + 1];
    const bool last = (b == p.level_off[p.lc + 1]);
    const uint64_t leaf_base = p.level_off[p.depth];
    for (int l = p.lc; l < p.depth; ++l) {
        if (threadIdx.x < 32) {
            const uint32_t pa = prefix_at_warp(p.B, p.chunk_prefix, a);
            if (threadIdx.x == 0) s_p = pa;
        }
        __syncthreads();
        const uint32_t pa = s_p;
        const bool to_leaves = (l + 1 == p.depth);
        uint32_t total = 0;
        for (uint64_t c0 = a; c0 < b; c0 += kLvlTile) {
            const uint64_t c1 = c0 + kLvlTile < b ? c0 + kLvlTile : b;
            total += expand_chunk(p.B, c0, c1, pa + total, p.codes_all, base, p.codes_all, base,
                                  p.level_off[l + 2], to_leaves ? &p.leaf : nullptr, leaf_base, sm,
                                  p.status);
        }
        const uint64_t na = 1ull + pa, nb = na + total;
        if (threadIdx.x == 0 && (na < p.level_off[l + 1] || nb > p.level_off[l + 2] ||
                                 (last && nb != p.level_off[l + 2]) ||
                                 (blockIdx.x == 0 && na != p.level_off[l + 1])))
            set_status(p.status, SGS_E_CORRUPT);
        a = na < p.level_off[l + 1] ? p.level_off[l + 1] : na;
        b = nb > p.level_off[l + 2] ? p.level_off[l + 2] : nb;
        if (a > b) a = b;
        __syncthreads();
    }
}

// First level of the subtree walk: the shallowest level >= l1 below which every level grows
// by at most 5/4 (chain-like); D if there is none.
int octree_subtree_level(const GeoPlan &plan, int l1) {
    const int D = plan.depth;
    int lc = D;
    for (int l = D - 1; l >= l1; --l) {
        if ((uint64_t)plan.n_level[l + 1] * 4 > (uint64_t)plan.n_level[l] * 5) break;
        lc = l;
    }
    return lc;
}

int octree_top_level(const GeoPlan &plan) {
    int l1 = 1;
    while (l1 < plan.depth && plan.n_level[l1] <= kTopCap) ++l1;
    return l1;
}

// ------------------------------------------------------------------ launcher

cudaError_t launch_octree(const uint8_t *B, const sgs_scene_info &info, const GeoPlan &plan,
                          const uint8_t *bits, const Scratch &s, const sgs_scene_out &out,
                          int *status, cudaStream_t st, cudaStream_t st2, cudaEvent_t ev_a,
                          cudaEvent_t ev_b) {
    if (info.n_rows == 0 || info.n_leaves == 0) return cudaSuccess;
    const int D = plan.depth;
    LeafOut lo;
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
    cudaError_t e;
    if (info.n_dup) {
        k_dup_prefix<<<1, 256, 0, st>>>(lo.dup, info.n_dup, info.n_leaves, info.n_rows,
                                        s.dup_prefix, status);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const uint64_t n_chunks = (info.n_geo + kChunk - 1) / kChunk;
    const uint64_t n_tiles = (info.n_geo + kScanTile - 1) / kScanTile;
    const int l1 = octree_top_level(plan);
    const int lc = octree_subtree_level(plan, l1);
    uint64_t *codes_all = s.codes[2];
    auto dst = [&](int l) -> uint64_t * { return l >= lc ? codes_all : s.codes[l & 1]; };
    auto dst_base = [&](int l) -> uint64_t { return l >= lc ? plan.level_off[lc] : plan.level_off[l]; };
    // the top levels need no prefix: they run on st2 while the scan runs on st
    if (st2 != st) {
        if (cudaEventRecord(ev_a, st) != cudaSuccess || cudaStreamWaitEvent(st2, ev_a, 0) != cudaSuccess)
            return cudaErrorUnknown;
    }
    TopParams tp;
    tp.B = B;
    tp.plan = plan;
    tp.l1 = l1;
    tp.codes_out = (l1 < D) ? dst(l1) + (plan.level_off[l1] - dst_base(l1)) : nullptr;
    tp.leaf = lo;
    tp.status = status;
    k_octree_top<<<1, kTopThreads, 0, st2>>>(tp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (st2 != st && cudaEventRecord(ev_b, st2) != cudaSuccess) return cudaErrorUnknown;
    k_octree_scan<<<(unsigned)n_tiles, kScanThreads, 0, st>>>(B, info.n_geo, s.chunk_prefix,
                                                              n_chunks, s.scan_flags, s.ticket,
                                                              status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (st2 != st && cudaStreamWaitEvent(st, ev_b, 0) != cudaSuccess) return cudaErrorUnknown;
    for (int l = l1; l < lc; ++l) {
        LevelParams lp;
        lp.B = B;
        lp.chunk_prefix = s.chunk_prefix;
        lp.lo = plan.level_off[l];
        lp.n = plan.n_level[l];
        lp.next_lo = plan.level_off[l + 1];
        lp.n_next = plan.n_level[l + 1];
        lp.codes_in = dst(l);
        lp.in_base = dst_base(l);
        lp.codes_out = (l + 1 < D) ? dst(l + 1) : nullptr;
        lp.out_base = (l + 1 < D) ? dst_base(l + 1) : 0;
        lp.leaf = lo;
        lp.status = status;
        const unsigned grid = (unsigned)((lp.n + kLvlTile - 1) / kLvlTile);
        if (grid) k_octree_level<<<grid, kLvlThreads, 0, st>>>(lp);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (lc < D) {
        SubtreeParams sp;
        sp.B = B;
        sp.chunk_prefix = s.chunk_prefix;
        sp.lc = lc;
        sp.depth = D;
        for (int l = 0; l <= D; ++l) sp.level_off[l] = plan.level_off[l];
        sp.level_off[D + 1] = plan.level_off[D] + plan.n_level[D];
        sp.codes_all = codes_all;
        sp.leaf = lo;
        sp.status = status;
        const unsigned grid = (unsigned)((plan.n_level[lc] + kLvlTile - 1) / kLvlTile);
        k_octree_subtree<<<grid, kLvlThreads, 0, st>>>(sp);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Scratch of the octree stage (bytes of the three code buffers).
void octree_code_buffers(const sgs_scene_info &info, const GeoPlan &plan, uint64_t *pingpong,
                         uint64_t *all) {
    const int l1 = octree_top_level(plan);
    const int lc = octree_subtree_level(plan, l1);
    uint64_t m = 1, a = 1;
    for (int l = l1; l < lc && l < plan.depth; ++l) m = m > plan.n_level[l] ? m : plan.n_level[l];
    for (int l = lc; l < plan.depth; ++l) a += plan.n_level[l];
    if (info.n_rows == 0) m = a = 1;
    *pingpong = 8 * m;
    *all = 8 * a;
}

// Kernels launch_octree enqueues for a non-empty scene.
int octree_launches(const sgs_scene_info &info, const GeoPlan &plan) {
    const int l1 = octree_top_level(plan);
    const int lc = octree_subtree_level(plan, l1);
    return (info.n_dup ? 1 : 0) + 2 + (lc - l1) + (lc < plan.depth ? 1 : 0);
}

size_t octree_scan_tiles(uint64_t n_geo) { return (n_geo + kScanTile - 1) / kScanTile; }
size_t octree_chunks(uint64_t n_geo) { return (n_geo + kChunk - 1) / kChunk; }

}  // namespace sgs
