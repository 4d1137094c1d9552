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
    if (threadIdx.x == 0) {
        uint32_t prefix = 0;
        volatile unsigned long long *vf = reinterpret_cast<volatile unsigned long long *>(flags);
        if (tile == 0) {
            __threadfence();
            vf[0] = (2ull << 32) | agg;
        } else {
            vf[tile] = (1ull << 32) | agg;
            __threadfence();
            int64_t i = (int64_t)tile - 1;
            uint32_t spins = 0;
            while (i >= 0) {
                const unsigned long long v = vf[i];
                const uint32_t flag = (uint32_t)(v >> 32);
                if (flag == 0) {
                    if (++spins > kSpinLimit) { set_status(status, SGS_E_TIMEOUT); break; }
                    __nanosleep(32);
                    continue;
                }
                prefix += (uint32_t)v;
                if (flag == 2) break;
                --i;
            }
            __threadfence();
            vf[tile] = (2ull << 32) | (uint64_t)(prefix + agg);
        }
        s_prefix = prefix;
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

__global__ void __launch_bounds__(kTopThreads) k_octree_top(TopParams p) {
    __shared__ uint64_t codes[2][kTopCap];
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t s_carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) codes[0][0] = 0;
    __syncthreads();
    int cur = 0;
    for (int l = 0; l < p.l1; ++l) {
        const uint32_t n = p.plan.n_level[l];
        const uint32_t n_next = p.plan.n_level[l + 1];
        const bool to_leaves = (l + 1 == p.plan.depth);
        const bool to_global = (l + 1 == p.l1) && !to_leaves;
        const uint8_t *Bl = p.B + p.plan.level_off[l];
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

// ------------------------------------------------------------------ one deep level

struct LevelParams {
    const uint8_t *B;
    const uint32_t *chunk_prefix;
    uint64_t lo, n;          // level's BFS offset and node count
    uint32_t n_next;
    const uint64_t *codes_in;
    uint64_t *codes_out;     // NULL when the next level is the leaves
    LeafOut leaf;
    int *status;
};

__global__ void __launch_bounds__(kLvlThreads) k_octree_level(LevelParams p) {
    __shared__ uint32_t sm[8];
    __shared__ uint32_t s_base;
    const uint64_t t0 = (uint64_t)blockIdx.x * kLvlTile;
    if (threadIdx.x < 32) {
        const uint32_t p_lo = prefix_at_warp(p.B, p.chunk_prefix, p.lo);
        const uint32_t p_g0 = prefix_at_warp(p.B, p.chunk_prefix, p.lo + t0);
        if (threadIdx.x == 0) s_base = p_g0 - p_lo;
        if (blockIdx.x == 0) {
            const uint32_t p_hi = prefix_at_warp(p.B, p.chunk_prefix, p.lo + p.n);
            if (threadIdx.x == 0 && p_hi - p_lo != p.n_next) set_status(p.status, SGS_E_CORRUPT);
        }
    }
    const uint64_t i0 = t0 + (uint64_t)threadIdx.x * kLvlPer;
    uint32_t bytes[kLvlPer];
    uint32_t cnt = 0;
#pragma unroll
    for (int q = 0; q < kLvlPer; ++q) {
        bytes[q] = (i0 + q < p.n) ? p.B[p.lo + i0 + q] : 0u;
        cnt += __popc(bytes[q]);
    }
    uint32_t tot;
    const uint32_t ex = block_excl_scan_256(cnt, &tot, sm);  // also orders s_base
    uint32_t idx = s_base + ex;
#pragma unroll
    for (int q = 0; q < kLvlPer; ++q) {
        if (i0 + q >= p.n) break;
        const uint64_t pc = p.codes_in[i0 + q];
        uint32_t b = bytes[q];
        while (b) {
            const uint32_t k = __ffs(b) - 1;
            b &= b - 1;
            if (idx >= p.n_next) { set_status(p.status, SGS_E_CORRUPT); b = 0; break; }
            const uint64_t cc = child_code(pc, k);
            if (p.codes_out) p.codes_out[idx] = cc;
            else write_leaf(p.leaf, idx, cc, p.status);
            ++idx;
        }
    }
}

// ------------------------------------------------------------------ launcher

cudaError_t launch_octree(const uint8_t *B, const sgs_scene_info &info, const GeoPlan &plan,
                          const uint8_t *bits, const Scratch &s, const sgs_scene_out &out,
                          int *status, cudaStream_t st) {
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
    // popcount prefix over all tokens
    const uint64_t n_chunks = (info.n_geo + kChunk - 1) / kChunk;
    const uint64_t n_tiles = (info.n_geo + kScanTile - 1) / kScanTile;
    k_octree_scan<<<(unsigned)n_tiles, kScanThreads, 0, st>>>(B, info.n_geo, s.chunk_prefix,
                                                              n_chunks, s.scan_flags, s.ticket,
                                                              status);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // top levels in one CTA
    int l1 = 1;
    while (l1 < D && plan.n_level[l1] <= kTopCap) ++l1;
    TopParams tp;
    tp.B = B;
    tp.plan = plan;
    tp.l1 = l1;
    tp.codes_out = s.codes[0];
    tp.leaf = lo;
    tp.status = status;
    k_octree_top<<<1, kTopThreads, 0, st>>>(tp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int cur = 0;
    for (int l = l1; l < D; ++l) {
        LevelParams lp;
        lp.B = B;
        lp.chunk_prefix = s.chunk_prefix;
        lp.lo = plan.level_off[l];
        lp.n = plan.n_level[l];
        lp.n_next = plan.n_level[l + 1];
        lp.codes_in = s.codes[cur];
        lp.codes_out = (l + 1 < D) ? s.codes[cur ^ 1] : nullptr;
        lp.leaf = lo;
        lp.status = status;
        const unsigned grid = (unsigned)((lp.n + kLvlTile - 1) / kLvlTile);
        if (grid) k_octree_level<<<grid, kLvlThreads, 0, st>>>(lp);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        cur ^= 1;
    }
    return cudaSuccess;
}

// Kernels launch_octree enqueues for a non-empty scene.
int octree_launches(const sgs_scene_info &info, const GeoPlan &plan) {
    int l1 = 1;
    while (l1 < plan.depth && plan.n_level[l1] <= kTopCap) ++l1;
    return (info.n_dup ? 1 : 0) + 2 + (plan.depth - l1);
}

size_t octree_scan_tiles(uint64_t n_geo) { return (n_geo + kScanTile - 1) / kScanTile; }
size_t octree_chunks(uint64_t n_geo) { return (n_geo + kChunk - 1) / kChunk; }

}  // namespace sgs
