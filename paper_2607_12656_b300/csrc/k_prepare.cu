// Scene preparation for the encoder on the device (Sec. 3.3 structural formation, Sec. 3.4
// serialization): prune the floor(n/10) Gaussians of lowest opacity (ties: lower index
// first), voxelize at depth D, order the kept rows by (Morton code, original index), find
// the unique voxels and the duplicate counts, build the octree's occupancy bytes per level
// and quantize every channel uniformly between its minimum and maximum.  The results are the
// host `prepare`'s exactly (every tie-break is fixed); they are copied back for the
// bitstream writer.
//
// Orders come from stable LSD radix sorts (k_sort.cu): the prune sorts (opacity, index) keys,
// the rows sort their Morton code's low word, then its high word; runs of equal codes give the
// voxels and duplicates, runs of equal code prefixes the nodes of each level.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "encode_prep.h"
#include "sgs_device.cuh"
#include "sgs_internal.h"

namespace sgs {
namespace {

constexpr int kPT = 256;

inline uint32_t blocks(uint64_t n) { return (uint32_t)((n + kPT - 1) / kPT); }

// Inputs `prepare` refuses: a position outside [0, 1) or a non-finite attribute.
__global__ void k_prep_check(const float *pos, const float *attr, uint32_t n, int *bad) {
    const uint64_t np = 3ull * n, na = (uint64_t)kNChan * n;
    bool b = false;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < np + na;
         i += (uint64_t)gridDim.x * blockDim.x) {
        if (i < np) {
            const float p = pos[i];
            b |= !(p >= 0.0f && p < 1.0f);
        } else {
            b |= !isfinite(attr[i - np]);
        }
    }
    if (__any_sync(0xffffffffu, b) && (threadIdx.x & 31) == 0) atomicOr(bad, 1);
}

// A float's order as an unsigned key (-0 and +0 equal, as the comparison `<` has them).
__device__ __forceinline__ uint32_t float_key(float f) {
    uint32_t u = __float_as_uint(f);
    if (u == 0x80000000u) u = 0u;
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__global__ void k_prune_keys(const float *opacity, uint32_t n, uint32_t *key, uint32_t *val) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    key[i] = float_key(opacity[i]);
    val[i] = i;
}

// flag[i] = 1 for the Gaussians after the first `drop` of the (opacity, index) order
__global__ void k_keep_flags(const uint32_t *sorted_idx, uint32_t n, uint32_t drop, uint32_t *flag) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) flag[sorted_idx[j]] = j >= drop ? 1u : 0u;
}

// keep[pos[i]] = i for flagged i: the kept indices, ascending
__global__ void k_compact_idx(const uint32_t *flag, const uint32_t *pos, uint32_t n, uint32_t *keep) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) keep[pos[i]] = i;
}

// Bits of v spread to every third bit (bit b -> 3 b).
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
    uint64_t x = v & 0x1FFFFFull;
    x = (x | (x << 32)) & 0x1F00000000FFFFull;
    x = (x | (x << 16)) & 0x1F0000FF0000FFull;
    x = (x | (x << 8)) & 0x100F00F00F00F00Full;
    x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// Row r (kept index keep[r]): voxel v = min(floor(p 2^D), 2^D - 1) per axis (exact: the
// product by a power of two rounds nothing) and its Morton code, x the most significant bit
// of each triple.
__global__ void k_morton(const float *pos, uint32_t n, const uint32_t *keep, uint32_t R, uint32_t D, uint32_t *lo,
                         uint32_t *hi, uint32_t *row) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const uint32_t i = keep[r];
    const float scale = ldexpf(1.0f, (int)D);
    const uint32_t vmax = (1u << D) - 1u;
    uint32_t v[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] = min((uint32_t)floorf(pos[(uint64_t)k * n + i] * scale), vmax);
    const uint64_t code = (spread3(v[0]) << 2) | (spread3(v[1]) << 1) | spread3(v[2]);
    lo[r] = (uint32_t)code;
    hi[r] = (uint32_t)(code >> 32);
    row[r] = r;
}

__global__ void k_gather_u32(const uint32_t *src, const uint32_t *idx, uint32_t n, uint32_t *dst) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) dst[j] = src[idx[j]];
}

// The sorted rows: original index, 64-bit code, voxel coordinates.
__global__ void k_rows(const uint32_t *ord, const uint32_t *keep, const uint32_t *lo, const uint32_t *hi, uint32_t R,
                       uint32_t D, uint32_t *keep_s, uint64_t *code_s, uint32_t *coord) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= R) return;
    const uint32_t r = ord[j];
    keep_s[j] = keep[r];
    const uint64_t code = ((uint64_t)hi[r] << 32) | lo[r];
    code_s[j] = code;
    uint32_t v[3] = {0u, 0u, 0u};
    for (uint32_t b = 0; b < D; ++b)
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] |= (uint32_t)((code >> (3 * b + 2 - k)) & 1u) << b;
#pragma unroll
    for (int k = 0; k < 3; ++k) coord[(uint64_t)k * R + j] = v[k];
}

// flag[i] = 1 where code >> sh differs from the previous item's (a run's first item)
__global__ void k_run_flags(const uint64_t *code, uint32_t n, uint32_t sh, uint32_t *flag) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    flag[i] = (i == 0 || (code[i] >> sh) != (code[i - 1] >> sh)) ? 1u : 0u;
}

// The unique voxels and where each one's run of rows starts
__global__ void k_leaves(const uint64_t *code, const uint32_t *flag, const uint32_t *pos, uint32_t R, uint64_t *leaves,
                         uint32_t *start) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R || !flag[i]) return;
    leaves[pos[i]] = code[i];
    start[pos[i]] = i;
}

// dflag[u] = 1 if voxel u holds more than one row
__global__ void k_dup_flags(const uint32_t *start, uint32_t U, uint32_t R, uint32_t *dflag) {
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= U) return;
    const uint32_t end = u + 1 < U ? start[u + 1] : R;
    dflag[u] = end - start[u] > 1 ? 1u : 0u;
}

__global__ void k_dups(const uint32_t *start, const uint32_t *dflag, const uint32_t *dpos, uint32_t U, uint32_t R,
                       uint32_t *dups) {
    const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= U || !dflag[u]) return;
    const uint32_t end = u + 1 < U ? start[u + 1] : R;
    dups[2 * dpos[u]] = u;
    dups[2 * dpos[u] + 1] = end - start[u] - 1;
}

// Level l's occupancy: leaf i lies in node pos[i] + flag[i] - 1 (pos the exclusive scan of the
// run-start flags over runs of leaves sharing code >> sn) and sets its child (code >> sk) & 7
__global__ void k_occupancy(const uint64_t *leaves, const uint32_t *flag, const uint32_t *pos, uint32_t U, uint32_t sk,
                            uint32_t *occ) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < U) atomicOr(&occ[pos[i] + flag[i] - 1u], 1u << ((leaves[i] >> sk) & 7u));
}

__global__ void k_pack_bytes(const uint32_t *occ, uint32_t m, uint8_t *bytes) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) bytes[j] = (uint8_t)occ[j];
}

// Per channel, the first row (in row order) holding the minimum and the first holding the
// maximum, as 64-bit keys (value order, then row) reduced with atomics: the host's running
// min/max keeps the first of equal values, and so the zero's sign it finds.
__global__ void k_chan_extrema(const float *attr, uint32_t n, const uint32_t *keep_s, uint32_t R,
                               unsigned long long *kmin, unsigned long long *kmax) {
    const uint32_t c = blockIdx.y;
    unsigned long long lo = ~0ull, hi = 0ull;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < R; j += gridDim.x * blockDim.x) {
        const uint64_t key = float_key(attr[(uint64_t)c * n + keep_s[j]]);
        lo = min(lo, (unsigned long long)((key << 32) | j));
        hi = max(hi, (unsigned long long)((key << 32) | (0xFFFFFFFFu - j)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&kmin[c], lo);
        atomicMax(&kmax[c], hi);
    }
}

struct QuantParams {
    double mn[kNChan], step[kNChan];
    uint32_t top[kNChan];
};

// q[j][c] = clamp(rint((v - min) / step), 0, 2^b - 1) in fp64 (0 for a constant channel)
__global__ void k_quantize(const float *attr, uint32_t n, const uint32_t *keep_s, uint32_t R, QuantParams Q,
                           uint16_t *q) {
    const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (t >= (uint64_t)R * kNChan) return;
    const uint32_t j = (uint32_t)(t / kNChan), c = (uint32_t)(t - (uint64_t)j * kNChan);
    uint16_t out = 0;
    if (Q.step[c] != 0.0) {
        double x = rint(((double)attr[(uint64_t)c * n + keep_s[j]] - Q.mn[c]) / Q.step[c]);
        x = fmin(fmax(x, 0.0), (double)Q.top[c]);
        out = (uint16_t)x;
    }
    q[t] = out;
}

// Device allocations of one preparation, freed together.
struct Pool {
    std::vector<void *> p;
    bool failed = false;
    template <typename T>
    T *get(uint64_t count) {
        void *q = nullptr;
        if (cudaMalloc(&q, std::max<uint64_t>(count, 1) * sizeof(T)) != cudaSuccess) {
            failed = true;
            return nullptr;
        }
        p.push_back(q);
        return static_cast<T *>(q);
    }
    ~Pool() {
        for (void *q : p) cudaFree(q);
    }
};

}  // namespace

int prepare_device(int device, const float *pos, const float *attr, uint32_t n, uint32_t D, const uint32_t *bits,
                   Prepared &P) {
    if (D < 1 || D > SGS_MAX_DEPTH) return SGS_E_INVALID;
    for (int c = 0; c < kNChan; ++c)
        if (bits[c] < 1 || bits[c] > 16) return SGS_E_INVALID;
    if (cudaSetDevice(device) != cudaSuccess) return SGS_E_CUDA;
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return SGS_E_CUDA;
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamDestroy(s); }
    } guard{st};
    Pool pool;
    const uint32_t R = n - n / 10;
    float *dpos = pool.get<float>(3ull * n);
    float *dattr = pool.get<float>((uint64_t)kNChan * n);
    int *dbad = pool.get<int>(1);
    // sort buffers (two of each, ping-pong), scan sums, flags and positions
    const uint32_t nmax = std::max(n, 1u);
    uint32_t *k2[2] = {pool.get<uint32_t>(nmax), pool.get<uint32_t>(nmax)};
    uint32_t *v2[2] = {pool.get<uint32_t>(nmax), pool.get<uint32_t>(nmax)};
    const uint64_t nb = (nmax + kSortChunk - 1) / kSortChunk;
    uint32_t *cnt = pool.get<uint32_t>(256 * nb), *cnt_off = pool.get<uint32_t>(256 * nb);
    const uint64_t scan_words = std::max<uint64_t>(256 * nb, nmax) / kScanBlock + 2;
    uint32_t *sums = pool.get<uint32_t>(scan_words);
    uint32_t *flag = pool.get<uint32_t>(nmax), *fpos = pool.get<uint32_t>(nmax);
    uint32_t *keep = pool.get<uint32_t>(nmax), *keep_s = pool.get<uint32_t>(nmax);
    uint32_t *lo = pool.get<uint32_t>(nmax), *hi = pool.get<uint32_t>(nmax), *row = pool.get<uint32_t>(nmax);
    uint64_t *code_s = pool.get<uint64_t>(nmax), *leaves = pool.get<uint64_t>(nmax);
    uint32_t *coord = pool.get<uint32_t>(3ull * nmax), *start = pool.get<uint32_t>(nmax);
    uint32_t *dflag = pool.get<uint32_t>(nmax), *dup_pos = pool.get<uint32_t>(nmax), *dups = pool.get<uint32_t>(2ull * nmax);
    uint32_t *occ = pool.get<uint32_t>(nmax);
    uint8_t *bytes = pool.get<uint8_t>(nmax);
    unsigned long long *kmin = pool.get<unsigned long long>(kNChan), *kmax = pool.get<unsigned long long>(kNChan);
    uint16_t *q = pool.get<uint16_t>((uint64_t)R * kNChan);
    if (pool.failed) {
        cudaGetLastError();  // the failed allocation's error is answered here
        return SGS_E_NOMEM;
    }
    auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    // upload and check the inputs
    if (!ok(cudaMemcpyAsync(dpos, pos, 12ull * n, cudaMemcpyHostToDevice, st)) ||
        !ok(cudaMemcpyAsync(dattr, attr, 4ull * kNChan * n, cudaMemcpyHostToDevice, st)) ||
        !ok(cudaMemsetAsync(dbad, 0, sizeof(int), st)))
        return SGS_E_CUDA;
    if (n) k_prep_check<<<148 * 8, kPT, 0, st>>>(dpos, dattr, n, dbad);
    int bad = 0;
    if (!ok(cudaMemcpyAsync(&bad, dbad, sizeof(int), cudaMemcpyDeviceToHost, st)) || !ok(cudaStreamSynchronize(st)))
        return SGS_E_CUDA;
    if (bad) return SGS_E_INVALID;
    P.depth = D;
    P.n_in = n;
    memcpy(P.bits, bits, sizeof(P.bits));
    auto radix = [&](uint32_t count, int lo_bit, int hi_bit, int &cur) -> bool {
        for (int sh = lo_bit; sh < hi_bit; sh += 8) {
            if (!ok(radix_pass(k2[cur], v2[cur], count, sh, cnt, cnt_off, sums, k2[cur ^ 1], v2[cur ^ 1], st)))
                return false;
            cur ^= 1;
        }
        return true;
    };
    // prune: (opacity, index) order, the first n / 10 dropped; the rest, ascending
    int cur = 0;
    if (n) {
        k_prune_keys<<<blocks(n), kPT, 0, st>>>(dattr + 48ull * n, n, k2[0], v2[0]);
        if (!radix(n, 0, 32, cur)) return SGS_E_CUDA;
        k_keep_flags<<<blocks(n), kPT, 0, st>>>(v2[cur], n, n / 10, flag);
        if (!ok(scan_u32(flag, n, sums, fpos, st))) return SGS_E_CUDA;
        k_compact_idx<<<blocks(n), kPT, 0, st>>>(flag, fpos, n, keep);
    }
    // rows in (Morton code, original index) order: stable sorts on the low word, then the high
    if (R) {
        k_morton<<<blocks(R), kPT, 0, st>>>(dpos, n, keep, R, D, k2[0], hi, v2[0]);
        cur = 0;
        const int bits_total = 3 * (int)D;
        if (!radix(R, 0, std::min(bits_total, 32), cur)) return SGS_E_CUDA;
        if (bits_total > 32) {
            k_gather_u32<<<blocks(R), kPT, 0, st>>>(hi, v2[cur], R, k2[cur]);
            if (!radix(R, 0, bits_total - 32, cur)) return SGS_E_CUDA;
        }
        // lo of each original row again (k2 now holds the last sort's keys)
        k_morton<<<blocks(R), kPT, 0, st>>>(dpos, n, keep, R, D, lo, hi, row);
        k_rows<<<blocks(R), kPT, 0, st>>>(v2[cur], keep, lo, hi, R, D, keep_s, code_s, coord);
        // unique voxels and duplicates
        k_run_flags<<<blocks(R), kPT, 0, st>>>(code_s, R, 0, flag);
        if (!ok(scan_u32(flag, R, sums, fpos, st))) return SGS_E_CUDA;
        k_leaves<<<blocks(R), kPT, 0, st>>>(code_s, flag, fpos, R, leaves, start);
        uint32_t last_pos = 0, last_flag = 0;
        if (!ok(cudaMemcpyAsync(&last_pos, fpos + R - 1, 4, cudaMemcpyDeviceToHost, st)) ||
            !ok(cudaMemcpyAsync(&last_flag, flag + R - 1, 4, cudaMemcpyDeviceToHost, st)) ||
            !ok(cudaStreamSynchronize(st)))
            return SGS_E_CUDA;
        const uint32_t U = last_pos + last_flag;
        k_dup_flags<<<blocks(U), kPT, 0, st>>>(start, U, R, dflag);
        if (!ok(scan_u32(dflag, U, sums, dup_pos, st))) return SGS_E_CUDA;
        k_dups<<<blocks(U), kPT, 0, st>>>(start, dflag, dup_pos, U, R, dups);
        uint32_t nd_pos = 0, nd_flag = 0;
        if (!ok(cudaMemcpyAsync(&nd_pos, dup_pos + U - 1, 4, cudaMemcpyDeviceToHost, st)) ||
            !ok(cudaMemcpyAsync(&nd_flag, dflag + U - 1, 4, cudaMemcpyDeviceToHost, st)) || !ok(cudaStreamSynchronize(st)))
            return SGS_E_CUDA;
        const uint32_t n_dup = nd_pos + nd_flag;
        P.leaves.resize(U);
        P.dups.resize(2ull * n_dup);
        if (!ok(cudaMemcpyAsync(P.leaves.data(), leaves, 8ull * U, cudaMemcpyDeviceToHost, st)) ||
            (n_dup && !ok(cudaMemcpyAsync(P.dups.data(), dups, 8ull * n_dup, cudaMemcpyDeviceToHost, st))))
            return SGS_E_CUDA;
        // octree levels: nodes of level l = runs of leaves sharing code >> 3 (D - l)
        P.levels.assign(D, {});
        for (uint32_t l = 0; l < D; ++l) {
            const uint32_t sn = 3 * (D - l), sk = 3 * (D - l - 1);
            k_run_flags<<<blocks(U), kPT, 0, st>>>(leaves, U, sn, flag);
            if (!ok(scan_u32(flag, U, sums, fpos, st))) return SGS_E_CUDA;
            uint32_t lp = 0, lf = 0;
            if (!ok(cudaMemcpyAsync(&lp, fpos + U - 1, 4, cudaMemcpyDeviceToHost, st)) ||
                !ok(cudaMemcpyAsync(&lf, flag + U - 1, 4, cudaMemcpyDeviceToHost, st)) || !ok(cudaStreamSynchronize(st)))
                return SGS_E_CUDA;
            const uint32_t m = lp + lf;
            if (!ok(cudaMemsetAsync(occ, 0, 4ull * m, st))) return SGS_E_CUDA;
            k_occupancy<<<blocks(U), kPT, 0, st>>>(leaves, flag, fpos, U, sk, occ);
            k_pack_bytes<<<blocks(m), kPT, 0, st>>>(occ, m, bytes);
            P.levels[l].resize(m);
            if (!ok(cudaMemcpyAsync(P.levels[l].data(), bytes, m, cudaMemcpyDeviceToHost, st)) ||
                !ok(cudaStreamSynchronize(st)))
                return SGS_E_CUDA;
        }
        // per-channel extrema (first of equal values in row order) and quantization
        if (!ok(cudaMemsetAsync(kmin, 0xFF, 8 * kNChan, st)) || !ok(cudaMemsetAsync(kmax, 0, 8 * kNChan, st)))
            return SGS_E_CUDA;
        k_chan_extrema<<<dim3(std::min<uint32_t>(blocks(R), 64), kNChan), kPT, 0, st>>>(dattr, n, keep_s, R, kmin, kmax);
        unsigned long long hmin[kNChan], hmax[kNChan];
        std::vector<uint32_t> ks(R);
        if (!ok(cudaMemcpyAsync(hmin, kmin, sizeof(hmin), cudaMemcpyDeviceToHost, st)) ||
            !ok(cudaMemcpyAsync(hmax, kmax, sizeof(hmax), cudaMemcpyDeviceToHost, st)) ||
            !ok(cudaMemcpyAsync(ks.data(), keep_s, 4ull * R, cudaMemcpyDeviceToHost, st)) || !ok(cudaStreamSynchronize(st)))
            return SGS_E_CUDA;
        QuantParams Q;
        for (int c = 0; c < kNChan; ++c) {
            const uint32_t jmin = (uint32_t)(hmin[c] & 0xFFFFFFFFu), jmax = 0xFFFFFFFFu - (uint32_t)(hmax[c] & 0xFFFFFFFFu);
            const float mn = attr[(uint64_t)c * n + ks[jmin]], mx = attr[(uint64_t)c * n + ks[jmax]];
            const uint32_t top = (1u << bits[c]) - 1u;
            const float step = (mx == mn) ? 0.0f : (float)(((double)mx - (double)mn) / (double)top);
            P.step[c] = step;
            P.offset[c] = mn;
            Q.mn[c] = (double)mn;
            Q.step[c] = (double)step;
            Q.top[c] = top;
        }
        const uint64_t nq = (uint64_t)R * kNChan;
        k_quantize<<<(uint32_t)((nq + kPT - 1) / kPT), kPT, 0, st>>>(dattr, n, keep_s, R, Q, q);
        P.keep.swap(ks);
        P.q16.resize(nq);
        P.coord.resize(3ull * R);
        if (!ok(cudaMemcpyAsync(P.q16.data(), q, 2 * nq, cudaMemcpyDeviceToHost, st)) ||
            !ok(cudaMemcpyAsync(P.coord.data(), coord, 12ull * R, cudaMemcpyDeviceToHost, st)) ||
            !ok(cudaStreamSynchronize(st)) || !ok(cudaGetLastError()))
            return SGS_E_CUDA;
    } else {
        P.keep.clear();
        P.leaves.clear();
        P.dups.clear();
        P.levels.assign(D, {});
        P.q16.clear();
        P.coord.clear();
        for (int c = 0; c < kNChan; ++c) P.step[c] = P.offset[c] = 0.0f;
        if (!ok(cudaStreamSynchronize(st)) || !ok(cudaGetLastError())) return SGS_E_CUDA;
    }
    return SGS_OK;
}

}  // namespace sgs
