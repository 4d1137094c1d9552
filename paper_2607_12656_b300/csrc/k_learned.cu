// Learned-model attribute decoding on sm_103a: rANS driven by the local autoregressive
// context model (Sec. 3.4.2 "Autoregressive Prediction Coding", made small and integer).
//
// Model (frozen, integer): for token (i, c) of a lane, u_j = s_{i-j,c} - 128 (j = 1..4, 0 past
// the lane start), h1 = rq(W1 u + B1[c]), h2 = rq(W2 h1 + b2), z = W3 h2 + b3 with
// rq(a) = clamp((a m + 2^(sh-1)) >> sh, 0, 127); integer softmax
//   t_k = min(((zmax - z_k) ms) >> ss, 6144),  e_k = EXP2Q[t_k & 255] >> (t_k >> 8),
//   R = floor(65280 * 2^32 / sum e),  f_k = 1 + floor(e_k R / 2^32),  remainder to argmax z.
//
// Decoder: one CTA of 8 warps per group of 32 lanes; it walks the group's tokens in stream
// order (Gaussian i, channel c).  Per (i, c) step the 32 lanes' rows go through layer 1 on
// the ALU, layers 2-3 as int8 mma.sync m16n8k32 with exact int32 accumulation (sm_103a has
// no tcgen05 int8 kind), the softmax reductions across the 4 column quarters, a CDF search
// restricted to the quarter holding each lane's slot, and finally warp 0 advances the 32
// rANS states and refills them from the group's shared word stream.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "exp2q_table.h"
#include "sgs_device.cuh"
#include "sgs_internal.h"

namespace sgs {

__constant__ uint32_t kExp2Q[256] = {SGS_EXP2Q_VALUES};

constexpr int kLThreads = 256;
constexpr int kRS = 80;  // smem row stride (bytes) of int8 rows of 64: conflict-free fragments

// Frozen model blob offsets (bytes).
constexpr int kMB_B1 = 32, kMB_B2 = 14368, kMB_B3 = 14624, kMB_W1 = 15648, kMB_W2 = 15904,
              kMB_W3 = 20000;

struct LSmem {
    int8_t w1[64 * 4];
    int32_t b1[kNChan * 64];
    int8_t w2[64 * kRS];
    int32_t b2[64];
    int8_t w3[256 * kRS];
    int32_t b3[256];
    uint32_t exp2q[256];
    int8_t h1[32 * kRS];
    int8_t h2[32 * kRS];
    uint8_t ctx[32 * 4 * kNChan];  // [lane][ring row][channel]
    alignas(16) uint16_t win[kWinWords];  // word-stream window of warp 0
    int32_t red_max[4][32];
    int32_t red_idx[4][32];
    uint32_t red_sum[4][32];
    uint32_t red_T[4][32];
    uint32_t R[32];
    uint32_t slot[32];
    uint32_t res_s[32], res_f[32], res_c[32];
    uint32_t nrows[32];
    uint64_t row0[32];
    float step[kNChan], offset[kNChan];
    int32_t m1, sh1, m2, sh2;
    uint32_t ms, ss;
    int bad;
};

__device__ __forceinline__ int32_t requant(int32_t acc, int32_t m, int32_t sh) {
    int64_t v = ((int64_t)acc * (int64_t)m + ((int64_t)1 << (sh - 1))) >> sh;
    v = v < 0 ? 0 : v;
    return (int32_t)(v > 127 ? 127 : v);
}

__device__ __forceinline__ void mma_s8(int32_t (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                       uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t lds32(const int8_t *p) {
    return *reinterpret_cast<const uint32_t *>(p);
}

// acc(16 x 8 tile at rows r0.., cols n0..) += A[r0.., 0..63] * W[n0.., 0..63]^T (both int8 rows
// of stride kRS in smem).
__device__ __forceinline__ void tile_16x8x64(int32_t (&acc)[4], const int8_t *A, int r0,
                                             const int8_t *W, int n0, int g, int t) {
#pragma unroll
    for (int kk = 0; kk < 64; kk += 32) {
        const uint32_t a0 = lds32(A + (r0 + g) * kRS + kk + 4 * t);
        const uint32_t a1 = lds32(A + (r0 + g + 8) * kRS + kk + 4 * t);
        const uint32_t a2 = lds32(A + (r0 + g) * kRS + kk + 16 + 4 * t);
        const uint32_t a3 = lds32(A + (r0 + g + 8) * kRS + kk + 16 + 4 * t);
        const uint32_t b0 = lds32(W + (n0 + g) * kRS + kk + 4 * t);
        const uint32_t b1 = lds32(W + (n0 + g) * kRS + kk + 16 + 4 * t);
        mma_s8(acc, a0, a1, a2, a3, b0, b1);
    }
}

// Loads and validates the frozen model; returns false (and marks the stream) if invalid.
__device__ bool load_model(LSmem &S, const uint8_t *m, int *status) {
    const int tid = threadIdx.x;
    if (tid == 0) {
        const int32_t *h = reinterpret_cast<const int32_t *>(m);
        S.m1 = h[0]; S.sh1 = h[1]; S.m2 = h[2]; S.sh2 = h[3];
        S.ms = (uint32_t)h[4]; S.ss = (uint32_t)h[5];
        S.bad = !(S.sh1 >= 1 && S.sh1 <= 47 && S.sh2 >= 1 && S.sh2 <= 47 && S.m1 >= 0 && S.m2 >= 0 &&
                  S.ms >= 1 && S.ms < (1u << 24) && S.ss <= 24);
    }
    const int32_t *b1 = reinterpret_cast<const int32_t *>(m + kMB_B1);
    const int32_t *b2 = reinterpret_cast<const int32_t *>(m + kMB_B2);
    const int32_t *b3 = reinterpret_cast<const int32_t *>(m + kMB_B3);
    bool badb = false;
    for (int i = tid; i < kNChan * 64; i += kLThreads) {
        S.b1[i] = b1[i];
        badb |= (b1[i] >= (1 << 24) || b1[i] <= -(1 << 24));
    }
    for (int i = tid; i < 64; i += kLThreads) {
        S.b2[i] = b2[i];
        badb |= (b2[i] >= (1 << 24) || b2[i] <= -(1 << 24));
    }
    for (int i = tid; i < 256; i += kLThreads) {
        S.b3[i] = b3[i];
        badb |= (b3[i] >= (1 << 24) || b3[i] <= -(1 << 24));
        S.exp2q[i] = kExp2Q[i];
    }
    for (int i = tid; i < 256; i += kLThreads) S.w1[i] = (int8_t)m[kMB_W1 + i];
    for (int i = tid; i < 64 * 64; i += kLThreads) S.w2[(i >> 6) * kRS + (i & 63)] = (int8_t)m[kMB_W2 + i];
    for (int i = tid; i < 256 * 64; i += kLThreads) S.w3[(i >> 6) * kRS + (i & 63)] = (int8_t)m[kMB_W3 + i];
    __syncthreads();
    if (badb) atomicOr(&S.bad, 1);
    __syncthreads();
    if (S.bad) {
        if (tid == 0) set_status(status, SGS_E_CORRUPT);
        return false;
    }
    return true;
}

static_assert(offsetof(LSmem, win) % 16 == 0, "window must be 16-byte aligned");

struct LearnedParams {
    const uint8_t *bits;
    uint64_t model_off, chan_off, grp_sec, pay_off, pay_len;
    uint32_t L, G, n_rows;
    float *out;
    const uint32_t *out_index;
    int *status;
};

__global__ void __launch_bounds__(kLThreads, 1) k_learned_decode(LearnedParams p) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    LSmem &S = *reinterpret_cast<LSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const uint32_t grp = blockIdx.x;
    const int nl = (int)min(32u, p.L - grp * 32);
    if (!load_model(S, p.bits + p.model_off, p.status)) return;
    if (tid < kNChan) {
        S.step[tid] = ld_f32(p.bits + p.chan_off + 4 * tid);
        S.offset[tid] = ld_f32(p.bits + p.chan_off + 4 * (kNChan + tid));
    }
    if (tid < 32) {
        uint64_t r0 = 0, r1 = 0;
        if (tid < nl) {
            const uint64_t j = (uint64_t)grp * 32 + tid;
            r0 = j * p.n_rows / p.L;
            r1 = (j + 1) * p.n_rows / p.L;
        }
        S.row0[tid] = r0;
        S.nrows[tid] = (uint32_t)(r1 - r0);
    }
    for (int i = tid; i < 32 * 4 * kNChan; i += kLThreads) S.ctx[i] = 0;
    GroupStream gs;
    uint32_t x = 0x10000u;
    if (warp == 0) {
        group_open(p.bits, p.grp_sec, p.pay_off, p.pay_len, p.G, grp, nl, lane, gs, x, S.win);
        S.slot[lane] = x & 0xFFFFu;
    }
    __syncthreads();
    uint32_t maxrows = 0;
    for (int r = 0; r < 32; ++r) maxrows = max(maxrows, S.nrows[r]);

    for (uint32_t i = 0; i < maxrows; ++i) {
        for (int c = 0; c < kNChan; ++c) {
            // ---- layer 1 (ALU): row r = tid >> 3, outputs 8 (tid & 7) .. +7
            {
                const int r = tid >> 3, o0 = (tid & 7) * 8;
                int32_t u[4];
#pragma unroll
                for (int j = 1; j <= 4; ++j)
                    u[j - 1] = (i >= (uint32_t)j) ? (int32_t)S.ctx[(r * 4 + ((i - j) & 3)) * kNChan + c] - 128 : 0;
#pragma unroll
                for (int o = o0; o < o0 + 8; ++o) {
                    int32_t acc = S.b1[c * 64 + o];
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc += (int32_t)S.w1[o * 4 + j] * u[j];
                    S.h1[r * kRS + o] = (int8_t)requant(acc, S.m1, S.sh1);
                }
            }
            __syncthreads();
            // ---- layer 2 (mma): warp -> rows 16 (warp & 1), cols 16 (warp >> 1) .. +15
            {
                const int r0 = (warp & 1) * 16;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int n0 = (warp >> 1) * 16 + q * 8;
                    int32_t acc[4] = {0, 0, 0, 0};
                    tile_16x8x64(acc, S.h1, r0, S.w2, n0, g, t);
                    const int col = n0 + 2 * t;
                    S.h2[(r0 + g) * kRS + col] = (int8_t)requant(acc[0] + S.b2[col], S.m2, S.sh2);
                    S.h2[(r0 + g) * kRS + col + 1] = (int8_t)requant(acc[1] + S.b2[col + 1], S.m2, S.sh2);
                    S.h2[(r0 + g + 8) * kRS + col] = (int8_t)requant(acc[2] + S.b2[col], S.m2, S.sh2);
                    S.h2[(r0 + g + 8) * kRS + col + 1] = (int8_t)requant(acc[3] + S.b2[col + 1], S.m2, S.sh2);
                }
            }
            __syncthreads();
            // ---- layer 3 (mma): warp -> rows 16 (warp & 1), column quarter qw = warp >> 1
            const int r0 = (warp & 1) * 16, qw = warp >> 1;
            const int rA = r0 + g, rB = r0 + g + 8;
            int32_t z[8][4];
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const int n0 = qw * 64 + nt * 8;
                z[nt][0] = z[nt][1] = z[nt][2] = z[nt][3] = 0;
                tile_16x8x64(z[nt], S.h2, r0, S.w3, n0, g, t);
                const int col = n0 + 2 * t;
                z[nt][0] += S.b3[col];
                z[nt][1] += S.b3[col + 1];
                z[nt][2] += S.b3[col];
                z[nt][3] += S.b3[col + 1];
            }
            // (a) row max and lowest argmax
            {
                int32_t mA = z[0][0], mB = z[0][2];
                int32_t iA = qw * 64 + 2 * t, iB = iA;
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
                    for (int v = 0; v < 2; ++v) {
                        const int32_t col = qw * 64 + nt * 8 + 2 * t + v;
                        if (z[nt][v] > mA) { mA = z[nt][v]; iA = col; }
                        if (z[nt][2 + v] > mB) { mB = z[nt][2 + v]; iB = col; }
                    }
                }
#pragma unroll
                for (int o = 1; o <= 2; o <<= 1) {
                    const int32_t omA = __shfl_xor_sync(0xffffffffu, mA, o), oiA = __shfl_xor_sync(0xffffffffu, iA, o);
                    const int32_t omB = __shfl_xor_sync(0xffffffffu, mB, o), oiB = __shfl_xor_sync(0xffffffffu, iB, o);
                    if (omA > mA || (omA == mA && oiA < iA)) { mA = omA; iA = oiA; }
                    if (omB > mB || (omB == mB && oiB < iB)) { mB = omB; iB = oiB; }
                }
                if (t == 0) {
                    S.red_max[qw][rA] = mA; S.red_idx[qw][rA] = iA;
                    S.red_max[qw][rB] = mB; S.red_idx[qw][rB] = iB;
                }
            }
            __syncthreads();
            int32_t zmA = S.red_max[0][rA], amA = S.red_idx[0][rA];
            int32_t zmB = S.red_max[0][rB], amB = S.red_idx[0][rB];
#pragma unroll
            for (int q = 1; q < 4; ++q) {
                if (S.red_max[q][rA] > zmA) { zmA = S.red_max[q][rA]; amA = S.red_idx[q][rA]; }
                if (S.red_max[q][rB] > zmB) { zmB = S.red_max[q][rB]; amB = S.red_idx[q][rB]; }
            }
            // (b) e_k (kept in z) and partial sums
            {
                uint32_t sA = 0, sB = 0;
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const uint32_t d = (uint32_t)((v < 2 ? zmA : zmB) - z[nt][v]);
                        uint64_t tt = ((uint64_t)d * S.ms) >> S.ss;
                        const uint32_t tk = tt > 6144 ? 6144u : (uint32_t)tt;
                        const uint32_t e = S.exp2q[tk & 255] >> (tk >> 8);
                        z[nt][v] = (int32_t)e;
                        if (v < 2) sA += e; else sB += e;
                    }
                }
                sA += __shfl_xor_sync(0xffffffffu, sA, 1);
                sA += __shfl_xor_sync(0xffffffffu, sA, 2);
                sB += __shfl_xor_sync(0xffffffffu, sB, 1);
                sB += __shfl_xor_sync(0xffffffffu, sB, 2);
                if (t == 0) { S.red_sum[qw][rA] = sA; S.red_sum[qw][rB] = sB; }
            }
            __syncthreads();
            if (tid < 32) {
                const uint64_t E = (uint64_t)S.red_sum[0][tid] + S.red_sum[1][tid] + S.red_sum[2][tid] + S.red_sum[3][tid];
                S.R[tid] = (uint32_t)((65280ull << 32) / E);
            }
            __syncthreads();
            // (c) floor terms f_k - 1 = umulhi(e_k, R), per-quarter sums
            const uint32_t RA = S.R[rA], RB = S.R[rB];
            {
                uint32_t TA = 0, TB = 0;
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const uint32_t fl = __umulhi((uint32_t)z[nt][v], v < 2 ? RA : RB);
                        z[nt][v] = (int32_t)fl;
                        if (v < 2) TA += fl; else TB += fl;
                    }
                }
                TA += __shfl_xor_sync(0xffffffffu, TA, 1);
                TA += __shfl_xor_sync(0xffffffffu, TA, 2);
                TB += __shfl_xor_sync(0xffffffffu, TB, 1);
                TB += __shfl_xor_sync(0xffffffffu, TB, 2);
                if (t == 0) { S.red_T[qw][rA] = TA; S.red_T[qw][rB] = TB; }
            }
            __syncthreads();
            // (d) CDF search inside the quarter that holds the lane's slot
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int r = half ? rB : rA;
                const int32_t am = half ? amB : amA;
                const bool live = r < nl && i < S.nrows[r];
                const uint32_t T0 = S.red_T[0][r], T1 = S.red_T[1][r], T2 = S.red_T[2][r], T3 = S.red_T[3][r];
                const uint32_t rem = 65536u - 256u - (T0 + T1 + T2 + T3);
                const uint32_t Tq[4] = {T0, T1, T2, T3};
                uint32_t base = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (q < qw) base += 64u + Tq[q] + ((am >> 6) == q ? rem : 0u);
                const uint32_t qtot = 64u + Tq[qw] + ((am >> 6) == qw ? rem : 0u);
                const uint32_t slot = S.slot[r];
                // uniform per quad; the loop runs in every thread so the shuffles see the whole warp
                const bool mine = live && slot >= base && slot < base + qtot;
                uint32_t cum = base;
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) {
                    const int k0 = qw * 64 + nt * 8 + 2 * t;
                    const uint32_t f0 = 1u + (uint32_t)z[nt][2 * half] + (k0 == am ? rem : 0u);
                    const uint32_t f1 = 1u + (uint32_t)z[nt][2 * half + 1] + (k0 + 1 == am ? rem : 0u);
                    const uint32_t mine_sum = f0 + f1;
                    uint32_t incl = mine_sum;
                    const uint32_t n1 = __shfl_up_sync(0xffffffffu, incl, 1, 4);
                    if (t >= 1) incl += n1;
                    const uint32_t n2 = __shfl_up_sync(0xffffffffu, incl, 2, 4);
                    if (t >= 2) incl += n2;
                    const uint32_t tsum = __shfl_sync(0xffffffffu, incl, 3, 4);
                    const uint32_t start = cum + incl - mine_sum;
                    if (mine && slot >= start && slot < start + mine_sum) {
                        const bool first = slot < start + f0;
                        S.res_s[r] = first ? (uint32_t)k0 : (uint32_t)k0 + 1;
                        S.res_f[r] = first ? f0 : f1;
                        S.res_c[r] = first ? start : start + f0;
                    }
                    cum += tsum;
                }
            }
            __syncthreads();
            // (e) warp 0: advance the 32 rANS states, emit tokens, refill from the stream
            if (warp == 0) {
                const bool live = lane < nl && i < S.nrows[lane];
                if (live) {
                    const uint32_t s = S.res_s[lane];
                    x = S.res_f[lane] * (x >> 16) + S.slot[lane] - S.res_c[lane];
                    S.ctx[(lane * 4 + (i & 3)) * kNChan + c] = (uint8_t)s;
                    const uint64_t row = S.row0[lane] + i;
                    const uint64_t col = p.out_index ? (uint64_t)p.out_index[row] : row;
                    p.out[(uint64_t)c * p.n_rows + col] = dequant(s, S.step[c], S.offset[c]);
                }
                group_refill(gs, x, live);
                S.slot[lane] = x & 0xFFFFu;
            }
            __syncthreads();
        }
    }
    if (warp == 0) {
        const bool bad = gs.bad || (lane < nl && x != 0x10000u) || (gs.ptr != gs.n_words);
        if (bad) set_status(p.status, SGS_E_CORRUPT);
    }
}

size_t learned_work_bytes(const sgs_scene_info &) { return 0; }

cudaError_t launch_learned_decode(const uint8_t *bits, const sgs_scene_info &info,
                                  const sgs_scene_out &out, uint8_t *, int *status, cudaStream_t st) {
    if (info.n_rows == 0) return cudaSuccess;
    LearnedParams p;
    p.bits = bits;
    p.model_off = info.off[S_ATTR_TAB];
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
    const size_t smem = sizeof(LSmem);
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_learned_decode, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_learned_decode<<<p.G, kLThreads, smem, st>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ encoder side

// Frequency and cumulative of every token under the model: thread per (row, channel).  All
// contexts are known at encode time, so the rows are independent.  The 256 logits are
// recomputed in three passes (max, sum, floor terms + cumulative) to stay in registers.
__global__ void __launch_bounds__(256) k_learned_fc(const uint8_t *model, const uint8_t *tok,
                                                    uint32_t n_rows, uint32_t L, uint32_t *f_out,
                                                    uint32_t *c_out) {
    __shared__ __align__(16) int8_t w3[256 * 64];
    __shared__ __align__(16) int8_t w2[64 * 64];
    __shared__ int8_t w1[256];
    __shared__ int32_t b2[64], b3[256];
    __shared__ uint32_t ex[256];
    for (int i = threadIdx.x; i < 256 * 64; i += blockDim.x) w3[i] = (int8_t)model[kMB_W3 + i];
    for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) w2[i] = (int8_t)model[kMB_W2 + i];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        w1[i] = (int8_t)model[kMB_W1 + i];
        b3[i] = reinterpret_cast<const int32_t *>(model + kMB_B3)[i];
        ex[i] = kExp2Q[i];
    }
    for (int i = threadIdx.x; i < 64; i += blockDim.x) b2[i] = reinterpret_cast<const int32_t *>(model + kMB_B2)[i];
    __syncthreads();
    const int32_t *hdr = reinterpret_cast<const int32_t *>(model);
    const int32_t m1 = hdr[0], sh1 = hdr[1], m2 = hdr[2], sh2 = hdr[3];
    const uint32_t ms = (uint32_t)hdr[4], ss = (uint32_t)hdr[5];
    const int32_t *B1 = reinterpret_cast<const int32_t *>(model + kMB_B1);
    const uint64_t nt = (uint64_t)n_rows * kNChan;
    for (uint64_t id = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; id < nt;
         id += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t row = id / kNChan;
        const int c = (int)(id - row * kNChan);
        // lane of the row: largest j with floor(j n / L) <= row
        const uint64_t j = ((row + 1) * L + n_rows - 1) / n_rows - 1;
        const uint64_t row0 = j * n_rows / L;
        int32_t u[4];
#pragma unroll
        for (int q = 1; q <= 4; ++q)
            u[q - 1] = (row >= row0 + q) ? (int32_t)tok[(row - q) * kNChan + c] - 128 : 0;
        uint32_t h1w[16], h2w[16];
#pragma unroll
        for (int o4 = 0; o4 < 16; ++o4) {
            uint32_t packed = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int o = o4 * 4 + b;
                int32_t acc = B1[c * 64 + o];
#pragma unroll
                for (int q = 0; q < 4; ++q) acc += (int32_t)w1[o * 4 + q] * u[q];
                packed |= (uint32_t)requant(acc, m1, sh1) << (8 * b);
            }
            h1w[o4] = packed;
        }
#pragma unroll
        for (int o4 = 0; o4 < 16; ++o4) {
            uint32_t packed = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int o = o4 * 4 + b;
                int32_t acc = b2[o];
                const uint32_t *wr = reinterpret_cast<const uint32_t *>(w2 + o * 64);
#pragma unroll
                for (int k = 0; k < 16; ++k) acc = __dp4a((int)wr[k], (int)h1w[k], acc);
                packed |= (uint32_t)requant(acc, m2, sh2) << (8 * b);
            }
            h2w[o4] = packed;
        }
        auto logit = [&](int k) {
            int32_t acc = b3[k];
            const uint32_t *wr = reinterpret_cast<const uint32_t *>(w3 + k * 64);
#pragma unroll
            for (int q = 0; q < 16; ++q) acc = __dp4a((int)wr[q], (int)h2w[q], acc);
            return acc;
        };
        int32_t zmax = logit(0);
        int amax = 0;
        for (int k = 1; k < 256; ++k) {
            const int32_t zk = logit(k);
            if (zk > zmax) { zmax = zk; amax = k; }
        }
        auto ek = [&](int32_t zk) {
            const uint64_t tt = ((uint64_t)(uint32_t)(zmax - zk) * ms) >> ss;
            const uint32_t tk = tt > 6144 ? 6144u : (uint32_t)tt;
            return ex[tk & 255] >> (tk >> 8);
        };
        uint64_t E = 0;
        for (int k = 0; k < 256; ++k) E += ek(logit(k));
        const uint32_t R = (uint32_t)((65280ull << 32) / E);
        const uint32_t s = tok[row * kNChan + c];
        uint32_t S = 0, cum = 0, fs = 0;
        for (int k = 0; k < 256; ++k) {
            const uint32_t fl = __umulhi(ek(logit(k)), R);
            if (k < (int)s) cum += 1u + fl;
            if (k == (int)s) fs = 1u + fl;
            S += fl;
        }
        const uint32_t rem = 65536u - 256u - S;
        if ((int)s == amax) fs += rem;
        if (amax < (int)s) cum += rem;
        f_out[id] = fs;
        c_out[id] = cum;
    }
}

int learned_token_fc(sgs_ctx *, const uint8_t *model, const uint8_t *tokens, uint32_t n_rows,
                     uint32_t lanes, std::vector<uint32_t> &f, std::vector<uint32_t> &cum) {
    const uint64_t n = (uint64_t)n_rows * kNChan;
    f.assign(n, 0);
    cum.assign(n, 0);
    if (n == 0) return SGS_OK;
    uint8_t *dm = nullptr, *dt = nullptr;
    uint32_t *df = nullptr, *dc = nullptr;
    int rc = SGS_OK;
    if (cudaMalloc(&dm, SGS_MODEL_BYTES) != cudaSuccess || cudaMalloc(&dt, n) != cudaSuccess ||
        cudaMalloc(&df, 4 * n) != cudaSuccess || cudaMalloc(&dc, 4 * n) != cudaSuccess) {
        rc = SGS_E_NOMEM;
    } else {
        cudaMemcpy(dm, model, SGS_MODEL_BYTES, cudaMemcpyHostToDevice);
        cudaMemcpy(dt, tokens, n, cudaMemcpyHostToDevice);
        const uint64_t blocks = (n + 255) / 256;
        k_learned_fc<<<(unsigned)(blocks < 148 * 64 ? blocks : 148 * 64), 256>>>(dm, dt, n_rows, lanes, df, dc);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) rc = SGS_E_CUDA;
        else {
            cudaMemcpy(f.data(), df, 4 * n, cudaMemcpyDeviceToHost);
            cudaMemcpy(cum.data(), dc, 4 * n, cudaMemcpyDeviceToHost);
        }
    }
    cudaFree(dm);
    cudaFree(dt);
    cudaFree(df);
    cudaFree(dc);
    return rc;
}

}  // namespace sgs
