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
#include <string.h>
#include <cuda_bf16.h>

#include <vector>

#include "exp2q_table.h"
#include "sgs_device.cuh"
#include "sgs_internal.h"

namespace sgs {

__constant__ uint32_t kExp2Q[256] = {SGS_EXP2Q_VALUES};


// Frozen model blob offsets (bytes).
constexpr int kMB_B1 = 32, kMB_B2 = 14368, kMB_B3 = 14624, kMB_W1 = 15648, kMB_W2 = 15904,
              kMB_W3 = 20000;

__device__ __forceinline__ int32_t requant(int32_t acc, int32_t m, int32_t sh) {
    int64_t v = ((int64_t)acc * (int64_t)m + ((int64_t)1 << (sh - 1))) >> sh;
    v = v < 0 ? 0 : v;
    return (int32_t)(v > 127 ? 127 : v);
}

// Layers 2-3 on the tensor cores in bf16 with fp32 accumulation.  This is exact: int8
// weights and activations in [0, 127] are exact in bf16, their products exact in fp32, and
// every partial sum of 64 products is an integer below 2^21 < 2^24.  (B300 has no tcgen05
// int8 kind and a far slower int8 mma path.)
constexpr int kBS = 72;  // smem row stride in bf16 elements (64 used): conflict-free fragments

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t lds32(const __nv_bfloat16 *p) {
    return *reinterpret_cast<const uint32_t *>(p);
}

// acc(16 x 8 tile at rows r0.., cols n0..) += A[r0.., 0..63] * W[n0.., 0..63]^T, both bf16
// rows of stride kBS in shared memory; returns the exact integer sums.
__device__ __forceinline__ void tile_16x8x64(int32_t (&out)[4], const __nv_bfloat16 *A, int r0,
                                             const __nv_bfloat16 *W, int n0, int g, int t) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kk = 0; kk < 64; kk += 16) {
        const uint32_t a0 = lds32(A + (r0 + g) * kBS + kk + 2 * t);
        const uint32_t a1 = lds32(A + (r0 + g + 8) * kBS + kk + 2 * t);
        const uint32_t a2 = lds32(A + (r0 + g) * kBS + kk + 8 + 2 * t);
        const uint32_t a3 = lds32(A + (r0 + g + 8) * kBS + kk + 8 + 2 * t);
        const uint32_t b0 = lds32(W + (n0 + g) * kBS + kk + 2 * t);
        const uint32_t b1 = lds32(W + (n0 + g) * kBS + kk + 8 + 2 * t);
        mma_bf16(acc, a0, a1, a2, a3, b0, b1);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) out[i] = __float2int_rn(acc[i]);
}

__device__ __forceinline__ __nv_bfloat16 bf(int v) { return __int2bfloat16_rn(v); }

struct LearnedParams {
    const uint8_t *bits;
    uint64_t model_off, chan_off, grp_sec, pay_off, pay_len;
    uint32_t L, G, n_rows;
    float *out;
    const uint32_t *out_index;
    int *status;
};

// Pipelined decoder: 16 producer warps compute, step by step (Gaussian i, channel c), the
// 32 lanes' frequency tables -- layer 1 on the ALU, layers 2-3 as int8 mma.sync, the
// integer softmax -- and store them as u16 cumulative tables in a ring of kNB buffers; one
// consumer warp runs the 32 rANS chains, binary-searching its lane's table.  Only the search
// is on the sequential chain; the context of step (i+1, c) needs only (i, c), 56 steps back,
// so producers run up to kNB steps ahead.  Hand-offs use mbarriers with bounded waits.
constexpr int kPW = 16;                  // producer warps
constexpr int kPT = 32 * kPW;            // producer threads
constexpr int kLT = kPT + 32;            // + consumer warp
constexpr int kNB = 4;                   // pipeline depth (steps)
constexpr uint32_t kWaitLimit = 1u << 24;

struct LSmem2 {
    int8_t w1[64 * 4];
    int32_t b1[kNChan * 64];
    alignas(16) __nv_bfloat16 w2[64 * kBS];
    int32_t b2[64];
    alignas(16) __nv_bfloat16 w3[256 * kBS];
    int32_t b3[256];
    uint32_t exp2q[256];
    alignas(16) __nv_bfloat16 h1[32 * kBS];
    alignas(16) __nv_bfloat16 h2[32 * kBS];
    uint8_t ctx[32 * 4 * kNChan];            // [lane][ring row][channel]
    alignas(16) uint16_t cdf[kNB][32][256];  // cumulative frequency of each symbol
    alignas(16) uint16_t win[kWinWords];     // consumer's word-stream window
    int32_t red_max[8][32];
    int32_t red_idx[8][32];
    uint32_t red_sum[8][32];
    uint32_t red_T[8][32];
    uint32_t R[32];
    uint32_t nrows[32];
    uint64_t row0[32];
    float step[kNChan], offset[kNChan];
    alignas(8) uint64_t full[kNB], empty[kNB];
    int32_t m1, sh1, m2, sh2;
    uint32_t ms, ss;
    int bad;
    int abort_;
};
static_assert(offsetof(LSmem2, cdf) % 16 == 0 && offsetof(LSmem2, win) % 16 == 0, "alignment");

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase of `parity` to complete; false on timeout or abort.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_) {
    for (uint32_t it = 0; it < kWaitLimit; ++it) {
        if (mbar_test(bar, parity)) return true;
        if (*abort_) return false;
        if (it > 64) __nanosleep(64);
    }
    return false;
}
__device__ __forceinline__ void producer_sync() {
    asm volatile("bar.sync 1, %0;" ::"r"(kPT) : "memory");
}

__device__ bool load_model2(LSmem2 &S, const uint8_t *m, int *status) {
    const int tid = threadIdx.x;
    if (tid == 0) {
        const int32_t *h = reinterpret_cast<const int32_t *>(m);
        S.m1 = h[0]; S.sh1 = h[1]; S.m2 = h[2]; S.sh2 = h[3];
        S.ms = (uint32_t)h[4]; S.ss = (uint32_t)h[5];
        S.bad = !(S.sh1 >= 1 && S.sh1 <= 47 && S.sh2 >= 1 && S.sh2 <= 47 && S.m1 >= 0 && S.m2 >= 0 &&
                  S.ms >= 1 && S.ms < (1u << 24) && S.ss <= 24);
        S.abort_ = 0;
    }
    const int32_t *b1 = reinterpret_cast<const int32_t *>(m + kMB_B1);
    const int32_t *b2 = reinterpret_cast<const int32_t *>(m + kMB_B2);
    const int32_t *b3 = reinterpret_cast<const int32_t *>(m + kMB_B3);
    bool badb = false;
    for (int i = tid; i < kNChan * 64; i += kLT) {
        S.b1[i] = b1[i];
        badb |= (b1[i] >= (1 << 24) || b1[i] <= -(1 << 24));
    }
    for (int i = tid; i < 64; i += kLT) {
        S.b2[i] = b2[i];
        badb |= (b2[i] >= (1 << 24) || b2[i] <= -(1 << 24));
    }
    for (int i = tid; i < 256; i += kLT) {
        S.b3[i] = b3[i];
        badb |= (b3[i] >= (1 << 24) || b3[i] <= -(1 << 24));
        S.exp2q[i] = kExp2Q[i];
        S.w1[i] = (int8_t)m[kMB_W1 + i];
    }
    for (int i = tid; i < 64 * 64; i += kLT) S.w2[(i >> 6) * kBS + (i & 63)] = bf((int8_t)m[kMB_W2 + i]);
    for (int i = tid; i < 256 * 64; i += kLT) S.w3[(i >> 6) * kBS + (i & 63)] = bf((int8_t)m[kMB_W3 + i]);
    __syncthreads();
    if (badb) atomicOr(&S.bad, 1);
    __syncthreads();
    if (S.bad) {
        if (tid == 0) set_status(status, SGS_E_CORRUPT);
        return false;
    }
    return true;
}

// One producer step: frequency tables of the 32 lanes' rows for (i, c) into cdf[b].
__device__ __forceinline__ void produce_step(LSmem2 &S, uint32_t i, int c, int b) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    // layer 1 (ALU): row r = tid >> 4, outputs 4 (tid & 15) .. +3
    {
        const int r = tid >> 4, o0 = (tid & 15) * 4;
        int32_t u[4];
#pragma unroll
        for (int j = 1; j <= 4; ++j)
            u[j - 1] = (i >= (uint32_t)j) ? (int32_t)S.ctx[(r * 4 + ((i - j) & 3)) * kNChan + c] - 128 : 0;
#pragma unroll
        for (int o = o0; o < o0 + 4; ++o) {
            int32_t acc = S.b1[c * 64 + o];
#pragma unroll
            for (int j = 0; j < 4; ++j) acc += (int32_t)S.w1[o * 4 + j] * u[j];
            S.h1[r * kBS + o] = bf(requant(acc, S.m1, S.sh1));
        }
    }
    producer_sync();
    // layer 2: warp -> rows 16 (warp & 1), cols 8 (warp >> 1)
    {
        const int r0 = (warp & 1) * 16, n0 = (warp >> 1) * 8;
        int32_t acc[4] = {0, 0, 0, 0};
        tile_16x8x64(acc, S.h1, r0, S.w2, n0, g, t);
        const int col = n0 + 2 * t;
        S.h2[(r0 + g) * kBS + col] = bf(requant(acc[0] + S.b2[col], S.m2, S.sh2));
        S.h2[(r0 + g) * kBS + col + 1] = bf(requant(acc[1] + S.b2[col + 1], S.m2, S.sh2));
        S.h2[(r0 + g + 8) * kBS + col] = bf(requant(acc[2] + S.b2[col], S.m2, S.sh2));
        S.h2[(r0 + g + 8) * kBS + col + 1] = bf(requant(acc[3] + S.b2[col + 1], S.m2, S.sh2));
    }
    producer_sync();
    // layer 3: warp -> rows 16 (warp & 1), column slice cs = warp >> 1 (32 columns)
    const int r0 = (warp & 1) * 16, cs = warp >> 1;
    const int rA = r0 + g, rB = r0 + g + 8;
    int32_t z[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        const int n0 = cs * 32 + nt * 8;
        z[nt][0] = z[nt][1] = z[nt][2] = z[nt][3] = 0;
        tile_16x8x64(z[nt], S.h2, r0, S.w3, n0, g, t);
        const int col = n0 + 2 * t;
        z[nt][0] += S.b3[col];
        z[nt][1] += S.b3[col + 1];
        z[nt][2] += S.b3[col];
        z[nt][3] += S.b3[col + 1];
    }
    // (a) row max, lowest argmax
    {
        int32_t mA = z[0][0], mB = z[0][2];
        int32_t iA = cs * 32 + 2 * t, iB = iA;
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                const int32_t col = cs * 32 + nt * 8 + 2 * t + v;
                if (z[nt][v] > mA) { mA = z[nt][v]; iA = col; }
                if (z[nt][2 + v] > mB) { mB = z[nt][2 + v]; iB = col; }
            }
#pragma unroll
        for (int o = 1; o <= 2; o <<= 1) {
            const int32_t omA = __shfl_xor_sync(0xffffffffu, mA, o), oiA = __shfl_xor_sync(0xffffffffu, iA, o);
            const int32_t omB = __shfl_xor_sync(0xffffffffu, mB, o), oiB = __shfl_xor_sync(0xffffffffu, iB, o);
            if (omA > mA || (omA == mA && oiA < iA)) { mA = omA; iA = oiA; }
            if (omB > mB || (omB == mB && oiB < iB)) { mB = omB; iB = oiB; }
        }
        if (t == 0) {
            S.red_max[cs][rA] = mA; S.red_idx[cs][rA] = iA;
            S.red_max[cs][rB] = mB; S.red_idx[cs][rB] = iB;
        }
    }
    producer_sync();
    int32_t zmA = S.red_max[0][rA], amA = S.red_idx[0][rA];
    int32_t zmB = S.red_max[0][rB], amB = S.red_idx[0][rB];
#pragma unroll
    for (int q = 1; q < 8; ++q) {
        if (S.red_max[q][rA] > zmA) { zmA = S.red_max[q][rA]; amA = S.red_idx[q][rA]; }
        if (S.red_max[q][rB] > zmB) { zmB = S.red_max[q][rB]; amB = S.red_idx[q][rB]; }
    }
    // (b) e_k and partial sums
    {
        uint32_t sA = 0, sB = 0;
        const uint32_t ms = S.ms, ss = S.ss;
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const uint32_t d = (uint32_t)((v < 2 ? zmA : zmB) - z[nt][v]);
                const uint64_t tt = ((uint64_t)d * ms) >> ss;
                const uint32_t tk = tt > 6144 ? 6144u : (uint32_t)tt;
                const uint32_t e = S.exp2q[tk & 255] >> (tk >> 8);
                z[nt][v] = (int32_t)e;
                if (v < 2) sA += e; else sB += e;
            }
        sA += __shfl_xor_sync(0xffffffffu, sA, 1);
        sA += __shfl_xor_sync(0xffffffffu, sA, 2);
        sB += __shfl_xor_sync(0xffffffffu, sB, 1);
        sB += __shfl_xor_sync(0xffffffffu, sB, 2);
        if (t == 0) { S.red_sum[cs][rA] = sA; S.red_sum[cs][rB] = sB; }
    }
    producer_sync();
    // R = floor(65280 * 2^32 / E) once per row (32 threads), then shared
    if (tid < 32) {
        uint64_t E = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) E += S.red_sum[q][tid];
        S.R[tid] = (uint32_t)((65280ull << 32) / E);
    }
    producer_sync();
    const uint32_t RA = S.R[rA], RB = S.R[rB];
    // (c) floor terms and per-slice sums
    {
        uint32_t TA = 0, TB = 0;
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const uint32_t fl = __umulhi((uint32_t)z[nt][v], v < 2 ? RA : RB);
                z[nt][v] = (int32_t)fl;
                if (v < 2) TA += fl; else TB += fl;
            }
        TA += __shfl_xor_sync(0xffffffffu, TA, 1);
        TA += __shfl_xor_sync(0xffffffffu, TA, 2);
        TB += __shfl_xor_sync(0xffffffffu, TB, 1);
        TB += __shfl_xor_sync(0xffffffffu, TB, 2);
        if (t == 0) { S.red_T[cs][rA] = TA; S.red_T[cs][rB] = TB; }
    }
    producer_sync();
    // (d) cumulative frequencies: f_k = 1 + floor term (+ remainder at the argmax)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        const int r = half ? rB : rA;
        const int32_t am = half ? amB : amA;
        uint32_t T[8], Tsum = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) { T[q] = S.red_T[q][r]; Tsum += T[q]; }
        const uint32_t rem = 65536u - 256u - Tsum;
        uint32_t cum = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (q < cs) cum += 32u + T[q] + ((am >> 5) == q ? rem : 0u);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int k0 = cs * 32 + nt * 8 + 2 * t;
            const uint32_t f0 = 1u + (uint32_t)z[nt][2 * half] + (k0 == am ? rem : 0u);
            const uint32_t f1 = 1u + (uint32_t)z[nt][2 * half + 1] + (k0 + 1 == am ? rem : 0u);
            const uint32_t mine = f0 + f1;
            uint32_t incl = mine;
            const uint32_t n1 = __shfl_up_sync(0xffffffffu, incl, 1, 4);
            if (t >= 1) incl += n1;
            const uint32_t n2 = __shfl_up_sync(0xffffffffu, incl, 2, 4);
            if (t >= 2) incl += n2;
            const uint32_t tsum = __shfl_sync(0xffffffffu, incl, 3, 4);
            const uint32_t start = cum + incl - mine;
            // cdf[k] <= 65535 for every k <= 255 since every f >= 1
            *reinterpret_cast<uint32_t *>(&S.cdf[b][r][k0]) = (start & 0xFFFFu) | ((start + f0) << 16);
            cum += tsum;
        }
    }
}

// The consumer warp: the group's 32 rANS chains over K steps.
__device__ __forceinline__ void consume(const LearnedParams &p, LSmem2 &S, uint32_t grp, int nl,
                                        uint32_t K, volatile int *abort_) {
    const int lane = threadIdx.x & 31;
    GroupStream gs;
    uint32_t x = 0x10000u;
    group_open(p.bits, p.grp_sec, p.pay_off, p.pay_len, p.G, grp, nl, lane, gs, x, S.win);
    bool aborted = false;
    for (uint32_t k = 0; k < K; ++k) {
        const int b = (int)(k % kNB);
        // every lane acquires the producers' release of buffer b
        const bool ok = __all_sync(0xffffffffu, mbar_wait(&S.full[b], (k / kNB) & 1, abort_));
        if (!ok) {
            if (lane == 0) { *abort_ = 1; set_status(p.status, SGS_E_TIMEOUT); }
            aborted = true;
            break;
        }
        const uint32_t i = k / kNChan;
        const int c = (int)(k - i * kNChan);
        const bool live = lane < nl && i < S.nrows[lane];
        if (live) {
            const uint32_t slot = x & 0xFFFFu;
            const uint16_t *cdf = S.cdf[b][lane];
            uint32_t s = 0;
#pragma unroll
            for (uint32_t st = 128; st > 0; st >>= 1)
                if (cdf[s + st] <= slot) s += st;
            const uint32_t lo = cdf[s];
            const uint32_t hi = s < 255 ? cdf[s + 1] : 65536u;
            x = (hi - lo) * (x >> 16) + slot - lo;
            S.ctx[(lane * 4 + (i & 3)) * kNChan + c] = (uint8_t)s;
            const uint64_t row = S.row0[lane] + i;
            const uint64_t col = p.out_index ? (uint64_t)p.out_index[row] : row;
            p.out[(uint64_t)c * p.n_rows + col] = dequant(s, S.step[c], S.offset[c]);
        }
        group_refill(gs, x, live);
        __syncwarp();
        if (lane == 0 && k + kNB < K) mbar_arrive(&S.empty[b]);
    }
    if (!aborted) {
        const bool bad = gs.bad || (lane < nl && x != 0x10000u) || (gs.ptr != gs.n_words);
        if (bad) set_status(p.status, SGS_E_CORRUPT);
    }
}

__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// One group of 32 lanes.  reload = false: the CTA's previous group was of the same scene,
// whose model is still in shared memory (S.bad records whether it was refused).
__device__ __forceinline__ void learned_body(const LearnedParams &p, uint32_t grp, bool reload) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    LSmem2 &S = *reinterpret_cast<LSmem2 *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nl = (int)min(32u, p.L - grp * 32);
    if (reload) {
        if (!load_model2(S, p.bits + p.model_off, p.status)) return;
    } else {
        if (S.bad) return;
        if (tid == 0) S.abort_ = 0;
    }
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
    for (int i = tid; i < 32 * 4 * kNChan; i += kLT) S.ctx[i] = 0;
    if (tid == 0) {
        for (int b = 0; b < kNB; ++b) {
            mbar_init(&S.full[b], kPW);
            mbar_init(&S.empty[b], 1);
        }
    }
    __syncthreads();
    uint32_t maxrows = 0;
    for (int r = 0; r < 32; ++r) maxrows = max(maxrows, S.nrows[r]);
    const uint32_t K = maxrows * kNChan;  // steps
    volatile int *abort_ = &S.abort_;

    if (warp < kPW) {
        // ---------------- producers
        for (uint32_t k = 0; k < K; ++k) {
            const int b = (int)(k % kNB);
            // every producer thread acquires the consumer's release of buffer b (and with it
            // the tokens the consumer wrote into the context ring)
            if (k >= (uint32_t)kNB && !mbar_wait(&S.empty[b], ((k / kNB) - 1) & 1, abort_)) {
                *abort_ = 1;
                if (tid == 0) set_status(p.status, SGS_E_TIMEOUT);
            }
            producer_sync();  // uniform exit: every producer sees the same abort flag
            if (*abort_) break;
            const uint32_t i = k / kNChan;
            produce_step(S, i, (int)(k - i * kNChan), b);
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.full[b]);
        }
    } else {
        consume(p, S, grp, nl, K, abort_);
    }
    // every hand-off is over: retire the barriers (a persistent CTA initialises them again)
    __syncthreads();
    if (tid == 0)
        for (int b = 0; b < kNB; ++b) {
            mbar_inval(&S.full[b]);
            mbar_inval(&S.empty[b]);
        }
}

__global__ void __launch_bounds__(kLT, 1) k_learned_decode(LearnedParams p) { learned_body(p, blockIdx.x, true); }

__global__ void __launch_bounds__(kLT, 1) k_learned_multi(MultiArgs m) {
    run_items<LearnedParams>(m, [](const LearnedParams &p, uint32_t vb, uint32_t, bool same) {
        learned_body(p, vb, !same);
    });
}

size_t learned_work_bytes(const sgs_scene_info &) { return 0; }


static uint32_t make_learned(const uint8_t *bits, const sgs_scene_info &info, const sgs_scene_out &out,
                             int *status, LearnedParams *pp) {
    LearnedParams &p = *pp;
    memset(&p, 0, sizeof(p));
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
    return info.n_rows ? p.G : 0;
}

static cudaError_t learned_smem_limit(const void *kernel, bool *done) {
    if (*done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(LSmem2));
    if (e == cudaSuccess) *done = true;
    return e;
}

cudaError_t launch_learned_decode(const uint8_t *bits, const sgs_scene_info &info,
                                  const sgs_scene_out &out, uint8_t *, int *status, cudaStream_t st) {
    LearnedParams p;
    const uint32_t grid = make_learned(bits, info, out, status, &p);
    if (grid == 0) return cudaSuccess;
    static bool set = false;
    cudaError_t e = learned_smem_limit(reinterpret_cast<const void *>(k_learned_decode), &set);
    if (e != cudaSuccess) return e;
    k_learned_decode<<<grid, kLT, sizeof(LSmem2), st>>>(p);
    return cudaGetLastError();
}

uint32_t stage_learned(const SceneRef &r, void *par) {
    if (r.info->mode != SGS_MODE_LEARNED) return 0;
    LearnedParams p;
    const uint32_t n = make_learned(r.bits, *r.info, *r.out, r.status, &p);
    memcpy(par, &p, sizeof(p));
    return n;
}
size_t stage_learned_bytes() { return sizeof(LearnedParams); }
cudaError_t launch_learned_multi(const MultiArgs &m, cudaStream_t st) {
    static bool set = false;
    cudaError_t e = learned_smem_limit(reinterpret_cast<const void *>(k_learned_multi), &set);
    if (e != cudaSuccess) return e;
    return launch_persistent(k_learned_multi, kLT, sizeof(LSmem2), m, st);
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
