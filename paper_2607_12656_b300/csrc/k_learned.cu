// Learned-model attribute decoding on sm_103a: rANS driven by the local autoregressive
// context model (Sec. 3.4.2 "Autoregressive Prediction Coding", made small and integer).
//
// Model (frozen, integer): for token (i, c) of a lane, u_j = s_{i-j,c} - 128 (j = 1..4, 0 past
// the lane start), h1 = rq(W1 u + B1[c]), h2 = rq(W2 h1 + b2), z = W3 h2 + b3 with
// rq(a) = clamp((a m + 2^(sh-1)) >> sh, 0, 127); integer softmax
//   t_k = min(((zmax - z_k) ms) >> ss, 6144),  e_k = EXP2Q[t_k & 255] >> (t_k >> 8),
//   R = floor(65280 * 2^32 / sum e),  f_k = 1 + floor(e_k R / 2^32),  remainder to argmax z.
//
// Decoder: one CTA per group of 32 lanes, walking the group's tokens in stream order
// (Gaussian i, channel c): 12 producer warps compute the steps' cumulative tables ahead of
// one consumer warp that advances the 32 rANS states and refills them from the group's
// shared word stream (details at the pipeline's constants below).
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>
#include <cuda_bf16.h>

#include <vector>

#include "exp2q_table.h"
#include "sgs_device.cuh"
#include "sgs_mma.cuh"
#include "sgs_internal.h"

namespace sgs {

__constant__ uint32_t kExp2Q[256] = {SGS_EXP2Q_VALUES};

// The decoder expands e(t) = EXP2Q[t & 255] >> (t >> 8) into one table over t = 0 .. kETop:
// e(t) = 0 for every t >= kETop (EXP2Q[0] = 2^23 is the only entry that survives a shift by
// 23, and nothing survives 24), so clamping t at kETop instead of 6144 leaves every e_k as
// it is and turns the lookup into a single load.
constexpr int kETop = 23 * 256 + 1;
constexpr uint32_t kExp2QHost[256] = {SGS_EXP2Q_VALUES};
constexpr bool exp_tail_zero() {
    for (int t = kETop; t <= 6144; ++t)
        if ((kExp2QHost[t & 255] >> (t >> 8)) != 0u) return false;
    return (kExp2QHost[0] >> 23) == 1u;
}
static_assert(exp_tail_zero(), "EXP2Q vanishes from 23 * 256 + 1 on");


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

__device__ __forceinline__ uint32_t lds32(const __nv_bfloat16 *p) {
    return *reinterpret_cast<const uint32_t *>(p);
}

// The four A fragments of one m16n8k16 tile (16 x 16 bf16, row-major, rows kBS apart) with
// one ldmatrix: lane L gives the address of row (L & 7) + 8 ((L >> 3) & 1), columns
// 8 (L >> 4) .. +7, of the tile starting at A.
__device__ __forceinline__ void ldsm_a(const __nv_bfloat16 *A, uint32_t &a0, uint32_t &a1, uint32_t &a2,
                                       uint32_t &a3) {
    const int lane = threadIdx.x & 31;
    const __nv_bfloat16 *p = A + ((lane & 7) + 8 * ((lane >> 3) & 1)) * kBS + 8 * (lane >> 4);
    const uint32_t addr = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(a0), "=r"(a1), "=r"(a2), "=r"(a3)
                 : "r"(addr));
}

struct LearnedParams {
    const uint8_t *bits;
    uint64_t model_off, chan_off, grp_sec, pay_off, pay_len;
    uint32_t L, G, n_rows;
    float *out;
    const uint32_t *out_index;
    int *status;
    uint32_t wait_limit;  // polls of each bounded mbarrier wait before it gives up
};

// Pipelined decoder: kPW producer warps compute the frequency tables of the steps (Gaussian i,
// channel c) ahead of one consumer warp that runs the group's 32 rANS chains.  Each producer
// warp owns 8 of a step's 32 contexts and computes them end to end on its own -- layer 1 on
// the ALU, layers 2-3 as bf16 mma.sync with the contexts as the N dimension, the integer
// softmax reduced with shuffles among the 8 lanes that share a context -- so producers never
// synchronise with each other.  Four warps make one step; the kPW warps work on kSW steps
// at once, writing u16 cumulative tables into a ring of kNB steps.  The context of step (i, c)
// needs only (i-1 .. i-4, c), at least 56 steps back, so the ring's release by the consumer
// also publishes the tokens a producer reads.  Hand-offs are mbarriers with bounded waits.
constexpr int kPW = 12;                  // producer warps
constexpr int kPT = 32 * kPW;            // producer threads
constexpr int kLT = kPT + 32;            // + consumer warp
constexpr int kNB = 7;                   // ring depth (steps)
constexpr int kQW = 4;                   // warps per step (8 contexts each)
constexpr int kSW = kPW / kQW;           // steps in flight
constexpr uint32_t kWaitLimit = kDefaultWaitPolls;
constexpr int kCS = 264;                 // cdf row stride (u16): rows 528 B apart spread the banks
static_assert(kNB >= kSW && kNB <= kNChan, "ring");

struct LSmem2 {
    int8_t w1[64 * 4];
    int32_t b1[kNChan * 64];
    alignas(16) __nv_bfloat16 w2[64 * kBS];
    int32_t b2[64];
    alignas(16) __nv_bfloat16 w3[256 * kBS];
    int32_t b3m[256];                           // b3 - 0x4B400000 (see layer 3)
    uint32_t etab[kETop + 1];                   // e(t), t = 0 .. kETop
    alignas(16) __nv_bfloat16 h2t[kPW][8 * kBS];  // per warp: layer-2 output, [context][unit]
    uint8_t ctx[32 * 4 * kNChan];               // [lane][ring row][channel]
    alignas(16) uint16_t cdf[kNB][32][kCS];     // cumulative frequency of each symbol
    alignas(16) uint16_t win[kWinWords];        // consumer's word-stream window
    uint32_t nrows[32];
    uint64_t row0[32];
    float step[kNChan], offset[kNChan];
    alignas(8) uint64_t full[kNB], empty[kNB];
    int32_t m1, sh1, m2, sh2;
    uint32_t ms, ss;
    uint32_t dcap;  // smallest d with (d ms) >> ss >= kETop, saturated at 2^32 - 1
    int bad;
    int abort_;
};
static_assert(offsetof(LSmem2, cdf) % 16 == 0 && offsetof(LSmem2, win) % 16 == 0 &&
              offsetof(LSmem2, h2t) % 16 == 0, "alignment");
static_assert(sizeof(LSmem2) <= 227 * 1024, "shared memory");

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
// Bounded wait for the phase of `parity` to complete: at most `limit` polls; false on
// timeout or abort.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_,
                                          uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it) {
        if (mbar_test(bar, parity)) return true;
        if (*abort_) return false;
        if (it > 64) __nanosleep(64);
    }
    return false;
}
__device__ bool load_model2(LSmem2 &S, const uint8_t *m, int *status) {
    const int tid = threadIdx.x;
    if (tid == 0) {
        const int32_t *h = reinterpret_cast<const int32_t *>(m);
        S.m1 = h[0]; S.sh1 = h[1]; S.m2 = h[2]; S.sh2 = h[3];
        S.ms = (uint32_t)h[4]; S.ss = (uint32_t)h[5];
        S.bad = !(S.sh1 >= 1 && S.sh1 <= 47 && S.sh2 >= 1 && S.sh2 <= 47 && S.m1 >= 0 && S.m2 >= 0 &&
                  S.ms >= 1 && S.ms < (1u << 24) && S.ss <= 24);
        if (!S.bad) {
            const uint64_t dc = (((uint64_t)kETop << S.ss) + S.ms - 1) / S.ms;
            S.dcap = dc > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)dc;
        }
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
        S.b3m[i] = b3[i] - 0x4B400000;
        badb |= (b3[i] >= (1 << 24) || b3[i] <= -(1 << 24));
        S.w1[i] = (int8_t)m[kMB_W1 + i];
    }
    for (int t = tid; t <= kETop; t += kLT) S.etab[t] = kExp2Q[t & 255] >> (t >> 8);
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

// One warp's share of step (i, c): the frequency tables of lanes 8q .. 8q+7 into cdf[b].
// mma.sync m16n8k16 fragments: lane = 4 g + t; A rows g, g+8, B column g, D rows g, g+8 x
// columns 2t, 2t+1.  Layers 2 and 3 compute W h^T, so the 8 contexts are the columns.
__device__ __forceinline__ void produce_pass(LSmem2 &S, uint32_t i, int c, int b, int q) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    // ---- layer 1 for context g: the 16 units this lane feeds into layer 2's B fragments
    uint32_t bf2[4][2];
    {
        const int L = 8 * q + g;
        // u_j = token_{i-j} - 128 as packed int8 (0 before the lane's first row)
        uint32_t up = 0;
#pragma unroll
        for (int j = 1; j <= 4; ++j) {
            const uint32_t tok = (i >= (uint32_t)j) ? S.ctx[(L * 4 + ((i - j) & 3)) * kNChan + c] : 128u;
            up |= (tok ^ 0x80u) << (8 * (j - 1));
        }
        const int32_t *b1 = S.b1 + c * 64;
        const int32_t *w1 = reinterpret_cast<const int32_t *>(S.w1);  // row o: 4 int8 weights
        const int32_t m1 = S.m1, sh1 = S.sh1;
#pragma unroll
        for (int kt = 0; kt < 4; ++kt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                int32_t v[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int o = 16 * kt + 8 * h + 2 * t + e;
                    v[e] = requant(__dp4a(w1[o], (int32_t)up, b1[o]), m1, sh1);
                }
                bf2[kt][h] = pack_bf16(v[0], v[1]);
            }
    }
    // ---- layer 2: D[unit][context] = W2 h1^T; requantised into this warp's transpose buffer
    __nv_bfloat16 *h2t = S.h2t[warp];
    {
        const int32_t m2 = S.m2, sh2 = S.sh2;
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int kt = 0; kt < 4; ++kt) {
                uint32_t a0, a1, a2, a3;
                ldsm_a(S.w2 + 16 * mt * kBS + 16 * kt, a0, a1, a2, a3);
                mma_bf16(acc, a0, a1, a2, a3, bf2[kt][0], bf2[kt][1]);
            }
            const int r0 = 16 * mt + g, r1 = r0 + 8;
            h2t[(2 * t) * kBS + r0] = bf(requant(__float2int_rn(acc[0]) + S.b2[r0], m2, sh2));
            h2t[(2 * t + 1) * kBS + r0] = bf(requant(__float2int_rn(acc[1]) + S.b2[r0], m2, sh2));
            h2t[(2 * t) * kBS + r1] = bf(requant(__float2int_rn(acc[2]) + S.b2[r1], m2, sh2));
            h2t[(2 * t + 1) * kBS + r1] = bf(requant(__float2int_rn(acc[3]) + S.b2[r1], m2, sh2));
        }
    }
    __syncwarp();
    uint32_t bf3[4][2];
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
        bf3[kt][0] = lds32(h2t + g * kBS + 16 * kt + 2 * t);
        bf3[kt][1] = lds32(h2t + g * kBS + 16 * kt + 2 * t + 8);
    }
    // ---- layer 3: z[symbol][context]; this lane holds symbols 16 mt + g (+8) of contexts
    //      2t (z[mt][0], z[mt][2]) and 2t+1 (z[mt][1], z[mt][3])
    int32_t z[16][4];
#pragma unroll
    for (int mt = 0; mt < 16; ++mt) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < 4; ++kt) {
            uint32_t a0, a1, a2, a3;
            ldsm_a(S.w3 + 16 * mt * kBS + 16 * kt, a0, a1, a2, a3);
            mma_bf16(acc, a0, a1, a2, a3, bf3[kt][0], bf3[kt][1]);
        }
        // acc is an integer of magnitude below 2^21, so acc + 1.5 2^23 is exact and its bit
        // pattern is 0x4B400000 + acc: the conversion is one full-rate add
        const int32_t b30 = S.b3m[16 * mt + g], b31 = S.b3m[16 * mt + g + 8];
#pragma unroll
        for (int v = 0; v < 4; ++v)
            z[mt][v] = __float_as_int(__fadd_rn(acc[v], 12582912.0f)) + (v < 2 ? b30 : b31);
    }
    // ---- integer softmax of contexts 2t (e = 0) and 2t+1 (e = 1); the 8 lanes g = 0..7 with
    //      this t hold all 256 symbols of both
    int32_t zmax[2], amax[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        zmax[e] = z[0][e];
        amax[e] = g;
#pragma unroll
        for (int mt = 0; mt < 16; ++mt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int32_t v = z[mt][2 * h + e];
                const int32_t k = 16 * mt + 8 * h + g;  // ascending over (mt, h): strict > keeps the lowest
                if (v > zmax[e]) { zmax[e] = v; amax[e] = k; }
            }
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) {
            const int32_t om = __shfl_xor_sync(0xffffffffu, zmax[e], o);
            const int32_t oa = __shfl_xor_sync(0xffffffffu, amax[e], o);
            if (om > zmax[e] || (om == zmax[e] && oa < amax[e])) { zmax[e] = om; amax[e] = oa; }
        }
    }
    // e_k = etab[min((min(d_k, dcap) ms) >> ss, kETop)]: for d_k >= dcap both t_k and the
    // clamped t are at least kETop, where e vanishes; below dcap the product shifted by ss is
    // under 2^32 and the clamp does nothing.  z is overwritten with e_k.
    const uint32_t ms = S.ms, ss = S.ss, dcap = S.dcap;
    uint32_t E[2] = {0u, 0u};
#pragma unroll
    for (int mt = 0; mt < 16; ++mt)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int e = v & 1;
            const uint32_t d = min((uint32_t)(zmax[e] - z[mt][v]), dcap);
            const uint32_t tt = (uint32_t)(((uint64_t)d * ms) >> ss);
            const uint32_t ek = S.etab[min(tt, (uint32_t)kETop)];
            z[mt][v] = (int32_t)ek;
            E[e] += ek;
        }
    uint32_t R[2], Tf[2] = {0u, 0u};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) E[e] += __shfl_xor_sync(0xffffffffu, E[e], o);
        R[e] = (uint32_t)((65280ull << 32) / E[e]);
    }
    // f_k = 1 + floor(e_k R / 2^32) stored in symbol order; their sum gives the remainder,
    // which one lane per context then adds at the argmax
    uint16_t *cdfw = &S.cdf[b][8 * q][0];  // this warp's 8 contexts, rows kCS apart
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        uint16_t *row = cdfw + (2 * t + e) * kCS;
#pragma unroll
        for (int mt = 0; mt < 16; ++mt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t f = __umulhi((uint32_t)z[mt][2 * h + e], R[e]) + 1u;
                Tf[e] += f;
                row[16 * mt + 8 * h + g] = (uint16_t)f;
            }
    }
    uint32_t pk[2];  // (remainder << 8) | argmax of context 2t + e
#pragma unroll
    for (int e = 0; e < 2; ++e) {
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) Tf[e] += __shfl_xor_sync(0xffffffffu, Tf[e], o);
        pk[e] = ((65536u - Tf[e]) << 8) | (uint32_t)amax[e];
    }
    {
        // context n = lane (lanes 0..7) is held by the lanes with t = n / 2, component n % 2
        const uint32_t p0 = __shfl_sync(0xffffffffu, pk[0], (lane & 7) >> 1);
        const uint32_t p1 = __shfl_sync(0xffffffffu, pk[1], (lane & 7) >> 1);
        const uint32_t p = (lane & 1) ? p1 : p0;
        __syncwarp();
        if (lane < 8) {
            uint16_t *fa = cdfw + lane * kCS + (p & 255u);
            *fa = (uint16_t)(*fa + (p >> 8));  // f <= 65281
        }
    }
    __syncwarp();
    {
        // lane -> context lane & 7, quarter lane >> 3 (64 symbols, 8 uint4); the 8 lanes of a
        // quarter-warp touch 8 rows at the same column: 528-byte rows put them in 8 bank groups
        const int n = lane & 7, qq = lane >> 3;
        uint16_t *seg = cdfw + n * kCS + qq * 64;
        // Every f >= 1 and a context's f sum to 2^16, so the even and the odd halves of a
        // segment each sum below 2^16: the words add without carries between the halves, and
        // so do the two halves of one word (f0 + f1 < 2^16).
        uint4 w[8];
        uint32_t sw = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            w[j] = reinterpret_cast<const uint4 *>(seg)[j];
            sw += (w[j].x + w[j].y) + (w[j].z + w[j].w);
        }
        const uint32_t sum = (sw & 0xFFFFu) + (sw >> 16);
        uint32_t incl = sum;  // scan over the 4 quarters of context n (lanes n, n+8, n+16, n+24)
        const uint32_t n1 = __shfl_up_sync(0xffffffffu, incl, 8);
        if (qq >= 1) incl += n1;
        const uint32_t n2 = __shfl_up_sync(0xffffffffu, incl, 16);
        if (qq >= 2) incl += n2;
        uint32_t run = incl - sum;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            uint32_t *h = reinterpret_cast<uint32_t *>(&w[j]);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                // (run, run + f0) with run + f0 <= 65535 below symbol 256; then run += f0 + f1
                const uint32_t hv = h[k];
                h[k] = run * 0x10001u + (hv << 16);
                run += (hv * 0x10001u) >> 16;
            }
            reinterpret_cast<uint4 *>(seg)[j] = w[j];
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
        const bool ok = __all_sync(0xffffffffu, mbar_wait(&S.full[b], (k / kNB) & 1, abort_, p.wait_limit));
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
        if (k + kNB < K) mbar_arrive(&S.empty[b]);
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
            mbar_init(&S.full[b], 32 * kQW);  // every lane of the step's producer warps
            mbar_init(&S.empty[b], 32);       // every consumer lane
        }
    }
    __syncthreads();
    uint32_t maxrows = 0;
    for (int r = 0; r < 32; ++r) maxrows = max(maxrows, S.nrows[r]);
    const uint32_t K = maxrows * kNChan;  // steps
    volatile int *abort_ = &S.abort_;

    if (warp < kPW) {
        // ---------------- producers: warp w makes contexts 8 (w % 4) .. +7 of steps w / 4 + 4 j
        const int q = warp % kQW;
        for (uint32_t k = warp / kQW; k < K; k += kSW) {
            const int b = (int)(k % kNB);
            // every lane acquires the consumer's release of buffer b (and with it the tokens
            // the consumer wrote into the context ring)
            const bool ok = k < (uint32_t)kNB || mbar_wait(&S.empty[b], ((k / kNB) - 1) & 1, abort_, p.wait_limit);
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0) { *abort_ = 1; set_status(p.status, SGS_E_TIMEOUT); }
                break;
            }
            const uint32_t i = k / kNChan;
            produce_pass(S, i, (int)(k - i * kNChan), b, q);
            mbar_arrive(&S.full[b]);
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
                             int *status, LearnedParams *pp, uint32_t wait_limit = kWaitLimit) {
    LearnedParams &p = *pp;
    memset(&p, 0, sizeof(p));
    p.wait_limit = wait_limit ? wait_limit : kWaitLimit;
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
                                  const sgs_scene_out &out, uint8_t *, int *status, cudaStream_t st,
                                  uint32_t wait_limit) {
    LearnedParams p;
    const uint32_t grid = make_learned(bits, info, out, status, &p, wait_limit);
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

int rans_encode_device(const uint32_t *f, const uint32_t *cum, const std::vector<uint64_t> &lane_start,
                       std::vector<uint8_t> &grp, std::vector<uint8_t> &pay);

// Learned attribute coding on the device: the frozen model's f and cum of every token stay on
// the device for the interleaved rANS encoder.
int learned_encode_device(const uint8_t *model, const uint8_t *tokens, uint32_t n_rows, uint32_t lanes,
                          const std::vector<uint64_t> &lane_start, std::vector<uint8_t> &grp,
                          std::vector<uint8_t> &pay) {
    const uint64_t n = (uint64_t)n_rows * kNChan;
    uint8_t *dm = nullptr, *dt = nullptr;
    uint32_t *df = nullptr, *dc = nullptr;
    int rc = SGS_OK;
    if (cudaMalloc(&dm, SGS_MODEL_BYTES) != cudaSuccess || cudaMalloc(&dt, n ? n : 1) != cudaSuccess ||
        cudaMalloc(&df, 4 * (n ? n : 1)) != cudaSuccess || cudaMalloc(&dc, 4 * (n ? n : 1)) != cudaSuccess) {
        rc = SGS_E_NOMEM;
    } else if (cudaMemcpy(dm, model, SGS_MODEL_BYTES, cudaMemcpyHostToDevice) != cudaSuccess ||
               (n && cudaMemcpy(dt, tokens, n, cudaMemcpyHostToDevice) != cudaSuccess)) {
        rc = SGS_E_CUDA;
    } else {
        if (n) {
            const uint64_t blocks = (n + 255) / 256;
            k_learned_fc<<<(unsigned)(blocks < 148 * 64 ? blocks : 148 * 64), 256>>>(dm, dt, n_rows, lanes, df, dc);
            if (cudaGetLastError() != cudaSuccess) rc = SGS_E_CUDA;
        }
        if (rc == SGS_OK) rc = rans_encode_device(df, dc, lane_start, grp, pay);
    }
    cudaFree(dm);
    cudaFree(dt);
    cudaFree(df);
    cudaFree(dc);
    return rc;
}

}  // namespace sgs
