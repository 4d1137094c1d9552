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
// (Gaussian i, channel c).  Layer 3 of 128 contexts at a time runs on the fifth-generation
// tensor cores (tcgen05) into tensor memory, where a thread reads its context's 256 logits as
// one row; a consumer warp advances the 32 rANS states (roles at the decoder's constants below).
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>
#include <cuda_bf16.h>

#include <vector>

#include "exp2q_table.h"
#include "sgs_device.cuh"
#include "sgs_mma.cuh"
#include "sgs_tc.cuh"
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

// Layers 2 and 3 run on the tensor cores in bf16 with fp32 accumulation, and exactly so:
// int8 weights and activations in [0, 127] are exact in bf16, their products exact in fp32,
// and every partial sum of layer 2 (64 products) is an integer below 2^21.  Layer 3
// accumulates onto 1.5 2^23 in tensor memory, so every partial sum lies in [2^23, 2^24),
// where fp32 holds every integer, and the result's bit pattern is 0x4B400000 + the sum.
// (B300 has no tcgen05 int8 kind.)
constexpr int kBS = 72;  // layer-2 weight rows in shared memory (bf16, 64 used): conflict-free

__device__ __forceinline__ uint32_t lds32(const __nv_bfloat16 *p) {
    return *reinterpret_cast<const uint32_t *>(p);
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

// Decoder: one CTA per group of 32 lanes.  A tile is the 128 contexts of 4 channels x 32 lanes
// at one row i (tile (i, j): channels 4 j .. 4 j + 3), TMEM lane 32 q + l = channel 4 j + q of
// lane l.  Roles:
//   warp 0      the consumer: the group's 32 rANS chains in stream order (i, c), each step's
//               32 tables read from a ring of kNS steps; it writes the tokens, the outputs and
//               the token history the contexts of later rows read;
//   warp 1      allocates the tensor memory; its lane 0 issues layer 3 of every tile;
//   warps 2-5   layers 1 and 2 of a tile, warp w taking channel 4 j + w: layer 1 on the ALU,
//               layer 2 as mma.sync, requantised into one of two bf16 operand buffers of
//               layer 3 (tile t uses buffer t % 2), so they run up to two tiles ahead;
//   warps 6-13  two softmax teams: team T takes the tiles of parity T, their logits in tensor
//               memory columns 256 T .. 256 T + 255.  A thread per context makes three passes
//               over its row (max; e_k and their sum; floor terms and cumulative table) and
//               writes the context's table without the remainder, with a record (argmax,
//               remainder) that the consumer applies when it looks a slot up.
// Tile (i, j) needs rows i-1 .. i-4 of its channels: the consumer publishes row i-1 of a
// channel quad with one mbarrier per quad, and every step it finishes with a counter that
// the teams read before they overwrite a table slot.  Waits are bounded.
//
// Two exact shortcuts apply when the model's integers allow them (checked per model; the
// general forms run otherwise): with |b3| < 2^21 the layer-3 bias is preloaded into the
// accumulator with the 1.5 2^23 offset, so the logits arrive biased; with sh <= 32, m <= 2^sh
// (both requantisations) and |b2| < 2^21, layer 2's bias enters the mma.sync accumulator the
// same way and each requantisation is one clamp, one wide multiply-add and one funnel shift.
constexpr int kNQ = kNChan / 4;        // tiles per row
constexpr int kNS = 6;                 // table ring (steps): step k uses slot k % kNS
constexpr int kNA = 2;                 // layer-3 operand buffers
constexpr int kWL12 = 2;               // first layer-1/2 warp
constexpr int kWTeam = 6;              // first softmax warp
constexpr int kLT = 14 * 32;           // threads
constexpr int kCS = 264;               // table row stride (u16): 528-byte rows spread the banks
constexpr uint32_t kWaitLimit = kDefaultWaitPolls;
constexpr uint32_t kAccBias = 0x4B400000u;  // bit pattern of 1.5 2^23
constexpr int32_t kFastBias = 1 << 21;      // |bias| below this keeps every partial sum in [2^23, 2^24)
// A row has an even number of tiles, so tile (i, j) goes to team j % 2 and to operand
// buffer j % 2.
static_assert(kNQ % 2 == 0 && kNA == 2, "tile parity");

struct LSmem4 {
    alignas(1024) uint8_t w3t[256 * 64 * 2];     // layer 3 B operand: W3 (symbol x unit), canonical layout
    alignas(1024) uint8_t at[kNA][128 * 64 * 2]; // layer 3 A operands: a tile's h2 (context x unit)
    alignas(16) __nv_bfloat16 w2[64 * kBS];      // W2 (out x in) for layer 2's B fragments
    alignas(16) int32_t b3m[256];                // b3 - 0x4B400000 (general form: added in pass 1)
    alignas(16) uint32_t b3f[256];               // 0x4B400000 + b3: 1.5 2^23 + b3 as fp32 bits
    float b2f[64];                               // 1.5 2^23 + b2 (layer 2 accumulator input)
    int32_t b2m[64];                             // b2 - 0x4B400000 (general form)
    int32_t b1[kNChan * 64];
    alignas(16) int8_t w1[64 * 4];
    uint32_t etab[kETop + 1];                    // e(t), t = 0 .. kETop
    uint8_t ctx[32 * 4 * kNChan];                // token history [lane][row % 4][channel]
    alignas(16) uint16_t cdf[kNS][32][kCS];      // cumulative table without the remainder
    uint2 meta[kNS][32];                         // (cdf[a] | (f_a + r) << 16, r | a << 16), a = argmax
    alignas(16) uint16_t win[kWinWords];         // consumer's word-stream window
    uint64_t row0[32];
    uint32_t nrows[32];
    float step[kNChan], offset[kNChan];
    alignas(8) uint64_t a_full[kNA], a_empty[kNA], t_full[2], t_empty[2], c_full[kNS], tok[kNQ];
    uint32_t consumed;                           // steps the consumer has finished
    int32_t m1, sh1, m2, sh2, ahi1, ahi2;
    uint32_t ms, ss, dcap, mq;
    int fast12, fast3;
    int bad;
    int abort_;
    uint32_t tmem;
};
static_assert(offsetof(LSmem4, at) % 1024 == 0 && offsetof(LSmem4, cdf) % 16 == 0 &&
              offsetof(LSmem4, win) % 16 == 0 && offsetof(LSmem4, b3m) % 16 == 0 &&
              offsetof(LSmem4, b3f) % 16 == 0, "alignment");
static_assert(sizeof(LSmem4) + 256 <= 227 * 1024, "shared memory");

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
// timeout or abort (abort_ may be NULL: then only the limit ends it).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_,
                                          uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it) {
        if (mbar_test(bar, parity)) return true;
        if (abort_ && *abort_) return false;
        if (it > 64) __nanosleep(64);
    }
    return false;
}
__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
    asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}

// Requantisation rq(a) = clamp((a m + 2^(sh-1)) >> sh, 0, 127) (m >= 0, 1 <= sh <= 47), on a
// clamped to [0, ahi]: every a <= 0 gives 0, and ahi is the least a giving 127 or more, so the
// shifted sum stays below 2^32 and the 64-bit shift is one funnel shift and one shift.
struct Rq {
    uint64_t half;
    uint32_t m, sh_lo, sh_hi;
    int32_t ahi;
};
__device__ __forceinline__ Rq make_rq(int32_t m, int32_t sh, int32_t ahi) {
    Rq q;
    q.half = 1ull << (sh - 1);
    q.m = (uint32_t)m;
    q.sh_lo = (uint32_t)min(sh, 32);
    q.sh_hi = (uint32_t)max(sh - 32, 0);
    q.ahi = ahi;
    return q;
}
__device__ __forceinline__ uint32_t rq32(int32_t a, const Rq &q) {
    const uint32_t ac = (uint32_t)min(max(a, 0), q.ahi);
    const uint64_t P = (uint64_t)ac * q.m + q.half;
    const uint32_t v = __funnelshift_rc((uint32_t)P, (uint32_t)(P >> 32), q.sh_lo) >> q.sh_hi;
    return min(v, 127u);
}
// The least a >= 0 with (a m + 2^(sh-1)) >> sh >= 127, capped at 2^31 - 1.
__device__ __forceinline__ int32_t rq_ahi(int32_t m, int32_t sh) {
    if (m <= 0) return 0x7FFFFFFF;
    const uint64_t need = 253ull << (sh - 1);  // 127 2^sh - 2^(sh-1)
    const uint64_t a = (need + (uint64_t)m - 1) / (uint64_t)m;
    return a > 0x7FFFFFFFull ? 0x7FFFFFFF : (int32_t)a;
}
// The short form for sh <= 32 and m <= 2^sh, of an input x = a + base (base 0, or the fp32 bit
// offset 0x4B400000 of an accumulator that carries it): clamping x to [base, base + ahi] makes
// the result land in [0, 127] (at ahi it is 127 exactly: it rises by at most 1 per unit of a),
// and (x - base) m + 2^(sh-1) = x m + (2^(sh-1) - base m) modulo 2^64.
struct RqF {
    uint64_t add;
    uint32_t m, sh;
    int32_t lo, hi;
};
__device__ __forceinline__ RqF make_rqf(int32_t m, int32_t sh, int32_t ahi, uint32_t base) {
    RqF q;
    q.m = (uint32_t)m;
    q.sh = (uint32_t)sh;
    q.add = (1ull << (sh - 1)) - (uint64_t)base * (uint64_t)(uint32_t)m;
    q.lo = (int32_t)base;
    const int64_t hi = (int64_t)base + ahi;
    q.hi = hi > 0x7FFFFFFF ? 0x7FFFFFFF : (int32_t)hi;
    return q;
}
__device__ __forceinline__ uint32_t rqf(int32_t x, const RqF &q) {
    const uint32_t xc = (uint32_t)min(max(x, q.lo), q.hi);
    const uint64_t P = (uint64_t)xc * q.m + q.add;
    return __funnelshift_rc((uint32_t)P, (uint32_t)(P >> 32), q.sh);
}

// Two integers in [0, 127] as a bf16 pair, the first in the low half.
__device__ __forceinline__ uint32_t pack2(uint32_t lo, uint32_t hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn((float)lo, (float)hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

// floor(65280 2^32 / E) for 2^23 <= E <= 2^31, from a float estimate and two integer
// corrections: the estimate is within 7 of the quotient, the second one within 1.
__device__ __forceinline__ uint32_t softmax_scale(uint32_t E) {
    const uint64_t N = 65280ull << 32;
    const float rf = __frcp_rn((float)E);
    uint32_t q = (uint32_t)__fmul_rn(280375465082880.0f, rf);  // 65280 2^32 = 255 2^40, exact in fp32
    int64_t rem = (int64_t)(N - (uint64_t)q * E);
    const int32_t dq = (int32_t)floorf(__fmul_rn((float)rem, rf));
    q += (uint32_t)dq;
    rem -= (int64_t)dq * (int64_t)E;
    if (rem < 0) q -= 1;
    else if (rem >= (int64_t)E) q += 1;
    return q;
}

__device__ bool load_model4(LSmem4 &S, const uint8_t *m, int *status) {
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
            // t = floor(d ms / 2^ss) = floor(d mq / 2^32) when ms < 2^ss (then t rises by at
            // most 1 per unit of d, so t(dcap) = kETop exactly); else mq = 0 and t is taken in 64
            // bits and clamped
            S.mq = (S.ss >= 1 && S.ms < (1u << S.ss)) ? (S.ms << (32 - S.ss)) : 0u;
            S.ahi1 = rq_ahi(S.m1, S.sh1);
            S.ahi2 = rq_ahi(S.m2, S.sh2);
            S.fast12 = S.sh1 <= 32 && S.sh2 <= 32 && (uint64_t)S.m1 <= (1ull << S.sh1) &&
                       (uint64_t)S.m2 <= (1ull << S.sh2);
            S.fast3 = 1;
        }
        S.abort_ = 0;
    }
    const int32_t *b1 = reinterpret_cast<const int32_t *>(m + kMB_B1);
    const int32_t *b2 = reinterpret_cast<const int32_t *>(m + kMB_B2);
    const int32_t *b3 = reinterpret_cast<const int32_t *>(m + kMB_B3);
    bool badb = false, wide2 = false, wide3 = false;
    for (int i = tid; i < kNChan * 64; i += kLT) {
        S.b1[i] = b1[i];
        badb |= (b1[i] >= (1 << 24) || b1[i] <= -(1 << 24));
    }
    for (int i = tid; i < 64; i += kLT) {
        S.b2m[i] = b2[i] - (int32_t)kAccBias;
        S.b2f[i] = __int_as_float((int32_t)kAccBias + b2[i]);  // 1.5 2^23 + b2 when |b2| < 2^22
        badb |= (b2[i] >= (1 << 24) || b2[i] <= -(1 << 24));
        wide2 |= (b2[i] >= kFastBias || b2[i] <= -kFastBias);
    }
    for (int i = tid; i < 256; i += kLT) {
        S.b3m[i] = b3[i] - (int32_t)kAccBias;
        S.b3f[i] = kAccBias + (uint32_t)b3[i];
        badb |= (b3[i] >= (1 << 24) || b3[i] <= -(1 << 24));
        wide3 |= (b3[i] >= kFastBias || b3[i] <= -kFastBias);
        S.w1[i] = (int8_t)m[kMB_W1 + i];
    }
    for (int t = tid; t <= kETop; t += kLT) S.etab[t] = kExp2Q[t & 255] >> (t >> 8);
    for (int i = tid; i < 64 * 64; i += kLT) S.w2[(i >> 6) * kBS + (i & 63)] = bf((int8_t)m[kMB_W2 + i]);
    for (int i = tid; i < 256 * 64; i += kLT)
        *reinterpret_cast<__nv_bfloat16 *>(S.w3t + tc_off(i >> 6, i & 63)) = bf((int8_t)m[kMB_W3 + i]);
    tc_fence_proxy();  // W3 is read by the tensor cores
    __syncthreads();
    if (badb) atomicOr(&S.bad, 1);
    if (wide2) atomicAnd(&S.fast12, 0);
    if (wide3) atomicAnd(&S.fast3, 0);
    __syncthreads();
    if (S.bad) {
        if (tid == 0) set_status(status, SGS_E_CORRUPT);
        return false;
    }
    return true;
}

// Every lane's wait, agreed across the warp; on failure the first lane raises the abort.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, volatile int *abort_, const LearnedParams &p) {
    const bool ok = __all_sync(0xffffffffu, mbar_wait(bar, parity, abort_, p.wait_limit));
    if (!ok && (threadIdx.x & 31) == 0) {
        if (!*abort_) set_status(p.status, SGS_E_TIMEOUT);
        *abort_ = 1;
    }
    return ok;
}

// ---- layers 1-2: warp w makes rows 32 w .. 32 w + 31 of the operand (channel 4 j + w).
// mma.sync m16n8k16 with the contexts as M: lane 4 g + t holds contexts 16 mt + g (+ 8) and
// layer-1 units 16 kt + 8 h + 2 t + e (its A fragments); layer 2's accumulators hold the same
// contexts at out units 8 nt + 2 t + e.
template <bool kFast>
__device__ void l12_run(const LearnedParams &p, LSmem4 &S, uint32_t NT, volatile int *abort_) {
    const int lane = threadIdx.x & 31, w = (threadIdx.x >> 5) - kWL12;
    const int g = lane >> 2, t4 = lane & 3;
    const Rq R1 = make_rq(S.m1, S.sh1, S.ahi1), R2 = make_rq(S.m2, S.sh2, S.ahi2);
    const RqF F1 = make_rqf(S.m1, S.sh1, S.ahi1, 0u), F2 = make_rqf(S.m2, S.sh2, S.ahi2, kAccBias);
    const int32_t *w1w = reinterpret_cast<const int32_t *>(S.w1);
    int32_t w1r[4][2][2];
    float b2c[8][2];  // kFast: the layer-2 accumulator input; else b2 - 0x4B400000 as bits
#pragma unroll
    for (int kt = 0; kt < 4; ++kt)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int e = 0; e < 2; ++e) w1r[kt][h][e] = w1w[16 * kt + 8 * h + 2 * t4 + e];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int e = 0; e < 2; ++e)
            b2c[nt][e] = kFast ? S.b2f[8 * nt + 2 * t4 + e] : __int_as_float(S.b2m[8 * nt + 2 * t4 + e]);
    for (uint32_t tau = 0; tau < NT; ++tau) {
        const uint32_t i = tau / kNQ, j = tau - i * kNQ;
        const int c = 4 * (int)j + w;
        const int b = (int)(tau & 1);
        if (i >= 1 && !warp_wait(&S.tok[j], (i - 1) & 1, abort_, p)) break;
        if (tau >= 2 && !warp_wait(&S.a_empty[b], ((tau >> 1) - 1) & 1, abort_, p)) break;
        const int32_t *b1c = S.b1 + c * 64;
        // layer 1 into A fragments: afr[mt][kt][r + 2 h] = units 16 kt + 8 h + 2 t4 (+1) of
        // context 16 mt + 8 r + g
        uint32_t afr[2][4][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int l = 16 * mt + 8 * r + g;
                uint32_t up = 0;  // u_jj = token_{i-jj} - 128 as packed int8, 0 before the lane's start
#pragma unroll
                for (int jj = 1; jj <= 4; ++jj) {
                    const uint32_t tok = (i >= (uint32_t)jj) ? S.ctx[(l * 4 + ((i - jj) & 3)) * kNChan + c] : 128u;
                    up |= (tok ^ 0x80u) << (8 * (jj - 1));
                }
#pragma unroll
                for (int kt = 0; kt < 4; ++kt)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int o = 16 * kt + 8 * h + 2 * t4;
                        const int32_t a0 = __dp4a(w1r[kt][h][0], (int32_t)up, b1c[o]);
                        const int32_t a1 = __dp4a(w1r[kt][h][1], (int32_t)up, b1c[o + 1]);
                        const uint32_t v0 = kFast ? rqf(a0, F1) : rq32(a0, R1);
                        const uint32_t v1 = kFast ? rqf(a1, F1) : rq32(a1, R1);
                        afr[mt][kt][r + 2 * h] = pack2(v0, v1);
                    }
            }
        // layer 2, requantised into the operand tile
        uint8_t *at = S.at[b];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            uint32_t bfr[4][2];
#pragma unroll
            for (int kt = 0; kt < 4; ++kt) {
                const __nv_bfloat16 *wr = S.w2 + (8 * nt + g) * kBS + 16 * kt + 2 * t4;
                bfr[kt][0] = lds32(wr);
                bfr[kt][1] = lds32(wr + 8);
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                float acc[4];
                if (kFast) {
                    // accumulated onto 1.5 2^23 + b2: every partial sum stays in [2^23, 2^24)
                    const float c4[4] = {b2c[nt][0], b2c[nt][1], b2c[nt][0], b2c[nt][1]};
                    mma_bf16_c(acc, c4, afr[mt][0][0], afr[mt][0][1], afr[mt][0][2], afr[mt][0][3], bfr[0][0], bfr[0][1]);
                } else {
                    acc[0] = acc[1] = acc[2] = acc[3] = 0.f;
                    mma_bf16(acc, afr[mt][0][0], afr[mt][0][1], afr[mt][0][2], afr[mt][0][3], bfr[0][0], bfr[0][1]);
                }
#pragma unroll
                for (int kt = 1; kt < 4; ++kt)
                    mma_bf16(acc, afr[mt][kt][0], afr[mt][kt][1], afr[mt][kt][2], afr[mt][kt][3], bfr[kt][0], bfr[kt][1]);
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    uint32_t v0, v1;
                    if (kFast) {
                        v0 = rqf(__float_as_int(acc[2 * r]), F2);
                        v1 = rqf(__float_as_int(acc[2 * r + 1]), F2);
                    } else {
                        // acc is an integer below 2^21 in magnitude: acc + 1.5 2^23 is exact
                        // and its bit pattern is 0x4B400000 + acc
                        v0 = rq32(__float_as_int(__fadd_rn(acc[2 * r], 12582912.0f)) + __float_as_int(b2c[nt][0]), R2);
                        v1 = rq32(__float_as_int(__fadd_rn(acc[2 * r + 1], 12582912.0f)) + __float_as_int(b2c[nt][1]), R2);
                    }
                    const int l = 16 * mt + 8 * r + g;
                    *reinterpret_cast<uint32_t *>(at + tc_off(32 * w + l, 8 * nt + 2 * t4)) = pack2(v0, v1);
                }
            }
        }
        tc_fence_proxy();
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.a_full[b]);
    }
}

// ---- layer 3 issue (one thread)
__device__ void mma_run(const LearnedParams &p, LSmem4 &S, uint32_t NT, volatile int *abort_) {
    const uint32_t idesc = tc_idesc_bf16(128, 256);
    const uint32_t b0 = smem_addr(S.w3t);
    uint32_t issued = 0;
    for (uint32_t tau = 0; tau < NT; ++tau) {
        const int T = (int)(tau & 1);  // team and operand buffer
        const uint32_t n = tau >> 1;
        bool ok = mbar_wait(&S.a_full[T], n & 1, abort_, p.wait_limit) &&
                  mbar_wait(&S.t_empty[T], n & 1, abort_, p.wait_limit);
        if (!ok) {
            if (!*abort_) set_status(p.status, SGS_E_TIMEOUT);
            *abort_ = 1;
            break;
        }
        tc_fence_after();
        const uint32_t a0 = smem_addr(S.at[T]);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
            tc_mma_bf16(S.tmem + 256u * T, tc_desc(a0 + 256u * kk), tc_desc(b0 + 256u * kk), idesc, 1u);
        tc_commit(&S.t_full[T]);
        tc_commit(&S.a_empty[T]);
        ++issued;
    }
    // the last commit's arrival (its tile's and every earlier tile's work complete) precedes
    // the CTA's next use of the barriers and the release of the tensor memory, also after an
    // abort: an issued MMA ends within microseconds, so this wait keeps the default limit
    // whatever limit the caller set for the hand-offs
    if (issued) {
        const uint32_t last = issued - 1;
        if (!mbar_wait(&S.a_empty[last & 1], (last >> 1) & 1, nullptr, kWaitLimit)) {
            set_status(p.status, SGS_E_TIMEOUT);
            *abort_ = 1;
        }
    }
}

// ---- softmax teams
__device__ __forceinline__ int32_t max32(const uint32_t (&v)[32]) {
    int32_t m[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) m[j] = max((int32_t)v[j], (int32_t)v[j + 16]);
#pragma unroll
    for (int s = 8; s > 0; s >>= 1)
#pragma unroll
        for (int j = 0; j < s; ++j) m[j] = max(m[j], m[j + s]);
    return m[0];
}

// The team's columns are set up for the next tile's layer 3 (1.5 2^23, plus b3 in the short
// form); then the buffer is free.
template <bool kFast3>
__device__ __forceinline__ void team_release(LSmem4 &S, uint32_t tb, int T) {
    uint32_t v[32];
#pragma unroll 1
    for (int ch = 0; ch < 8; ++ch) {
        if (kFast3) {
            const uint4 *src = reinterpret_cast<const uint4 *>(S.b3f + 32 * ch);
#pragma unroll
            for (int j4 = 0; j4 < 8; ++j4) {
                const uint4 b = src[j4];
                v[4 * j4] = b.x; v[4 * j4 + 1] = b.y; v[4 * j4 + 2] = b.z; v[4 * j4 + 3] = b.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = kAccBias;
        }
        tc_st32(tb + 32 * ch, v);
    }
    tc_wait_st();
    tc_fence_before();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&S.t_empty[T]);
}

// Bounded wait until the consumer has finished `need` steps.
__device__ __forceinline__ bool wait_consumed(LSmem4 &S, uint32_t need, volatile int *abort_, const LearnedParams &p) {
    bool ok = false;
    for (uint32_t it = 0; it < p.wait_limit; ++it) {
        if (ld_acquire(&S.consumed) >= need) { ok = true; break; }
        if (*abort_) break;
        if (it > 64) __nanosleep(64);
    }
    ok = __all_sync(0xffffffffu, ok);
    if (!ok && (threadIdx.x & 31) == 0) {
        if (!*abort_) set_status(p.status, SGS_E_TIMEOUT);
        *abort_ = 1;
    }
    return ok;
}

template <bool kSmallScale, bool kFast3>
__device__ void team_run(const LearnedParams &p, LSmem4 &S, int T, uint32_t NT, volatile int *abort_) {
    const int lane = threadIdx.x & 31, q = (threadIdx.x >> 5) & 3;
    const uint32_t tb = tc_taddr(S.tmem, q, 256u * T);
    const uint32_t dcap = S.dcap, mq = S.mq, ms = S.ms, ss = S.ss;
    const int4 *b3v = reinterpret_cast<const int4 *>(S.b3m);
    team_release<kFast3>(S, tb, T);
    for (uint32_t tau = T; tau < NT; tau += 2) {
        if (!warp_wait(&S.t_full[T], (tau >> 1) & 1, abort_, p)) break;
        tc_fence_after();
        uint32_t v[32];
        // pass 1: zmax (the general form adds the bias and writes the logits back)
        int32_t zmax = INT32_MIN;
#pragma unroll 1
        for (int ch = 0; ch < 8; ++ch) {
            tc_ld32(tb + 32 * ch, v);
            tc_wait_ld();
            if (!kFast3) {
#pragma unroll
                for (int j4 = 0; j4 < 8; ++j4) {
                    const int4 bb = b3v[8 * ch + j4];
                    v[4 * j4] += bb.x; v[4 * j4 + 1] += bb.y; v[4 * j4 + 2] += bb.z; v[4 * j4 + 3] += bb.w;
                }
                tc_st32(tb + 32 * ch, v);
            }
            zmax = max(zmax, max32(v));
        }
        if (!kFast3) tc_wait_st();
        // pass 2: e_k = etab[t(min(zmax - z_k, dcap))] (e vanishes from d = dcap on), their
        // sum, and the lowest k with z_k = zmax (symbols visited in descending order).  The
        // short form's logits carry a common offset, which no difference sees.
        const int64_t zl = (int64_t)zmax - (int64_t)dcap;
        const int32_t zlo = zl < (int64_t)INT32_MIN ? INT32_MIN : (int32_t)zl;
        uint32_t E = 0, am = 0;
#pragma unroll 1
        for (int ch = 7; ch >= 0; --ch) {
            tc_ld32(tb + 32 * ch, v);
            tc_wait_ld();
#pragma unroll
            for (int j = 31; j >= 0; --j) {
                const int32_t z = (int32_t)v[j];
                const uint32_t d = (uint32_t)(zmax - max(z, zlo));
                if (z == zmax) am = 32 * ch + j;
                uint32_t t;
                if (kSmallScale) t = __umulhi(d, mq);
                else t = min((uint32_t)(((uint64_t)d * ms) >> ss), (uint32_t)kETop);
                v[j] = S.etab[t];
                E += v[j];
            }
            tc_st32(tb + 32 * ch, v);
        }
        tc_wait_st();
        const uint32_t R = softmax_scale(E);  // E >= e(0) = 2^23
        // pass 3: cumulative table of f_k = 1 + floor(e_k R / 2^32), without the remainder,
        // into the slot of step k once the consumer has finished step k - kNS
        const uint32_t i = tau / kNQ, jq = tau - i * kNQ;
        const uint32_t c = 4 * jq + q, k = i * kNChan + c, slot = k % kNS;
        if (k >= (uint32_t)kNS && !wait_consumed(S, k - kNS + 1, abort_, p)) break;
        uint16_t *row = &S.cdf[slot][lane][0];
        uint32_t run = 0;
#pragma unroll 1
        for (int ch = 0; ch < 8; ++ch) {
            tc_ld32(tb + 32 * ch, v);
            tc_wait_ld();
#pragma unroll
            for (int o = 0; o < 32; o += 8) {
                uint32_t wv[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const uint32_t c0 = run;
                    run += __umulhi(v[o + 2 * h], R) + 1u;
                    const uint32_t c1 = run;
                    run += __umulhi(v[o + 2 * h + 1], R) + 1u;
                    wv[h] = __byte_perm(c0, c1, 0x5410);
                }
                *reinterpret_cast<uint4 *>(row + 32 * ch + o) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            }
        }
        // the remainder r = 2^16 - sum f goes to the argmax: its interval becomes
        // [cdf[a], cdf[a + 1] + r) and every later entry moves up by r
        const uint32_t r = 65536u - run;
        const uint32_t lo_a = row[am], nx = am < 255 ? row[am + 1] : run;
        S.meta[slot][lane] = make_uint2(lo_a | ((nx - lo_a + r) << 16), r | (am << 16));
        __syncwarp();
        if (lane == 0) mbar_arrive(&S.c_full[slot]);
        team_release<kFast3>(S, tb, T);
    }
}

// Symbol of `y` (the state's low 16 bits) under a table without its remainder and the
// record (cdf[a], f_a + r, r, a): slots inside a's widened interval are a's; above it the
// table is searched for y - r and the interval moved up by r.
__device__ __forceinline__ uint32_t table_sym(const uint16_t *row, uint2 mt, uint32_t y, uint32_t &lo, uint32_t &hi) {
    const uint32_t lo_a = mt.x & 0xFFFFu, fr = mt.x >> 16, r = mt.y & 0xFFFFu, a = mt.y >> 16;
    const bool in_a = (y - lo_a) < fr;
    const bool up = y >= lo_a + fr;
    const uint32_t y2 = up ? y - r : y;
    uint32_t s = 0;
#pragma unroll
    for (uint32_t st = 128; st > 0; st >>= 1) s += (row[s + st] <= y2) ? st : 0u;
    uint32_t l = row[s], h = s < 255 ? row[s + 1] : 65536u - r;
    if (up) { l += r; h += r; }
    if (in_a) { s = a; l = lo_a; h = lo_a + fr; }
    lo = l;
    hi = h;
    return s;
}

__device__ void consume4(const LearnedParams &p, LSmem4 &S, uint32_t grp, int nl, uint32_t K,
                         uint32_t maxrows, volatile int *abort_) {
    const int lane = threadIdx.x & 31;
    GroupStream gs;
    uint32_t x = 0x10000u;
    group_open(p.bits, p.grp_sec, p.pay_off, p.pay_len, p.G, grp, nl, lane, gs, x, S.win);
    const uint32_t my_rows = lane < nl ? S.nrows[lane] : 0u;
    float *out_lane = p.out + (p.out_index ? 0 : S.row0[lane]);
    const uint32_t *idx_lane = p.out_index ? p.out_index + S.row0[lane] : nullptr;
    bool aborted = false;
    uint32_t i = 0, c = 0, slot = 0, u = 0;  // step k = i kNChan + c, slot = k % kNS, u = k / kNS
    for (uint32_t k = 0; k < K; ++k) {
        if (!warp_wait(&S.c_full[slot], u & 1, abort_, p)) {
            aborted = true;
            break;
        }
        const bool live = i < my_rows;
        if (live) {
            const uint32_t y = x & 0xFFFFu;
            uint32_t lo, hi;
            const uint32_t s = table_sym(S.cdf[slot][lane], S.meta[slot][lane], y, lo, hi);
            x = (hi - lo) * (x >> 16) + y - lo;
            S.ctx[(lane * 4 + (i & 3)) * kNChan + c] = (uint8_t)s;
            const uint64_t col = idx_lane ? (uint64_t)idx_lane[i] : (uint64_t)i;
            out_lane[(uint64_t)c * p.n_rows + col] = dequant(s, S.step[c], S.offset[c]);
        }
        group_refill(gs, x, live);
        __syncwarp();
        if (lane == 0) {
            st_release(&S.consumed, k + 1);
            if ((c & 3) == 3 && i + 1 < maxrows) mbar_arrive(&S.tok[c >> 2]);
        }
        if (++c == (uint32_t)kNChan) { c = 0; ++i; }
        if (++slot == (uint32_t)kNS) { slot = 0; ++u; }
    }
    if (!aborted) {
        const bool bad = gs.bad || (lane < nl && x != 0x10000u) || (gs.ptr != gs.n_words);
        if (bad) set_status(p.status, SGS_E_CORRUPT);
    }
}

// Tensor memory of the CTA: 512 columns (two teams x 256), allocated by warp 1.  One CTA fits
// an SM (the shared memory above), so the allocation never waits for another CTA's.
__device__ __forceinline__ void learned_tmem_alloc(LSmem4 &S) {
    if ((threadIdx.x >> 5) == 1) tc_alloc(&S.tmem, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}
__device__ __forceinline__ void learned_tmem_free(LSmem4 &S) {
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if ((threadIdx.x >> 5) == 1) {
        __syncwarp();
        tc_dealloc(S.tmem, 512);
    }
}

// One group of 32 lanes.  reload = false: the CTA's previous group was of the same scene,
// whose model is still in shared memory (S.bad records whether it was refused).
__device__ __forceinline__ void learned_body(const LearnedParams &p, LSmem4 &S, uint32_t grp, bool reload) {
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nl = (int)min(32u, p.L - grp * 32);
    if (reload) {
        if (!load_model4(S, p.bits + p.model_off, p.status)) return;
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
    if (tid == 0) {
        for (int b = 0; b < kNA; ++b) {
            mbar_init(&S.a_full[b], 4);
            mbar_init(&S.a_empty[b], 1);
        }
        for (int T = 0; T < 2; ++T) {
            mbar_init(&S.t_full[T], 1);
            mbar_init(&S.t_empty[T], 4);
        }
        for (int b = 0; b < kNS; ++b) mbar_init(&S.c_full[b], 1);
        for (int b = 0; b < kNQ; ++b) mbar_init(&S.tok[b], 1);
        S.consumed = 0;
    }
    __syncthreads();
    uint32_t maxrows = 0;
    for (int r = 0; r < 32; ++r) maxrows = max(maxrows, S.nrows[r]);
    const uint32_t K = maxrows * kNChan, NT = maxrows * kNQ;
    volatile int *abort_ = &S.abort_;
    if (warp == 0) {
        consume4(p, S, grp, nl, K, maxrows, abort_);
    } else if (warp == 1) {
        if ((tid & 31) == 0) mma_run(p, S, NT, abort_);
    } else if (warp < kWTeam) {
        if (S.fast12) l12_run<true>(p, S, NT, abort_);
        else l12_run<false>(p, S, NT, abort_);
    } else {
        const int T = (warp - kWTeam) >> 2;
        if (S.mq) {
            if (S.fast3) team_run<true, true>(p, S, T, NT, abort_);
            else team_run<true, false>(p, S, T, NT, abort_);
        } else {
            if (S.fast3) team_run<false, true>(p, S, T, NT, abort_);
            else team_run<false, false>(p, S, T, NT, abort_);
        }
    }
    // every hand-off is over: retire the barriers (a persistent CTA initialises them again)
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
        for (int b = 0; b < kNA; ++b) {
            mbar_inval(&S.a_full[b]);
            mbar_inval(&S.a_empty[b]);
        }
        for (int T = 0; T < 2; ++T) {
            mbar_inval(&S.t_full[T]);
            mbar_inval(&S.t_empty[T]);
        }
        for (int b = 0; b < kNS; ++b) mbar_inval(&S.c_full[b]);
        for (int b = 0; b < kNQ; ++b) mbar_inval(&S.tok[b]);
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kLT, 1) k_learned_decode(LearnedParams p) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    LSmem4 &S = *reinterpret_cast<LSmem4 *>(smem_raw);
    learned_tmem_alloc(S);
    learned_body(p, S, blockIdx.x, true);
    learned_tmem_free(S);
}

__global__ void __launch_bounds__(kLT, 1) k_learned_multi(MultiArgs m) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    LSmem4 &S = *reinterpret_cast<LSmem4 *>(smem_raw);
    learned_tmem_alloc(S);
    run_items<LearnedParams>(m, [&S](const LearnedParams &p, uint32_t vb, uint32_t, bool same) {
        learned_body(p, S, vb, !same);
    });
    learned_tmem_free(S);
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
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(LSmem4));
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
    k_learned_decode<<<grid, kLT, sizeof(LSmem4), st>>>(p);
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
    return launch_persistent(k_learned_multi, kLT, sizeof(LSmem4), m, st);
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
