// Position-aware learned attribute coding on sm_103a: rANS driven by the local autoregressive
// model of Sec. 3.4.2 with its Fourier positional embedding (Sec. 3.4.2, "Fourier-based
// Positional Embedding": phi(mu) = [mu; sin(2 pi F mu); cos(2 pi F mu)], L = 12 octave bands,
// projected to d = 32) and a conditional Laplace entropy model (Sec. 3.2, "Rate Proxy").
//
// Integer model (frozen, the bitstream's model section):
//   x = [u (4); phi_q (75); 0],  u_j = s_{i-j,c} - 128 (0 past the lane start),
//   phi_q = [floor(128 mu) (3); SIN8[theta_k] (36); SIN8[theta_k + 64] (36)] of the row's
//   voxel v at depth D, mu = (v + 1/2) / 2^D, theta_k = floor(256 frac(2^k mu));
//   h1 = q(W1 x + B1[c], s1), h2 = q(W2 h1 + b2, s2), (z0, z1) = W3 h2 + b3 with
//   q(a, s) = clamp(rint(fl32(a * s)), 0, 127) (every accumulator is an integer below 2^24,
//   exact in fp32, so one fp32 multiply and round-half-even decide each activation);
//   mean mu8 = 32640 + clamp(rint(z0 * smu), +-32640) in 1/256 symbol,
//   n = 4096 + clamp(rint(z1 * slr), -2048, 1536) (log2 of the rate in 1/256, plus 16);
//   cdf(s) = s + floor(65280 F(s - 1/2) / 2^23), F from EXP2Q (pe_cdf below).
//
// Decoder: a team of two warps per group of 32 lanes.  For each row step i the team first runs
// the model for all 56 channels of its 32 lanes, each warp one half -- 112 tiles of 16
// contexts, each three bf16 mma.sync
// layers with the contexts as M, so a layer's accumulator fragments are the next layer's A
// fragments without any data movement; layer 1's embedding part depends on the row only and
// is computed once per row -- and keeps each (mean, rate) in shared memory; then
// one warp decodes the row's 56 tokens, each lane searching its CDF with 8 evaluations.  The
// context of (i, c) needs only rows i-1 .. i-4, so the whole row's model runs before its
// tokens are decoded.  The encoder's frequency kernel runs the same tile code with 32
// consecutive rows as its contexts.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "exp2q_table.h"
#include "sin8_table.h"
#include "sgs_device.cuh"
#include "sgs_internal.h"
#include "sgs_mma.cuh"

namespace sgs {

namespace {

__constant__ uint32_t kPeExp2Q[256] = {SGS_EXP2Q_VALUES};
__constant__ int8_t kPeSin8[256] = {SGS_SIN8_VALUES};

// Model section offsets (bytes).
constexpr int kPB_B1 = 32, kPB_B2 = 14368, kPB_B3 = 14624, kPB_W1 = 14640, kPB_W2 = 19760, kPB_W3 = 23856;
static_assert(kPB_W3 + 128 == SGS_MODEL_PE_BYTES, "model layout");
constexpr int kKin = 80;      // layer-1 inputs
constexpr int kPeGroups = 3;  // groups per CTA
constexpr int kPeTeam = 2;    // warps per group: each runs one 16-lane half of the model tiles
constexpr int kPeThreads = 32 * kPeGroups * kPeTeam;

struct PeSmem {
    alignas(16) uint16_t win[kPeGroups][kWinWords];  // group stream windows (filled by 16-byte stores)
    uint4 w1f[5][4][32];  // layer-1 B fragments (W1 transposed) [k tile][n tile pair][lane]: n tiles 2p, 2p + 1
    uint4 w2f[4][4][32];  // layer-2 B fragments, likewise
    uint2 w3f[4][32];    // layer-3 B fragments (outputs 0, 1; the other six columns zero)
    float b1[kNChan * 64];
    float b2[64];
    uint32_t exq[256];
    int8_t sin8[256];
    float step[kNChan], offset[kNChan];
    float b3[2], s1, s2, smu, slr;
    int bad;
    uint32_t hist[kPeGroups][kNChan * 32];  // per channel and lane: s_{i-1} .. s_{i-4}, one byte each
    uint32_t hist2[kPeGroups][kNChan * 32]; // the four tokens before those (s_{i-5} .. s_{i-8})
    uint32_t par[kPeGroups][kNChan * 32];   // per channel and lane: mu8 | n << 16
};
static_assert(offsetof(PeSmem, win) % 16 == 0 && sizeof(PeSmem::win[0]) % 16 == 0, "16-byte window stores");
static_assert(offsetof(PeSmem, b1) % 8 == 0 && offsetof(PeSmem, b2) % 8 == 0, "float2 bias loads");
static_assert(offsetof(PeSmem, w1f) % 16 == 0 && offsetof(PeSmem, w2f) % 16 == 0, "16-byte fragment loads");

__device__ __forceinline__ int32_t ld_i32(const uint8_t *p) { return *reinterpret_cast<const int32_t *>(p); }

// Loads and checks the model (all threads of the CTA).  False (and the CTA's S.bad) if the
// model breaks the bounds the decoder relies on.
__device__ bool pe_load_model(PeSmem &S, const uint8_t *m) {
    const int tid = threadIdx.x;
    int bad = 0;
    for (int i = tid; i < kNChan * 64; i += blockDim.x) {
        const int32_t v = ld_i32(m + kPB_B1 + 4 * i);
        bad |= (v <= -(1 << 23) || v >= (1 << 23));
        S.b1[i] = (float)v;
    }
    if (tid < 64) {
        const int32_t v = ld_i32(m + kPB_B2 + 4 * tid);
        bad |= (v <= -(1 << 23) || v >= (1 << 23));
        S.b2[tid] = (float)v;
    }
    if (tid < 2) {
        const int32_t v = ld_i32(m + kPB_B3 + 4 * tid);
        bad |= (v <= -(1 << 23) || v >= (1 << 23));
        S.b3[tid] = (float)v;
    }
    if (tid == 0) {
        const float s1 = ld_f32(m), s2 = ld_f32(m + 4), smu = ld_f32(m + 8), slr = ld_f32(m + 12);
        // (the comparisons are false for NaN: a NaN scale is refused)
        const bool ok = s1 > 0.0f && s1 <= 127.0f && s2 > 0.0f && s2 <= 127.0f && smu > 0.0f &&
                        smu < 3.0e38f && slr > 0.0f && slr < 3.0e38f;
        bad |= !ok;
        S.s1 = s1; S.s2 = s2; S.smu = smu; S.slr = slr;
    }
    const int8_t *w1 = reinterpret_cast<const int8_t *>(m + kPB_W1);
    const int8_t *w2 = reinterpret_cast<const int8_t *>(m + kPB_W2);
    const int8_t *w3 = reinterpret_cast<const int8_t *>(m + kPB_W3);
    // B fragment of n tile nt, k tile kt for lane (g, t): rows k0, k0 + 1 and k0 + 8, k0 + 9 of
    // column n = 8 nt + g of W^T, i.e. row n of W
    auto frag = [](const int8_t *w, int ld, int kt, int nt, int ln) {
        const int8_t *r = w + (8 * nt + (ln >> 2)) * ld;
        const int k0 = 16 * kt + 2 * (ln & 3);
        return make_uint2(pack_bf16(r[k0], r[k0 + 1]), pack_bf16(r[k0 + 8], r[k0 + 9]));
    };
    for (int f = tid; f < 5 * 4 * 32; f += blockDim.x) {
        const int kt = f >> 7, np = (f >> 5) & 3, ln = f & 31;
        const uint2 a = frag(w1, kKin, kt, 2 * np, ln), b = frag(w1, kKin, kt, 2 * np + 1, ln);
        S.w1f[kt][np][ln] = make_uint4(a.x, a.y, b.x, b.y);
    }
    for (int f = tid; f < 4 * 4 * 32; f += blockDim.x) {
        const int kt = f >> 7, np = (f >> 5) & 3, ln = f & 31;
        const uint2 a = frag(w2, 64, kt, 2 * np, ln), b = frag(w2, 64, kt, 2 * np + 1, ln);
        S.w2f[kt][np][ln] = make_uint4(a.x, a.y, b.x, b.y);
    }
    for (int f = tid; f < 4 * 32; f += blockDim.x) {
        const int kt = f >> 5, ln = f & 31, g = ln >> 2, t = ln & 3, k0 = 16 * kt + 2 * t;
        uint2 v = make_uint2(0u, 0u);
        if (g < 2) {
            const int8_t *r = w3 + g * 64;
            v = make_uint2(pack_bf16(r[k0], r[k0 + 1]), pack_bf16(r[k0 + 8], r[k0 + 9]));
        }
        S.w3f[kt][ln] = v;
    }
    for (int i = tid; i < 256; i += blockDim.x) {
        S.exq[i] = kPeExp2Q[i];
        S.sin8[i] = kPeSin8[i];
    }
    bad = __syncthreads_or(bad);
    if (tid == 0) S.bad = bad;
    return !bad;
}

// x_q[k] of the layer-1 input for k >= 4 (embedding part) of voxel (v0, v1, v2) at depth D.
__device__ __forceinline__ float pe_x(const int8_t *sin8, uint32_t v0, uint32_t v1, uint32_t v2, int D, int k) {
    if (k < 4 || k >= 79) return 0.0f;
    const int j = k - 4;
    if (j < 3) {
        const uint32_t va = j == 0 ? v0 : (j == 1 ? v1 : v2);
        return (float)(uint32_t)(((2ull * va + 1ull) << 6) >> D);
    }
    const int jj = j - 3;
    const bool cosine = jj >= 36;
    const int r = cosine ? jj - 36 : jj;
    const int band = r / 3, a = r - 3 * band;
    const uint32_t va = a == 0 ? v0 : (a == 1 ? v1 : v2);
    uint32_t th = (uint32_t)((((2ull * va + 1ull) << (band + 8)) >> (D + 1)) & 255ull);
    if (cosine) th = (th + 64u) & 255u;
    return (float)sin8[th];
}

// Two activations clamp(rint(fl32(acc * s)), 0, 127) packed as a bf16 pair (a in the low
// half): rint and the upper clamp in fp32, the clamp at 0 by the conversion's relu.
__device__ __forceinline__ uint32_t pe_rq2(float a, float b, float s) {
    const float ra = fminf(rintf(__fmul_rn(a, s)), 127.0f), rb = fminf(rintf(__fmul_rn(b, s)), 127.0f);
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(rb), "f"(ra));
    return d;
}

__device__ __forceinline__ uint32_t pe_head(float zm, float zl, float smu, float slr) {
    const float vm = fminf(fmaxf(rintf(__fmul_rn(zm, smu)), -32640.0f), 32640.0f);
    const float vl = fminf(fmaxf(rintf(__fmul_rn(zl, slr)), -2048.0f), 1536.0f);
    return (uint32_t)(32640 + (int)vm) | ((uint32_t)(4096 + (int)vl) << 16);
}

// Cumulative count below symbol m (1..255) of the Laplace with mean mu8 and rate R.
__device__ __forceinline__ uint32_t pe_cdf(const uint32_t *exq, int mu8, uint32_t R, uint32_t m) {
    const int d = 256 * (int)m - 128 - mu8;
    const uint32_t ad = (uint32_t)(d < 0 ? -d : d);
    const uint32_t t = min((uint32_t)(((uint64_t)ad * R) >> 16), 6144u);
    const uint32_t e = exq[t & 255u] >> (t >> 8);
    const uint32_t F = d < 0 ? (e >> 1) : ((1u << 23) - (e >> 1));
    return m + (uint32_t)(((uint64_t)F * 65280ull) >> 23);
}

__device__ __forceinline__ uint32_t pe_rate(const uint32_t *exq, uint32_t n) {
    const uint32_t q = (n + 255u) >> 8;  // 8 .. 22
    return exq[(0u - n) & 255u] >> (23u - q);
}

// The model for 16 of a group's 32 contexts (context = lane; half h: lanes 16h .. 16h + 15)
// and all 56 channels: hist holds each context's packed history per channel, (v0, v1, v2)
// the calling lane's voxel; writes par[c * 32 + context].
__device__ __forceinline__ void pe_model_half(const PeSmem &S, const uint32_t *hist, uint32_t *par, uint32_t v0,
                                              uint32_t v1, uint32_t v2, int D, int h) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    uint32_t w3b[4][2];
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
        const uint2 b = S.w3f[kt][lane];
        w3b[kt][0] = b.x;
        w3b[kt][1] = b.y;
    }
    {
        const int ga = 16 * h + g, gb = ga + 8;  // the tile's rows g and g + 8
        const uint32_t a0 = __shfl_sync(0xffffffffu, v0, ga), a1 = __shfl_sync(0xffffffffu, v1, ga),
                       a2 = __shfl_sync(0xffffffffu, v2, ga);
        const uint32_t c0 = __shfl_sync(0xffffffffu, v0, gb), c1 = __shfl_sync(0xffffffffu, v1, gb),
                       c2 = __shfl_sync(0xffffffffu, v2, gb);
        // Layer 1 splits into the embedding part, which depends on the row only, and the
        // context part (columns 0-3, the tokens u): the embedding part P of the tile's 16
        // contexts is computed once per row (k tiles 0-4 with the u columns zero) and reused
        // for all 56 channels.  Every partial sum is an integer below 2^24: exact in fp32.
        float P[8][4];
        {
            uint32_t A[5][4];
#pragma unroll
            for (int kt = 0; kt < 5; ++kt) {
                const int k = 16 * kt + 2 * t;
                A[kt][0] = pack_bf16f(pe_x(S.sin8, a0, a1, a2, D, k), pe_x(S.sin8, a0, a1, a2, D, k + 1));
                A[kt][1] = pack_bf16f(pe_x(S.sin8, c0, c1, c2, D, k), pe_x(S.sin8, c0, c1, c2, D, k + 1));
                A[kt][2] = pack_bf16f(pe_x(S.sin8, a0, a1, a2, D, k + 8), pe_x(S.sin8, a0, a1, a2, D, k + 9));
                A[kt][3] = pack_bf16f(pe_x(S.sin8, c0, c1, c2, D, k + 8), pe_x(S.sin8, c0, c1, c2, D, k + 9));
            }
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) P[nt][0] = P[nt][1] = P[nt][2] = P[nt][3] = 0.0f;
#pragma unroll
            for (int kt = 0; kt < 5; ++kt)
#pragma unroll
                for (int np = 0; np < 4; ++np) {
                    const uint4 b = S.w1f[kt][np][lane];
                    mma_bf16(P[2 * np], A[kt][0], A[kt][1], A[kt][2], A[kt][3], b.x, b.y);
                    mma_bf16(P[2 * np + 1], A[kt][0], A[kt][1], A[kt][2], A[kt][3], b.z, b.w);
                }
        }
#pragma unroll 1
        for (int c = 0; c < kNChan; ++c) {
            // context part: columns 2t, 2t + 1 (t < 2) of k tile 0 are the tokens u_2t, u_2t+1
            uint32_t u0 = 0u, u1 = 0u;
            if (t < 2) {
                const uint32_t ha = hist[c * 32 + ga] >> (16 * t), hb = hist[c * 32 + gb] >> (16 * t);
                u0 = pack_bf16((int)(ha & 255u) - 128, (int)((ha >> 8) & 255u) - 128);
                u1 = pack_bf16((int)(hb & 255u) - 128, (int)((hb >> 8) & 255u) - 128);
            }
            uint32_t H[4][4];
            {
                float d[8][4];
                // the embedding part enters as the accumulator: every partial sum stays below 2^22
#pragma unroll
                for (int np = 0; np < 4; ++np) {
                    const uint4 b = S.w1f[0][np][lane];
                    mma_bf16_c(d[2 * np], P[2 * np], u0, u1, 0u, 0u, b.x, b.y);
                    mma_bf16_c(d[2 * np + 1], P[2 * np + 1], u0, u1, 0u, 0u, b.z, b.w);
                }
                const float *b1 = S.b1 + c * 64;
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) {
                    const float2 bb = *reinterpret_cast<const float2 *>(b1 + 8 * nt + 2 * t);
                    const int j = (nt & 1) * 2;
                    H[nt >> 1][j] = pe_rq2(d[nt][0] + bb.x, d[nt][1] + bb.y, S.s1);
                    H[nt >> 1][j + 1] = pe_rq2(d[nt][2] + bb.x, d[nt][3] + bb.y, S.s1);
                }
            }
            uint32_t H2[4][4];
            {
                float d[8][4];
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) d[nt][0] = d[nt][1] = d[nt][2] = d[nt][3] = 0.0f;
#pragma unroll
                for (int kt = 0; kt < 4; ++kt)
#pragma unroll
                    for (int np = 0; np < 4; ++np) {
                        const uint4 b = S.w2f[kt][np][lane];
                        mma_bf16(d[2 * np], H[kt][0], H[kt][1], H[kt][2], H[kt][3], b.x, b.y);
                        mma_bf16(d[2 * np + 1], H[kt][0], H[kt][1], H[kt][2], H[kt][3], b.z, b.w);
                    }
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) {
                    const float2 bb = *reinterpret_cast<const float2 *>(S.b2 + 8 * nt + 2 * t);
                    const int j = (nt & 1) * 2;
                    H2[nt >> 1][j] = pe_rq2(d[nt][0] + bb.x, d[nt][1] + bb.y, S.s2);
                    H2[nt >> 1][j + 1] = pe_rq2(d[nt][2] + bb.x, d[nt][3] + bb.y, S.s2);
                }
            }
            float z[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int kt = 0; kt < 4; ++kt) mma_bf16(z, H2[kt][0], H2[kt][1], H2[kt][2], H2[kt][3], w3b[kt][0], w3b[kt][1]);
            if (t == 0) {  // columns 0 (mean) and 1 (rate) of rows g and g + 8
                par[c * 32 + ga] = pe_head(z[0] + S.b3[0], z[1] + S.b3[1], S.smu, S.slr);
                par[c * 32 + gb] = pe_head(z[2] + S.b3[0], z[3] + S.b3[1], S.smu, S.slr);
            }
        }
    }
}

struct PeParams {
    const uint8_t *bits;
    uint64_t model_off, chan_off, grp_sec, pay_off, pay_len;
    uint32_t L, G, n_rows, depth;
    const uint32_t *coord;   // [3][n_rows] voxel coordinates (the octree's output, columns as
                             // the attributes: out_index[row] when a permutation is given)
    float *out;
    const uint32_t *out_index;
    int *status;
    int vec;  // no out_index, 16-byte aligned channels (n_rows % 4 == 0): 8-row stores
};

// The two warps of a group's team synchronise on a named barrier of their own (ids 1..3;
// __syncthreads uses 0).  Both execute the same sequence of barriers.
__device__ __forceinline__ void team_sync(int slot) {
    static_assert(kPeGroups == 3 && kPeTeam == 2, "one barrier id per team, 64 threads each");
    if (slot == 0) asm volatile("bar.sync 1, 64;" ::: "memory");
    else if (slot == 1) asm volatile("bar.sync 2, 64;" ::: "memory");
    else asm volatile("bar.sync 3, 64;" ::: "memory");
}

// One group of 32 lanes, decoded by a team of two warps: per row step each warp runs the
// model for one half of the lanes, then member 0 decodes the row's tokens (the group's word
// stream is read by one warp, in lane order).
__device__ void pe_group(const PeParams &p, PeSmem &S, uint32_t grp, int slot, int member) {
    const int lane = threadIdx.x & 31;
    uint32_t *hist = S.hist[slot], *hist2 = S.hist2[slot], *par = S.par[slot];
    const int nl = (int)min(32u, p.L - grp * 32);
    uint64_t r0 = 0, r1 = 0;
    if (lane < nl) {
        const uint64_t j = (uint64_t)grp * 32 + lane;
        r0 = j * p.n_rows / p.L;
        r1 = (j + 1) * p.n_rows / p.L;
    }
    // A lane's rows are contiguous, so at one row step the warp's stores are W rows apart: each
    // 32-byte sector would fill over 8 steps and leave L2 partly written in between.  Rows in
    // the aligned 8-row blocks inside [r0, r1) are therefore stored when a block's last row is
    // decoded, 8 values (hist2, hist) of each channel as two 16-byte stores; the rows outside
    // those blocks, and every row when the outputs are scattered or unaligned, one by one.
    const uint32_t b0 = ((uint32_t)r0 + 7u) & ~7u, b1 = (uint32_t)r1 & ~7u;  // [b0, b1): rows of whole blocks
    const uint32_t nrows = (uint32_t)(r1 - r0);
    uint32_t maxrows = nrows;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxrows = max(maxrows, __shfl_xor_sync(0xffffffffu, maxrows, o));
    GroupStream gs;
    uint32_t x = 0x10000u;
    if (member == 0) {
        for (int c = 0; c < kNChan; ++c) hist[c * 32 + lane] = 0x80808080u;
        group_open(p.bits, p.grp_sec, p.pay_off, p.pay_len, p.G, grp, nl, lane, gs, x, S.win[slot]);
    }
    team_sync(slot);
    const int D = (int)p.depth;
    for (uint32_t i = 0; i < maxrows; ++i) {
        const bool live = lane < nl && i < nrows;
        const uint64_t row = r0 + i;
        // the octree wrote row r's coordinates, like every output, at column out_index[r]
        const uint64_t col = live ? (p.out_index ? (uint64_t)p.out_index[row] : row) : 0;
        uint32_t v0 = 0, v1 = 0, v2 = 0;
        if (live) {
            v0 = p.coord[col];
            v1 = p.coord[(uint64_t)p.n_rows + col];
            v2 = p.coord[2ull * p.n_rows + col];
        }
        pe_model_half(S, hist, par, v0, v1, v2, D, member);
        team_sync(slot);  // both halves of the row's (mean, rate) are in par
        if (member == 0) {
            const bool defer = p.vec && live && (uint32_t)row >= b0 && (uint32_t)row < b1;
            for (int c = 0; c < kNChan; ++c) {
                if (live) {
                    const uint32_t pr = par[c * 32 + lane];
                    const int mu8 = (int)(pr & 0xFFFFu);
                    const uint32_t R = pe_rate(S.exq, pr >> 16);
                    const uint32_t slot_ = x & 0xFFFFu;
                    // 4-ary search: cdf(s) = lo <= slot < hi = cdf(s + 4 st); three independent
                    // evaluations per level, four levels
                    uint32_t s = 0, lo = 0, hi = 65536u;
#pragma unroll
                    for (uint32_t st = 64; st > 0; st >>= 2) {
                        const uint32_t c1 = pe_cdf(S.exq, mu8, R, s + st), c2 = pe_cdf(S.exq, mu8, R, s + 2 * st),
                                       c3 = pe_cdf(S.exq, mu8, R, s + 3 * st);
                        if (c3 <= slot_) { s += 3 * st; lo = c3; }
                        else if (c2 <= slot_) { s += 2 * st; lo = c2; hi = c3; }
                        else if (c1 <= slot_) { s += st; lo = c1; hi = c2; }
                        else { hi = c1; }
                    }
                    x = (hi - lo) * (x >> 16) + slot_ - lo;
                    const uint32_t h = hist[c * 32 + lane];
                    hist[c * 32 + lane] = (h << 8) | s;
                    hist2[c * 32 + lane] = (hist2[c * 32 + lane] << 8) | (h >> 24);
                    if (!defer) p.out[(uint64_t)c * p.n_rows + col] = dequant(s, S.step[c], S.offset[c]);
                }
                group_refill(gs, x, live);
            }
            if (defer && (row & 7) == 7) {  // rows row - 7 .. row, oldest in hist2's top byte
#pragma unroll 1
                for (int c = 0; c < kNChan; ++c) {
                    const uint32_t ha = hist2[c * 32 + lane], hb = hist[c * 32 + lane];
                    const float st = S.step[c], of = S.offset[c];
                    float4 *dst = reinterpret_cast<float4 *>(p.out + (uint64_t)c * p.n_rows + row - 7);
                    dst[0] = make_float4(dequant(ha >> 24, st, of), dequant((ha >> 16) & 0xFFu, st, of),
                                         dequant((ha >> 8) & 0xFFu, st, of), dequant(ha & 0xFFu, st, of));
                    dst[1] = make_float4(dequant(hb >> 24, st, of), dequant((hb >> 16) & 0xFFu, st, of),
                                         dequant((hb >> 8) & 0xFFu, st, of), dequant(hb & 0xFFu, st, of));
                }
            }
        }
        team_sync(slot);  // the row's tokens are in hist before the next row's model
    }
    if (member == 0) {
        const bool bad = gs.bad || (lane < nl && x != 0x10000u) || (gs.ptr != gs.n_words);
        if (bad) set_status(p.status, SGS_E_CORRUPT);
    }
}

// CTA work unit: groups [vb * kPeGroups, +kPeGroups), one team of two warps each.
__device__ __forceinline__ void pe_body(const PeParams &p, uint32_t vb, bool reload) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    PeSmem &S = *reinterpret_cast<PeSmem *>(smem_raw);
    if (reload) {
        if (!pe_load_model(S, p.bits + p.model_off)) {
            if (threadIdx.x == 0) set_status(p.status, SGS_E_CORRUPT);
            return;
        }
        if (threadIdx.x < kNChan) {
            S.step[threadIdx.x] = ld_f32(p.bits + p.chan_off + 4 * threadIdx.x);
            S.offset[threadIdx.x] = ld_f32(p.bits + p.chan_off + 4 * (kNChan + threadIdx.x));
        }
        __syncthreads();
    } else if (S.bad) {
        return;
    }
    const int warp = threadIdx.x >> 5, slot = warp / kPeTeam;
    const uint32_t grp = vb * kPeGroups + slot;
    if (grp < p.G) pe_group(p, S, grp, slot, warp % kPeTeam);
}

__global__ void __launch_bounds__(kPeThreads, 2) k_learned_pe(PeParams p) { pe_body(p, blockIdx.x, true); }

__global__ void __launch_bounds__(kPeThreads, 2) k_learned_pe_multi(MultiArgs m) {
    run_items<PeParams>(m, [](const PeParams &p, uint32_t vb, uint32_t, bool same) { pe_body(p, vb, !same); });
}

// ------------------------------------------------------------------ encoder side

// f and cum of every token (row-major = lane-major order): one team of two warps per 32
// consecutive rows, each row a context of the model tiles.  A token's context restarts at
// its lane's first row.
__global__ void __launch_bounds__(kPeThreads, 2) k_pe_fc(const uint8_t *model, const uint8_t *tok,
                                                         const uint32_t *coord, int D, uint32_t n_rows,
                                                         uint32_t L, uint32_t *f, uint32_t *cum, int *status) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    PeSmem &S = *reinterpret_cast<PeSmem *>(smem_raw);
    if (!pe_load_model(S, model)) {
        if (threadIdx.x == 0) set_status(status, SGS_E_INVALID);
        return;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, slot = warp / kPeTeam, member = warp % kPeTeam;
    uint32_t *hist = S.hist[slot], *par = S.par[slot];
    const uint64_t first = ((uint64_t)blockIdx.x * kPeGroups + slot) * 32;
    if (first >= n_rows) return;  // the whole team
    const uint64_t row = first + lane;
    const bool live = row < n_rows;
    uint64_t row0 = 0;
    if (live) {
        const uint64_t j = ((row + 1) * L + n_rows - 1) / n_rows - 1;  // the lane holding row
        row0 = j * n_rows / L;
    }
    for (int c = member; c < kNChan; c += kPeTeam) {
        uint32_t h = 0x80808080u;
        if (live)
            for (int j = 4; j >= 1; --j)
                h = (h << 8) | (row >= row0 + (uint64_t)j ? (uint32_t)tok[(row - j) * kNChan + c] : 0x80u);
        hist[c * 32 + lane] = h;
    }
    uint32_t v0 = 0, v1 = 0, v2 = 0;
    if (live) {
        v0 = coord[row];
        v1 = coord[(uint64_t)n_rows + row];
        v2 = coord[2ull * n_rows + row];
    }
    team_sync(slot);
    pe_model_half(S, hist, par, v0, v1, v2, D, member);
    team_sync(slot);
    if (!live) return;
    for (int c = member; c < kNChan; c += kPeTeam) {
        const uint32_t pr = par[c * 32 + lane];
        const int mu8 = (int)(pr & 0xFFFFu);
        const uint32_t R = pe_rate(S.exq, pr >> 16);
        const uint32_t s = tok[row * kNChan + c];
        const uint32_t lo = s == 0 ? 0u : pe_cdf(S.exq, mu8, R, s);
        const uint32_t hi = s == 255 ? 65536u : pe_cdf(S.exq, mu8, R, s + 1);
        f[row * kNChan + c] = hi - lo;
        cum[row * kNChan + c] = lo;
    }
}

uint32_t make_pe(const uint8_t *bits, const sgs_scene_info &info, const sgs_scene_out &out,
                 const uint32_t *coord, int *status, PeParams *pp) {
    PeParams &p = *pp;
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
    p.depth = info.depth;
    p.coord = coord;
    p.out = out.attr;
    p.out_index = out.out_index;
    p.status = status;
    p.vec = !out.out_index && info.n_rows % 4 == 0 && ((uintptr_t)out.attr & 15) == 0;
    return info.n_rows ? (p.G + kPeGroups - 1) / kPeGroups : 0;
}

cudaError_t pe_smem_limit(const void *kernel, bool *done) {
    if (*done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(PeSmem));
    if (e == cudaSuccess) *done = true;
    return e;
}

}  // namespace

cudaError_t launch_learned_pe_decode(const uint8_t *bits, const sgs_scene_info &info, const sgs_scene_out &out,
                                     const uint32_t *coord, int *status, cudaStream_t st) {
    PeParams p;
    const uint32_t grid = make_pe(bits, info, out, coord, status, &p);
    if (grid == 0) return cudaSuccess;
    static bool set = false;
    cudaError_t e = pe_smem_limit(reinterpret_cast<const void *>(k_learned_pe), &set);
    if (e != cudaSuccess) return e;
    k_learned_pe<<<grid, kPeThreads, sizeof(PeSmem), st>>>(p);
    return cudaGetLastError();
}

uint32_t stage_learned_pe(const SceneRef &r, void *par) {
    if (r.info->mode != SGS_MODE_LEARNED_PE) return 0;
    PeParams p;
    const uint32_t n = make_pe(r.bits, *r.info, *r.out, r.out->coord, r.status, &p);
    memcpy(par, &p, sizeof(p));
    return n;
}
size_t stage_learned_pe_bytes() { return sizeof(PeParams); }
cudaError_t launch_learned_pe_multi(const MultiArgs &m, cudaStream_t st) {
    static bool set = false;
    cudaError_t e = pe_smem_limit(reinterpret_cast<const void *>(k_learned_pe_multi), &set);
    if (e != cudaSuccess) return e;
    return launch_persistent(k_learned_pe_multi, kPeThreads, sizeof(PeSmem), m, st);
}

cudaError_t launch_pe_fc(const uint8_t *model_dev, const uint8_t *tok_dev, const uint32_t *coord_dev, int depth,
                         uint32_t n_rows, uint32_t lanes, uint32_t *f_dev, uint32_t *cum_dev, int *status,
                         cudaStream_t st) {
    if (n_rows == 0) return cudaSuccess;
    static bool set = false;
    cudaError_t e = pe_smem_limit(reinterpret_cast<const void *>(k_pe_fc), &set);
    if (e != cudaSuccess) return e;
    const uint32_t teams = (n_rows + 31) / 32;
    k_pe_fc<<<(teams + kPeGroups - 1) / kPeGroups, kPeThreads, sizeof(PeSmem), st>>>(
        model_dev, tok_dev, coord_dev, depth, n_rows, lanes, f_dev, cum_dev, status);
    return cudaGetLastError();
}

int rans_encode_device(const uint32_t *f, const uint32_t *cum, const std::vector<uint64_t> &lane_start,
                       std::vector<uint8_t> &grp, std::vector<uint8_t> &pay);

// The bounds the decoder checks (host copy of pe_load_model's test).
bool pe_model_valid(const uint8_t *m) {
    float sc[4];
    memcpy(sc, m, sizeof(sc));
    if (!(sc[0] > 0.0f && sc[0] <= 127.0f && sc[1] > 0.0f && sc[1] <= 127.0f && sc[2] > 0.0f && sc[2] < 3.0e38f &&
          sc[3] > 0.0f && sc[3] < 3.0e38f))
        return false;
    auto ok = [&](int off, int count) {
        for (int i = 0; i < count; ++i) {
            int32_t v;
            memcpy(&v, m + off + 4 * i, 4);
            if (v <= -(1 << 23) || v >= (1 << 23)) return false;
        }
        return true;
    };
    return ok(kPB_B1, kNChan * 64) && ok(kPB_B2, 64) && ok(kPB_B3, 2);
}

// Position-aware attribute coding on the device: f and cum of every token from the frozen
// model (k_pe_fc), then the interleaved rANS coder.  tokens row-major [n_rows][56], coord
// [3][n_rows] (host).
int learned_pe_encode_device(const uint8_t *model, const uint8_t *tokens, const uint32_t *coord, uint32_t depth,
                             uint32_t n_rows, uint32_t lanes, const std::vector<uint64_t> &lane_start,
                             std::vector<uint8_t> &grp, std::vector<uint8_t> &pay) {
    const uint64_t n = (uint64_t)n_rows * kNChan;
    uint8_t *dm = nullptr, *dt = nullptr;
    uint32_t *dcrd = nullptr, *df = nullptr, *dc = nullptr;
    int *dst = nullptr;
    int rc = SGS_OK;
    if (cudaMalloc(&dm, SGS_MODEL_PE_BYTES) != cudaSuccess || cudaMalloc(&dt, n ? n : 1) != cudaSuccess ||
        cudaMalloc(&dcrd, 12ull * (n_rows ? n_rows : 1)) != cudaSuccess ||
        cudaMalloc(&df, 4 * (n ? n : 1)) != cudaSuccess || cudaMalloc(&dc, 4 * (n ? n : 1)) != cudaSuccess ||
        cudaMalloc(&dst, sizeof(int)) != cudaSuccess) {
        rc = SGS_E_NOMEM;
    } else if (cudaMemcpy(dm, model, SGS_MODEL_PE_BYTES, cudaMemcpyHostToDevice) != cudaSuccess ||
               (n && cudaMemcpy(dt, tokens, n, cudaMemcpyHostToDevice) != cudaSuccess) ||
               (n_rows && cudaMemcpy(dcrd, coord, 12ull * n_rows, cudaMemcpyHostToDevice) != cudaSuccess) ||
               cudaMemset(dst, 0, sizeof(int)) != cudaSuccess) {
        rc = SGS_E_CUDA;
    } else {
        if (launch_pe_fc(dm, dt, dcrd, (int)depth, n_rows, lanes, df, dc, dst, 0) != cudaSuccess) rc = SGS_E_CUDA;
        int st = 0;
        if (rc == SGS_OK && cudaMemcpy(&st, dst, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = SGS_E_CUDA;
        if (rc == SGS_OK && st != 0) rc = st;
        if (rc == SGS_OK) rc = rans_encode_device(df, dc, lane_start, grp, pay);
    }
    cudaFree(dm);
    cudaFree(dt);
    cudaFree(dcrd);
    cudaFree(df);
    cudaFree(dc);
    cudaFree(dst);
    return rc;
}

}  // namespace sgs
