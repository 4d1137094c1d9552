// Scene encoder of the sgs library (host C++; given a context, the scene's preparation --
// prune, Morton sort, octree, quantization -- and the attribute coding run on the device).  Pipeline (Sec. 3.3-3.4):
//   prune floor(n/10) Gaussians of lowest opacity (ties: lower index first) -> voxelize at
//   depth D -> sort rows by (Morton code, original index) -> sparse-octree occupancy tokens
//   per level, duplicate counts as metadata -> per-channel uniform quantization
//   (offset = min, step = fl32((max-min)/(2^b-1)), q = clamp(rint((v-offset)/step))) ->
//   channel-wise fixed-length packing, static-frequency rANS, or learned-model rANS (the
//   plain model or the position-aware one).
// The output bytes are fully determined by the inputs (all tie-breaks fixed), so any two
// correct encoders produce identical bitstreams.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "exp2q_table.h"
#include "sgs_ctx.h"
#include "sgs_internal.h"
#include "encode_prep.h"

namespace sgs {
namespace {

constexpr uint32_t kM = 1u << 16;


uint64_t morton3(uint32_t x, uint32_t y, uint32_t z, uint32_t D) {
    uint64_t m = 0;
    for (uint32_t b = 0; b < D; ++b) {
        m |= (uint64_t)((x >> b) & 1u) << (3 * b + 2);
        m |= (uint64_t)((y >> b) & 1u) << (3 * b + 1);
        m |= (uint64_t)((z >> b) & 1u) << (3 * b);
    }
    return m;
}

int prepare(const float *pos, const float *attr, uint32_t n, uint32_t D, const uint32_t *bits,
            Prepared &P) {
    if (D < 1 || D > SGS_MAX_DEPTH) return SGS_E_INVALID;
    for (int c = 0; c < kNChan; ++c)
        if (bits[c] < 1 || bits[c] > 16) return SGS_E_INVALID;
    for (uint64_t i = 0; i < 3ull * n; ++i)
        if (!(pos[i] >= 0.0f && pos[i] < 1.0f)) return SGS_E_INVALID;
    for (uint64_t i = 0; i < (uint64_t)kNChan * n; ++i)
        if (!isfinite(attr[i])) return SGS_E_INVALID;
    P.depth = D;
    P.n_in = n;
    memcpy(P.bits, bits, sizeof(P.bits));
    // prune: order by (opacity, index), drop the first floor(n/10)
    const float *op = attr + 48ull * n;
    std::vector<uint32_t> idx(n);
    std::iota(idx.begin(), idx.end(), 0u);
    std::sort(idx.begin(), idx.end(), [&](uint32_t a, uint32_t b) {
        return op[a] < op[b] || (op[a] == op[b] && a < b);
    });
    std::vector<uint32_t> keep(idx.begin() + n / 10, idx.end());
    std::sort(keep.begin(), keep.end());
    // voxelize + Morton
    const double scale = (double)(1u << D);
    const double vmax = (double)((1u << D) - 1);
    std::vector<uint64_t> code(keep.size());
    for (size_t r = 0; r < keep.size(); ++r) {
        uint32_t v[3];
        for (int k = 0; k < 3; ++k) {
            double t = floor((double)pos[(uint64_t)k * n + keep[r]] * scale);
            v[k] = (uint32_t)std::min(t, vmax);
        }
        code[r] = morton3(v[0], v[1], v[2], D);
    }
    std::vector<uint32_t> ord(keep.size());
    std::iota(ord.begin(), ord.end(), 0u);
    std::sort(ord.begin(), ord.end(), [&](uint32_t a, uint32_t b) {
        return code[a] < code[b] || (code[a] == code[b] && keep[a] < keep[b]);
    });
    P.keep.resize(keep.size());
    std::vector<uint64_t> sc(keep.size());
    P.coord.assign(3 * keep.size(), 0);
    for (size_t r = 0; r < ord.size(); ++r) {
        P.keep[r] = keep[ord[r]];
        sc[r] = code[ord[r]];
        for (uint32_t b = 0; b < D; ++b)
            for (int k = 0; k < 3; ++k)
                P.coord[k * keep.size() + r] |= (uint32_t)((sc[r] >> (3 * b + 2 - k)) & 1u) << b;
    }
    // unique voxels and duplicate counts
    for (size_t r = 0; r < sc.size();) {
        size_t e = r + 1;
        while (e < sc.size() && sc[e] == sc[r]) ++e;
        if (e - r > 1) {
            P.dups.push_back((uint32_t)P.leaves.size());
            P.dups.push_back((uint32_t)(e - r - 1));
        }
        P.leaves.push_back(sc[r]);
        r = e;
    }
    // octree tokens per level
    P.levels.assign(D, {});
    for (uint32_t l = 0; l < D && !P.leaves.empty(); ++l) {
        const uint32_t sn = 3 * (D - l), sk = 3 * (D - l - 1);
        auto &lv = P.levels[l];
        uint64_t cur = P.leaves[0] >> sn;
        uint8_t byte = 0;
        for (uint64_t m : P.leaves) {
            const uint64_t node = m >> sn;
            if (node != cur) {
                lv.push_back(byte);
                byte = 0;
                cur = node;
            }
            byte |= (uint8_t)(1u << ((m >> sk) & 7u));
        }
        lv.push_back(byte);
    }
    // per-channel quantization
    const uint32_t R = P.rows();
    P.q16.assign((size_t)R * kNChan, 0);
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < kNChan; ++c) {
        const float *v = attr + (uint64_t)c * n;
        if (R == 0) {
            P.step[c] = 0.0f;
            P.offset[c] = 0.0f;
            continue;
        }
        float mn = v[P.keep[0]], mx = mn;
        for (uint32_t r = 1; r < R; ++r) {
            const float a = v[P.keep[r]];
            mn = a < mn ? a : mn;
            mx = a > mx ? a : mx;
        }
        const uint32_t top = (1u << bits[c]) - 1u;
        const float step = (mx == mn) ? 0.0f : (float)(((double)mx - (double)mn) / (double)top);
        P.step[c] = step;
        P.offset[c] = mn;
        if (step == 0.0f) continue;
        for (uint32_t r = 0; r < R; ++r) {
            double t = nearbyint(((double)v[P.keep[r]] - (double)mn) / (double)step);
            t = std::min(std::max(t, 0.0), (double)top);
            P.q16[(size_t)r * kNChan + c] = (uint16_t)t;
        }
    }
    return SGS_OK;
}

// Static 16-bit table: f = 1 + floor(h (2^16 - K) / sum) for present symbols, remainder to
// the most frequent symbol (lowest index on ties).
void normalize(const uint64_t *h, uint32_t *f) {
    uint64_t tot = 0, K = 0;
    int amax = 0;
    for (int s = 0; s < kNSym; ++s) {
        tot += h[s];
        K += h[s] > 0;
        if (h[s] > h[amax]) amax = s;
    }
    uint64_t sum = 0;
    for (int s = 0; s < kNSym; ++s) {
        f[s] = h[s] ? (uint32_t)(1 + h[s] * (kM - K) / tot) : 0u;
        sum += f[s];
    }
    if (tot) f[amax] += (uint32_t)(kM - sum);
}

void put_table(std::vector<uint8_t> &o, const uint32_t *f) {
    uint8_t mask[32] = {0};
    for (int s = 0; s < kNSym; ++s)
        if (f[s]) mask[s >> 3] |= (uint8_t)(1u << (s & 7));
    o.insert(o.end(), mask, mask + 32);
    for (int s = 0; s < kNSym; ++s)
        if (f[s]) {
            const uint32_t v = f[s] - 1;
            o.push_back((uint8_t)v);
            o.push_back((uint8_t)(v >> 8));
        }
    while (o.size() % 16) o.push_back(0);
}

// Interleaved rANS: lanes of 32 share a stream; per group, encode steps in reverse (t and
// lane descending), push the final states as (lo, hi) for lanes descending, reverse.
// sym_f / sym_c: frequency and cumulative of every token, lane-major (lane_start offsets).
void rans_encode(const std::vector<uint64_t> &lane_start, const uint32_t *sym_f,
                 const uint32_t *sym_c, std::vector<uint8_t> &grp, std::vector<uint8_t> &pay) {
    const int64_t L = (int64_t)lane_start.size() - 1;
    const int64_t G = (L + 31) / 32;
    std::vector<std::vector<uint16_t>> words(G);  // each group's stream, in emission order
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t g = 0; g < G; ++g) {
        const int64_t j0 = 32 * g, j1 = std::min(L, j0 + 32);
        const int nl = (int)(j1 - j0);
        uint64_t maxn = 0;
        for (int64_t j = j0; j < j1; ++j) maxn = std::max(maxn, lane_start[j + 1] - lane_start[j]);
        std::vector<uint16_t> &w = words[g];
        uint32_t x[32];
        for (int j = 0; j < nl; ++j) x[j] = kM;
        for (uint64_t tt = maxn; tt-- > 0;) {
            for (int j = nl - 1; j >= 0; --j) {
                const uint64_t n = lane_start[j0 + j + 1] - lane_start[j0 + j];
                if (tt >= n) continue;
                const uint64_t p = lane_start[j0 + j] + tt;
                const uint32_t f = sym_f[p], cu = sym_c[p];
                if ((uint64_t)x[j] >= ((uint64_t)f << 16)) {
                    w.push_back((uint16_t)(x[j] & 0xFFFFu));
                    x[j] >>= 16;
                }
                x[j] = ((x[j] / f) << 16) + (x[j] % f) + cu;
            }
        }
        for (int j = nl - 1; j >= 0; --j) {
            w.push_back((uint16_t)(x[j] & 0xFFFFu));
            w.push_back((uint16_t)(x[j] >> 16));
        }
    }
    // assemble: each group's words reversed, little endian, padded to 16 bytes
    std::vector<uint64_t> goff(G + 1, 0);
    std::vector<uint32_t> gw(G, 0);
    for (int64_t g = 0; g < G; ++g) {
        gw[g] = (uint32_t)words[g].size();
        goff[g + 1] = goff[g] + ((2ull * gw[g] + 15) & ~15ull);
    }
    const size_t base = pay.size();
    pay.resize(base + goff[G], 0);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t g = 0; g < G; ++g) {
        uint8_t *o = pay.data() + base + goff[g];
        const std::vector<uint16_t> &w = words[g];
        for (size_t k = w.size(), i = 0; k-- > 0; ++i) {
            o[2 * i] = (uint8_t)(w[k] & 0xFF);
            o[2 * i + 1] = (uint8_t)(w[k] >> 8);
        }
    }
    for (int64_t g = 0; g <= G; ++g) goff[g] += base;
    grp.resize(8 * (G + 1) + 4 * G);
    memcpy(grp.data(), goff.data(), 8 * (G + 1));
    memcpy(grp.data() + 8 * (G + 1), gw.data(), 4 * G);
    while (grp.size() % 16) grp.push_back(0);
}

// Static-table coding (attribute rows, octree tokens): group g of 32 lanes owns the items
// its lanes would own as contiguous chunks and deals them round robin to its lanes (lane j:
// items R_g + j + k n_g), so the 32 lanes of a group always hold 32 consecutive items.
// Returns the items in lane-major coding order and each lane's start offset.
void static_row_order(uint64_t n, uint64_t L, std::vector<uint32_t> &perm, std::vector<uint64_t> &start) {
    perm.resize(n);
    start.assign(L + 1, 0);
    uint64_t pos = 0;
    for (uint64_t j0 = 0; j0 < L; j0 += 32) {
        const uint64_t j1 = std::min(L, j0 + 32), nl = j1 - j0;
        const uint64_t R0 = j0 * n / L, R1 = j1 * n / L;
        for (uint64_t jj = 0; jj < nl; ++jj) {
            for (uint64_t r = R0 + jj; r < R1; r += nl) perm[pos++] = (uint32_t)r;
            start[j0 + jj + 1] = pos;
        }
    }
}

std::vector<uint64_t> lane_bounds(uint64_t n, uint64_t L, uint64_t mul) {
    std::vector<uint64_t> b(L + 1);
    for (uint64_t j = 0; j <= L; ++j) b[j] = (j * n / L) * mul;
    return b;
}

void pack_fixed(const Prepared &P, int c, std::vector<uint8_t> &o) {
    const uint32_t b = P.bits[c], R = P.rows();
    if (R == 0) return;
    const uint64_t nw = ((uint64_t)R * b + 31) / 32;
    std::vector<uint32_t> w(nw, 0);
    for (uint32_t r = 0; r < R; ++r) {
        const uint64_t v = P.q16[(size_t)r * kNChan + c];
        const uint64_t bit = (uint64_t)r * b;
        const uint64_t wi = bit >> 5, sh = bit & 31;
        w[wi] |= (uint32_t)(v << sh);
        if (sh + b > 32) w[wi + 1] |= (uint32_t)(v >> (32 - sh));
    }
    const size_t at = o.size();
    o.resize(at + 4 * nw);
    memcpy(o.data() + at, w.data(), 4 * nw);
    while (o.size() % 16) o.push_back(0);
}

void pad16(std::vector<uint8_t> &v) {
    while (v.size() % 16) v.push_back(0);
}

template <typename T>
void put(std::vector<uint8_t> &o, T v) {
    const uint8_t *p = reinterpret_cast<const uint8_t *>(&v);
    o.insert(o.end(), p, p + sizeof(T));
}

uint32_t default_geo_lanes(uint64_t n) {
    const uint64_t per = 128ull * 32;
    return (uint32_t)std::max<uint64_t>(32, (n + per - 1) / per * 32);
}

// ---- the learned model's integer frequencies on the host (for the learned geometry coder)
//
// Frozen model blob (SGS_MODEL_BYTES, little endian): i32 m1, sh1, m2, sh2, ms, ss, then 8
// zero bytes; i32 B1[56][64]; i32 b2[64]; i32 b3[256]; i8 W1[64][4]; i8 W2[64][64];
// i8 W3[256][64].  Inference: acc1 = W1 u + B1[c], h1 = rq(acc1; m1, sh1), acc2 = W2 h1 + b2,
// h2 = rq(acc2; m2, sh2), z = W3 h2 + b3, rq(a; m, sh) = clamp((a m + 2^(sh-1)) >> sh, 0, 127)
// in 64-bit arithmetic; then the integer softmax: d_k = zmax - z_k, t_k = min((d_k ms) >> ss,
// 6144), e_k = EXP2Q[t_k & 255] >> (t_k >> 8), R = floor(65280 2^32 / sum e), f_k = 1 +
// floor(e_k R / 2^32), and the remainder 2^16 - sum f added at the lowest index of max z.
constexpr size_t kMB1 = 32, kMb2 = 14368, kMb3 = 14624, kMW1 = 15648, kMW2 = 15904, kMW3 = 20000;
constexpr uint32_t kExp2QTab[256] = {SGS_EXP2Q_VALUES};
static_assert(kMW3 + 256 * 64 == SGS_MODEL_BYTES, "model layout");

int32_t rdi(const uint8_t *m, size_t off) {
    int32_t v;
    memcpy(&v, m + off, 4);
    return v;
}

struct HostModel {
    const uint8_t *m = nullptr;
    int32_t m1 = 0, sh1 = 0, m2 = 0, sh2 = 0;
    uint32_t ms = 0, ss = 0;
};

// Reads the header scalars and checks the ranges every decoder relies on (shifts, multipliers,
// biases below 2^24 in magnitude).
bool host_model(const uint8_t *m, HostModel &H) {
    if (!m) return false;
    H.m = m;
    H.m1 = rdi(m, 0); H.sh1 = rdi(m, 4); H.m2 = rdi(m, 8); H.sh2 = rdi(m, 12);
    H.ms = (uint32_t)rdi(m, 16); H.ss = (uint32_t)rdi(m, 20);
    if (!(H.sh1 >= 1 && H.sh1 <= 47 && H.sh2 >= 1 && H.sh2 <= 47 && H.m1 >= 0 && H.m2 >= 0 && H.ms >= 1 &&
          H.ms < (1u << 24) && H.ss <= 24))
        return false;
    auto ok = [&](size_t off, int n) {
        for (int i = 0; i < n; ++i) {
            const int32_t v = rdi(m, off + 4 * (size_t)i);
            if (v >= (1 << 24) || v <= -(1 << 24)) return false;
        }
        return true;
    };
    return ok(kMB1, kNChan * 64) && ok(kMb2, 64) && ok(kMb3, 256);
}

int64_t requant_host(int64_t a, int32_t m, int32_t sh) {
    const int64_t v = (a * (int64_t)m + ((int64_t)1 << (sh - 1))) >> sh;
    return v < 0 ? 0 : (v > 127 ? 127 : v);
}

void learned_freq_host(const HostModel &H, const int32_t u[4], int c, uint32_t *f) {
    const int8_t *W1 = reinterpret_cast<const int8_t *>(H.m + kMW1);
    const int8_t *W2 = reinterpret_cast<const int8_t *>(H.m + kMW2);
    const int8_t *W3 = reinterpret_cast<const int8_t *>(H.m + kMW3);
    int64_t h1[64], h2[64];
    for (int o = 0; o < 64; ++o) {
        int64_t a = rdi(H.m, kMB1 + 4 * ((size_t)c * 64 + o));
        for (int j = 0; j < 4; ++j) a += (int64_t)W1[4 * o + j] * u[j];
        h1[o] = requant_host(a, H.m1, H.sh1);
    }
    for (int o = 0; o < 64; ++o) {
        int64_t a = rdi(H.m, kMb2 + 4 * (size_t)o);
        for (int k = 0; k < 64; ++k) a += (int64_t)W2[64 * o + k] * h1[k];
        h2[o] = requant_host(a, H.m2, H.sh2);
    }
    int64_t z[kNSym];
    int amax = 0;
    for (int s = 0; s < kNSym; ++s) {
        int64_t a = rdi(H.m, kMb3 + 4 * (size_t)s);
        for (int k = 0; k < 64; ++k) a += (int64_t)W3[64 * s + k] * h2[k];
        z[s] = a;
        if (a > z[amax]) amax = s;
    }
    uint64_t e[kNSym], E = 0;
    for (int s = 0; s < kNSym; ++s) {
        const uint64_t t = std::min<uint64_t>(((uint64_t)(z[amax] - z[s]) * H.ms) >> H.ss, 6144);
        e[s] = kExp2QTab[t & 255] >> (t >> 8);
        E += e[s];
    }
    const uint64_t R = (65280ull << 32) / E;
    uint32_t sum = 0;
    for (int s = 0; s < kNSym; ++s) {
        f[s] = 1u + (uint32_t)((e[s] * R) >> 32);
        sum += f[s];
    }
    f[amax] += kM - sum;
}

// Learned geometry (SGS_GEO_LEARNED): level l's nodes, in order, are the set bits k (ascending)
// of each byte b of level l - 1; node context 8 b + k; the model's inputs of a context.
void geo_inputs(uint32_t ctx, int32_t u[4]) {
    const uint32_t b = ctx >> 3, k = ctx & 7;
    u[0] = (int32_t)b - 128;
    u[1] = 32 * (int32_t)k - 112;
    u[2] = 16 * __builtin_popcount(b) - 64;
    u[3] = 32 * __builtin_popcount(b & ((1u << k) - 1u)) - 112;
}

}  // namespace

// Interleaved rANS coding of the attribute streams on the device (k_encode.cu; the learned
// model's frequencies in k_learned.cu), byte for byte as rans_encode above.
int rans_encode_static_device(const uint8_t *tok_lane_major, uint64_t nsym, const uint32_t *ftab,
                              const std::vector<uint64_t> &lane_start, std::vector<uint8_t> &grp,
                              std::vector<uint8_t> &pay);
int learned_encode_device(const uint8_t *model, const uint8_t *tokens, uint32_t n_rows, uint32_t lanes,
                          const std::vector<uint64_t> &lane_start, std::vector<uint8_t> &grp,
                          std::vector<uint8_t> &pay);
bool pe_model_valid(const uint8_t *model);
int learned_pe_encode_device(const uint8_t *model, const uint8_t *tokens, const uint32_t *coord, uint32_t depth,
                             uint32_t n_rows, uint32_t lanes, const std::vector<uint64_t> &lane_start,
                             std::vector<uint8_t> &grp, std::vector<uint8_t> &pay);

}  // namespace sgs

using namespace sgs;

extern "C" int scene_tokens(const float *pos, const float *attr, uint32_t n, uint32_t depth,
                            uint8_t *tokens, size_t cap, uint32_t *n_rows) {
    if (!pos || !attr || !n_rows) return SGS_E_INVALID;
    uint32_t bits[kNChan];
    for (int c = 0; c < kNChan; ++c) bits[c] = 8;
    Prepared P;
    int r = prepare(pos, attr, n, depth, bits, P);
    if (r) return r;
    *n_rows = P.rows();
    if (cap < (size_t)P.rows() * kNChan || (!tokens && P.rows())) return SGS_E_INVALID;
    for (size_t i = 0; i < (size_t)P.rows() * kNChan; ++i) tokens[i] = (uint8_t)P.q16[i];
    return SGS_OK;
}

extern "C" int scene_rows(const float *pos, const float *attr, uint32_t n, uint32_t depth, uint8_t *tokens,
                          uint32_t *coord, uint32_t cap, uint32_t *n_rows) {
    if (!pos || !attr || !n_rows) return SGS_E_INVALID;
    uint32_t bits[kNChan];
    for (int c = 0; c < kNChan; ++c) bits[c] = 8;
    Prepared P;
    int r = prepare(pos, attr, n, depth, bits, P);
    if (r) return r;
    const uint32_t R = P.rows();
    *n_rows = R;
    if (cap < R || ((!tokens || !coord) && R)) return SGS_E_INVALID;
    for (size_t i = 0; i < (size_t)R * kNChan; ++i) tokens[i] = (uint8_t)P.q16[i];
    for (int k = 0; k < 3; ++k) memcpy(coord + (size_t)k * R, P.coord.data() + (size_t)k * R, 4ull * R);
    return SGS_OK;
}

extern "C" int scene_geo_samples(const float *pos, const float *attr, uint32_t n, uint32_t depth, int32_t *u,
                                 uint32_t *chan, uint8_t *sym, uint64_t cap, uint64_t *n_samples) {
    if (!pos || !attr || !n_samples) return SGS_E_INVALID;
    uint32_t bits[kNChan];
    for (int c = 0; c < kNChan; ++c) bits[c] = 8;
    Prepared P;
    int r = prepare(pos, attr, n, depth, bits, P);
    if (r) return r;
    uint64_t total = 0;
    for (uint32_t l = 1; l < depth; ++l)
        if (P.levels[l].size() >= kGeoRansMinLevel) total += P.levels[l].size();
    *n_samples = total;
    if (cap < total || ((!u || !chan || !sym) && total)) return SGS_E_INVALID;
    uint64_t k = 0;
    for (uint32_t l = 1; l < depth; ++l) {
        if (P.levels[l].size() < kGeoRansMinLevel) continue;
        uint64_t j = 0;
        for (uint8_t b : P.levels[l - 1])
            for (uint32_t kk = 0; kk < 8; ++kk)
                if ((b >> kk) & 1u) {
                    if (j >= P.levels[l].size()) return SGS_E_INVALID;
                    geo_inputs(8u * b + kk, u + 4 * (k + j));
                    chan[k + j] = l;
                    sym[k + j] = P.levels[l][j];
                    ++j;
                }
        if (j != P.levels[l].size()) return SGS_E_INVALID;
        k += j;
    }
    return SGS_OK;
}

extern "C" int scene_encode(sgs_ctx *ctx, const float *pos, const float *attr, uint32_t n,
                            const sgs_encode_params *prm, uint8_t *out, size_t cap,
                            size_t *out_len) {
    if (!prm || !out_len || (n && (!pos || !attr))) return SGS_E_INVALID;
    if (prm->mode > SGS_MODE_LEARNED_PE || prm->geo_mode > SGS_GEO_LEARNED) return SGS_E_INVALID;
    uint32_t bits[kNChan];
    for (int c = 0; c < kNChan; ++c) bits[c] = prm->mode == SGS_MODE_FIXED ? prm->bits[c] : 8u;
    if (prm->mode != SGS_MODE_FIXED && prm->lanes < 1) return SGS_E_INVALID;
    if (prm->mode == SGS_MODE_LEARNED && (!prm->model || !ctx)) return SGS_E_INVALID;
    if (prm->mode == SGS_MODE_LEARNED_PE &&
        (!prm->model || !ctx || !pe_model_valid(static_cast<const uint8_t *>(prm->model))))
        return SGS_E_INVALID;
    // with a context the scene is prepared on its device (k_prepare.cu), else on the host:
    // the same rows, octree and quantized values either way
    Prepared P;
    int r = ctx ? prepare_device(ctx->device, pos, attr, n, prm->depth, bits, P) : prepare(pos, attr, n, prm->depth, bits, P);
    if (r) return r;
    const uint32_t D = prm->depth, R = P.rows();
    // geometry
    std::vector<uint8_t> s_levels, s_dup, s_chan, s_graw, s_gtab, s_ggrp, s_gpay;
    std::vector<int> coded_levels;
    uint64_t n_geo = 0, n_coded = 0;
    for (uint32_t l = 0; l < D; ++l) {
        const uint32_t nl = (uint32_t)P.levels[l].size();
        put<uint32_t>(s_levels, nl);
        n_geo += nl;
        if (prm->geo_mode != SGS_GEO_RAW && nl >= kGeoRansMinLevel) {
            coded_levels.push_back((int)l);
            n_coded += nl;
        } else {
            s_graw.insert(s_graw.end(), P.levels[l].begin(), P.levels[l].end());
        }
    }
    uint32_t Lg = 0;
    if (n_coded && prm->geo_mode == SGS_GEO_LEARNED) {
        // one model for every coded level (the geometry table section); each level's tokens
        // in lanes of contiguous chunks, about 128 tokens per lane, coded with the frequency
        // tables of their contexts; the levels' group tables follow one another and point
        // into one payload
        HostModel H;
        if (!host_model(static_cast<const uint8_t *>(prm->geo_model), H)) return SGS_E_INVALID;
        const uint8_t *gm = static_cast<const uint8_t *>(prm->geo_model);
        s_gtab.assign(gm, gm + SGS_MODEL_BYTES);
        std::vector<uint32_t> F((size_t)2048 * kNSym), C((size_t)2048 * kNSym);
        for (int l : coded_levels) {
            const std::vector<uint8_t> &par = P.levels[l - 1], &cur = P.levels[l];
            std::vector<uint16_t> ctx;
            ctx.reserve(cur.size());
            for (uint8_t b : par)
                for (uint32_t k = 0; k < 8; ++k)
                    if ((b >> k) & 1u) ctx.push_back((uint16_t)(8u * b + k));
            if (ctx.size() != cur.size()) return SGS_E_INVALID;
            std::vector<uint8_t> present(2048, 0);
            for (uint16_t x : ctx) present[x] = 1;
            std::vector<int> ids;
            for (int x = 0; x < 2048; ++x)
                if (present[x]) ids.push_back(x);
#pragma omp parallel for schedule(dynamic, 8)
            for (int64_t i = 0; i < (int64_t)ids.size(); ++i) {
                int32_t u[4];
                geo_inputs((uint32_t)ids[i], u);
                uint32_t *f = &F[(size_t)ids[i] * kNSym], *cu = &C[(size_t)ids[i] * kNSym];
                learned_freq_host(H, u, l, f);
                uint32_t acc = 0;
                for (int s2 = 0; s2 < kNSym; ++s2) { cu[s2] = acc; acc += f[s2]; }
            }
            std::vector<uint32_t> tf(cur.size()), tcu(cur.size());
            for (size_t p = 0; p < cur.size(); ++p) {
                tf[p] = F[(size_t)ctx[p] * kNSym + cur[p]];
                tcu[p] = C[(size_t)ctx[p] * kNSym + cur[p]];
            }
            const uint32_t Ll = default_geo_lanes(cur.size());
            Lg += Ll;
            std::vector<uint8_t> grp;
            rans_encode(lane_bounds(cur.size(), Ll, 1), tf.data(), tcu.data(), grp, s_gpay);
            s_ggrp.insert(s_ggrp.end(), grp.begin(), grp.end());
        }
    } else if (n_coded) {
        Lg = prm->geo_lanes ? prm->geo_lanes : default_geo_lanes(n_coded);
        std::vector<uint32_t> tf(n_coded), tcu(n_coded);  // in token order
        uint64_t p = 0;
        for (int l : coded_levels) {
            uint64_t h[kNSym] = {0};
            for (uint8_t b : P.levels[l]) h[b]++;
            uint32_t f[kNSym], cu[kNSym];
            normalize(h, f);
            put_table(s_gtab, f);
            uint32_t acc = 0;
            for (int s = 0; s < kNSym; ++s) { cu[s] = acc; acc += f[s]; }
            for (uint8_t b : P.levels[l]) { tf[p] = f[b]; tcu[p] = cu[b]; ++p; }
        }
        // tokens dealt round robin to the lanes of each group, as for static attributes
        std::vector<uint32_t> perm, sf(n_coded), scu(n_coded);
        std::vector<uint64_t> gstart;
        static_row_order(n_coded, Lg, perm, gstart);
        for (uint64_t i = 0; i < n_coded; ++i) { sf[i] = tf[perm[i]]; scu[i] = tcu[perm[i]]; }
        rans_encode(gstart, sf.data(), scu.data(), s_ggrp, s_gpay);
    }
    for (size_t i = 0; i < P.dups.size(); ++i) put<uint32_t>(s_dup, P.dups[i]);
    for (int c = 0; c < kNChan; ++c) put<float>(s_chan, P.step[c]);
    for (int c = 0; c < kNChan; ++c) put<float>(s_chan, P.offset[c]);
    for (int c = 0; c < kNChan; ++c) put<uint32_t>(s_chan, P.bits[c]);
    // attributes
    std::vector<uint8_t> s_atab, s_agrp, s_apay;
    uint32_t L = 0;
    if (prm->mode == SGS_MODE_FIXED) {
        std::vector<uint64_t> offs;
        for (int c = 0; c < kNChan; ++c) {
            offs.push_back(s_apay.size());
            pack_fixed(P, c, s_apay);
        }
        offs.push_back(s_apay.size());
        for (uint64_t o : offs) put<uint64_t>(s_atab, o);
    } else {
        L = prm->lanes;
        const uint64_t nsym = (uint64_t)R * kNChan;
        std::vector<uint32_t> sf, scu;  // host coding only
        if (!ctx) {
            sf.resize(nsym);
            scu.resize(nsym);
        }
        std::vector<uint64_t> starts = lane_bounds(R, L, kNChan);
        if (prm->mode == SGS_MODE_STATIC) {
            std::vector<uint32_t> perm;
            std::vector<uint64_t> rstart;
            static_row_order(R, L, perm, rstart);
            for (uint64_t j = 0; j <= L; ++j) starts[j] = rstart[j] * kNChan;
            std::vector<uint32_t> ftab((size_t)kNChan * kNSym);
#pragma omp parallel for schedule(dynamic, 1)
            for (int c = 0; c < kNChan; ++c) {
                uint64_t h[kNSym] = {0};
                for (uint32_t rr = 0; rr < R; ++rr) h[P.q16[(size_t)rr * kNChan + c]]++;
                uint32_t *f = &ftab[(size_t)c * kNSym];
                uint32_t cu[kNSym];
                normalize(h, f);
                uint32_t acc = 0;
                for (int s = 0; s < kNSym; ++s) { cu[s] = acc; acc += f[s]; }
                if (!ctx)
                    for (uint64_t p = 0; p < R; ++p) {
                        const uint32_t q = P.q16[(size_t)perm[p] * kNChan + c];
                        sf[p * kNChan + c] = f[q];
                        scu[p * kNChan + c] = cu[q];
                    }
            }
            for (int c = 0; c < kNChan; ++c) put_table(s_atab, &ftab[(size_t)c * kNSym]);
            if (ctx) {  // the interleaved rANS coding on the context's device
                std::vector<uint8_t> tok(nsym);
#pragma omp parallel for schedule(static)
                for (int64_t p = 0; p < (int64_t)R; ++p)
                    for (int c = 0; c < kNChan; ++c) tok[(size_t)p * kNChan + c] = (uint8_t)P.q16[(size_t)perm[p] * kNChan + c];
                if (cudaSetDevice(ctx->device) != cudaSuccess) return SGS_E_CUDA;
                r = rans_encode_static_device(tok.data(), nsym, ftab.data(), starts, s_agrp, s_apay);
                if (r) return r;
            } else {
                rans_encode(starts, sf.data(), scu.data(), s_agrp, s_apay);
            }
        } else if (prm->mode == SGS_MODE_LEARNED) {
            const uint8_t *m = static_cast<const uint8_t *>(prm->model);
            s_atab.assign(m, m + SGS_MODEL_BYTES);
            std::vector<uint8_t> tok(nsym);
            for (uint64_t i = 0; i < nsym; ++i) tok[i] = (uint8_t)P.q16[i];
            if (cudaSetDevice(ctx->device) != cudaSuccess) return SGS_E_CUDA;
            r = learned_encode_device(m, tok.data(), R, L, starts, s_agrp, s_apay);
            if (r) return r;
        } else {
            const uint8_t *m = static_cast<const uint8_t *>(prm->model);
            s_atab.assign(m, m + SGS_MODEL_PE_BYTES);
            std::vector<uint8_t> tok(nsym);
            for (uint64_t i = 0; i < nsym; ++i) tok[i] = (uint8_t)P.q16[i];
            if (cudaSetDevice(ctx->device) != cudaSuccess) return SGS_E_CUDA;
            r = learned_pe_encode_device(m, tok.data(), P.coord.data(), D, R, L, starts, s_agrp, s_apay);
            if (r) return r;
        }
    }
    // assemble
    std::vector<uint8_t> *secs[10] = {&s_levels, &s_dup, &s_chan, &s_graw, &s_gtab,
                                      &s_ggrp, &s_gpay, &s_atab, &s_agrp, &s_apay};
    uint64_t offs[11];
    uint64_t pos_ = kHeaderBytes;
    for (int i = 0; i < 10; ++i) {
        pad16(*secs[i]);
        offs[i] = pos_;
        pos_ += secs[i]->size();
    }
    offs[10] = pos_;
    *out_len = pos_;
    if (cap < pos_ || !out) return SGS_E_INVALID;
    std::vector<uint8_t> hdr;
    const uint32_t h32[12] = {kMagic, kVersion, prm->mode, prm->geo_mode, n, R, D,
                              (uint32_t)P.leaves.size(), (uint32_t)(P.dups.size() / 2),
                              (uint32_t)kNChan, L, Lg};
    for (uint32_t v : h32) put<uint32_t>(hdr, v);
    put<uint64_t>(hdr, n_geo);
    put<uint64_t>(hdr, n_coded);
    for (int i = 0; i < 11; ++i) put<uint64_t>(hdr, offs[i]);
    hdr.resize(kHeaderBytes, 0);
    memcpy(out, hdr.data(), kHeaderBytes);
    for (int i = 0; i < 10; ++i)
        if (!secs[i]->empty()) memcpy(out + offs[i], secs[i]->data(), secs[i]->size());
    return SGS_OK;
}
