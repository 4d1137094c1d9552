// Training and freezing of the position-aware context model (Sec. 3.4.2 with its Fourier
// positional embedding; Laplace entropy model of Sec. 3.2).
//
// Float model: phi = phi_q / 128 (the integer embedding inputs of the row's voxel),
// PE = Wp phi + bp (32), x = [u / 128 (4), emb[c] (16), PE (32)], h1 = ReLU(W1 x + b1),
// h2 = ReLU(W2 h1 + b2), (z0, z1) = W3 h2 + b3; mean m = clip(127.5 + 64 z0, 0, 255),
// log2 rate lam = clip(z1, -8, 6), r = 2^lam; F(x) = 2^(-r (m - x)) / 2 below the mean and
// 1 - 2^(-r (x - m)) / 2 above it; P(s) = F(s + 1/2) - F(s - 1/2) with the tails folded into
// symbols 0 and 255; p = (1 + 65280 P) / 65536; loss = mean -log2 p (bits per token).
//
// One step: k_train_pe_rows (thread per token: forward, head, backward to the token's
// activation gradients, stored transposed [feature][batch]) -> weight gradients as fixed-split
// outer-product sums -> Adam.  fp32 throughout, deterministic.
//
// Freeze (host, fp64 with a fixed operation order): the projection folded into layer 1
// (W1_pe Wp over phi, W1_pe bp into the bias), the channel embedding into a per-channel bias,
// int8 weights, requantisation scales from an integer calibration pass over 65,536 tokens.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "sgs_internal.h"
#include "sgs_train.cuh"
#include "sin8_table.h"

namespace sgs {

namespace {

// Flat weight layout (floats).
constexpr int kP_EMB = 0, kP_WP = 896, kP_BP = 3296, kP_W1 = 3328, kP_B1 = 6656, kP_W2 = 6720, kP_B2 = 10816,
              kP_W3 = 10880, kP_B3 = 11008, kP_TOTAL = 11010;
static_assert(kP_TOTAL == SGS_WEIGHTS_PE_FLOATS, "weight layout");
constexpr int kNPhi = 75, kXF = 52, kBands = 12;
constexpr int kTP = 128;  // tokens per CTA

__constant__ int8_t kTrainSin8[256] = {SGS_SIN8_VALUES};
const int8_t kHostSin8[256] = {SGS_SIN8_VALUES};

// phi_q[j] of voxel v (3 coordinates) at depth D (host and device).
__host__ __device__ __forceinline__ int phi_q(const int8_t *sin8, const uint32_t *v, int D, int j) {
    if (j < 3) return (int)(((2ull * v[j] + 1ull) << 6) >> D);
    const int jj = j - 3;
    const bool cosine = jj >= 3 * kBands;
    const int r = cosine ? jj - 3 * kBands : jj;
    const int band = r / 3, a = r - 3 * band;
    uint32_t th = (uint32_t)((((2ull * v[a] + 1ull) << (band + 8)) >> (D + 1)) & 255ull);
    if (cosine) th = (th + 64u) & 255u;
    return sin8[th];
}

struct PeWs {
    float *phiT, *xT, *h1T, *h2T, *dzT, *da2T, *da1T, *dxeT, *dpeT;  // [features][B]
    int32_t *cidx;
    float *loss_part;
    float *part;
    float *grad;
};

struct PeRowParams {
    const uint8_t *tok;
    const uint32_t *coord;
    uint64_t n_rows, L;
    int depth;
    const float *w;
    uint32_t B, seed, step;
    const int64_t *pos;
    PeWs ws;
};

// Code length of symbol s and its derivatives with respect to (z0, z1).
__device__ __forceinline__ float pe_head_grad(float z0, float z1, int s, float &dz0, float &dz1) {
    const float LN2 = 0.69314718055994531f;
    const float mu_raw = 127.5f + 64.0f * z0;
    const float mu = fminf(fmaxf(mu_raw, 0.0f), 255.0f);
    const float lam = fminf(fmaxf(z1, -8.0f), 6.0f);
    const float r = exp2f(lam);
    const bool first = s == 0, last = s == 255;
    const float lo = (float)s - 0.5f, hi = (float)s + 0.5f;
    float e_lo = 0.0f, dlo_mu = 0.0f, dlo_r = 0.0f, e_hi = 0.0f, dhi_mu = 0.0f, dhi_r = 0.0f;
    if (!first) {
        const float d = fabsf(lo - mu), sg = (mu > lo) - (mu < lo);
        e_lo = exp2f(-r * d);
        dlo_mu = -r * LN2 * sg * e_lo;
        dlo_r = -LN2 * d * e_lo;
    }
    if (!last) {
        const float d = fabsf(hi - mu), sg = (mu > hi) - (mu < hi);
        e_hi = exp2f(-r * d);
        dhi_mu = -r * LN2 * sg * e_hi;
        dhi_r = -LN2 * d * e_hi;
    }
    const bool lo_below = first || lo < mu, hi_above = last || hi >= mu;
    const bool straddle = lo_below && hi_above, below = !hi_above;
    float P, c_hi, c_lo;
    if (straddle) { P = 1.0f - 0.5f * (e_hi + e_lo); c_hi = -0.5f; c_lo = -0.5f; }
    else if (below) { P = 0.5f * (e_hi - e_lo); c_hi = 0.5f; c_lo = -0.5f; }
    else { P = 0.5f * (e_lo - e_hi); c_hi = -0.5f; c_lo = 0.5f; }
    const float p = (1.0f + 65280.0f * P) / 65536.0f;
    const float dL_dP = -(65280.0f / 65536.0f) / (p * LN2);
    dz0 = dL_dP * (c_hi * dhi_mu + c_lo * dlo_mu) * 64.0f * ((mu_raw > 0.0f && mu_raw < 255.0f) ? 1.0f : 0.0f);
    dz1 = dL_dP * (c_hi * dhi_r + c_lo * dlo_r) * r * LN2 * ((z1 > -8.0f && z1 < 6.0f) ? 1.0f : 0.0f);
    return -log2f(p);
}

__global__ void __launch_bounds__(kTP) k_train_pe_rows(PeRowParams p) {
    extern __shared__ __align__(16) float sw[];
    for (int i = threadIdx.x; i < kP_TOTAL; i += kTP) sw[i] = p.w[i];
    __shared__ float red[kTP / 32];
    __syncthreads();
    const float *emb = sw + kP_EMB, *Wp = sw + kP_WP, *bp = sw + kP_BP, *W1 = sw + kP_W1, *b1 = sw + kP_B1,
                *W2 = sw + kP_W2, *b2 = sw + kP_B2, *W3 = sw + kP_W3, *b3 = sw + kP_B3;
    const uint32_t b = blockIdx.x * kTP + threadIdx.x;
    const uint32_t B = p.B;
    float loss = 0.0f;
    if (b < B) {
        const uint64_t n_total = p.n_rows * kNChan;
        const uint64_t pos = p.pos ? (uint64_t)p.pos[b] : sample_pos(p.seed, p.step, b, n_total);
        const uint64_t row = pos / kNChan;
        const int c = (int)(pos - row * kNChan);
        const uint64_t row0 = lane_row0(row, p.n_rows, p.L);
        const int s = p.tok[row * kNChan + c];
        const uint32_t v[3] = {p.coord[row], p.coord[p.n_rows + row], p.coord[2 * p.n_rows + row]};
        float x[kXF];
#pragma unroll
        for (int q = 1; q <= 4; ++q)
            x[q - 1] = (row >= row0 + q) ? ((float)((int)p.tok[(row - q) * kNChan + c] - 128)) / 128.0f : 0.0f;
#pragma unroll
        for (int e = 0; e < 16; ++e) x[4 + e] = emb[c * 16 + e];
#pragma unroll
        for (int o = 0; o < 32; ++o) x[20 + o] = bp[o];
        for (int j = 0; j < kNPhi; ++j) {
            const float ph = (float)phi_q(kTrainSin8, v, p.depth, j) / 128.0f;
            p.ws.phiT[(size_t)j * B + b] = ph;
#pragma unroll
            for (int o = 0; o < 32; ++o) x[20 + o] = fmaf(Wp[o * kNPhi + j], ph, x[20 + o]);
        }
#pragma unroll
        for (int j = 0; j < kXF; ++j) p.ws.xT[(size_t)j * B + b] = x[j];
        p.ws.cidx[b] = c;
        float h2[64];
        {
            float h1[64];
#pragma unroll
            for (int o = 0; o < 64; ++o) {
                float a = b1[o];
#pragma unroll
                for (int j = 0; j < kXF; ++j) a = fmaf(W1[o * kXF + j], x[j], a);
                h1[o] = a > 0.0f ? a : 0.0f;
                p.ws.h1T[(size_t)o * B + b] = h1[o];
            }
#pragma unroll 4
            for (int o = 0; o < 64; ++o) {
                float a = b2[o];
#pragma unroll
                for (int k = 0; k < 64; ++k) a = fmaf(W2[o * 64 + k], h1[k], a);
                h2[o] = a > 0.0f ? a : 0.0f;
            }
        }
#pragma unroll
        for (int k = 0; k < 64; ++k) p.ws.h2T[(size_t)k * B + b] = h2[k];
        float z0 = b3[0], z1 = b3[1];
#pragma unroll
        for (int k = 0; k < 64; ++k) {
            z0 = fmaf(W3[k], h2[k], z0);
            z1 = fmaf(W3[64 + k], h2[k], z1);
        }
        float dz0, dz1;
        loss = pe_head_grad(z0, z1, s, dz0, dz1);
        dz0 /= (float)B;
        dz1 /= (float)B;
        p.ws.dzT[b] = dz0;
        p.ws.dzT[(size_t)B + b] = dz1;
        float dh2[64];
#pragma unroll
        for (int k = 0; k < 64; ++k) {
            const float d = fmaf(dz1, W3[64 + k], dz0 * W3[k]);
            dh2[k] = h2[k] > 0.0f ? d : 0.0f;
            p.ws.da2T[(size_t)k * B + b] = dh2[k];
        }
        float dh1[64];
#pragma unroll
        for (int k = 0; k < 64; ++k) dh1[k] = 0.0f;
#pragma unroll 4
        for (int o = 0; o < 64; ++o) {
            const float d = dh2[o];
#pragma unroll
            for (int k = 0; k < 64; ++k) dh1[k] = fmaf(d, W2[o * 64 + k], dh1[k]);
        }
        float dx[kXF];
#pragma unroll
        for (int j = 0; j < kXF; ++j) dx[j] = 0.0f;
#pragma unroll 4
        for (int o = 0; o < 64; ++o) {
            const float h1o = p.ws.h1T[(size_t)o * B + b];
            const float d = h1o > 0.0f ? dh1[o] : 0.0f;
            p.ws.da1T[(size_t)o * B + b] = d;
#pragma unroll
            for (int j = 0; j < kXF; ++j) dx[j] = fmaf(d, W1[o * kXF + j], dx[j]);
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) p.ws.dxeT[(size_t)e * B + b] = dx[4 + e];
#pragma unroll
        for (int o = 0; o < 32; ++o) p.ws.dpeT[(size_t)o * B + b] = dx[20 + o];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = loss;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int i = 0; i < kTP / 32; ++i) t += red[i];
        p.ws.loss_part[blockIdx.x] = t;
    }
}

struct PeBufs {
    PeWs ws;
    void *base = nullptr;
    uint32_t B = 0;
    int n_cta = 0;
};

int pe_alloc(PeBufs &t, uint32_t B) {
    t.B = B;
    t.n_cta = (int)((B + kTP - 1) / kTP);
    const size_t feats = kNPhi + kXF + 64 + 64 + 2 + 64 + 64 + 16 + 32;
    const size_t part = (size_t)kTrainSplits * 64 * (kNPhi + 1);
    const size_t bytes = 4 * (feats * B + B + t.n_cta + part + kP_TOTAL) + 1024;
    if (cudaMalloc(&t.base, bytes) != cudaSuccess) return SGS_E_NOMEM;
    float *f = reinterpret_cast<float *>(t.base);
    t.ws.phiT = f; f += (size_t)kNPhi * B;
    t.ws.xT = f; f += (size_t)kXF * B;
    t.ws.h1T = f; f += 64ull * B;
    t.ws.h2T = f; f += 64ull * B;
    t.ws.dzT = f; f += 2ull * B;
    t.ws.da2T = f; f += 64ull * B;
    t.ws.da1T = f; f += 64ull * B;
    t.ws.dxeT = f; f += 16ull * B;
    t.ws.dpeT = f; f += 32ull * B;
    t.ws.cidx = reinterpret_cast<int32_t *>(f); f += B;
    t.ws.loss_part = f; f += t.n_cta;
    t.ws.part = f; f += part;
    t.ws.grad = f;
    return SGS_OK;
}

cudaError_t pe_grad_step(const PeBufs &t, const uint8_t *tok, const uint32_t *coord, int depth, uint32_t n_rows,
                         uint32_t L, const float *w, uint32_t seed, uint32_t step, const int64_t *pos,
                         float *loss_dev, cudaStream_t st) {
    static bool attr = false;
    const int smem = kP_TOTAL * 4;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_train_pe_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    PeRowParams rp{tok, coord, n_rows, L, depth, w, t.B, seed, step, pos, t.ws};
    k_train_pe_rows<<<t.n_cta, kTP, smem, st>>>(rp);
    cudaError_t e;
    const PeWs &ws = t.ws;
    auto outer = [&](const float *A, const int32_t *cidx, const float *Bm, int M, int N, int bias, int wo, int bo) {
        return train_outer_reduce(A, cidx, Bm, M, N, bias, t.B, ws.part, ws.grad, wo, bo, st);
    };
    if ((e = outer(ws.dzT, nullptr, ws.h2T, 2, 64, 1, kP_W3, kP_B3))) return e;
    if ((e = outer(ws.da2T, nullptr, ws.h1T, 64, 64, 1, kP_W2, kP_B2))) return e;
    if ((e = outer(ws.da1T, nullptr, ws.xT, 64, kXF, 1, kP_W1, kP_B1))) return e;
    if ((e = outer(ws.dpeT, nullptr, ws.phiT, 32, kNPhi, 1, kP_WP, kP_BP))) return e;
    if ((e = outer(nullptr, ws.cidx, ws.dxeT, kNChan, 16, 0, kP_EMB, 0))) return e;
    if (loss_dev) return train_loss(ws.loss_part, t.n_cta, t.B, loss_dev, st);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ freeze (host)

void q8d(const std::vector<double> &w, int rows, int cols, std::vector<int8_t> &q, double &s) {
    double mx = 0.0;
    for (double v : w) mx = std::max(mx, fabs(v));
    s = mx / 127.0;
    if (s == 0.0) s = 1.0;
    q.resize((size_t)rows * cols);
    for (size_t i = 0; i < q.size(); ++i) q[i] = (int8_t)std::min(127.0, std::max(-127.0, nearbyint(w[i] / s)));
}

int32_t clamp23(double v) {
    const double lim = (double)((1 << 23) - 1);
    return (int32_t)std::min(lim, std::max(-lim, v));
}

int32_t rq_f32(int64_t acc, float s) {
    const float v = rintf((float)acc * s);
    return (int32_t)std::min(127.0f, std::max(0.0f, v));
}

}  // namespace

}  // namespace sgs

using namespace sgs;

extern "C" int sgs_train_pe(sgs_ctx *ctx, const uint8_t *tok, const uint32_t *coord, uint32_t depth,
                            uint32_t n_rows, uint32_t lanes, const sgs_train_params *prm, uint32_t step0,
                            float *w, float *adam, float *loss_dev) {
    if (!ctx || !tok || !coord || !prm || !w || !adam || n_rows == 0 || lanes == 0 || depth < 1 ||
        depth > SGS_MAX_DEPTH || prm->batch == 0 || prm->batch > (1u << 20) ||
        (uint64_t)n_rows * kNChan >= (1ull << 32))
        return SGS_E_INVALID;
    PeBufs t;
    int rc = pe_alloc(t, prm->batch);
    if (rc) return rc;
    cudaStream_t st = 0;
    cudaError_t e = cudaSuccess;
    for (uint32_t k = 0; k < prm->steps && e == cudaSuccess; ++k) {
        const uint32_t step = step0 + k;
        e = pe_grad_step(t, tok, coord, (int)depth, n_rows, lanes, w, prm->seed, step, nullptr,
                         loss_dev ? loss_dev + k : nullptr, st);
        if (e != cudaSuccess) break;
        const double tt = (double)step + 1.0;
        e = train_adam(w, adam, t.ws.grad, kP_TOTAL, prm->lr, (float)(1.0 - pow(0.9, tt)),
                       (float)(1.0 - pow(0.999, tt)), st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(t.base);
    return e == cudaSuccess ? SGS_OK : SGS_E_CUDA;
}

extern "C" int sgs_train_pe_grad(sgs_ctx *ctx, const uint8_t *tok, const uint32_t *coord, uint32_t depth,
                                 uint32_t n_rows, uint32_t lanes, const int64_t *pos, uint32_t batch,
                                 const float *w, float *grad, float *loss_host) {
    if (!ctx || !tok || !coord || !pos || !w || !grad || batch == 0 || n_rows == 0 || lanes == 0 || depth < 1 ||
        depth > SGS_MAX_DEPTH)
        return SGS_E_INVALID;
    PeBufs t;
    int rc = pe_alloc(t, batch);
    if (rc) return rc;
    float *lbuf = nullptr;
    if (cudaMalloc(&lbuf, 4) != cudaSuccess) { cudaFree(t.base); return SGS_E_NOMEM; }
    cudaError_t e = pe_grad_step(t, tok, coord, (int)depth, n_rows, lanes, w, 0, 0, pos, lbuf, 0);
    if (e == cudaSuccess) e = cudaMemcpy(grad, t.ws.grad, 4 * kP_TOTAL, cudaMemcpyDeviceToDevice);
    float l = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&l, lbuf, 4, cudaMemcpyDeviceToHost);
    if (loss_host) *loss_host = l;
    cudaFree(lbuf);
    cudaFree(t.base);
    return e == cudaSuccess ? SGS_OK : SGS_E_CUDA;
}

extern "C" int sgs_freeze_pe(const float *wf, const uint8_t *tok, const uint32_t *coord, uint32_t depth,
                             uint32_t n_rows, uint32_t lanes, uint32_t seed, uint8_t *out) {
    if (!wf || !tok || !coord || !out || n_rows == 0 || lanes == 0 || depth < 1 || depth > SGS_MAX_DEPTH)
        return SGS_E_INVALID;
    for (int i = 0; i < kP_TOTAL; ++i)
        if (!isfinite(wf[i])) return SGS_E_INVALID;
    auto W = [&](int off, int i) { return (double)wf[off + i]; };
    // fold the projection: W1_pe (Wp phi + bp) = (W1_pe Wp) phi + W1_pe bp
    std::vector<double> w1cat((size_t)64 * 80, 0.0);
    for (int o = 0; o < 64; ++o) {
        for (int j = 0; j < 4; ++j) w1cat[o * 80 + j] = W(kP_W1, o * kXF + j);
        for (int k = 0; k < kNPhi; ++k) {
            double acc = 0.0;
            for (int e = 0; e < 32; ++e) acc = acc + W(kP_W1, o * kXF + 20 + e) * W(kP_WP, e * kNPhi + k);
            w1cat[o * 80 + 4 + k] = acc;
        }
    }
    std::vector<int8_t> w1q, w2q, w3m, w3l;
    double s_w1, s_w2, s_w3m, s_w3l;
    q8d(w1cat, 64, 80, w1q, s_w1);
    const double s_a1 = s_w1 / 128.0;
    std::vector<int32_t> B1(kNChan * 64);
    for (int c = 0; c < kNChan; ++c)
        for (int o = 0; o < 64; ++o) {
            double t = W(kP_B1, o);
            for (int e = 0; e < 16; ++e) t = t + W(kP_W1, o * kXF + 4 + e) * W(kP_EMB, c * 16 + e);
            for (int e = 0; e < 32; ++e) t = t + W(kP_W1, o * kXF + 20 + e) * W(kP_BP, e);
            B1[c * 64 + o] = clamp23(nearbyint(t / s_a1));
        }
    // integer calibration over 65,536 tokens drawn at step 2^20 - 1
    const uint64_t n_total = (uint64_t)n_rows * kNChan;
    const int n_cal = 65536;
    std::vector<int32_t> xq((size_t)n_cal * 80);
    std::vector<int> cc(n_cal);
    for (int k = 0; k < n_cal; ++k) {
        const uint64_t pos = sample_pos(seed, (1u << 20) - 1, (uint32_t)k, n_total);
        const uint64_t row = pos / kNChan;
        const int c = (int)(pos % kNChan);
        const uint64_t row0 = lane_row0(row, n_rows, lanes);
        cc[k] = c;
        int32_t *x = &xq[(size_t)k * 80];
        for (int q = 1; q <= 4; ++q) x[q - 1] = (row >= row0 + q) ? (int32_t)tok[(row - q) * kNChan + c] - 128 : 0;
        const uint32_t v[3] = {coord[row], coord[n_rows + row], coord[2ull * n_rows + row]};
        for (int j = 0; j < kNPhi; ++j) x[4 + j] = phi_q(kHostSin8, v, (int)depth, j);
        x[79] = 0;
    }
    std::vector<int64_t> a1((size_t)n_cal * 64);
    int64_t A1 = INT64_MIN;
#pragma omp parallel for reduction(max : A1)
    for (int k = 0; k < n_cal; ++k)
        for (int o = 0; o < 64; ++o) {
            int64_t a = B1[cc[k] * 64 + o];
            for (int j = 0; j < 80; ++j) a += (int64_t)w1q[o * 80 + j] * xq[(size_t)k * 80 + j];
            a1[(size_t)k * 64 + o] = a;
            A1 = std::max(A1, a);
        }
    A1 = std::max<int64_t>(A1, 1);
    const float s1 = (float)(127.0 / (double)A1);
    const double s_h1 = s_a1 * (double)A1 / 127.0;
    std::vector<float> w2f(64 * 64);
    for (int i = 0; i < 64 * 64; ++i) w2f[i] = wf[kP_W2 + i];
    q8(w2f.data(), 64, 64, 64, w2q, s_w2);
    const double s_a2 = s_h1 * s_w2;
    std::vector<int32_t> b2q(64);
    for (int o = 0; o < 64; ++o) b2q[o] = clamp23(nearbyint(W(kP_B2, o) / s_a2));
    int64_t A2 = INT64_MIN;
#pragma omp parallel for reduction(max : A2)
    for (int k = 0; k < n_cal; ++k) {
        int32_t h1[64];
        for (int o = 0; o < 64; ++o) h1[o] = rq_f32(a1[(size_t)k * 64 + o], s1);
        for (int o = 0; o < 64; ++o) {
            int64_t a = b2q[o];
            for (int j = 0; j < 64; ++j) a += (int64_t)w2q[o * 64 + j] * h1[j];
            A2 = std::max(A2, a);
        }
    }
    A2 = std::max<int64_t>(A2, 1);
    const float s2 = (float)(127.0 / (double)A2);
    const double s_h2 = s_a2 * (double)A2 / 127.0;
    q8(wf + kP_W3, 1, 64, 64, w3m, s_w3m);
    q8(wf + kP_W3 + 64, 1, 64, 64, w3l, s_w3l);
    const double s_zm = s_h2 * s_w3m, s_zl = s_h2 * s_w3l;
    const int32_t b3q[4] = {clamp23(nearbyint(W(kP_B3, 0) / s_zm)), clamp23(nearbyint(W(kP_B3, 1) / s_zl)), 0, 0};
    const float hdr[4] = {s1, s2, (float)(64.0 * 256.0 * s_zm), (float)(256.0 * s_zl)};
    // serialize (layout of the bitstream's model section)
    memset(out, 0, SGS_MODEL_PE_BYTES);
    memcpy(out, hdr, 16);
    memcpy(out + 32, B1.data(), 4 * B1.size());
    memcpy(out + 14368, b2q.data(), 256);
    memcpy(out + 14624, b3q, 16);
    memcpy(out + 14640, w1q.data(), 64 * 80);
    memcpy(out + 19760, w2q.data(), 64 * 64);
    memcpy(out + 23856, w3m.data(), 64);
    memcpy(out + 23920, w3l.data(), 64);
    return SGS_OK;
}
