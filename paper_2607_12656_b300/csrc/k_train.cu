// Training and freezing of the context model (the learned part of Sec. 3.4.2).
//
// Float model: x = [u / 128 (4), emb[c] (16)], h1 = ReLU(W1 x + b1), h2 = ReLU(W2 h1 + b2),
// z = W3 h2 + b3, p = softmax(z) over 256 symbols; loss = mean -log2 p(s) (the attribute rate
// of Eq. 9 in bits per token).  Adam (beta 0.9 / 0.999, eps 1e-8).
//
// One step on the device: k_train_rows (thread per token: forward, softmax, backward to the
// token's activation gradients, stored transposed [feature][batch]) -> k_outer (weight
// gradients as sums over the batch of outer products, in fixed batch splits) -> k_reduce
// (sums the splits in order: deterministic) -> k_adam.  fp32 throughout.
//
// Freeze (host): int8 weights, int32 biases with the channel embedding folded into the
// per-channel layer-1 bias, requantization multipliers from an integer calibration pass.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "sgs_internal.h"
#include "sgs_train.cuh"

namespace sgs {

// Flat weight layout (floats).
constexpr int kW_EMB = 0, kW_W1 = 896, kW_B1 = 2176, kW_W2 = 2240, kW_B2 = 6336, kW_W3 = 6400,
              kW_B3 = 22784, kW_TOTAL = 23040;
static_assert(kW_TOTAL == SGS_WEIGHTS_FLOATS, "weight layout");

constexpr int kTR = 128;  // tokens per CTA in k_train_rows

struct TrainWs {
    float *xT, *h1T, *h2T, *dzT, *da2T, *da1T, *dxeT;  // [features][B]
    int32_t *cidx;
    float *loss_part;
    float *part;  // split partial sums of the weight gradients
    float *grad;  // [kW_TOTAL]
};

struct RowParams {
    const uint8_t *tok;
    uint64_t n_rows, L;
    const float *w;
    uint32_t B, seed, step;
    const int64_t *pos;  // explicit positions (gradient checks) or NULL
    TrainWs ws;
};

__global__ void __launch_bounds__(kTR) k_train_rows(RowParams p) {
    extern __shared__ __align__(16) float sw[];
    for (int i = threadIdx.x; i < kW_TOTAL; i += kTR) sw[i] = p.w[i];
    __shared__ float red[kTR / 32];
    __syncthreads();
    const float *emb = sw + kW_EMB, *W1 = sw + kW_W1, *b1 = sw + kW_B1, *W2 = sw + kW_W2,
                *b2 = sw + kW_B2, *W3 = sw + kW_W3, *b3 = sw + kW_B3;
    const uint32_t b = blockIdx.x * kTR + threadIdx.x;
    const uint32_t B = p.B;
    float loss = 0.0f;
    if (b < B) {
        const uint64_t n_total = p.n_rows * kNChan;
        const uint64_t pos = p.pos ? (uint64_t)p.pos[b] : sample_pos(p.seed, p.step, b, n_total);
        const uint64_t row = pos / kNChan;
        const int c = (int)(pos - row * kNChan);
        const uint64_t row0 = lane_row0(row, p.n_rows, p.L);
        const int s = p.tok[row * kNChan + c];
        float x[20];
#pragma unroll
        for (int q = 1; q <= 4; ++q)
            x[q - 1] = (row >= row0 + q) ? ((float)((int)p.tok[(row - q) * kNChan + c] - 128)) / 128.0f : 0.0f;
#pragma unroll
        for (int e = 0; e < 16; ++e) x[4 + e] = emb[c * 16 + e];
#pragma unroll
        for (int j = 0; j < 20; ++j) p.ws.xT[(size_t)j * B + b] = x[j];
        p.ws.cidx[b] = c;
        float h2[64];
        {
            float h1[64];
#pragma unroll
            for (int o = 0; o < 64; ++o) {
                float a = b1[o];
#pragma unroll
                for (int j = 0; j < 20; ++j) a = fmaf(W1[o * 20 + j], x[j], a);
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
        // softmax over 256 logits: online max/sum, then a second pass for the gradient
        float m = -INFINITY, ssum = 0.0f, zs = 0.0f;
        for (int o = 0; o < 256; ++o) {
            float z = b3[o];
#pragma unroll
            for (int k = 0; k < 64; ++k) z = fmaf(W3[o * 64 + k], h2[k], z);
            if (o == s) zs = z;
            if (z > m) {
                ssum = ssum * expf(m - z) + 1.0f;
                m = z;
            } else {
                ssum += expf(z - m);
            }
        }
        const float lse = m + logf(ssum);
        const float inv = 1.0f / ((float)B * 0.69314718055994531f);
        loss = (lse - zs) * 1.4426950408889634f;
        float dh2[64];
#pragma unroll
        for (int k = 0; k < 64; ++k) dh2[k] = 0.0f;
        for (int o = 0; o < 256; ++o) {
            float z = b3[o];
#pragma unroll
            for (int k = 0; k < 64; ++k) z = fmaf(W3[o * 64 + k], h2[k], z);
            const float d = (expf(z - lse) - (o == s ? 1.0f : 0.0f)) * inv;
            p.ws.dzT[(size_t)o * B + b] = d;
#pragma unroll
            for (int k = 0; k < 64; ++k) dh2[k] = fmaf(d, W3[o * 64 + k], dh2[k]);
        }
        // da2 = dh2 * [h2 > 0] (kept in dh2)
#pragma unroll
        for (int k = 0; k < 64; ++k) {
            dh2[k] = h2[k] > 0.0f ? dh2[k] : 0.0f;
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
        float dx[20];
#pragma unroll
        for (int j = 0; j < 20; ++j) dx[j] = 0.0f;
#pragma unroll
        for (int o = 0; o < 64; ++o) {
            const float h1o = p.ws.h1T[(size_t)o * B + b];
            const float d = h1o > 0.0f ? dh1[o] : 0.0f;
            p.ws.da1T[(size_t)o * B + b] = d;
#pragma unroll
            for (int j = 0; j < 20; ++j) dx[j] = fmaf(d, W1[o * 20 + j], dx[j]);
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) p.ws.dxeT[(size_t)e * B + b] = dx[4 + e];
    }
    // per-CTA loss sum (fixed order)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = loss;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int i = 0; i < kTR / 32; ++i) t += red[i];
        p.ws.loss_part[blockIdx.x] = t;
    }
}

// part[split][m][n] = sum over b in split of A[m][b] * Bm[n][b]; column n == N is the bias
// (Bm = 1).  If onehot, A[m][b] = (cidx[b] == m).  CTA: 32 x 32 outputs, 256 threads.
constexpr int kOT = 32, kOK = 64, kSplits = kTrainSplits;

struct OuterParams {
    const float *A;
    const int32_t *cidx;
    const float *Bm;
    int M, N;  // output is M x (N + bias)
    int bias;
    uint32_t B;
    float *part;  // [kSplits][M][N + bias]
};

__global__ void __launch_bounds__(256) k_outer(OuterParams p) {
    __shared__ float sa[kOK][kOT + 1];
    __shared__ float sb[kOK][kOT + 1];
    const int m0 = blockIdx.x * kOT, n0 = blockIdx.y * kOT, split = blockIdx.z;
    const int NC = p.N + p.bias;
    const uint32_t per = (p.B + kSplits - 1) / kSplits;
    const uint32_t bb0 = split * per, bb1 = min(p.B, bb0 + per);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 2 x 2 outputs each
    float acc[2][2] = {{0, 0}, {0, 0}};
    for (uint32_t k0 = bb0; k0 < bb1; k0 += kOK) {
        for (int i = threadIdx.x; i < kOT * kOK; i += 256) {
            const int r = i / kOK, kk = i - r * kOK;
            const uint32_t bidx = k0 + kk;
            const int m = m0 + r, n = n0 + r;
            float av = 0.0f, bv = 0.0f;
            if (bidx < bb1) {
                if (m < p.M) av = p.cidx ? (p.cidx[bidx] == m ? 1.0f : 0.0f) : p.A[(size_t)m * p.B + bidx];
                if (n < p.N) bv = p.Bm[(size_t)n * p.B + bidx];
                else if (n < NC) bv = 1.0f;
            }
            sa[kk][r] = av;
            sb[kk][r] = bv;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kOK; ++kk) {
            const float a0 = sa[kk][ty * 2], a1 = sa[kk][ty * 2 + 1];
            const float c0 = sb[kk][tx * 2], c1 = sb[kk][tx * 2 + 1];
            acc[0][0] = fmaf(a0, c0, acc[0][0]);
            acc[0][1] = fmaf(a0, c1, acc[0][1]);
            acc[1][0] = fmaf(a1, c0, acc[1][0]);
            acc[1][1] = fmaf(a1, c1, acc[1][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int m = m0 + ty * 2 + i, n = n0 + tx * 2 + j;
            if (m < p.M && n < NC) p.part[((size_t)split * p.M + m) * NC + n] = acc[i][j];
        }
}

// grad[w_off + m*N + n] / grad[b_off + m] = sum over splits, in split order.
__global__ void k_reduce(const float *part, int M, int N, int bias, float *grad, int w_off,
                         int b_off) {
    const int NC = N + bias;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * NC) return;
    float s = 0.0f;
    for (int k = 0; k < kSplits; ++k) s += part[(size_t)k * M * NC + i];
    const int m = i / NC, n = i - m * NC;
    if (n < N) grad[w_off + m * N + n] = s;
    else grad[b_off + m] = s;
}

__global__ void k_adam(float *w, float *mom, const float *g, int n, float lr, float bc1, float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float *m = mom, *v = mom + n;
    const float gi = g[i];
    m[i] = 0.9f * m[i] + 0.1f * gi;
    v[i] = 0.999f * v[i] + 0.001f * gi * gi;
    const float mh = m[i] / bc1, vh = v[i] / bc2;
    w[i] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

__global__ void k_loss(const float *part, int n, uint32_t B, float *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        float s = 0.0f;
        for (int i = 0; i < n; ++i) s += part[i];
        *out = s / (float)B;
    }
}

struct TrainBufs {
    TrainWs ws;
    void *base = nullptr;
    uint32_t B = 0;
    int n_cta = 0;
};

static int train_alloc(TrainBufs &t, uint32_t B) {
    t.B = B;
    t.n_cta = (int)((B + kTR - 1) / kTR);
    const size_t feats = 20 + 64 + 64 + 256 + 64 + 64 + 16;
    const size_t part = (size_t)kSplits * 256 * 65;
    const size_t bytes = 4 * (feats * B + B + t.n_cta + part + kW_TOTAL) + 1024;
    if (cudaMalloc(&t.base, bytes) != cudaSuccess) return SGS_E_NOMEM;
    float *f = reinterpret_cast<float *>(t.base);
    t.ws.xT = f; f += 20ull * B;
    t.ws.h1T = f; f += 64ull * B;
    t.ws.h2T = f; f += 64ull * B;
    t.ws.dzT = f; f += 256ull * B;
    t.ws.da2T = f; f += 64ull * B;
    t.ws.da1T = f; f += 64ull * B;
    t.ws.dxeT = f; f += 16ull * B;
    t.ws.cidx = reinterpret_cast<int32_t *>(f); f += B;
    t.ws.loss_part = f; f += t.n_cta;
    t.ws.part = f; f += part;
    t.ws.grad = f;
    return SGS_OK;
}

cudaError_t train_outer_reduce(const float *A, const int32_t *cidx, const float *Bm, int M, int N, int bias,
                               uint32_t B, float *part, float *grad, int w_off, int b_off, cudaStream_t st) {
    OuterParams op{A, cidx, Bm, M, N, bias, B, part};
    dim3 grid((M + kOT - 1) / kOT, (N + bias + kOT - 1) / kOT, kSplits);
    k_outer<<<grid, 256, 0, st>>>(op);
    const int n = M * (N + bias);
    k_reduce<<<(n + 255) / 256, 256, 0, st>>>(part, M, N, bias, grad, w_off, b_off);
    return cudaGetLastError();
}

cudaError_t train_adam(float *w, float *mom, const float *g, int n, float lr, float bc1, float bc2, cudaStream_t st) {
    k_adam<<<(n + 255) / 256, 256, 0, st>>>(w, mom, g, n, lr, bc1, bc2);
    return cudaGetLastError();
}

cudaError_t train_loss(const float *part, int n, uint32_t B, float *out, cudaStream_t st) {
    k_loss<<<1, 32, 0, st>>>(part, n, B, out);
    return cudaGetLastError();
}

static cudaError_t outer_and_reduce(const TrainBufs &t, const float *A, const int32_t *cidx,
                                    const float *Bm, int M, int N, int bias, int w_off, int b_off,
                                    cudaStream_t st) {
    return train_outer_reduce(A, cidx, Bm, M, N, bias, t.B, t.ws.part, t.ws.grad, w_off, b_off, st);
}

// One forward/backward: gradients into t.ws.grad, mean loss into *loss_dev (if non-null).
static cudaError_t train_grad_step(const TrainBufs &t, const uint8_t *tok, uint32_t n_rows,
                                   uint32_t L, const float *w, uint32_t seed, uint32_t step,
                                   const int64_t *pos, float *loss_dev, cudaStream_t st) {
    static bool attr = false;
    const int smem = kW_TOTAL * 4;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_train_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    RowParams rp{tok, n_rows, L, w, t.B, seed, step, pos, t.ws};
    k_train_rows<<<t.n_cta, kTR, smem, st>>>(rp);
    cudaError_t e;
    if ((e = outer_and_reduce(t, t.ws.dzT, nullptr, t.ws.h2T, 256, 64, 1, kW_W3, kW_B3, st))) return e;
    if ((e = outer_and_reduce(t, t.ws.da2T, nullptr, t.ws.h1T, 64, 64, 1, kW_W2, kW_B2, st))) return e;
    if ((e = outer_and_reduce(t, t.ws.da1T, nullptr, t.ws.xT, 64, 20, 1, kW_W1, kW_B1, st))) return e;
    if ((e = outer_and_reduce(t, nullptr, t.ws.cidx, t.ws.dxeT, kNChan, 16, 0, kW_EMB, 0, st))) return e;
    if (loss_dev) k_loss<<<1, 32, 0, st>>>(t.ws.loss_part, t.n_cta, t.B, loss_dev);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ freeze (host)

void q8(const float *w, int n, int stride, int cols, std::vector<int8_t> &q, double &s) {
    double mx = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < cols; ++j) mx = std::max(mx, fabs((double)w[i * stride + j]));
    s = mx / 127.0;
    if (s == 0.0) s = 1.0;
    q.resize((size_t)n * cols);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < cols; ++j) {
            double v = nearbyint((double)w[i * stride + j] / s);
            v = std::min(127.0, std::max(-127.0, v));
            q[(size_t)i * cols + j] = (int8_t)v;
        }
}

int32_t clamp24(double v) {
    const double lim = (double)((1 << 24) - 1);
    return (int32_t)std::min(lim, std::max(-lim, v));
}

static void requant_params(int64_t A, int32_t &m, int32_t &sh) {
    A = std::max<int64_t>(A, 1);
    for (int s = 31; s >= 1; --s) {
        const int64_t mm = (int64_t)(((uint64_t)127 << s) / (uint64_t)A);
        if (mm < (1ll << 31)) { m = (int32_t)mm; sh = s; return; }
    }
    m = (int32_t)(254 / A);
    sh = 1;
}

static int32_t rq_host(int32_t acc, int32_t m, int32_t sh) {
    int64_t v = ((int64_t)acc * m + ((int64_t)1 << (sh - 1))) >> sh;
    return (int32_t)std::min<int64_t>(127, std::max<int64_t>(0, v));
}

}  // namespace sgs

using namespace sgs;

namespace sgs {
namespace {

// The freeze's arithmetic (fp64, fixed operation order): per-tensor int8 weights, the channel
// embedding folded into the layer-1 bias, requantisation multipliers from the layer maxima
// over the n_cal calibration contexts (u [n_cal][4], channel cc [n_cal]), biases at the
// layers' scales, the softmax multiplier; then the model blob.
void freeze_common(const float *w, const std::vector<int32_t> &u, const std::vector<int> &cc, uint8_t *out) {
    const float *emb = w + kW_EMB, *W1 = w + kW_W1, *b1 = w + kW_B1, *W2 = w + kW_W2, *b2 = w + kW_B2,
                *W3 = w + kW_W3, *b3 = w + kW_B3;
    const int n_cal = (int)cc.size();
    const double s_u = 1.0 / 128.0;
    std::vector<int8_t> w1q, w2q, w3q;
    double s_w1, s_w2, s_w3;
    q8(W1, 64, 20, 4, w1q, s_w1);
    const double s_a1 = s_u * s_w1;
    std::vector<int32_t> B1(kNChan * 64);
    for (int c = 0; c < kNChan; ++c)
        for (int o = 0; o < 64; ++o) {
            double t = (double)b1[o];
            for (int e = 0; e < 16; ++e) t = t + (double)W1[o * 20 + 4 + e] * (double)emb[c * 16 + e];
            B1[c * 64 + o] = clamp24(nearbyint(t / s_a1));
        }
    q8(W2, 64, 64, 64, w2q, s_w2);
    q8(W3, 256, 64, 64, w3q, s_w3);
    auto acc1 = [&](int k, int o) {
        int32_t a = B1[cc[k] * 64 + o];
        for (int j = 0; j < 4; ++j) a += (int32_t)w1q[o * 4 + j] * u[4 * k + j];
        return a;
    };
    int64_t A1 = INT64_MIN;
    for (int k = 0; k < n_cal; ++k)
        for (int o = 0; o < 64; ++o) A1 = std::max<int64_t>(A1, acc1(k, o));
    A1 = std::max<int64_t>(A1, 1);
    int32_t m1, sh1, m2, sh2;
    requant_params(A1, m1, sh1);
    const double s_h1 = s_a1 * (double)A1 / 127.0;
    const double s_a2 = s_h1 * s_w2;
    std::vector<int32_t> b2q(64), b3q(256);
    for (int o = 0; o < 64; ++o) b2q[o] = clamp24(nearbyint((double)b2[o] / s_a2));
    int64_t A2 = INT64_MIN;
    int32_t h1[64];
    for (int k = 0; k < n_cal; ++k) {
        for (int o = 0; o < 64; ++o) h1[o] = rq_host(acc1(k, o), m1, sh1);
        for (int o = 0; o < 64; ++o) {
            int32_t a = b2q[o];
            for (int q = 0; q < 64; ++q) a += (int32_t)w2q[o * 64 + q] * h1[q];
            A2 = std::max<int64_t>(A2, a);
        }
    }
    A2 = std::max<int64_t>(A2, 1);
    requant_params(A2, m2, sh2);
    const double s_h2 = s_a2 * (double)A2 / 127.0;
    const double s_z = s_h2 * s_w3;
    for (int o = 0; o < 256; ++o) b3q[o] = clamp24(nearbyint((double)b3[o] / s_z));
    double msd = nearbyint(s_z * 1.4426950408889634 * 256.0 * 65536.0);
    msd = std::min((double)((1 << 24) - 1), std::max(1.0, msd));
    // serialize (layout of the bitstream's model section)
    memset(out, 0, SGS_MODEL_BYTES);
    const int32_t hdr[8] = {m1, sh1, m2, sh2, (int32_t)(uint32_t)msd, 16, 0, 0};
    memcpy(out, hdr, 32);
    memcpy(out + 32, B1.data(), 4 * B1.size());
    memcpy(out + 14368, b2q.data(), 256);
    memcpy(out + 14624, b3q.data(), 1024);
    memcpy(out + 15648, w1q.data(), 256);
    memcpy(out + 15904, w2q.data(), 4096);
    memcpy(out + 20000, w3q.data(), 16384);
}

bool weights_finite(const float *w) {
    for (int i = 0; i < kW_TOTAL; ++i)
        if (!isfinite(w[i])) return false;
    return true;
}

}  // namespace
}  // namespace sgs

extern "C" int sgs_freeze(const float *w, const uint8_t *tok, uint32_t n_rows, uint32_t lanes,
                          uint32_t seed, uint8_t *out) {
    if (!w || !out || !tok || n_rows == 0 || lanes == 0) return SGS_E_INVALID;
    if (!weights_finite(w)) return SGS_E_INVALID;
    // integer calibration over 65,536 tokens drawn at step 2^20 - 1
    const uint64_t n_total = (uint64_t)n_rows * kNChan;
    const int n_cal = 65536;
    std::vector<int32_t> u(4 * n_cal);
    std::vector<int> cc(n_cal);
    for (int k = 0; k < n_cal; ++k) {
        const uint64_t pos = sample_pos(seed, (1u << 20) - 1, (uint32_t)k, n_total);
        const uint64_t row = pos / kNChan;
        const int c = (int)(pos % kNChan);
        const uint64_t row0 = lane_row0(row, n_rows, lanes);
        cc[k] = c;
        for (int q = 1; q <= 4; ++q)
            u[4 * k + q - 1] = (row >= row0 + q) ? (int32_t)tok[(row - q) * kNChan + c] - 128 : 0;
    }
    freeze_common(w, u, cc, out);
    return SGS_OK;
}

extern "C" int sgs_freeze_samples(const float *w, const int32_t *u_in, const uint32_t *chan, uint64_t n,
                                  uint32_t seed, uint8_t *out) {
    if (!w || !out || !u_in || !chan || n == 0) return SGS_E_INVALID;
    if (!weights_finite(w)) return SGS_E_INVALID;
    for (uint64_t i = 0; i < n; ++i) {
        if (chan[i] >= (uint32_t)kNChan) return SGS_E_INVALID;
        for (int j = 0; j < 4; ++j)
            if (u_in[4 * i + j] < -128 || u_in[4 * i + j] > 127) return SGS_E_INVALID;
    }
    // calibration sample k = entry sample_pos(seed, 2^20 - 1, k, n) of the set
    const int n_cal = 65536;
    std::vector<int32_t> u(4 * n_cal);
    std::vector<int> cc(n_cal);
    for (int k = 0; k < n_cal; ++k) {
        const uint64_t i = sample_pos(seed, (1u << 20) - 1, (uint32_t)k, n);
        cc[k] = (int)chan[i];
        for (int j = 0; j < 4; ++j) u[4 * k + j] = u_in[4 * i + j];
    }
    freeze_common(w, u, cc, out);
    return SGS_OK;
}

extern "C" int sgs_train_grad(sgs_ctx *ctx, const uint8_t *tok, uint32_t n_rows, uint32_t lanes,
                              const int64_t *pos, uint32_t batch, const float *w, float *grad,
                              float *loss_host) {
    if (!ctx || !tok || !pos || !w || !grad || batch == 0 || n_rows == 0 || lanes == 0)
        return SGS_E_INVALID;
    TrainBufs t;
    int rc = train_alloc(t, batch);
    if (rc) return rc;
    float *lbuf = nullptr;
    if (cudaMalloc(&lbuf, 4) != cudaSuccess) { cudaFree(t.base); return SGS_E_NOMEM; }
    cudaError_t e = train_grad_step(t, tok, n_rows, lanes, w, 0, 0, pos, lbuf, 0);
    if (e == cudaSuccess) e = cudaMemcpy(grad, t.ws.grad, 4 * kW_TOTAL, cudaMemcpyDeviceToDevice);
    float l = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&l, lbuf, 4, cudaMemcpyDeviceToHost);
    if (loss_host) *loss_host = l;
    cudaFree(lbuf);
    cudaFree(t.base);
    return e == cudaSuccess ? SGS_OK : SGS_E_CUDA;
}

extern "C" int sgs_train(sgs_ctx *ctx, const uint8_t *tok, uint32_t n_rows, uint32_t lanes,
                         const sgs_train_params *prm, uint32_t step0, float *w, float *adam,
                         float *loss_dev) {
    if (!ctx || !tok || !prm || !w || !adam || n_rows == 0 || lanes == 0 || prm->batch == 0 ||
        prm->batch > (1u << 20) || (uint64_t)n_rows * kNChan >= (1ull << 32))
        return SGS_E_INVALID;
    TrainBufs t;
    int rc = train_alloc(t, prm->batch);
    if (rc) return rc;
    cudaStream_t st = 0;
    cudaError_t e = cudaSuccess;
    for (uint32_t k = 0; k < prm->steps && e == cudaSuccess; ++k) {
        const uint32_t step = step0 + k;
        e = train_grad_step(t, tok, n_rows, lanes, w, prm->seed, step, nullptr,
                            loss_dev ? loss_dev + k : nullptr, st);
        if (e != cudaSuccess) break;
        const double tt = (double)step + 1.0;
        const float bc1 = (float)(1.0 - pow(0.9, tt)), bc2 = (float)(1.0 - pow(0.999, tt));
        k_adam<<<(kW_TOTAL + 255) / 256, 256, 0, st>>>(w, adam, t.ws.grad, kW_TOTAL, prm->lr, bc1, bc2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(t.base);
    return e == cudaSuccess ? SGS_OK : SGS_E_CUDA;
}
