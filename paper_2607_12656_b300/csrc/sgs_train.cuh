// Shared pieces of the context-model trainers (k_train.cu, k_train_pe.cu): the counter-based
// batch sampler, lane starts, the fixed-split outer-product reduction and Adam.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace sgs {

// splitmix64 (Steele, Lea and Flood 2014), the counter-based generator of the batches.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Token position of sample k of a step: hi32(splitmix64(seed<<40 ^ step<<20 ^ k)) * n >> 32.
__host__ __device__ __forceinline__ uint64_t sample_pos(uint32_t seed, uint32_t step, uint32_t k,
                                                        uint64_t n_total) {
    const uint64_t key = ((uint64_t)seed << 40) ^ ((uint64_t)step << 20) ^ (uint64_t)k;
    return ((splitmix64(key) >> 32) * n_total) >> 32;
}

// First row of the lane holding `row` (lanes own rows [floor(j n / L), floor((j+1) n / L))).
__host__ __device__ __forceinline__ uint64_t lane_row0(uint64_t row, uint64_t n, uint64_t L) {
    const uint64_t j = ((row + 1) * L + n - 1) / n - 1;
    return j * n / L;
}

// Batch splits of the outer-product reduction (a fixed order: runs repeat bit for bit).
constexpr int kTrainSplits = 16;

// grad[w_off + m N + n] (and grad[b_off + m] for the bias column) = sum over the batch of
// A[m][b] Bm[n][b], A the one-hot of cidx when A is NULL; part holds kTrainSplits x M x
// (N + bias) floats.
cudaError_t train_outer_reduce(const float *A, const int32_t *cidx, const float *Bm, int M, int N, int bias,
                               uint32_t B, float *part, float *grad, int w_off, int b_off, cudaStream_t st);
// Adam (beta 0.9 / 0.999, eps 1e-8) over n weights; mom holds the two moments (2 n).
cudaError_t train_adam(float *w, float *mom, const float *g, int n, float lr, float bc1, float bc2, cudaStream_t st);
// Mean loss of a step from the per-CTA partial sums.
cudaError_t train_loss(const float *part, int n, uint32_t B, float *out, cudaStream_t st);

// Freeze helpers (host): symmetric int8 quantisation with scale max|w| / 127 (1 if all zero)
// and round half to even; clamp to +-(2^24 - 1).
void q8(const float *w, int n, int stride, int cols, std::vector<int8_t> &q, double &s);
int32_t clamp24(double v);

}  // namespace sgs
