// Warp-level bf16 tensor-core helpers (mma.sync m16n8k16, fp32 accumulation) shared by the
// learned-model kernels.  Fragment layout, lane = 4 g + t: A holds rows g and g + 8 at
// columns 2t, 2t + 1 (a0, a1) and 2t + 8, 2t + 9 (a2, a3); B holds column g at rows 2t, 2t + 1
// (b0) and 2t + 8, 2t + 9 (b1); the accumulator holds rows g, g + 8 at columns 2t, 2t + 1.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sgs {

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// d = A B + c with a separate accumulator input.
__device__ __forceinline__ void mma_bf16_c(float (&d)[4], const float (&c)[4], uint32_t a0, uint32_t a1,
                                           uint32_t a2, uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%11,%12,%13};"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1), "f"(c[0]), "f"(c[1]), "f"(c[2]), "f"(c[3]));
}

__device__ __forceinline__ __nv_bfloat16 bf(int v) { return __int2bfloat16_rn(v); }

// Two small integers as a bf16 pair, the first in the low half.
__device__ __forceinline__ uint32_t pack_bf16(int lo, int hi) {
    __nv_bfloat162 h = __halves2bfloat162(bf(lo), bf(hi));
    return *reinterpret_cast<uint32_t *>(&h);
}

// Two integer-valued floats (|v| <= 256: exact in bf16) as a bf16 pair.
__device__ __forceinline__ uint32_t pack_bf16f(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

}  // namespace sgs
