// Warp-level TF32 tensor products (mma.sync m16n8k8) and the hi / lo split of the 3xTF32
// scheme: x = hi + lo with hi = tf32(x) and lo = tf32(x - hi), both rounded to nearest; the
// three products hi*hi + hi*lo + lo*hi, accumulated in FP32, carry about 22 bits of each
// operand (internal header of the line sweep and the batched inversion).
#pragma once
#include <stdint.h>

namespace helm {

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
    hi = tf32_rna(x);
    lo = tf32_rna(x - __uint_as_float(hi));
}
// d += A (16 x 8, row) * B (8 x 8, col), TF32 inputs, FP32 accumulate.  Fragments of lane
// (g, t) = (lane / 4, lane % 4): a = {A(g, t), A(g + 8, t), A(g, t + 4), A(g + 8, t + 4)},
// b = {B(t, g), B(t + 4, g)}, d = {D(g, 2t), D(g, 2t + 1), D(g + 8, 2t), D(g + 8, 2t + 1)}.
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

}  // namespace helm
