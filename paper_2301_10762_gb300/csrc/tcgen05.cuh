// Fifth-generation tensor-core helpers shared by the GEMM and the batched inversion (internal
// header): the 128-byte-swizzled K-major shared-memory layout and its descriptor, the TF32
// instruction descriptor (M = 128), the 3xTF32 split, tcgen05 MMA / commit and tensor-memory
// loads and stores of 16 columns of a warp's 32 lanes.
#pragma once
#include <stdint.h>

#include "common.cuh"

namespace helm {

// byte offset of 16-byte chunk j of row r in a 128-byte-swizzled tile (tile base 1024-aligned)
__device__ __forceinline__ uint32_t sw128(int r, int j) { return (uint32_t)(r * 128 + (((j ^ r) & 7) << 4)); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu)        // start address
           | ((uint64_t)1 << 16)                      // leading byte offset (unused for this layout)
           | ((uint64_t)(1024 >> 4) << 32)            // stride byte offset: next 8-row group
           | ((uint64_t)1 << 46)                      // descriptor version of this architecture
           | ((uint64_t)2 << 61);                     // 128-byte swizzle
}

// instruction descriptor: FP32 accumulator, TF32 A and B, both K-major, M = 128, N = n_real
__host__ __device__ constexpr uint32_t idesc_tf32(int n_real) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n_real >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// x rounded to the TF32 grid (10 explicit mantissa bits), to nearest with ties away from zero:
// add half a unit of the 11th bit to the magnitude bits and clear the 13 low bits.  Integer
// operations at full rate (the conversion instruction runs on a low-rate pipe, and the operand
// warps round every element of every chunk).  Finite inputs; a carry into the exponent gives the
// correctly rounded next power of two.
__device__ __forceinline__ float tf32_round(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, float4 v) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

// hi / lo split of the four floats of v (s: the term's sign, exact)
__device__ __forceinline__ void split4(float4 v, float s, float4 &hi, float4 &lo) {
    v.x *= s; v.y *= s; v.z *= s; v.w *= s;
    hi = make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z), tf32_round(v.w));
    lo = make_float4(v.x - hi.x, v.y - hi.y, v.z - hi.z, v.w - hi.w);
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

// arrive on the mbarrier once every tcgen05 operation issued so far by this thread is complete
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive accumulator columns of this thread's lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive columns of this thread's lane from v (the warp's 32 lanes); tc_wait_st() before
// the columns are read by the tensor core or another thread
__device__ __forceinline__ void tc_st16(uint32_t taddr, const float (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
        "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
        "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
        : "memory");
}
__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

}  // namespace helm
