// FP32-pair split of an FP64 value from integer operations (internal header; host and device).
//
// hi = the float nearest to v (ties to even), lo = the float nearest to v - hi: the pair the
// refinement keeps its right-hand side in.  The FP64 form -- hi = (float)v, lo = (float)(v - hi)
// -- takes three conversions and a subtraction on the FP64 pipe, which on this GPU issues at a
// small fraction of the FP32 rate; here hi is rounded from v's 53-bit significand with integer
// operations, the remainder r (v - hi = r 2^(E - 52) exactly, |r| <= 2^28) is converted once and
// scaled by an exact power of two.  Wherever both results are normal floats (binary exponent of v
// in [-74, 126]) this gives the FP64 form's bits exactly, and so it does for zeros; other values
// (subnormal, tiny, huge, infinite, NaN) take the FP64 form.  pair_to_double is the exact inverse widening:
// (double)hi + (double)lo with the float-to-double widening done by bit operations.
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define PAIRSPLIT_HD __host__ __device__ __forceinline__
#else
#define PAIRSPLIT_HD inline
#endif

namespace helm {

PAIRSPLIT_HD uint64_t ps_bits64(double v) {
#if defined(__CUDA_ARCH__)
    return (uint64_t)__double_as_longlong(v);
#else
    uint64_t u;
    memcpy(&u, &v, 8);
    return u;
#endif
}
PAIRSPLIT_HD float ps_float(uint32_t u) {
#if defined(__CUDA_ARCH__)
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, 4);
    return f;
#endif
}
PAIRSPLIT_HD uint32_t ps_bits32(float f) {
#if defined(__CUDA_ARCH__)
    return __float_as_uint(f);
#else
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
#endif
}
PAIRSPLIT_HD double ps_double(uint64_t u) {
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)u);
#else
    double d;
    memcpy(&d, &u, 8);
    return d;
#endif
}

PAIRSPLIT_HD void split_double_int(double v, float &hi, float &lo) {
    const uint64_t u = ps_bits64(v);
    if ((u << 1) == 0) {   // +-0 (most entries of point-source right-hand sides): hi keeps the sign
        hi = ps_float((uint32_t)(u >> 63) << 31);
        lo = 0.f;
        return;
    }
    const int E = (int)((u >> 52) & 0x7FF) - 1023;   // binary exponent of a normal v
    if (E < -74 || E > 126) {                           // outside: the FP64 form
        hi = (float)v;
        lo = (float)(v - (double)hi);
        return;
    }
    const uint64_t m = (u & 0xFFFFFFFFFFFFFull) | (1ull << 52);   // 53-bit significand
    uint32_t q = (uint32_t)(m >> 29);                               // its top 24 bits
    const uint32_t rem = (uint32_t)(m & 0x1FFFFFFFu);               // and the 29 below
    int32_t r = (int32_t)rem;
    int Eh = E;
    if (rem > 0x10000000u || (rem == 0x10000000u && (q & 1u))) {   // round to nearest, ties to even
        ++q;
        r -= 0x20000000;
        if (q == 0x1000000u) {   // the carry reaches the exponent
            q >>= 1;
            ++Eh;
        }
    }
    const uint32_t sign = (uint32_t)(u >> 63) << 31;
    hi = ps_float(sign | ((uint32_t)(Eh + 127) << 23) | (q & 0x7FFFFFu));
    // v - hi = +-r 2^(E - 52) exactly; (float)r rounds it once, the scale is exact (normal range)
    const float scale = ps_float((uint32_t)(E - 52 + 127) << 23);
    const float lr = (float)r * scale;
    lo = r == 0 ? 0.f : (sign ? -lr : lr);   // an exact split leaves +0, as v - hi does
}

// (double)f exactly, by bit operations for normal floats and zero
PAIRSPLIT_HD double ps_widen(float f) {
    const uint32_t b = ps_bits32(f);
    const uint32_t ef = (b >> 23) & 0xFFu;
    if (ef == 0u || ef == 0xFFu) return (b & 0x7FFFFFFFu) == 0u ? ps_double((uint64_t)(b >> 31) << 63) : (double)f;
    return ps_double(((uint64_t)(b >> 31) << 63) | ((uint64_t)(ef - 127 + 1023) << 52) | ((uint64_t)(b & 0x7FFFFFu) << 29));
}

PAIRSPLIT_HD double pair_to_double(float hi, float lo) { return ps_widen(hi) + ps_widen(lo); }

}  // namespace helm
