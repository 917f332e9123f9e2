// Pivot-block inversion shared by the line factor and the batched dense inversion: one warp
// inverts a 16 x 16 complex block by Gauss-Jordan with partial pivoting (internal header).
#pragma once
#include "common.cuh"

namespace helm {

constexpr int PIV = 16;   // pivot-block size

template <typename T> __device__ __forceinline__ T recip(T x);
template <> __device__ __forceinline__ float recip<float>(float x) { return __frcp_rn(x); }
template <> __device__ __forceinline__ double recip<double>(double x) { return __drcp_rn(x); }

// 16 x 16 inverse (kb x kb block padded with the identity) of M (shared, row stride ld)
// by one warp; lane (r, h) holds row r, column half h of [M | I].  Partial pivoting
// without row swaps: the pivot of column q is found by one warp-wide max reduction over
// a key (|a_rq|^2 with its low mantissa bits replaced by the row), the pivot row is
// broadcast from the pivot lane's registers by shuffles and scaled by every lane, and the
// pivot order is applied when the inverse is written to P (row stride PIV, shared).  Returns
// false if a pivot was zero or not finite.
template <typename T>
__device__ bool warp_invert16(const cx_t<T> *M, int ld, int kb, cx_t<T> *P) {
    using V = cx_t<T>;
    const int lane = threadIdx.x & 31, r = lane & 15, h = lane >> 4;
    V a[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if (h == 0) a[j] = (r < kb && j < kb) ? M[r * ld + j] : mkc<T>(r == j ? T(1) : T(0), T(0));
        else a[j] = mkc<T>(r == j ? T(1) : T(0), T(0));
    }
    unsigned used = 0;
    int qinv = 0;   // step at which this lane's row was the pivot
    bool ok = true;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const float mag = fminf((float)(a[q].x * a[q].x + a[q].y * a[q].y), 3.0e38f);
        const bool cand = h == 0 && !((used >> r) & 1u);
        // a non-finite entry among the pivot candidates (a NaN or infinite input, or a blow-up
        // of the line recurrence) fails the inversion like a zero pivot
        if (__any_sync(0xffffffffu, cand && !(isfinite(a[q].x) && isfinite(a[q].y)))) ok = false;
        const unsigned key = cand ? ((__float_as_uint(mag) & ~0xFu) | (unsigned)(15 - r)) : 0u;
        const unsigned best = __reduce_max_sync(0xffffffffu, key);
        const int p = 15 - (int)(best & 0xFu);
        if ((best >> 4) == 0u || (best >> 23) >= 255u) ok = false;
        used |= 1u << p;
        if (r == p) qinv = q;
        V pv, f;
        pv.x = __shfl_sync(0xffffffffu, a[q].x, p);
        pv.y = __shfl_sync(0xffffffffu, a[q].y, p);
        f.x = __shfl_sync(0xffffffffu, a[q].x, r);
        f.y = __shfl_sync(0xffffffffu, a[q].y, r);
        const T rd = recip<T>(pv.x * pv.x + pv.y * pv.y);
        const V inv = ok ? mkc<T>(pv.x * rd, -pv.y * rd) : mkc<T>(T(1), T(0));
        // pivot row of this lane's half, scaled by 1 / pivot, straight from the pivot lane's
        // registers; the pivot row takes it, every other row subtracts f times it
        const int src = p + 16 * h;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            V pj;
            pj.x = __shfl_sync(0xffffffffu, a[j].x, src);
            pj.y = __shfl_sync(0xffffffffu, a[j].y, src);
            pj = cmul(pj, inv);
            if (r == p) a[j] = pj;
            else cfms(a[j], f, pj);
        }
    }
    if (h == 1 && qinv < kb) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (j < kb) P[qinv * PIV + j] = a[j];
    }
    return ok;
}


}  // namespace helm
