// Mixed-precision iterative refinement in FP32-pair arithmetic.
//
// The correction solves run on the complex-FP32 factor (sweep.cu); the iterate and the
// residual need about twice the precision of FP32 to take the relative residual to 1e-10
// and below.  On this GPU the FP64 pipe issues at 1/64 of the FP32 rate, so the iterate
// x, the right-hand side b and the diagonal of A are held as unevaluated sums of two
// FP32 numbers (hi + lo, about 48 significant bits), and the residual b - A x is formed
// with error-free transformations on the FP32 pipe: two_sum (Knuth) for sums and the
// fused multiply-add for the exact error of a product (Dekker's product with FMA).  FP64
// arithmetic is used only to split the FP64 input once per solve and to form the FP64
// result once at the end.
//
//   start:   bd = split(conj?(b)), r = hi(bd), ||b||^2
//   loop:    delta = A~^{-1} r                                 (sweep.cu, complex FP32)
//            x' = x + delta,  r = hi(bd - A x'),  ||r||^2      (one fused pass)
//   finish:  X = conj?(hi(x) + lo(x)) in FP64
// (x is the solution of A x = conj(b) for the adjoint solve, whose result is conj(x).)
// A pair holds 48 bits, and so does the pair form of A's diagonal, so the relative residual
// this loop reaches levels off near 2^-48 |A| |x| / |b| (about 1e-13 on the 128^2 workload,
// against about 6e-15 with FP64 residuals).  Tighter tolerances continue with FP64
// residuals on the FP64 iterate (residual_kernel, refine_accumulate_kernel).
#include <math.h>
#include "kernels.h"
#include "pairsplit.h"
#include "trace.h"

namespace helm {

namespace {

constexpr int RF_THREADS = 256;
constexpr int RF_NPT = 8;   // nodes per thread in the per-column kernels (a block covers 2048 nodes)

// ---------------------------------------------------------------- FP32-pair arithmetic
// The intrinsics keep the compiler from contracting or reassociating these sequences.
struct ff {
    float hi, lo;
};
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ ff quick_two_sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_add1(ff a, float b) {
    ff s = two_sum(a.hi, b);
    s.lo = __fadd_rn(s.lo, a.lo);
    return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);   // exact error of the leading product
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return quick_two_sum(p, e);
}
struct cff {
    ff re, im;
};
__device__ __forceinline__ cff cff_of(float4 v) { return {{v.x, v.z}, {v.y, v.w}}; }   // (hi.re, hi.im, lo.re, lo.im)
__device__ __forceinline__ float4 cff_pack(cff v) { return make_float4(v.re.hi, v.im.hi, v.re.lo, v.im.lo); }
__device__ __forceinline__ cff cff_add(cff a, cff b) { return {ff_add(a.re, b.re), ff_add(a.im, b.im)}; }
__device__ __forceinline__ cff cff_sub(cff a, cff b) { return {ff_add(a.re, ff_neg(b.re)), ff_add(a.im, ff_neg(b.im))}; }
__device__ __forceinline__ cff cff_scale(cff a, ff c) { return {ff_mul(a.re, c), ff_mul(a.im, c)}; }
__device__ __forceinline__ cff cff_mul(cff a, cff b) {
    return {ff_add(ff_mul(a.re, b.re), ff_neg(ff_mul(a.im, b.im))), ff_add(ff_mul(a.re, b.im), ff_mul(a.im, b.re))};
}

__host__ __device__ inline void split_double(double v, float &hi, float &lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

// block sum of one double (RF_THREADS threads), valid in thread 0
__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = 0.0;
    if (wid == 0) {
        v = lane < RF_THREADS / 32 ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}
__device__ __forceinline__ float block_sum(float v, float *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    v = 0.f;
    if (wid == 0) {
        v = lane < RF_THREADS / 32 ? sh[lane] : 0.f;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

__global__ void split_diag_kernel(size_t n, const double2 *diag, float4 *diag2) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const double2 d = diag[e];
        float4 v;
        split_double(d.x, v.x, v.z);
        split_double(d.y, v.y, v.w);
        diag2[e] = v;
    }
}

// grid: (node blocks of RF_THREADS * RF_NPT, columns)
__global__ void __launch_bounds__(RF_THREADS) refine_start_kernel(int N, int cols, const double2 *B, int conj,
                                                                  float4 *bd, float2 *r32, double *norms) {
    __shared__ double sh[RF_THREADS / 32];
    for (int c = blockIdx.y; c < cols; c += gridDim.y) {
        double bb = 0.0;
        const size_t base = (size_t)c * N;
        const int k0 = blockIdx.x * RF_THREADS * RF_NPT + threadIdx.x;
        double2 b[RF_NPT];
#pragma unroll
        for (int q = 0; q < RF_NPT; ++q) {   // all loads first: RF_NPT in flight per thread
            const int k = k0 + q * RF_THREADS;
            b[q] = k < N ? __ldcs(B + base + k) : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int q = 0; q < RF_NPT; ++q) {
            const int k = k0 + q * RF_THREADS;
            if (k < N) {
                double2 v2 = b[q];
                if (conj) v2.y = -v2.y;
                float4 v;
                split_double_int(v2.x, v.x, v.z);   // the FP64 split's bits, from integer operations
                split_double_int(v2.y, v.y, v.w);
                bd[base + k] = v;
                r32[base + k] = make_float2(v.x, v.y);
                // (the zeros of point sources skip the FP64 arithmetic, tested on the bits)
                if (((ps_bits64(v2.x) | ps_bits64(v2.y)) << 1) != 0) bb += v2.x * v2.x + v2.y * v2.y;
            }
        }
        bb = block_sum(bb, sh);
        if (threadIdx.x == 0) {
            atomicAdd(norms + 2 * (size_t)c + 1, bb);
            if (blockIdx.x == 0) norms[2 * (size_t)c] = 0.0;
        }
        __syncthreads();   // sh reused by the next column
    }
}

struct StencilPairs {   // grid couplings as FP32 pairs: x (between lines), z (within a line); interior, edge
    ff cx_in, cx_edge, cz_in, cz_edge;
};

// x' = x + delta at node k (x absent: x' = delta)
__device__ __forceinline__ cff iterate_at(const float4 *x, const float2 *d, size_t e) {
    const float2 dv = d[e];
    if (!x) return {{dv.x, 0.f}, {dv.y, 0.f}};
    const cff xv = cff_of(x[e]);
    return {ff_add1(xv.re, dv.x), ff_add1(xv.im, dv.y)};
}

// maximum in which a NaN operand wins (a column with a non-finite residual must not be hidden)
__device__ __forceinline__ double nan_max(double a, double b) { return (isnan(a) || isnan(b)) ? NAN : fmax(a, b); }

// Stopping test of the pair phase, one block: rel = max over columns of sqrt(rr / bb) (bb = 0: 0 if
// rr = 0 else inf; a non-finite bb or rr: NaN, which stops the loop unconverged); record it and
// decide; rr = 0 again for the next update.  The norms were accumulated by atomics of other
// blocks, so they are read from L2.  One warp per system, its lanes over the system's columns
// (the test is the serial tail of the update, so its L2 reads are issued 32 at a time).
__device__ void refine_stop_test(int cols, int nrhs, double *norms, RefineStop stop, RefineState *st, double *sh) {
    double mx = 0.0;
    int *sys = refine_sys(st);
    const int n_sys = cols / nrhs;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, n_warps = (int)blockDim.x >> 5;
    for (int q = wid; q < n_sys; q += n_warps) {
        double ms = 0.0;
        for (int j = lane; j < nrhs; j += 32) {
            const size_t c = (size_t)q * nrhs + j;
            const double rr = __ldcg(norms + 2 * c), bb = __ldcg(norms + 2 * c + 1);
            // a non-finite right-hand side (bb NaN or inf) or residual gives NaN: not converged
            const double rel = (isnan(rr) || !isfinite(bb)) ? NAN : (bb > 0.0 ? sqrt(rr / bb) : (rr > 0.0 ? INFINITY : 0.0));
            ms = nan_max(ms, rel);
            norms[2 * c] = 0.0;
        }
        for (int o = 16; o > 0; o >>= 1) ms = nan_max(ms, __shfl_xor_sync(0xffffffffu, ms, o));
        if (lane == 0 && !sys[2 * q + 1]) {   // this pass updated the system: count it, freeze it once converged
            sys[2 * q] += 1;
            if (ms <= stop.rtol) sys[2 * q + 1] = 1;
        }
        mx = nan_max(mx, ms);   // (a frozen system's columns were not updated: 0)
    }
    if (lane == 0) sh[wid] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double rel = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w)
            rel = nan_max(rel, sh[w]);
        const int it = st->iters + 1;
        const double prev = it > 1 ? st->rel : INFINITY;
        st->iters = it;
        st->prev = prev;
        st->rel = rel;
        if (rel <= stop.rtol) st->done = 1;
        else if (!(rel < INFINITY) || it >= stop.max_iter || rel <= stop.floor_rel || rel > 0.25 * prev) st->done = 2;
    }
}

// grid: (node blocks of RF_THREADS * RF_NPT, columns); norms[col][0] pre-zeroed, norms[col][1] = ||b||^2
// (the arrays are distinct: __restrict__ lets the loads of later nodes move above the stores of
// earlier ones, so that several nodes' loads are in flight)
__global__ void __launch_bounds__(RF_THREADS) refine_update_kernel(GridGeom g, int nrhs, int cols,
                                                                   const float4 *__restrict__ diag2,
                                                                   const float4 *__restrict__ bd,
                                                                   const float4 *__restrict__ x_in,
                                                                   const float2 *__restrict__ delta,
                                                                   float4 *__restrict__ x_out, float2 *__restrict__ r32,
                                                                   double *norms, StencilPairs cp,
                                                                   RefineState *state, RefineStop stop) {
    __shared__ float shf[RF_THREADS / 32];
    __shared__ int s_last;
    __shared__ double shd[32];
    if (state && state->done) return;   // the refinement has stopped: later passes do nothing
    const int nx = g.nx, nz = g.nz, N = nx * nz;
    const int *sysflags = state ? refine_sys(state) : nullptr;
    for (int c = blockIdx.y; c < cols; c += gridDim.y) {
        const int sys = c / nrhs;
        if (sysflags && sysflags[2 * sys + 1]) continue;   // frozen: its iterate stays (whole block)
        const double bb = norms[2 * (size_t)c + 1];
        // power-of-two scale 2^-ks, ks about half the binary exponent of ||b||^2: keeps the FP32
        // squares of r 2^-ks in range; the sum is scaled back exactly by 2^(2 ks) (no FP64
        // arithmetic in the block's way)
        const int eb = (int)(((unsigned long long)__double_as_longlong(bb) >> 52) & 0x7FF);
        const int ks = bb > 0.0 ? max(-62, min(62, (eb - 1023) / 2)) : 0;
        const float scale = __uint_as_float((unsigned)(127 - ks) << 23);
        float rr = 0.f;
        const size_t base = (size_t)c * N;
        const float4 *__restrict__ xc = x_in ? x_in + base : nullptr;
        const float2 *__restrict__ dc = delta + base;
        const int k0 = blockIdx.x * RF_THREADS * RF_NPT + threadIdx.x;
#pragma unroll 4
        for (int q = 0; q < RF_NPT; ++q) {
            const int k = k0 + q * RF_THREADS;
            if (k >= N) break;
            const int i = k / nz, j = k % nz;
            const cff xk = iterate_at(xc, dc, k);
            cff sx = {{0.f, 0.f}, {0.f, 0.f}}, sz = sx;
            if (i > 0) sx = cff_add(sx, iterate_at(xc, dc, k - nz));
            if (i < nx - 1) sx = cff_add(sx, iterate_at(xc, dc, k + nz));
            if (j > 0) sz = cff_add(sz, iterate_at(xc, dc, k - 1));
            if (j < nz - 1) sz = cff_add(sz, iterate_at(xc, dc, k + 1));
            const ff cxj = (j == 0 || j == nz - 1) ? cp.cx_edge : cp.cx_in;
            const ff czi = (i == 0 || i == nx - 1) ? cp.cz_edge : cp.cz_in;
            cff ax = cff_mul(cff_of(diag2[(size_t)sys * N + k]), xk);
            ax = cff_add(ax, cff_scale(sx, cxj));
            ax = cff_add(ax, cff_scale(sz, czi));
            const cff r = cff_sub(cff_of(__ldcs(bd + base + k)), ax);
            x_out[base + k] = cff_pack(xk);
            r32[base + k] = make_float2(r.re.hi, r.im.hi);
            const float sr = r.re.hi * scale, si = r.im.hi * scale;
            rr = fmaf(sr, sr, fmaf(si, si, rr));
        }
        rr = block_sum(rr, shf);
        if (threadIdx.x == 0) atomicAdd(norms + 2 * (size_t)c, ldexp((double)rr, 2 * ks));
        __syncthreads();   // shf reused by the next column
    }
    if (state) {   // the last block to finish applies the stopping test
        if (threadIdx.x == 0) {
            __threadfence();   // this block's norm contributions before its count
            s_last = atomicAdd(&state->blocks, 1u) == gridDim.x * gridDim.y - 1;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            refine_stop_test(cols, nrhs, norms, stop, state, shd);
            if (threadIdx.x == 0) state->blocks = 0;
        }
    }
}

__global__ void refine_accumulate_kernel(size_t n, const float2 *d, int conj, double2 *X) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const float2 v = d[e];
        double2 x = X[e];
        x.x += (double)v.x;
        x.y += conj ? -(double)v.y : (double)v.y;
        X[e] = x;
    }
}

__global__ void refine_finish_kernel(size_t n, int N, int nrhs, const float4 *xa, const float4 *xb,
                                     const RefineState *st, int conj, double2 *X) {
    const int *sys = refine_sys(st);
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    auto at = [&](size_t e) -> float4 {   // the newest iterate of this element's system
        const int q = (int)(e / N) / nrhs;
        return (sys[2 * q] & 1) ? __ldcs(xa + e) : __ldcs(xb + e);
    };
    size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    for (; e + 3 * stride < n; e += 4 * stride) {   // four loads in flight per thread
        float4 v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = at(e + q * stride);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const double re = pair_to_double(v[q].x, v[q].z), im = pair_to_double(v[q].y, v[q].w);
            X[e + q * stride] = make_double2(re, conj ? -im : im);
        }
    }
    for (; e < n; e += stride) {
        const float4 v = at(e);
        const double re = pair_to_double(v.x, v.z), im = pair_to_double(v.y, v.w);
        X[e] = make_double2(re, conj ? -im : im);
    }
}

ff pair_of(double v) {
    ff p;
    split_double(v, p.hi, p.lo);
    return p;
}

unsigned flat_blocks(size_t n) { return (unsigned)std::min<size_t>((n + 255) / 256, 152 * 16); }

}  // namespace

cudaError_t launch_split_diag(size_t n, const double2 *diag, float4 *diag2, cudaStream_t st) {
    HELM_TRACED(K_SPLITDIAG, st, (split_diag_kernel<<<flat_blocks(n), 256, 0, st>>>(n, diag, diag2)));
    return cudaGetLastError();
}

cudaError_t launch_refine_start(const GridGeom &g, int cols, const double2 *B, int conj, float4 *bd, float2 *r32,
                                double *norms, cudaStream_t st) {
    const int N = g.nx * g.nz;
    cudaError_t e = cudaMemsetAsync(norms, 0, (size_t)cols * 2 * sizeof(double), st);
    if (e != cudaSuccess) return e;
    dim3 grid((N + RF_THREADS * RF_NPT - 1) / (RF_THREADS * RF_NPT), std::min(cols, 65535));
    HELM_TRACED(K_REFSTART, st, (refine_start_kernel<<<grid, RF_THREADS, 0, st>>>(N, cols, B, conj, bd, r32, norms)));
    return cudaGetLastError();
}

cudaError_t launch_refine_update(const GridGeom &g, int n_sys, int nrhs, const float4 *diag2, const float4 *bd,
                                 const float4 *x_in, const float2 *delta, float4 *x_out, float2 *r32, double *norms,
                                 cudaStream_t st, RefineState *state, RefineStop stop) {
    const int N = g.nx * g.nz, cols = n_sys * nrhs;
    StencilPairs cp{pair_of(coup_x(g, 1)), pair_of(coup_x(g, 0)), pair_of(coup_z(g, 1)), pair_of(coup_z(g, 0))};
    dim3 grid((N + RF_THREADS * RF_NPT - 1) / (RF_THREADS * RF_NPT), std::min(cols, 65535));
    HELM_TRACED(K_REFUPDATE, st, (refine_update_kernel<<<grid, RF_THREADS, 0, st>>>(g, nrhs, cols, diag2, bd, x_in, delta,
                                                                                    x_out, r32, norms, cp, state, stop)));
    return cudaGetLastError();
}

cudaError_t launch_refine_finish(size_t n, int N, int nrhs, const float4 *xa, const float4 *xb,
                                 const RefineState *state, int conj, double2 *X, cudaStream_t st) {
    HELM_TRACED(K_REFFINISH, st, (refine_finish_kernel<<<flat_blocks(n), 256, 0, st>>>(n, N, nrhs, xa, xb, state, conj, X)));
    return cudaGetLastError();
}

cudaError_t launch_refine_accumulate(size_t n, const float2 *delta, int conj, double2 *X, cudaStream_t st) {
    HELM_TRACED(K_REFACCUM, st, (refine_accumulate_kernel<<<flat_blocks(n), 256, 0, st>>>(n, delta, conj, X)));
    return cudaGetLastError();
}

}  // namespace helm
