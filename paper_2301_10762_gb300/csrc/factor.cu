// Line Schur factorisation of the block-tridiagonal Helmholtz matrix.
//
// With lines of constant i (n_z nodes each, z fastest), A(m, w) of the Appendix
// ("Numerical forward model") is block tridiagonal: D_i tridiagonal (the five-point
// stiffness along z plus the diagonal mass and boundary terms) and C_i = diag(c) the
// couplings between lines i-1 and i.  Block LU without block pivoting gives
//     S_0 = D_0,   S_i = D_i - C_i S_{i-1}^{-1} C_i,
// and the factor stores G_i = S_i^{-1} for every line (used by the sweeps as dense
// GEMM operands).  Because C_i is diagonal the Schur update is elementwise:
// (C G C)_{ab} = c_a G_ab c_b.
//
// One thread-block cluster factors one system (one (model, frequency) pair); the
// recurrence over lines is sequential, so parallelism inside a system comes from
// splitting each line's n_z x n_z inversion over the CTAs of the cluster by column
// blocks.  The inversion is an in-place block Gauss-Jordan sweep with 16 x 16 blocks:
//   for k:  P = inv(W_kk)                       (partial pivoting inside the block)
//           W_kJ <- P W_kJ,  W_IJ <- W_IJ - W_Ik W_kJ,  W_Ik <- -W_Ik P,  W_kk <- P.
// The owner of column block k inverts W_kk and publishes P and the old column panel
// W_:k through a double-buffered exchange slot in global memory (L2 resident); one
// hardware cluster barrier per block step orders publish and use.  Each CTA only ever
// touches its own columns of W, which lives in the factor storage itself (G_i slot).
#include <stdlib.h>
#include "kernels.h"
#include "pivot16.cuh"
#include "trace.h"

namespace helm {

constexpr int FAC_THREADS = 256;

__host__ __device__ size_t factor_xch_elems(int nz) { return 2 * ((size_t)nz * NB + NB * NB); }

template <typename T> __device__ __forceinline__ cx_t<T> from_c128(double2 a);
template <> __device__ __forceinline__ double2 from_c128<double>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from_c128<float>(double2 a) { return to_c64(a); }

template <typename T> struct FactorArgs {
    GridGeom g;
    const double2 *diag;  // [n_sys][N]
    cx_t<T> *G;           // [n_sys][nx][nz][nz]
    cx_t<T> *xch;         // [n_sys][factor_xch_elems(nz)]
    int *status;
    int cs;               // CTAs per team (cluster = teams * cs)
    int mid;              // middle line of the twisted factorisation (nx - 1: one-sided)
    float flag_tol;       // complex FP32: a Gauss-Jordan pivot inverse with max |I - M X| above
                          // this is redone in FP64 (status[1] counts those blocks)
    uint32_t tries;       // polls of a bounded mbarrier wait before it gives up
};

// In-place Gauss-Jordan inversion of the kb x kb block M (row stride NB, shared memory)
// with partial pivoting; the inverse is written to out (row stride NB).  aug is a
// kb x 2kb scratch (row stride 2*NB), fcol a length-NB scratch.
template <typename T>
__device__ void invert_block(const cx_t<T> *M, int kb, cx_t<T> *out, cx_t<T> *aug, cx_t<T> *fcol,
                             int *s_piv, int *s_ok, int &bad) {
    using V = cx_t<T>;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int w2 = 2 * kb;
    for (int e = tid; e < kb * w2; e += nt) {
        int r = e / w2, c = e % w2;
        aug[r * 2 * NB + c] = (c < kb) ? M[r * NB + c] : mkc<T>((c - kb) == r ? T(1) : T(0), T(0));
    }
    __syncthreads();
    for (int q = 0; q < kb; ++q) {
        if (tid < 32) {
            T best = T(-1);
            int bi = q;
            for (int r = q + tid; r < kb; r += 32) {
                V a = aug[r * 2 * NB + q];
                T v = a.x * a.x + a.y * a.y;
                if (v > best) { best = v; bi = r; }
            }
            for (int off = 16; off > 0; off >>= 1) {
                T ob = __shfl_down_sync(0xffffffffu, best, off);
                int oi = __shfl_down_sync(0xffffffffu, bi, off);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (tid == 0) {
                *s_piv = bi;
                *s_ok = (best > T(0) && isfinite(best)) ? 1 : 0;
            }
        }
        __syncthreads();
        const int piv = *s_piv;
        const int ok = *s_ok;
        if (!ok) bad = 1;
        if (ok && piv != q && tid < w2) {
            V t = aug[q * 2 * NB + tid];
            aug[q * 2 * NB + tid] = aug[piv * 2 * NB + tid];
            aug[piv * 2 * NB + tid] = t;
        }
        __syncthreads();
        V pv = aug[q * 2 * NB + q];
        if (tid < kb) fcol[tid] = aug[tid * 2 * NB + q];
        __syncthreads();
        if (ok && tid < w2) {
            T den = pv.x * pv.x + pv.y * pv.y;
            V inv = mkc<T>(pv.x / den, -pv.y / den);
            aug[q * 2 * NB + tid] = cmul(aug[q * 2 * NB + tid], inv);
        }
        __syncthreads();
        if (ok) {
            for (int e = tid; e < kb * w2; e += nt) {
                int r = e / w2, c = e % w2;
                if (r != q) cfms(aug[r * 2 * NB + c], fcol[r], aug[q * 2 * NB + c]);
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < kb * kb; e += nt) {
        int r = e / kb, c = e % kb;
        out[r * NB + c] = aug[r * 2 * NB + kb + c];
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(FAC_THREADS) line_factor_kernel(FactorArgs<T> a) {
    using V = cx_t<T>;
    const GridGeom g = a.g;
    const int nx = g.nx, nz = g.nz, cs = a.cs;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int rank = (int)cluster_ctarank();
    const int sys = (int)cluster_id_x();
    const int p = (nz + NB - 1) / NB;
    const int bpc = (p + cs - 1) / cs;
    const int kb_lo = rank * bpc, kb_hi = min(p, kb_lo + bpc);
    const int c0 = min(nz, kb_lo * NB), c1 = min(nz, kb_hi * NB);
    const int ncol = max(0, c1 - c0);
    const int RS = bpc * NB;  // row stride of sR

    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *sPanel = reinterpret_cast<V *>(smem_raw);     // nz x NB
    V *sP = sPanel + (size_t)nz * NB;                // NB x NB
    V *sR = sP + NB * NB;                            // NB x RS
    V *sAug = sR + NB * RS;                          // NB x 2NB
    V *sF = sAug + 2 * NB * NB;                      // NB
    __shared__ int s_piv, s_ok;

    V *Gs = a.G + (size_t)sys * nx * nz * nz;
    const double2 *dg = a.diag + (size_t)sys * nx * nz;
    V *xch = a.xch + (size_t)sys * factor_xch_elems(nz);
    const size_t slot_elems = (size_t)nz * NB + NB * NB;
    int bad = 0;
    int step = 0;
    // grid couplings, converted once (no FP64 work in the per-element loops)
    const T cx_in = (T)coup_x(g, 1), cx_edge = (T)coup_x(g, 0);
    const T cz_in = (T)coup_z(g, 1), cz_edge = (T)coup_z(g, 0);

    for (int i = 0; i < nx; ++i) {
        V *W = Gs + (size_t)i * nz * nz;
        const V *Wp = Gs + (size_t)(i - 1) * nz * nz;
        const T cz = (i == 0 || i == nx - 1) ? cz_edge : cz_in;
        // S_i = D_i - C_i G_{i-1} C_i on this CTA's columns
        for (int e = tid; e < nz * ncol; e += nt) {
            const int r = e / ncol, c = c0 + e % ncol;
            V v = mkc<T>(T(0), T(0));
            if (r == c) v = from_c128<T>(dg[(size_t)i * nz + r]);
            else if (r == c + 1 || c == r + 1) v = mkc<T>(cz, T(0));
            if (i > 0) {
                const T s = ((r == 0 || r == nz - 1) ? cx_edge : cx_in) * ((c == 0 || c == nz - 1) ? cx_edge : cx_in);
                V gp = Wp[(size_t)r * nz + c];
                v.x -= s * gp.x;
                v.y -= s * gp.y;
            }
            W[(size_t)r * nz + c] = v;
        }
        __syncthreads();

        for (int k = 0; k < p; ++k, ++step) {
            const int k0 = k * NB, kb = min(NB, nz - k0);
            const int owner = k / bpc;
            V *slot = xch + (size_t)(step & 1) * slot_elems;
            V *slotPanel = slot;
            V *slotP = slot + (size_t)nz * NB;
            if (rank == owner) {
                for (int e = tid; e < nz * kb; e += nt) {
                    const int r = e / kb, q = e % kb;
                    sPanel[r * NB + q] = W[(size_t)r * nz + k0 + q];
                }
                __syncthreads();
                invert_block<T>(sPanel + (size_t)k0 * NB, kb, sP, sAug, sF, &s_piv, &s_ok, bad);
                for (int e = tid; e < nz * kb; e += nt) {
                    const int r = e / kb, q = e % kb;
                    slotPanel[r * NB + q] = sPanel[r * NB + q];
                }
                for (int e = tid; e < kb * kb; e += nt) {
                    const int r = e / kb, q = e % kb;
                    slotP[r * NB + q] = sP[r * NB + q];
                }
                // own column block k: W_Ik <- -W_Ik P, W_kk <- P
                for (int e = tid; e < nz * kb; e += nt) {
                    const int r = e / kb, q = e % kb;
                    V v;
                    if (r >= k0 && r < k0 + kb) {
                        v = sP[(r - k0) * NB + q];
                    } else {
                        V acc = mkc<T>(T(0), T(0));
                        for (int t = 0; t < kb; ++t) cfma(acc, sPanel[r * NB + t], sP[t * NB + q]);
                        v = mkc<T>(-acc.x, -acc.y);
                    }
                    W[(size_t)r * nz + k0 + q] = v;
                }
            }
            cluster_sync_all();
            if (rank != owner) {
                for (int e = tid; e < nz * kb; e += nt) {
                    const int r = e / kb, q = e % kb;
                    sPanel[r * NB + q] = ldcg(slotPanel + r * NB + q);
                }
                for (int e = tid; e < kb * kb; e += nt) {
                    const int r = e / kb, q = e % kb;
                    sP[r * NB + q] = ldcg(slotP + r * NB + q);
                }
            }
            __syncthreads();
            // Rk = P W[k rows, own columns != k block]
            for (int e = tid; e < kb * ncol; e += nt) {
                const int q = e / ncol, cc = e % ncol, c = c0 + cc;
                if (c >= k0 && c < k0 + kb) continue;
                V acc = mkc<T>(T(0), T(0));
                for (int t = 0; t < kb; ++t) cfma(acc, sP[q * NB + t], W[(size_t)(k0 + t) * nz + c]);
                sR[q * RS + cc] = acc;
            }
            __syncthreads();
            for (int e = tid; e < nz * ncol; e += nt) {
                const int r = e / ncol, cc = e % ncol, c = c0 + cc;
                if (c >= k0 && c < k0 + kb) continue;
                if (r >= k0 && r < k0 + kb) {
                    W[(size_t)r * nz + c] = sR[(r - k0) * RS + cc];
                } else {
                    V acc = W[(size_t)r * nz + c];
                    for (int t = 0; t < kb; ++t) cfms(acc, sPanel[r * NB + t], sR[t * RS + cc]);
                    W[(size_t)r * nz + c] = acc;
                }
            }
            __syncthreads();
        }
    }
    if (bad && tid == 0) atomicOr(a.status, ST_SINGULAR);
}

// ----------------------------------------------------------------------------------
// Shared-memory-resident variant (used whenever the slab fits): each CTA keeps its own
// columns of S_i / G_i in shared memory for the whole line recurrence, so the Schur
// update S_{i+1} = D_{i+1} - C G_i C of its columns is local.  Per 16-column block step
// the owner inverts the diagonal block in one warp (registers and shuffles, partial
// pivoting without row swaps: the pivot order is applied when the inverse is written)
// and pushes the old column panel and the block inverse into every CTA's receive
// buffer with distributed-shared-memory stores; one hardware cluster barrier per
// block step publishes them.  Receive buffers alternate, so the owner of step t+1 never
// overwrites data a slower CTA still reads at step t.

// Flagged pivot block, one warp: the FP32 kb x kb block M (row stride ld) promoted to FP64
// (identity outside kb), inverted by warp_invert16<double>, the inverse rounded into P (row
// stride NB, rows and columns < kb).  d64 is a 2 x 16 x 16 FP64 scratch.  Kept out of line so
// that the FP64 registers do not weigh on the factor's main loop.
__device__ __noinline__ bool fp64_pivot_inverse(const float2 *M, int ld, int kb, double2 *d64, float2 *P) {
    const int lane = threadIdx.x & 31;
    for (int e = lane; e < NB * NB; e += 32) {
        const int r = e >> 4, c = e & 15;
        const float2 v = M[(size_t)(r < kb ? r : 0) * ld + (c < kb ? c : 0)];
        d64[e] = (r < kb && c < kb) ? make_double2((double)v.x, (double)v.y) : make_double2(r == c ? 1.0 : 0.0, 0.0);
    }
    __syncwarp();
    const bool ok = warp_invert16<double>(d64, NB, kb, d64 + NB * NB);
    __syncwarp();
    for (int e = lane; e < NB * NB; e += 32) {
        const int r = e >> 4, c = e & 15;
        if (r < kb && c < kb) P[e] = to_c64(d64[NB * NB + e]);
    }
    return ok;
}

// Accurate residual correction of a complex-FP32 16 x 16 inverse, 256 threads (thread (r, c)):
// E = I - M X with every product exact (the FMA gives its rounding error) and the sums kept as
// FP32 pairs (Knuth's two-sum), then X <- X + X E in FP32.  E is about the inverse's rounding
// error, so one step brings X to the inverse of M rounded to FP32, whatever route (Newton-Schulz,
// Gauss-Jordan) produced it.  M shared with row stride ld, P (in and out) row stride NB; the
// kb x kb block is extended by the identity.
// hi + lo += a b exactly up to the final rounding of lo (intrinsics: no contraction into FMAs)
__device__ __forceinline__ void pair_add_prod(float &hi, float &lo, float a, float b) {
    const float p = __fmul_rn(a, b), pe = fmaf(a, b, -p);
    const float s = __fadd_rn(hi, p), bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    lo = __fadd_rn(lo, __fadd_rn(e, pe));
    hi = s;
}
__device__ void polish_inverse16(const float2 *M, int ld, int kb, float2 *P, float2 (*sM)[NB + 1],
                                 float2 (*sX)[NB + 1], float2 (*sE)[NB + 1]) {
    const int tid = threadIdx.x, r = tid >> 4, c = tid & 15;
    const bool in = r < kb && c < kb;
    sM[r][c] = in ? M[r * ld + c] : make_float2(r == c ? 1.f : 0.f, 0.f);
    sX[r][c] = in ? P[r * NB + c] : make_float2(r == c ? 1.f : 0.f, 0.f);
    __syncthreads();
    float erh = r == c ? 1.f : 0.f, erl = 0.f, eih = 0.f, eil = 0.f;
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        const float2 a = sM[r][u], b = sX[u][c];
        pair_add_prod(erh, erl, -a.x, b.x);   // Re(I - M X): - Re M Re X + Im M Im X
        pair_add_prod(erh, erl, a.y, b.y);
        pair_add_prod(eih, eil, -a.x, b.y);   // Im: - Re M Im X - Im M Re X
        pair_add_prod(eih, eil, -a.y, b.x);
    }
    sE[r][c] = make_float2(erh + erl, eih + eil);
    __syncthreads();
    float2 xe[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
    for (int u = 0; u < NB; ++u) cfma(xe[u & 3], sX[r][u], sE[u][c]);
    const float2 x0 = sX[r][c];
    const float2 x = make_float2(x0.x + ((xe[0].x + xe[1].x) + (xe[2].x + xe[3].x)),
                                 x0.y + ((xe[0].y + xe[1].y) + (xe[2].y + xe[3].y)));
    if (in) P[r * NB + c] = x;
    __syncthreads();
}

// max |I - M X| over the kb x kb block (M shared with row stride ld, X row stride NB), the rest
// of the 16 x 16 tile taken as the identity; every thread of the 256-thread CTA returns it.
template <typename T>
__device__ float block_residual(const cx_t<T> *M, int ld, const cx_t<T> *X, int kb, float *sred) {
    using V = cx_t<T>;
    const int tid = threadIdx.x, r = tid >> 4, c = tid & 15, lane = tid & 31, wid = tid >> 5;
    float a = 0.f;
    if (r < kb && c < kb) {
        V e = mkc<T>(r == c ? T(1) : T(0), T(0));
        for (int u = 0; u < kb; ++u) cfms(e, M[r * ld + u], X[u * NB + c]);
        a = (float)(e.x * e.x + e.y * e.y);
        a = isfinite(a) ? a : 3.0e38f;
    }
    for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
    if (lane == 0) sred[wid] = a;
    __syncthreads();
    float en2 = 0.f;
#pragma unroll
    for (int w = 0; w < FAC_THREADS / 32; ++w) en2 = fmaxf(en2, sred[w]);
    __syncthreads();   // sred reusable
    return sqrtf(en2);
}

// Inverse of the 16 x 16 block M (shared, row stride ld) by Newton-Schulz iteration from the
// seed X0 (row stride NB), one element per thread of a 256-thread CTA (thread (r, c) =
// (tid / 16, tid % 16)):  E = I - M X,  X <- X + X E  (quadratic convergence while |E| < 1).
// Consecutive lines have nearly equal Schur complements, so the inverse of the same pivot block
// on the previous line is a seed with |E| around 1e-3 (1e-2 at worst away from the first lines),
// and two or three iterations reach the FP32 floor: about ten times fewer dependent steps than
// the pivoted Gauss-Jordan of warp_invert16.  Returns false (P untouched) when the seed is too
// far (|E| > 1/4 at the start) or the iteration stalls above 1e-4; the caller then uses
// Gauss-Jordan.  |E| is the largest entry modulus; all threads take the same decisions.
template <typename T>
__device__ bool ns_invert16(const cx_t<T> *M, int ld, const cx_t<T> *X0, cx_t<T> *P, cx_t<T> (*sM)[NB + 1],
                            cx_t<T> (*sX)[NB + 1], cx_t<T> (*sE)[NB + 1], float *sred) {
    using V = cx_t<T>;
    const int tid = threadIdx.x, r = tid >> 4, c = tid & 15, lane = tid & 31, wid = tid >> 5;
    sM[r][c] = M[r * ld + c];
    sX[r][c] = X0[r * NB + c];
    __syncthreads();
    float eprev = 0.f;
    bool ok = false;
    for (int it = 0; it < 6; ++it) {
        V e = mkc<T>(r == c ? T(1) : T(0), T(0));
#pragma unroll
        for (int u = 0; u < NB; ++u) cfms(e, sM[r][u], sX[u][c]);
        sE[r][c] = e;
        float a = (float)(e.x * e.x + e.y * e.y);
        a = isfinite(a) ? a : 3.0e38f;
        for (int o = 16; o > 0; o >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, o));
        if (lane == 0) sred[wid] = a;
        __syncthreads();   // sE and sred complete
        float en2 = 0.f;
#pragma unroll
        for (int w = 0; w < FAC_THREADS / 32; ++w) en2 = fmaxf(en2, sred[w]);
        const float en = sqrtf(en2);
        if (it == 0 && !(en <= 0.25f)) break;                       // seed too far: Gauss-Jordan
        if (en < 1e-7f) { ok = true; break; }                        // converged
        if (it > 0 && en > 0.5f * eprev) { ok = eprev < 1e-4f; break; }   // FP32 floor (X of the last step)
        eprev = en;
        V x = sX[r][c];
#pragma unroll
        for (int u = 0; u < NB; ++u) cfma(x, sX[r][u], sE[u][c]);
        __syncthreads();   // every read of the old X and of sred done
        sX[r][c] = x;
        __syncthreads();
        // quadratic convergence: the new X leaves about |E|^2; below 1e-4 (|E| < 1e-2) the
        // exactly-summed correction that follows (polish_inverse16) takes it to the FP32 floor
        if (en < 1e-2f) { ok = true; break; }
    }
    if (ok) P[r * NB + c] = sX[r][c];
    __syncthreads();
    return ok;
}

__device__ __forceinline__ void st_cluster_c(uint32_t addr, float2 v) { st_cluster(addr, v); }
__device__ __forceinline__ void st_cluster_c(uint32_t addr, double2 v) { st_cluster(addr, v); }

// Twisted variant: the cluster holds two teams of `cs` CTAs.  The left team runs the
// Schur recurrence from the absorbing boundary x = 0 (S_0 = D_0, S_i = D_i - C G_{i-1} C,
// i < m), the right team from x = L (S_{nx-1} = D_{nx-1}, S_i = D_i - C G_{i+1} C, i > m),
// concurrently, and the left team then factors the middle line
//     S_m = D_m - C G_{m-1} C - C G_{m+1} C.
// The factor stores G_i = S_i^{-1} for every line (left inverses for i < m, right ones for
// i > m).  With teams == 1 and m = nx - 1 this is the plain one-sided factorisation.
// The two teams only meet at the middle line (G_{m+1} is read back from global memory);
// the panel exchange of each block step stays inside a team.
template <typename T>
__global__ void __launch_bounds__(FAC_THREADS, 1) line_factor_smem_kernel(FactorArgs<T> a) {
    using V = cx_t<T>;
    const GridGeom g = a.g;
    const int nx = g.nx, nz = g.nz, cs = a.cs;
    const int tid = threadIdx.x;
    const int crank = (int)cluster_ctarank();
    const int team = crank / cs, rank = crank % cs;
    const int sys = (int)cluster_id_x();
    const int p = (nz + NB - 1) / NB;
    const int bpc = (p + cs - 1) / cs;
    const int kb_lo = rank * bpc, kb_hi = min(p, kb_lo + bpc);
    const int c0 = min(nz, kb_lo * NB), c1 = min(nz, kb_hi * NB);
    const int ncol = max(0, c1 - c0);
    const int ncb = (ncol + NB - 1) / NB;     // own column blocks
    const int ldw = bpc * NB + 1;             // padded row stride of the slab
    const int ldr = bpc * NB + 1;
    const int m = a.mid;                      // middle line (nx - 1 without a right team)
    const int lenR = nx - 1 - m;              // lines of the right team
    unsigned cluster_ctas;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(cluster_ctas));

    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *sW = reinterpret_cast<V *>(smem_raw);                  // nz x ldw   own columns of S_i / G_i
    const size_t recv_off = ((size_t)nz * ldw * sizeof(V) + 15) & ~(size_t)15;
    V *sRecv = reinterpret_cast<V *>(smem_raw + recv_off);    // 2 x (nz*NB + NB*NB), 16-byte aligned
    const size_t recv_elems = (size_t)nz * NB + NB * NB;
    V *sR = sRecv + 2 * recv_elems;                           // NB x ldr
    __shared__ int s_bad;
    __shared__ int s_abort;                                   // a wait of the cluster gave up
    __shared__ __align__(8) uint64_t bars[2];                 // panel arrival, one per receive buffer
    // buffer release: the other CTAs of the team arrive on the empty barrier of the CTA that
    // next writes into a receive buffer (the owner of the step two later) once they are done
    // with it; that owner waits before it stages and sends the panel
    __shared__ __align__(8) uint64_t empty_bars[2];
    // Newton-Schulz pivot inversion (complex FP32): work blocks and the previous line's inverse of
    // each pivot block this CTA owns (the seed)
    constexpr bool kNS = sizeof(T) == 4;
    constexpr int kSeedBlocks = 4;
    __shared__ __align__(16) V s_nsM[kNS ? NB : 1][NB + 1], s_nsX[kNS ? NB : 1][NB + 1], s_nsE[kNS ? NB : 1][NB + 1];
    __shared__ __align__(16) V s_seed[kNS ? kSeedBlocks : 1][kNS ? NB * NB : 1];
    __shared__ float s_nsred[FAC_THREADS / 32];
    // flagged pivot blocks: the FP32 entries and the FP64 inverse
    __shared__ __align__(16) double2 s_d64[kNS ? 2 : 1][kNS ? NB * NB : 1];

    V *Gs = a.G + (size_t)sys * nx * nz * nz;
    const double2 *dg = a.diag + (size_t)sys * nx * nz;
    const T cx_in = (T)coup_x(g, 1), cx_edge = (T)coup_x(g, 0);
    const T cz_in = (T)coup_z(g, 1), cz_edge = (T)coup_z(g, 0);
    const int cl = tid & (NB - 1), rw = tid >> 4;   // (row group, column) of the 2D loops
    if (tid == 0) {
        s_bad = 0;
        s_abort = 0;
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&empty_bars[0], (uint32_t)max(cs - 1, 1));
        mbar_init(&empty_bars[1], (uint32_t)max(cs - 1, 1));
        fence_mbar_init_cluster();
    }
    __syncthreads();
    const uint32_t panel_bytes = (uint32_t)(recv_elems * sizeof(V));     // what a consumer receives per step
    const uint32_t panel_u_bytes = (uint32_t)((size_t)nz * NB * sizeof(V));   // old column panel
    const uint32_t panel_p_bytes = panel_bytes - panel_u_bytes;               // block inverse
    uint32_t ph0 = 0, ph1 = 0;   // completed panel phases per receive buffer (consumer side)
    uint32_t eph0 = 0, eph1 = 0;   // completed release phases of this CTA's empty barriers (thread 0)
    bool tmo = false;              // thread 0: a wait gave up; later waits are skipped
    // thread 0: after a give-up anywhere in the cluster it sends, expects and releases nothing
    // more, so that no barrier sees arrivals or bytes that nobody accounts for
    auto quiet = [&]() { return tmo || *(volatile int *)&s_abort != 0; };
    // whether this team works on a line at the given slot
    auto active_slot = [&](int sl) { return team == 0 ? sl <= m : sl < lenR; };
    int t = 0;

    for (int slot = 0; slot <= m; ++slot) {
        // line of this team at this slot (-1: idle); the left team ends with the middle line
        int i = -1, iprev = -1;
        if (team == 0) { i = slot; iprev = slot - 1; }
        else if (slot < lenR) { i = nx - 1 - slot; iprev = (slot == 0) ? -1 : i + 1; }
        const bool active = i >= 0;
        const bool middle = (team == 0 && slot == m && lenR > 0);
        // the previous slot's G write-out of both teams is visible (the middle line reads G_{m+1})
        cluster_sync_all();
        if (active) {
            const T cz = (i == 0 || i == nx - 1) ? cz_edge : cz_in;
            const V *Gright = Gs + (size_t)(m + 1) * nz * nz;   // G_{m+1}, written by the right team
            // S_i = D_i - C G_prev C (the slab holds G_prev), minus C G_{m+1} C on the middle line
            for (int cb = 0; cb < ncb; ++cb) {
                const int cc = cb * NB + cl, c = c0 + cc;
                if (c >= c1) continue;
                const T cxc = (c == 0 || c == nz - 1) ? cx_edge : cx_in;
                for (int r = rw; r < nz; r += FAC_THREADS / NB) {
                    const T cxr = (r == 0 || r == nz - 1) ? cx_edge : cx_in;
                    const T sc = cxr * cxc;
                    V v = mkc<T>(T(0), T(0));
                    if (iprev >= 0) {
                        const V gp = sW[(size_t)r * ldw + cc];
                        v = mkc<T>(-sc * gp.x, -sc * gp.y);
                    }
                    if (middle) {
                        const V gr = ldcg(Gright + (size_t)r * nz + c);
                        v.x -= sc * gr.x;
                        v.y -= sc * gr.y;
                    }
                    if (r == c) {
                        const V d = from_c128<T>(dg[(size_t)i * nz + r]);
                        v.x += d.x;
                        v.y += d.y;
                    } else if (r == c + 1 || c == r + 1) {
                        v.x += cz;
                    }
                    sW[(size_t)r * ldw + cc] = v;
                }
            }
        }
        __syncthreads();

        for (int k = 0; k < p; ++k, ++t) {
            const int k0 = k * NB, kb = min(NB, nz - k0);
            const int owner = k / bpc;
            const int buf = t & 1;
            V *recvU = sRecv + (size_t)buf * recv_elems;        // nz x NB: old column panel W_:k
            V *recvP = recvU + (size_t)nz * NB;                 // NB x NB: inverse of W_kk
            if (active) {
                if (rank == owner) {
                    // the other CTAs of the team are done with this buffer (its use two steps ago,
                    // including a bulk copy this CTA sent from it)
                    if (t >= 2 && cs > 1) {
                        if (tid == 0) {
                            const uint32_t par = buf ? eph1 : eph0;
                            if (!quiet() && !mbar_wait_or_abort(&empty_bars[buf], par, a.tries, &s_abort)) {
                                atomicOr(a.status, ST_TIMEOUT);
                                tmo = true;
                                if (atomicExch(&s_abort, 1) == 0) cluster_abort_broadcast(&s_abort, (unsigned)cluster_ctas);
                            }
                            if (buf) eph1 ^= 1u; else eph0 ^= 1u;
                        }
                        __syncthreads();
                    }
                    const int kc = k0 - c0;
                    // stage the old column panel and send it to the other CTAs of the team at once
                    // (the bulk-copy engine delivers it while the pivot block is inverted); the
                    // block inverse, staged right after it, follows on the same barrier.  Within a
                    // line (complex FP32, at most two blocks per CTA) the previous step's update
                    // has already written the panel here.
                    if (!(kNS && k > 0 && bpc <= 2)) {
                        for (int r = rw; r < nz; r += FAC_THREADS / NB)
                            if (cl < kb) recvU[(size_t)r * NB + cl] = sW[(size_t)r * ldw + kc + cl];
                        __syncthreads();
                    }
                    if (tid == 0 && !quiet()) {
                        fence_proxy_async_smem();
                        const uint32_t src = smem_u32(recvU), lbar = smem_u32(&bars[buf]);
                        for (int d = 0; d < cs; ++d)
                            if (d != rank) {
                                const uint32_t dst = (uint32_t)(team * cs + d);
                                bulk_copy_s2s(mapa_u32(src, dst), src, panel_u_bytes, mapa_u32(lbar, dst));
                            }
                    }
                    bool done = false;
                    if constexpr (kNS) {
                        // seeded by this block's inverse on the team's previous line
                        const int kl = k - kb_lo;
                        if (slot > 0 && kb == NB && bpc <= kSeedBlocks)
                            done = ns_invert16<T>(sW + (size_t)k0 * ldw + kc, ldw, s_seed[kl], recvP, s_nsM, s_nsX,
                                                  s_nsE, s_nsred);
                    }
                    if (!done) {
                        if (tid < 32) {
                            if (!warp_invert16<T>(sW + (size_t)k0 * ldw + kc, ldw, kb, recvP) && tid == 0) s_bad = 1;
                        }
                        __syncthreads();
                        if constexpr (kNS) {
                            // a flagged block (ill-conditioned pivot: the FP32 inverse leaves a large
                            // residual) is inverted again by Gauss-Jordan in FP64 on the same entries
                            const V *Mk = sW + (size_t)k0 * ldw + kc;
                            if (block_residual<T>(Mk, ldw, recvP, kb, s_nsred) > a.flag_tol) {
                                if (tid < 32) {
                                    if (!fp64_pivot_inverse(Mk, ldw, kb, &s_d64[0][0], recvP) && tid == 0) s_bad = 1;
                                    if (tid == 0) atomicAdd(a.status + 1, 1);
                                }
                                __syncthreads();
                            }
                        }
                    }
                    if constexpr (kNS) {
                        // FP32 inverse to the FP32 rounding of the exact one: the pivot inverses set
                        // the factor's accuracy, and so the refinement sweeps of every solve
                        polish_inverse16(sW + (size_t)k0 * ldw + kc, ldw, kb, recvP, s_nsM, s_nsX, s_nsE);
                        if (kb == NB && bpc <= kSeedBlocks) s_seed[k - kb_lo][tid] = recvP[tid];   // next line's seed
                    }
                    if (tid == 0 && !quiet()) {
                        fence_proxy_async_smem();
                        const uint32_t src = smem_u32(recvP), lbar = smem_u32(&bars[buf]);
                        for (int d = 0; d < cs; ++d)
                            if (d != rank) {
                                const uint32_t dst = (uint32_t)(team * cs + d);
                                bulk_copy_s2s(mapa_u32(src, dst), src, panel_p_bytes, mapa_u32(lbar, dst));
                            }
                    }
                } else {
                    if (tid == 0 && !quiet()) {
                        mbar_arrive_expect_tx(&bars[buf], panel_bytes);
                        const uint32_t par = buf ? ph1 : ph0;
                        if (!mbar_wait_or_abort(&bars[buf], par, a.tries, &s_abort)) {
                            atomicOr(a.status, ST_TIMEOUT);
                            tmo = true;
                            if (atomicExch(&s_abort, 1) == 0) cluster_abort_broadcast(&s_abort, (unsigned)cluster_ctas);
                        }
                    }
                    if (buf) ph1 ^= 1u; else ph0 ^= 1u;
                    __syncthreads();
                }
                // Rk = P W[k rows, own columns outside block k]
                for (int cb = 0; cb < ncb; ++cb) {
                    const int cc = cb * NB + cl, c = c0 + cc;
                    if (c >= c1 || (c >= k0 && c < k0 + kb)) continue;
                    for (int q = rw; q < kb; q += FAC_THREADS / NB) {
                        V acc = mkc<T>(T(0), T(0));
#pragma unroll 4
                        for (int u = 0; u < kb; ++u) cfma(acc, recvP[q * NB + u], sW[(size_t)(k0 + u) * ldw + cc]);
                        sR[q * ldr + cc] = acc;
                    }
                }
                __syncthreads();
                // rank-kb update of the own columns: W_Ik <- -W_Ik P and W_kk <- P in block column
                // k, W_Ij <- W_Ij - W_Ik Rk elsewhere, rows of block k <- Rk.  A thread keeps its
                // column's kb coefficients in registers; the 16 threads of a row read the old
                // panel row U[r][:] as broadcast 16-byte loads.
                for (int cb = 0; cb < ncb; ++cb) {
                    const int cc = cb * NB + cl, c = c0 + cc;
                    if (c >= c1) continue;
                    const bool inblk = (c >= k0 && c < k0 + kb);
                    V coef[NB];
#pragma unroll
                    for (int u = 0; u < NB; ++u)
                        coef[u] = (u < kb) ? (inblk ? recvP[u * NB + (c - k0)] : sR[u * ldr + cc]) : mkc<T>(T(0), T(0));
                    const int rstep = FAC_THREADS / NB;
                    if constexpr (sizeof(T) == 4) {
                        // owner of the next block step of this line: its old column panel is the
                        // block column k + 1 written here; stage it for the send as well.  With at
                        // most two blocks per CTA this CTA did not send from that buffer at the
                        // previous step, and other CTAs only copy into their own buffers.
                        const int kn = k + 1;
                        const bool stage_next = kn < p && bpc <= 2 && kn / bpc == rank && c >= kn * NB &&
                                                c < kn * NB + min(NB, nz - kn * NB);
                        V *recvUn = sRecv + (size_t)((t + 1) & 1) * recv_elems;
                        const int cn = c - kn * NB;
                        // two rows per pass; the 16 products of a row go into four partial sums
                        // that are combined pairwise and then subtracted from the old value once
                        // (the summation error of the update is what limits the factor's accuracy,
                        // and so the refinement sweeps a solve needs)
                        for (int r = rw; r < nz; r += 2 * rstep) {
                            const int r2 = r + rstep;
                            const bool has2 = r2 < nz;
                            const bool blk1 = r >= k0 && r < k0 + kb, blk2 = has2 && r2 >= k0 && r2 < k0 + kb;
                            V *w1 = sW + (size_t)r * ldw + cc, *w2 = sW + (size_t)(has2 ? r2 : r) * ldw + cc;
                            const V zero = mkc<T>(T(0), T(0));
                            V p1[4] = {zero, zero, zero, zero}, p2[4] = {zero, zero, zero, zero};
                            const float4 *u1 = reinterpret_cast<const float4 *>(recvU + (size_t)r * NB);
                            const float4 *u2 = reinterpret_cast<const float4 *>(recvU + (size_t)(has2 ? r2 : r) * NB);
#pragma unroll
                            for (int h = 0; h < NB / 2; ++h) {
                                const float4 q1 = u1[h], q2 = u2[h];
                                const int e = (2 * h) & 3, o = (2 * h + 1) & 3;
                                if (2 * h < kb) {
                                    cfma(p1[e], make_float2(q1.x, q1.y), coef[2 * h]);
                                    cfma(p2[e], make_float2(q2.x, q2.y), coef[2 * h]);
                                }
                                if (2 * h + 1 < kb) {
                                    cfma(p1[o], make_float2(q1.z, q1.w), coef[2 * h + 1]);
                                    cfma(p2[o], make_float2(q2.z, q2.w), coef[2 * h + 1]);
                                }
                            }
                            const V w1o = (inblk || blk1) ? zero : *w1, w2o = (!has2 || inblk || blk2) ? zero : *w2;
                            const V s1 = mkc<T>((p1[0].x + p1[1].x) + (p1[2].x + p1[3].x),
                                                (p1[0].y + p1[1].y) + (p1[2].y + p1[3].y));
                            const V s2 = mkc<T>((p2[0].x + p2[1].x) + (p2[2].x + p2[3].x),
                                                (p2[0].y + p2[1].y) + (p2[2].y + p2[3].y));
                            const V n1 = blk1 ? (inblk ? recvP[(r - k0) * NB + (c - k0)] : sR[(r - k0) * ldr + cc])
                                              : mkc<T>(w1o.x - s1.x, w1o.y - s1.y);
                            *w1 = n1;
                            if (stage_next) recvUn[(size_t)r * NB + cn] = n1;
                            if (has2) {
                                const V n2 = blk2 ? (inblk ? recvP[(r2 - k0) * NB + (c - k0)] : sR[(r2 - k0) * ldr + cc])
                                                  : mkc<T>(w2o.x - s2.x, w2o.y - s2.y);
                                *w2 = n2;
                                if (stage_next) recvUn[(size_t)r2 * NB + cn] = n2;
                            }
                        }
                    } else {
                        for (int r = rw; r < nz; r += rstep) {
                            V *w = sW + (size_t)r * ldw + cc;
                            if (r >= k0 && r < k0 + kb) {
                                *w = inblk ? recvP[(r - k0) * NB + (c - k0)] : sR[(r - k0) * ldr + cc];
                                continue;
                            }
                            V acc = inblk ? mkc<T>(T(0), T(0)) : *w;
                            const V *ur = recvU + (size_t)r * NB;
#pragma unroll
                            for (int u = 0; u < NB; ++u)
                                if (u < kb) cfms(acc, ur[u], coef[u]);
                            *w = acc;
                        }
                    }
                }
            }
            __syncthreads();
            // done with this step's buffer: release it to the owner of step t + 2, its next writer
            if (active && tid == 0 && cs > 1 && !quiet()) {
                const int t2 = t + 2, owner2 = (t2 % p) / bpc;
                if (active_slot(t2 / p) && owner2 != rank)
                    mbar_arrive_remote(mapa_u32(smem_u32(&empty_bars[buf]), (uint32_t)(team * cs + owner2)));
            }
        }
        if (active) {
            // G_i (own columns) to the factor storage
            V *W = Gs + (size_t)i * nz * nz;
            for (int cb = 0; cb < ncb; ++cb) {
                const int cc = cb * NB + cl, c = c0 + cc;
                if (c >= c1) continue;
                for (int r = rw; r < nz; r += FAC_THREADS / NB) W[(size_t)r * nz + c] = sW[(size_t)r * ldw + cc];
            }
        }
    }
    // no CTA leaves while the bulk-copy engine may still read its shared memory: every
    // consumer has waited for the last panel before arriving here.  After a give-up (the
    // waits of the cluster are skipped from then on, so every CTA reaches this barrier in
    // bounded time) copies may still be in flight: they are drained first.
    cluster_sync_all();
    if (*(volatile int *)&s_abort) abort_drain();
    if (tid == 0 && s_bad) atomicOr(a.status, ST_SINGULAR);
}

template <typename T> static size_t factor_smem_resident_bytes(int nz, int cs) {
    const int p = (nz + NB - 1) / NB;
    const int bpc = (p + cs - 1) / cs;
    const size_t ld = (size_t)bpc * NB + 1;
    const size_t v = sizeof(cx_t<T>);
    return ((v * (size_t)nz * ld + 15) & ~(size_t)15) + v * (2 * ((size_t)nz * NB + NB * NB) + NB * ld);
}

template <typename T> static size_t factor_smem_bytes(int nz, int cs) {
    const int p = (nz + NB - 1) / NB;
    const int bpc = (p + cs - 1) / cs;
    return sizeof(cx_t<T>) * ((size_t)nz * NB + NB * NB + (size_t)NB * bpc * NB + 2 * NB * NB + NB);
}

int pick_cluster_size(int nz) {
    const int p = (nz + NB - 1) / NB;
    return p >= 8 ? 8 : (p >= 4 ? 4 : (p >= 2 ? 2 : 1));
}

template <typename T>
cudaError_t launch_line_factor(const GridGeom &g, int n_sys, const double2 *diag, cx_t<T> *G, cx_t<T> *xch,
                               int *status, int cs, cudaStream_t st, int *mid_out) {
    const size_t smem_res = factor_smem_resident_bytes<T>(g.nz, cs);
    const bool resident = smem_res <= 200 * 1024;
    int teams = 1;
    cudaError_t e;
    // HELM_FACTOR_TEAMS=1 forces the one-sided factorisation (for comparisons)
    const char *force = getenv("HELM_FACTOR_TEAMS");
    const bool allow_twisted = !(force && force[0] == '1');
    if (resident) {
        e = ensure_dyn_smem((const void *)line_factor_smem_kernel<T>, smem_res);
        if (e != cudaSuccess) return e;
    }
    if (resident && allow_twisted) {
        // two teams (twisted) when a cluster of 2 cs CTAs can be scheduled
        if (2 * cs <= 16) {
            const bool ok = max_active_clusters((const void *)line_factor_smem_kernel<T>, 2 * cs, FAC_THREADS,
                                                smem_res) > 0;
            if (ok) teams = 2;
        }
    }
    const int mid = (teams == 2) ? g.nx / 2 : g.nx - 1;
    if (mid_out) *mid_out = mid;
    // HELM_FACTOR_FLAG_TOL overrides the residual above which a pivot inverse is redone in FP64
    const char *env_tol = getenv("HELM_FACTOR_FLAG_TOL");
    const float flag_tol = (env_tol && *env_tol) ? (float)atof(env_tol) : 1e-4f;
    FactorArgs<T> a{g, diag, G, xch, status, cs, mid, flag_tol, wait_tries()};
    const size_t smem = resident ? smem_res : factor_smem_bytes<T>(g.nz, cs);
    auto kern = resident ? line_factor_smem_kernel<T> : line_factor_kernel<T>;
    if (!resident) {
        e = ensure_dyn_smem((const void *)kern, smem);
        if (e != cudaSuccess) return e;
    }
    const int csz = teams * cs;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_sys * csz, 1, 1);
    cfg.blockDim = dim3(FAC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csz;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t le = cudaSuccess;
    HELM_TRACED(sizeof(T) == 8 ? K_FACTOR64 : K_FACTOR32, st, (le = cudaLaunchKernelEx(&cfg, kern, a)));
    return le;
}

template cudaError_t launch_line_factor<double>(const GridGeom &, int, const double2 *, double2 *, double2 *,
                                                int *, int, cudaStream_t, int *);
template cudaError_t launch_line_factor<float>(const GridGeom &, int, const double2 *, float2 *, float2 *,
                                               int *, int, cudaStream_t, int *);

}  // namespace helm
