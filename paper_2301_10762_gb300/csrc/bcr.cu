// Block cyclic reduction (BCR) of the block-tridiagonal line system, mixed precision.
//
// With lines of constant x (n_z nodes each) the discrete operator A(m, w) of the Appendix
// ("Numerical forward model") is block tridiagonal: diagonal blocks D_i (tridiagonal) and the
// diagonal horizontal couplings C between neighbouring lines; A is complex symmetric, so the
// coupling of line k to a line a is the transpose of that of a to k.  Where the line factor
// (factor.cu) runs the Schur recurrence line after line, BCR eliminates every other line of
// the current system at once, level by level (spacing s = 2^l):
//     eliminated j (j = s mod 2s):    Dinv_j = D_j^{-1}
//     kept k (k = 0 mod 2s), a = k - s, c = k + s:
//         D_k <- D_k - L_k Dinv_a U_a - U_k Dinv_c L_c
//         L_k <- -L_k Dinv_a L_a      (coupling to k - 2s)
//         U_k <- -U_k Dinv_c U_c      (coupling to k + 2s)
// until one line is left (line 0, whose inverse ends the factor).  Every level is a batch of
// independent dense block products and inversions over all lines and frequencies, which the
// tensor-core GEMM (zgemm_tc.cu) and the batched block inversion below run; the depth of the
// dependent chain is log2(n_x) levels instead of n_x lines.  By symmetry L_k = U_a^T and
// U_k = L_c^T, so every product is a GEMM of row-major operands:
//     W_a = L_k Dinv_a (= (Dinv_a U_a)^T),   V_c = U_k Dinv_c (= (Dinv_c L_c)^T),
//     D_k -= L_k W_a^T + U_k V_c^T,   L_k <- -L_k V_a^T,   U_k <- -U_k W_c^T,
// and the back substitution takes P_j = V_j^T = Dinv_j L_j, Q_j = W_j^T = Dinv_j U_j.
// Level 0 has the diagonal couplings C: its products are elementwise scalings.
//
// The solve of A x = b (all right-hand sides of a system as the GEMM N dimension):
//     forward, level 0:  y_j = Dinv_j b_j;  b_k -= C (y_a + y_c)
//     forward, level l:  b_k -= W_a b_a + V_c b_c
//     last line:         x_0 = Dinv_0 b_0
//     backward, level l: x_j = Dinv_j b_j - P_j x_{j-s} - Q_j x_{j+s}
//     backward, level 0: x_j = y_j - Dinv_j C (x_{j-1} + x_{j+1}).
// Everything is complex FP32 (3xTF32 tensor products): the factor is the preconditioner of
// the FP64-residual refinement of the mixed path, exactly as the line factor is.
//
// Dense inversion of a batch of n x n blocks: n <= 128 in shared memory, one CTA per block
// (block Gauss-Jordan over 16-column blocks, partial pivoting inside each pivot block, as in
// the line factor); larger n by the 2 x 2 block inverse of a symmetric matrix
//     [[D11, D21^T], [D21, D22]]^{-1}:  X11 = D11^{-1}, T = X11 D21^T, S = D22 - D21 T,
//     X22 = S^{-1}, X12 = -T X22, X21 = X12^T, X11 <- X11 - T X21,
// with the products on the tensor cores and the two half-size inverses recursive.
#include <math.h>
#include <stdlib.h>

#include <algorithm>
#include <functional>
#include <vector>

#include "abi_internal.h"
#include "kernels.h"
#include "pivot16.cuh"
#include "tcgen05.cuh"
#include "trace.h"

namespace helm {

namespace {

constexpr int INV_THREADS = 512;
constexpr int INV_MAX = 128;   // largest block inverted in one CTA's shared memory

// ------------------------------------------------------------------- kernels

// couplings of the grid in FP32: horizontal (between lines, row j) and vertical (within line
// i), each halved on a boundary edge; computed once on the host
struct Coup {
    float cx_in, cx_edge, cz_in, cz_edge;
    __device__ __forceinline__ float cx(int j, int nz) const { return (j == 0 || j == nz - 1) ? cx_edge : cx_in; }
    __device__ __forceinline__ float cz(int i, int nx) const { return (i == 0 || i == nx - 1) ? cz_edge : cz_in; }
};
Coup coup_of(const GridGeom &g) {
    return Coup{(float)coup_x(g, 1), (float)coup_x(g, 0), (float)coup_z(g, 1), (float)coup_z(g, 0)};
}

// dense D_i of every line and system (n_z > 256): the diagonal of A and the vertical couplings
// next to it; one float4 (two complex entries of a row) per thread and step
__global__ void bcr_form_kernel(GridGeom g, Coup cp, const double2 *diag, float2 *D) {
    const int nz = g.nz, nx = g.nx;
    const int i = blockIdx.y, s = blockIdx.z;
    const float cz = cp.cz(i, nx);
    float4 *Di = reinterpret_cast<float4 *>(D + ((size_t)s * nx + i) * nz * nz);
    const double2 *dg = diag + ((size_t)s * nx + i) * nz;
    const int nq = nz * nz / 2;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
        const int r = (2 * q) / nz, c = (2 * q) - r * nz;   // columns c, c + 1 of row r
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        const int c1 = c + 1;
        if (c == r) { const float2 d = to_c64(dg[r]); v.x = d.x; v.y = d.y; }
        else if (c == r + 1 || c + 1 == r) v.x = cz;
        if (c1 == r) { const float2 d = to_c64(dg[r]); v.z = d.x; v.w = d.y; }
        else if (c1 == r + 1 || c1 + 1 == r) v.z = cz;
        Di[q] = v;
    }
}

// level 0 (couplings C = diag(cx)): kept line k (even) with eliminated neighbours k - 1, k + 1:
//   D_k -= C Dinv_{k-1} C + C Dinv_{k+1} C,  L_k = -C Dinv_{k-1} C,  U_k = -C Dinv_{k+1} C
// implicit (diag != nullptr): D_k is not in memory yet and is taken from A's diagonal and the
// line's vertical coupling (the tridiagonal line block) before the update
__global__ void bcr_level0_kernel(GridGeom g, Coup cp, float2 *D, const float2 *Dinv, float2 *Lnew, float2 *Unew,
                                  int half, const double2 *diag) {
    const int nz = g.nz, nx = g.nx, nz2 = nz * nz;
    const int k = 2 * blockIdx.y, s = blockIdx.z;
    const bool ha = k >= 1, hc = k + 1 < nx;
    const float2 *Da = Dinv + ((size_t)s * nx + (ha ? k - 1 : 0)) * nz2;
    const float2 *Dc = Dinv + ((size_t)s * nx + (hc ? k + 1 : 0)) * nz2;
    float2 *Dk = D + ((size_t)s * nx + k) * nz2;
    float2 *Lk = Lnew + ((size_t)s * half + k / 2) * nz2;
    float2 *Uk = Unew + ((size_t)s * half + k / 2) * nz2;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nz2; e += gridDim.x * blockDim.x) {
        const int r = e / nz, c = e - r * nz;
        const float sc = cp.cx(r, nz) * cp.cx(c, nz);
        float2 ta = make_float2(0.f, 0.f), tc = ta;
        if (ha) { const float2 v = Da[e]; ta = make_float2(sc * v.x, sc * v.y); }
        if (hc) { const float2 v = Dc[e]; tc = make_float2(sc * v.x, sc * v.y); }
        float2 d;
        if (diag) {
            const float cz = cp.cz(k, nx);
            d = r == c ? to_c64(diag[((size_t)s * nx + k) * nz + r])
                       : ((r - c == 1 || c - r == 1) ? make_float2(cz, 0.f) : make_float2(0.f, 0.f));
        } else {
            d = Dk[e];
        }
        d.x -= ta.x + tc.x;
        d.y -= ta.y + tc.y;
        Dk[e] = d;
        if (k >= 2) Lk[e] = make_float2(-ta.x, -ta.y);
        if (k + 2 < nx) Uk[e] = make_float2(-tc.x, -tc.y);
    }
}

// Implicit tridiagonal input of the block inversion (the level-0 line blocks, never formed in
// memory): rows and columns row0 .. row0 + n - 1 of the block of line idx (input index = system
// * nx + line) with A's diagonal diag[idx][.] and the line's vertical coupling; with corr, entry
// (0, 0) less cz^2 X[corr_off] (X the output block: the Schur complement of the lower half).
struct TriIn {
    const double2 *diag = nullptr;   // [idx][nz]; nullptr: the input is a dense block
    int nz = 0, nx = 0, row0 = 0;
    float cz_in = 0.f, cz_edge = 0.f;
    int corr = 0;
    long long corr_off = 0;
    __device__ __forceinline__ float cz(int idx) const {
        const int line = idx % nx;
        return (line == 0 || line == nx - 1) ? cz_edge : cz_in;
    }
    // entry (r, c) of the block of input idx; x: the output block (for the corrected corner)
    __device__ __forceinline__ float2 entry(int idx, int r, int c, const float2 *x) const {
        if (r == c) {
            float2 v = to_c64(diag[(long long)idx * nz + row0 + r]);
            if (corr && r == 0) {
                const float c2 = cz(idx) * cz(idx);
                const float2 w = x[corr_off];
                v.x -= c2 * w.x;
                v.y -= c2 * w.y;
            }
            return v;
        }
        return (r - c == 1 || c - r == 1) ? make_float2(cz(idx), 0.f) : make_float2(0.f, 0.f);
    }
};

struct InvArgs {
    int n;
    ZOperand in;                 // row-major, ld = in.ld
    float2 *out;                 // row-major, ld = ldo
    long long out_stride, out_stride_hi;
    int out_div, ldo;
    const int *idx;              // [count][2]: input index, output index
    int *status;
    TriIn tri;                   // tri.diag set: implicit tridiagonal input instead of `in`
    uint32_t tries = 0;          // polls of a bounded mbarrier wait before it gives up
};

__device__ __forceinline__ long long op_off(int idx, int div, long long stride, long long stride_hi) {
    return div > 0 ? (long long)(idx / div) * stride_hi + (long long)(idx % div) * stride : (long long)idx * stride;
}

// X = M^{-1} of one n x n block (n <= 128) per CTA, in shared memory: block Gauss-Jordan over
// 16-column blocks; the pivot block is inverted by one warp with partial pivoting, the other
// rows get the rank-16 update from the staged old column panel U and R = P M[k rows, :].
__global__ void __launch_bounds__(INV_THREADS, 1) zinv_base_kernel(InvArgs a) {
    extern __shared__ __align__(16) unsigned char inv_smem[];
    const int n = a.n, ldw = n + 1, tid = threadIdx.x;
    float2 *W = reinterpret_cast<float2 *>(inv_smem);          // n x ldw
    float2 *U = W + (size_t)n * ldw;                             // n x 16: old column panel
    float2 *R = U + (size_t)n * PIV;                             // 16 x ldw: P times the pivot rows
    float2 *P = R + (size_t)PIV * ldw;                           // 16 x 16: pivot-block inverse
    __shared__ int s_bad;
    const int *ix = a.idx + 2 * (size_t)blockIdx.x;
    const float2 *M = a.in.base + op_off(ix[0], a.in.div, a.in.stride, a.in.stride_hi);
    float2 *X = a.out + op_off(ix[1], a.out_div, a.out_stride, a.out_stride_hi);
    if (tid == 0) s_bad = 0;
    for (int e = tid; e < n * n; e += INV_THREADS) {
        const int r = e / n, c = e % n;
        W[(size_t)r * ldw + c] = a.tri.diag ? a.tri.entry(ix[0], r, c, X) : M[(size_t)r * a.in.ld + c];
    }
    __syncthreads();
    // update mapping: thread -> column c, row group rg (rows rg, rg + ng, ...)
    const int ng = INV_THREADS / n, c = tid % n, rg = tid / n;
    const int nb = (n + PIV - 1) / PIV;
    for (int kb_i = 0; kb_i < nb; ++kb_i) {
        const int k0 = kb_i * PIV, kb = min(PIV, n - k0);
        for (int e = tid; e < n * PIV; e += INV_THREADS) {
            const int r = e / PIV, u = e % PIV;
            U[e] = u < kb ? W[(size_t)r * ldw + k0 + u] : make_float2(0.f, 0.f);
        }
        if (tid < 32) {
            if (!warp_invert16<float>(W + (size_t)k0 * ldw + k0, ldw, kb, P) && tid == 0) s_bad = 1;
        }
        __syncthreads();
        for (int e = tid; e < PIV * n; e += INV_THREADS) {
            const int q = e / n, cc = e % n;
            if (q < kb && (cc < k0 || cc >= k0 + kb)) {
                float2 acc = make_float2(0.f, 0.f);
                for (int u = 0; u < kb; ++u) cfma(acc, P[q * PIV + u], W[(size_t)(k0 + u) * ldw + cc]);
                R[(size_t)q * ldw + cc] = acc;
            }
        }
        __syncthreads();
        if (rg < ng) {
            const bool inblk = c >= k0 && c < k0 + kb;
            float2 col[PIV];   // the R (or P) column this thread multiplies with
#pragma unroll
            for (int u = 0; u < PIV; ++u)
                col[u] = u < kb ? (inblk ? P[u * PIV + (c - k0)] : R[(size_t)u * ldw + c]) : make_float2(0.f, 0.f);
            for (int r = rg; r < n; r += ng) {
                float2 *w = W + (size_t)r * ldw + c;
                if (r >= k0 && r < k0 + kb) {
                    *w = inblk ? P[(r - k0) * PIV + (c - k0)] : R[(size_t)(r - k0) * ldw + c];
                    continue;
                }
                const float4 *ur = reinterpret_cast<const float4 *>(U + (size_t)r * PIV);
                float2 p[4] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
                for (int h = 0; h < PIV / 2; ++h) {
                    const float4 q = ur[h];
                    cfma(p[(2 * h) & 3], make_float2(q.x, q.y), col[2 * h]);
                    cfma(p[(2 * h + 1) & 3], make_float2(q.z, q.w), col[2 * h + 1]);
                }
                const float2 sum = make_float2((p[0].x + p[1].x) + (p[2].x + p[3].x), (p[0].y + p[1].y) + (p[2].y + p[3].y));
                const float2 old = inblk ? make_float2(0.f, 0.f) : *w;
                *w = make_float2(old.x - sum.x, old.y - sum.y);
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < n * n; e += INV_THREADS) {
        const int r = e / n, cc = e % n;
        X[(size_t)r * a.ldo + cc] = W[(size_t)r * ldw + cc];
    }
    if (tid == 0 && s_bad) atomicOr(a.status, ST_SINGULAR);
}

// X = M^{-1} of one 128 x 128 block per CTA with the block in tensor memory: lane r holds row r,
// 256 FP32 columns (column 2c the real, 2c + 1 the imaginary part of entry c).  Each
// Gauss-Jordan step (16 pivot columns K = k0 .. k0 + 15) is
//     W <- W' + A' R'  (W' = W with the rows and columns K zeroed in tensor memory;
//                       A'[r][u] = -W[r][k0 + u] off the pivot rows, delta(r - k0, u) on them;
//                       R' = P W[K, :] off the pivot columns, P on them, P = W[K, K]^{-1}),
// one tcgen05 3xTF32 product of M = 128, N = 256 (R' expanded to real rows as in the GEMM),
// K = 32, accumulated into W itself.  Shared memory holds only the product's operands, the
// pivot rows and the 16 x 16 blocks (~103 KB), so that two CTAs share an SM and one's pivot
// chain (one warp) overlaps the other's work.  Warp w owns tensor-memory lanes 32 (w mod 4) ..
// + 31 and columns 128 (w / 4) .. + 127.
constexpr int ZT_THREADS = 256;
constexpr int ZT_WS = 129;   // pivot rows W[K, :] in shared memory: row stride (complex)
constexpr int ZT_PS = 17;    // padded copy of P
constexpr uint32_t ZT_A = 0, ZT_B = 32768, ZT_PK = 98304, ZT_P = ZT_PK + 2048, ZT_PPAD = ZT_P + 2048;
size_t zinv128_tm_smem_bytes() { return (size_t)ZT_PPAD + sizeof(float2) * PIV * ZT_PS + 1024; }

__global__ void __launch_bounds__(ZT_THREADS, 2) zinv128_tm_kernel(InvArgs a) {
    extern __shared__ __align__(16) unsigned char zt_smem[];
    __shared__ __align__(8) uint64_t mma_bar;
    __shared__ uint32_t s_tmem;
    __shared__ int s_bad;
    constexpr int n = 128;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, hh = warp >> 2, r = 32 * q + lane;
    const uint32_t base = (smem_u32(zt_smem) + 1023u) & ~1023u;
    unsigned char *gbase = zt_smem + (base - smem_u32(zt_smem));
    float2 *Wk = reinterpret_cast<float2 *>(gbase + ZT_A);      // [16][ZT_WS], aliases the A tiles
    float2 *Pk = reinterpret_cast<float2 *>(gbase + ZT_PK);     // [16][16]: the pivot block
    float2 *P = reinterpret_cast<float2 *>(gbase + ZT_P);       // [16][16]: its inverse
    float2 *Ps = reinterpret_cast<float2 *>(gbase + ZT_PPAD);   // [16][ZT_PS]: padded copy
    const uint32_t a_hi = base + ZT_A, a_lo = a_hi + 16384, b_hi = base + ZT_B, b_lo = b_hi + 32768;
    const int *ix = a.idx + 2 * (size_t)blockIdx.x;
    const float2 *M = a.in.base + op_off(ix[0], a.in.div, a.in.stride, a.in.stride_hi);
    float2 *X = a.out + op_off(ix[1], a.out_div, a.out_stride, a.out_stride_hi);
    if (tid == 0) {
        s_bad = 0;
        mbar_init(&mma_bar, 1);
        fence_mbar_init_cluster();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(256u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t trow = s_tmem + ((uint32_t)(32 * q) << 16);   // this warp's lanes, column 0
    // the block into tensor memory: lane r, columns 128 hh .. + 127
#pragma unroll 1
    for (int ch = 0; ch < 8; ++ch) {
        const int col = 128 * hh + 16 * ch, c0 = col / 2;
        float v[16];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float2 e = a.tri.diag ? a.tri.entry(ix[0], r, c0 + i, X) : M[(size_t)r * a.in.ld + c0 + i];
            v[2 * i] = e.x;
            v[2 * i + 1] = e.y;
        }
        tc_st16(trow + (uint32_t)col, v);
    }
    tc_wait_st();
    constexpr uint32_t idesc = idesc_tf32(256);
    int phase = 0;
    bool aborted = false;
#pragma unroll 1
    for (int kb = 0; kb < n / PIV; ++kb) {
        const int k0 = kb * PIV, qk = k0 >> 5, rk0 = k0 & 31;
        const bool krow = q == qk && lane >= rk0 && lane < rk0 + PIV;   // this lane's row is a pivot row
        tc_fence_before();
        __syncthreads();   // the previous step's tensor-memory reads and shared-memory reads are done
        tc_fence_after();
        // (a) the column panel W[r][k0 + u], u = 8 hh .. 8 hh + 7 (kept for A'); the pivot block
        float uf[16];
        tc_ld16(trow + (uint32_t)(2 * k0 + 16 * hh), uf);
        if (krow) {
#pragma unroll
            for (int i = 0; i < 8; ++i) Pk[(lane - rk0) * PIV + 8 * hh + i] = make_float2(uf[2 * i], uf[2 * i + 1]);
        }
        // (b) the pivot rows' quarter: rows K to shared memory, then W' (rows K and columns K
        // zeroed) back; (c) the other quarters: columns K zeroed
        if (q == qk) {
#pragma unroll 1
            for (int ch = 0; ch < 8; ++ch) {
                const int col = 128 * hh + 16 * ch;
                float v[16];
                tc_ld16(trow + (uint32_t)col, v);
                if (krow) {
#pragma unroll
                    for (int i = 0; i < 8; ++i) Wk[(lane - rk0) * ZT_WS + col / 2 + i] = make_float2(v[2 * i], v[2 * i + 1]);
                }
                const bool kcol = col >= 2 * k0 && col < 2 * k0 + 2 * PIV;
                if (krow || kcol) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = 0.f;
                }
                tc_st16(trow + (uint32_t)col, v);
            }
        } else {
            float z[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) z[i] = 0.f;
            tc_st16(trow + (uint32_t)(2 * k0 + 16 * hh), z);
        }
        tc_wait_st();
        __syncthreads();
        // (d) the pivot block's inverse (one warp), and its padded copy
        if (warp == 0) {
            if (!warp_invert16<float>(Pk, PIV, PIV, P) && lane == 0) s_bad = 1;
            __syncwarp();
            for (int e = lane; e < PIV * PIV; e += 32) Ps[(e >> 4) * ZT_PS + (e & 15)] = P[e];
        }
        __syncthreads();
        // (e) R' and the expanded B tiles: item (c, j), u = 2j, 2j + 1; B row 2c = (Re, -Im),
        // row 2c + 1 = (Im, Re) of R'[u][c], split into hi and lo
#pragma unroll 1
        for (int it = tid; it < n * 8; it += ZT_THREADS) {
            const int c = it >> 3, j = it & 7, u0 = 2 * j, u1 = u0 + 1;
            float2 r0, r1;
            if (c >= k0 && c < k0 + PIV) {
                r0 = Ps[u0 * ZT_PS + (c - k0)];
                r1 = Ps[u1 * ZT_PS + (c - k0)];
            } else {
                r0 = make_float2(0.f, 0.f);
                r1 = r0;
#pragma unroll
                for (int v = 0; v < PIV; ++v) {
                    const float2 w = Wk[v * ZT_WS + c];
                    cfma(r0, Ps[u0 * ZT_PS + v], w);
                    cfma(r1, Ps[u1 * ZT_PS + v], w);
                }
            }
            float4 hi, lo;
            split4(make_float4(r0.x, -r0.y, r1.x, -r1.y), 1.f, hi, lo);
            st_shared_v4(b_hi + sw128(2 * c, j), hi);
            st_shared_v4(b_lo + sw128(2 * c, j), lo);
            split4(make_float4(r0.y, r0.x, r1.y, r1.x), 1.f, hi, lo);
            st_shared_v4(b_hi + sw128(2 * c + 1, j), hi);
            st_shared_v4(b_lo + sw128(2 * c + 1, j), lo);
        }
        __syncthreads();   // the pivot rows read: their storage becomes the A tiles
        // (f) A' row r, chunks j = 4 hh .. 4 hh + 3 (u = 2j, 2j + 1 of this thread's panel part)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const int j = 4 * hh + jj, u0 = 2 * j;
            float4 v;
            if (krow) {
                v = make_float4(r - k0 == u0 ? 1.f : 0.f, 0.f, r - k0 == u0 + 1 ? 1.f : 0.f, 0.f);
            } else {
                v = make_float4(-uf[4 * jj], -uf[4 * jj + 1], -uf[4 * jj + 2], -uf[4 * jj + 3]);
            }
            float4 hi, lo;
            split4(v, 1.f, hi, lo);
            st_shared_v4(a_hi + sw128(r, j), hi);
            st_shared_v4(a_lo + sw128(r, j), lo);
        }
        fence_proxy_async_smem();   // the operand tiles, before the tensor core reads them
        tc_fence_before();
        __syncthreads();
        // (g) W' + A' R' into tensor memory
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int p = 0; p < 3; ++p) {   // hi*hi, hi*lo, lo*hi
                const uint32_t aa = p == 2 ? a_lo : a_hi, bb = p == 1 ? b_lo : b_hi;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    tc_mma(s_tmem, desc_sw128(aa + 32 * kk), desc_sw128(bb + 32 * kk), idesc, 1u);
            }
            tc_commit(&mma_bar);
        }
        const bool done = mbar_wait_bounded(&mma_bar, (uint32_t)phase, a.tries);
        if (__syncthreads_or(!done)) {   // uniform: every thread leaves the loop
            if (tid == 0) atomicOr(a.status, ST_TIMEOUT);
            aborted = true;
            break;
        }
        phase ^= 1;
        tc_fence_after();
    }
    // the inverse out of tensor memory: lane r, columns 128 hh .. + 127
    if (!aborted) {
#pragma unroll 1
        for (int ch = 0; ch < 8; ++ch) {
            const int col = 128 * hh + 16 * ch;
            float v[16];
            tc_ld16(trow + (uint32_t)col, v);
            float4 *xr = reinterpret_cast<float4 *>(X + (size_t)r * a.ldo + col / 2);
#pragma unroll
            for (int i = 0; i < 4; ++i) xr[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        }
    } else {
        mbar_wait_bounded(&mma_bar, (uint32_t)phase, a.tries);   // an MMA that may still be in flight
    }
    if (tid == 0 && s_bad) atomicOr(a.status, ST_SINGULAR);
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem), "r"(256u) : "memory");
}

size_t inv_smem_bytes(int n) {
    return sizeof(float2) * ((size_t)n * (n + 1) + (size_t)n * PIV + (size_t)PIV * (n + 1) + PIV * PIV);
}

// Inverse of complex symmetric tridiagonal blocks D (the level-0 line blocks) of size
// n = n1 + n2 by the 2 x 2 block inverse, whose off-diagonal block D21 = c e_0 e_{n1-1}^T has a
// single entry, the line's vertical coupling c: with x = X11[:, n1 - 1] (X11 = D11^{-1}),
//     S = D22 - c^2 X11[n1-1][n1-1] e_0 e_0^T,  X22 = S^{-1},
//     X12 = -c x X22[0, :],  X21 = X12^T,  X11 <- X11 + c^2 X22[0][0] x x^T,
// so that the four products of the general case are rank-one updates (the inversions read D11
// and S implicitly, TriIn).  Output blocks at out + idx * stride, rows ld apart; pairs
// [count][2] (input index = system * nx + line, output index).
__global__ void __launch_bounds__(512) tri_rank1_kernel(int n, int n1, TriIn tri, float2 *out, long long stride, int ld,
                                                        const int *pairs) {
    __shared__ float2 xs[INV_MAX], rs[INV_MAX];
    float2 *X = out + (long long)pairs[2 * blockIdx.x + 1] * stride;
    const int n2 = n - n1;
    const float2 c = make_float2(tri.cz(pairs[2 * blockIdx.x]), 0.f);
    for (int i = threadIdx.x; i < n1; i += blockDim.x) xs[i] = X[(long long)i * ld + n1 - 1];
    for (int j = threadIdx.x; j < n2; j += blockDim.x) rs[j] = X[(long long)n1 * ld + n1 + j];
    __syncthreads();
    const float2 c2d = cmul(cmul(c, c), rs[0]);           // c^2 X22[0][0]
    const float2 mc = make_float2(-c.x, -c.y);
    for (int e = threadIdx.x; e < n1 * n; e += blockDim.x) {   // rows 0 .. n1 - 1: X11 and X12
        const int i = e / n, j = e % n;
        float2 *w = X + (long long)i * ld + j;
        if (j < n1) {
            float2 v = *w;
            cfma(v, cmul(c2d, xs[i]), xs[j]);
            *w = v;
        } else {
            *w = cmul(cmul(mc, xs[i]), rs[j - n1]);
        }
    }
    for (int e = threadIdx.x; e < n2 * n1; e += blockDim.x) {   // rows n1 .. n - 1, columns 0 .. n1 - 1: X21
        const int i = e / n1, j = e % n1;
        X[(long long)(n1 + i) * ld + j] = cmul(cmul(mc, rs[i]), xs[j]);
    }
}

// out[idx_out] = in[idx_in]^T for n x n complex blocks (32 x 32 tiles through shared memory)
__global__ void ztranspose_kernel(int n, const float2 *in, float2 *out, long long stride_in, long long stride_out,
                                  const int *idx) {
    __shared__ float2 t[32][33];
    const int *ix = idx + 2 * (size_t)blockIdx.z;
    const float2 *A = in + (long long)ix[0] * stride_in;
    float2 *B = out + (long long)ix[1] * stride_out;
    const int nt = (n + 31) / 32;
    const int bi = blockIdx.x / nt, bj = blockIdx.x % nt;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = bi * 32 + y, c = bj * 32 + threadIdx.x;
        if (r < n && c < n) t[y][threadIdx.x] = A[(size_t)r * n + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = bj * 32 + y, c = bi * 32 + threadIdx.x;
        if (r < n && c < n) B[(size_t)r * n + c] = t[threadIdx.x][y];
    }
}

// solve, level 0 of the forward pass: b_k -= C (y_{k-1} + y_{k+1}) for even k, y in x.  Thread:
// two rows (one float4) of the line, for L0_COLS columns (frequency x right-hand side).
constexpr int L0_COLS = 8;
__global__ void bcr_solve_l0_fwd_kernel(GridGeom g, Coup cp, int cols, float2 *b, const float2 *x, const int *skip,
                                        const int *frozen, int nrhs) {
    if (skip && *skip) return;
    const int nz = g.nz, nx = g.nx, N = nx * nz;
    const int k = 2 * blockIdx.y, r = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (r >= nz) return;
    const float c0 = cp.cx(r, nz), c1 = cp.cx(r + 1, nz);
    for (int col = blockIdx.z * L0_COLS; col < min(cols, (int)(blockIdx.z + 1) * L0_COLS); ++col) {
        if (frozen && frozen[2 * (col / nrhs)]) continue;   // a converged system's correction is not needed
        const size_t off = (size_t)col * N + (size_t)k * nz + r;
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k >= 1) { const float4 v = *reinterpret_cast<const float4 *>(x + off - nz); t.x += v.x; t.y += v.y; t.z += v.z; t.w += v.w; }
        if (k + 1 < nx) { const float4 v = *reinterpret_cast<const float4 *>(x + off + nz); t.x += v.x; t.y += v.y; t.z += v.z; t.w += v.w; }
        float4 *bp = reinterpret_cast<float4 *>(b + off);
        float4 v = *bp;
        v.x -= c0 * t.x; v.y -= c0 * t.y; v.z -= c1 * t.z; v.w -= c1 * t.w;
        *bp = v;
    }
}

// solve, level 0 of the backward pass: b_j = C (x_{j-1} + x_{j+1}) for odd j
__global__ void bcr_solve_l0_bwd_kernel(GridGeom g, Coup cp, int cols, float2 *b, const float2 *x, const int *skip,
                                        const int *frozen, int nrhs) {
    if (skip && *skip) return;
    const int nz = g.nz, nx = g.nx, N = nx * nz;
    const int j = 2 * blockIdx.y + 1, r = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (r >= nz) return;
    const float c0 = cp.cx(r, nz), c1 = cp.cx(r + 1, nz);
    for (int col = blockIdx.z * L0_COLS; col < min(cols, (int)(blockIdx.z + 1) * L0_COLS); ++col) {
        if (frozen && frozen[2 * (col / nrhs)]) continue;
        const size_t off = (size_t)col * N + (size_t)j * nz + r;
        float4 t = *reinterpret_cast<const float4 *>(x + off - nz);
        if (j + 1 < nx) { const float4 v = *reinterpret_cast<const float4 *>(x + off + nz); t.x += v.x; t.y += v.y; t.z += v.z; t.w += v.w; }
        *reinterpret_cast<float4 *>(b + off) = make_float4(c0 * t.x, c0 * t.y, c1 * t.z, c1 * t.w);
    }
}

// ----------------------------------------------------------------- host side

struct TaskBuf {   // device copy of host-built task lists (freed on the stream when done)
    int *dev = nullptr;
    cudaStream_t st = nullptr;
    ~TaskBuf() { dev_free(dev, st); }
};

helm_status upload_ints(const std::vector<int> &h, TaskBuf &b, cudaStream_t st) {
    b.st = st;
    helm_status s = dev_alloc((void **)&b.dev, h.size() * sizeof(int), "bcr: task list", st);
    if (s != HELM_OK) return s;
    cudaError_t e = cudaMemcpyAsync(b.dev, h.data(), h.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) { helm_set_error("bcr: task upload", e); return HELM_ECUDA; }
    return HELM_OK;
}

// A recorded sequence of launches: every task list goes into one host array, uploaded with a
// single copy before the launches are enqueued (a copy from pageable host memory waits for the
// stream, so one copy per launch would serialise the host with the GPU at every launch).
// partial tiles of split-K GEMM launches: 64 MB for a factorisation (its deep levels: 8 tasks of
// 256 x 256 split 16 ways), 32 MB kept with a factor for its solves (64 tasks of 256 x 64 split 8 ways)
constexpr size_t kFactorSplitElems = (size_t)8 << 20, kSolveSplitElems = (size_t)4 << 20;

struct Plan {
    cudaStream_t st;
    std::vector<int> ints;
    std::vector<std::function<helm_status(const int *)>> ops;
    std::vector<void *> scratch;   // device scratch of the launches, released after the last one
    float2 *split = nullptr;       // split-K partial tiles shared by the plan's GEMM launches (one
    size_t split_cap = 0;          // stream: each launch's reduction reads them before the next writes)
    explicit Plan(cudaStream_t s) : st(s) {}
    helm_status with_split(size_t elems) {
        helm_status s = dev_alloc((void **)&split, elems * sizeof(float2), "bcr: split-K tiles", st);
        if (s != HELM_OK) return s;
        scratch.push_back(split);
        split_cap = elems;
        return HELM_OK;
    }
    ~Plan() {
        for (void *p : scratch) dev_free(p, st);
    }
    int add(const std::vector<int> &v) {
        const int off = (int)ints.size();
        ints.insert(ints.end(), v.begin(), v.end());
        return off;
    }
    helm_status run() {
        TaskBuf tb;
        helm_status s = HELM_OK;
        if (!ints.empty() && (s = upload_ints(ints, tb, st)) != HELM_OK) return s;
        for (auto &op : ops)
            if ((s = op(tb.dev)) != HELM_OK) return s;
        return HELM_OK;
    }
};

ZOperand zop(const float2 *base, long long stride, int ld, int div = 0, long long stride_hi = 0) {
    ZOperand o;
    o.base = base;
    o.stride = stride;
    o.ld = ld;
    o.div = div;
    o.stride_hi = stride_hi;
    return o;
}

std::vector<int> task8(int a0, int b0, int c0, int c, int a1 = -1, int b1 = -1, int a2 = -1, int b2 = -1) {
    return {a0, a1, a2, b0, b1, b2, c0, c};
}

// product terms of a task list (a term is present when its A index is not negative)
long long count_terms(const int *tasks, size_t n_tasks, int nterms) {
    long long t = 0;
    for (size_t i = 0; i < n_tasks; ++i)
        for (int u = 0; u < nterms; ++u) t += tasks[8 * i + u] >= 0;
    return t;
}

// family counts of a launch's operands from its (host) task list, where not given
void count_families(ZGemmArgs &a, const std::vector<int> &tasks) {
    for (int u = 0; u < a.nterms; ++u) {
        int ma = -1, mb = -1;
        for (size_t t = 0; t < tasks.size(); t += 8)
            if (tasks[t + u] >= 0) {
                ma = std::max(ma, tasks[t + u]);
                mb = std::max(mb, tasks[t + 3 + u]);
            }
        auto set = [](ZOperand &o, int mx) {
            if (o.count == 0 && mx >= 0) o.count = o.div > 0 ? mx / o.div + 1 : mx + 1;
        };
        set(a.A[u], ma);
        set(a.B[u], mb);
    }
}

helm_status gemm(const ZGemmArgs &a0, const std::vector<int> &tasks, Plan &pl) {
    if (tasks.empty()) return HELM_OK;
    const int off = pl.add(tasks), n = (int)(tasks.size() / 8);
    ZGemmArgs a = a0;
    count_families(a, tasks);
    a.tries = wait_tries();
    a.flops = 8.0 * a.M * a.N * a.K * (double)count_terms(tasks.data(), (size_t)n, a.nterms);
    a.part = pl.split;
    a.part_cap = pl.split_cap;
    const cudaStream_t st = pl.st;
    pl.ops.push_back([a, off, n, st](const int *dev) mutable -> helm_status {
        a.tasks = dev + off;
        const cudaError_t e = launch_zgemm(a, n, st);
        if (e != cudaSuccess) { helm_set_error("bcr: tensor-core GEMM", e); return HELM_ECUDA; }
        return HELM_OK;
    });
    return HELM_OK;
}

// A family of n x n row-major blocks within a family of larger row-major matrices: the block
// at (row r0, column c0) of matrix idx (the larger matrices have row stride ld).
struct Fam {
    float2 *base;
    long long stride;
    int ld;
    Fam sub(int r0, int c0) const { return Fam{base + (long long)r0 * ld + c0, stride, ld}; }
    ZOperand op() const { return zop(base, stride, ld); }
};

// out[p.second] = in[p.first]^{-1} for every index pair, n x n blocks (may be the same matrices)
helm_status invert_blocks(int n, Fam in, Fam out, const std::vector<int> &pairs, int *status, Plan &pl,
                          const TriIn *tri = nullptr) {
    const int count = (int)(pairs.size() / 2);
    if (count == 0) return HELM_OK;
    const cudaStream_t st = pl.st;
    helm_status s;
    if (n <= INV_MAX) {
        const int off = pl.add(pairs);
        // 128 x 128 blocks on 16-byte boundaries (two complex entries per access): the kernel
        // with the block in tensor memory
        const bool t128 = n == 128 && ((uintptr_t)in.base & 15) == 0 && ((uintptr_t)out.base & 15) == 0 &&
                          (in.ld & 1) == 0 && (out.ld & 1) == 0 && (in.stride & 1) == 0 && (out.stride & 1) == 0;
        const size_t smem = t128 ? zinv128_tm_smem_bytes() : inv_smem_bytes(n);
        const void *fn = t128 ? (const void *)zinv128_tm_kernel : (const void *)zinv_base_kernel;
        cudaError_t e = ensure_dyn_smem(fn, smem);
        if (e != cudaSuccess) { helm_set_error("bcr: block inversion", e); return HELM_ECUDA; }
        InvArgs a{n, in.op(), out.base, out.stride, 0, 0, out.ld, nullptr, status, tri ? *tri : TriIn{}};
        a.tries = wait_tries();
        pl.ops.push_back([a, off, count, smem, st, t128](const int *dev) mutable -> helm_status {
            a.idx = dev + off;
            if (t128) HELM_TRACED(K_ZINV, st, (zinv128_tm_kernel<<<count, ZT_THREADS, smem, st>>>(a)));
            else HELM_TRACED(K_ZINV, st, (zinv_base_kernel<<<count, INV_THREADS, smem, st>>>(a)));
            const cudaError_t e2 = cudaGetLastError();
            if (e2 != cudaSuccess) { helm_set_error("bcr: block inversion", e2); return HELM_ECUDA; }
            return HELM_OK;
        });
        return HELM_OK;
    }
    if (tri) return HELM_EINVAL;   // implicit input: base blocks only (invert_tridiag_blocks splits)
    const int n1 = INV_MAX * ((n / INV_MAX + 1) / 2), n2 = n - n1;
    // X11 = D11^{-1}
    if ((s = invert_blocks(n1, in, out, pairs, status, pl)) != HELM_OK) return s;
    // scratch T (n1 x n2) and Tt = T^T (n2 x n1) per block: allocated now (stream-ordered, usable
    // by the launches enqueued later), released on the stream after the last launch that reads it
    float2 *T = nullptr, *Tt = nullptr;
    const long long ts = (long long)n1 * n2;
    if ((s = dev_alloc((void **)&T, (size_t)count * ts * sizeof(float2), "bcr: inversion scratch", st)) != HELM_OK)
        return s;
    if ((s = dev_alloc((void **)&Tt, (size_t)count * ts * sizeof(float2), "bcr: inversion scratch", st)) != HELM_OK) {
        dev_free(T, st);
        return s;
    }
    // (released by the plan after its last launch)
    pl.scratch.push_back(T);
    pl.scratch.push_back(Tt);
    const Fam X11 = out.sub(0, 0), X12 = out.sub(0, n1), X21 = out.sub(n1, 0), X22 = out.sub(n1, n1);
    const Fam D21 = in.sub(n1, 0), D22 = in.sub(n1, n1);
    const Fam FT{T, ts, n2}, FTt{Tt, ts, n1};
    std::vector<int> tk;
    auto run = [&](int M, int N, int K, Fam A, Fam B, const Fam *C0, Fam C, float sign, int which_a, int which_b,
                   int which_c0, int which_c) -> helm_status {
        // which_*: 0 the input index, 1 the output index, 2 the block's position in the batch
        tk.clear();
        for (int t = 0; t < count; ++t) {
            const int id[3] = {pairs[2 * t], pairs[2 * t + 1], t};
            auto v = task8(id[which_a], id[which_b], C0 ? id[which_c0] : 0, id[which_c]);
            tk.insert(tk.end(), v.begin(), v.end());
        }
        ZGemmArgs g;
        g.M = M; g.N = N; g.K = K;
        g.nterms = 1;
        g.A[0] = A.op();
        g.B[0] = B.op();
        g.sign[0] = sign;
        if (C0) g.C0 = C0->op();
        g.C = C.base;
        g.c_stride = C.stride;
        g.ldc = C.ld;
        g.status = status;
        return gemm(g, tk, pl);
    };
    // T = X11 D12 = X11 D21^T;  Tt = D21 X11 (= T^T, X11 symmetric)
    if ((s = run(n1, n2, n1, X11, D21, nullptr, FT, 1.f, 1, 0, 0, 2)) != HELM_OK) return s;
    if ((s = run(n2, n1, n1, D21, X11, nullptr, FTt, 1.f, 0, 1, 0, 2)) != HELM_OK) return s;
    // S = D22 - D21 T  -> X22, then X22 = S^{-1} in place
    if ((s = run(n2, n2, n1, D21, FTt, &D22, X22, -1.f, 0, 2, 0, 1)) != HELM_OK) return s;
    std::vector<int> self(pairs.size());
    for (int t = 0; t < count; ++t) self[2 * t] = self[2 * t + 1] = pairs[2 * t + 1];
    if ((s = invert_blocks(n2, X22, X22, self, status, pl)) != HELM_OK) return s;
    // X12 = -T X22;  X21 = -X22 T^T;  X11 <- X11 - T X21
    if ((s = run(n1, n2, n2, FT, X22, nullptr, X12, -1.f, 2, 1, 0, 1)) != HELM_OK) return s;
    if ((s = run(n2, n1, n2, X22, FT, nullptr, X21, -1.f, 1, 2, 0, 1)) != HELM_OK) return s;
    if ((s = run(n1, n1, n2, FT, X12, &X11, X11, -1.f, 2, 1, 1, 1)) != HELM_OK) return s;
    return HELM_OK;
}

// out[p.second] = D^{-1} for the complex symmetric tridiagonal line blocks D given by `tri`
// (input index = system * nx + line), n <= 256: one implicit base inversion for n <= 128; else
// two and two rank-one kernels (tri_rank1_kernel)
helm_status invert_tridiag_blocks(int n, Fam in, Fam out, const std::vector<int> &pairs, int *status, Plan &pl,
                                  const TriIn &tri) {
    const int count = (int)(pairs.size() / 2);
    if (count == 0) return HELM_OK;
    if (n > 2 * INV_MAX) return HELM_EINVAL;
    TriIn t0 = tri;
    t0.row0 = 0;
    t0.corr = 0;
    if (n <= INV_MAX) return invert_blocks(n, in, out, pairs, status, pl, &t0);
    const int n1 = INV_MAX, n2 = n - n1;
    const cudaStream_t st = pl.st;
    helm_status s;
    if ((s = invert_blocks(n1, in, out, pairs, status, pl, &t0)) != HELM_OK) return s;   // X11 = D11^{-1}
    // X22 = S^{-1}, S read from the diagonal with the corner corrected by X11[n1-1][n1-1]
    TriIn t1 = tri;
    t1.row0 = n1;
    t1.corr = 1;
    t1.corr_off = -(long long)out.ld - 1;   // from X22's first entry to X11's last
    if ((s = invert_blocks(n2, in, out.sub(n1, n1), pairs, status, pl, &t1)) != HELM_OK) return s;
    const int off = pl.add(pairs);
    float2 *ob = out.base;
    const long long stride = out.stride;
    const int ld = out.ld;
    pl.ops.push_back([=](const int *dev) -> helm_status {   // X12, X21, X11 from rank-one updates
        HELM_TRACED(K_ZINV, st, (tri_rank1_kernel<<<count, 512, 0, st>>>(n, n1, t0, ob, stride, ld, dev + off)));
        const cudaError_t e2 = cudaGetLastError();
        if (e2 != cudaSuccess) { helm_set_error("bcr: block inversion", e2); return HELM_ECUDA; }
        return HELM_OK;
    });
    return HELM_OK;
}

helm_status transpose_blocks(int n, const float2 *in, float2 *out, long long stride, const std::vector<int> &pairs,
                             Plan &pl) {
    const int count = (int)(pairs.size() / 2);
    if (count == 0) return HELM_OK;
    const int off = pl.add(pairs);
    const cudaStream_t st = pl.st;
    pl.ops.push_back([=](const int *dev) -> helm_status {
        const int nt = (n + 31) / 32;
        HELM_TRACED(K_ZTRANS, st, (ztranspose_kernel<<<dim3(nt * nt, 1, count), dim3(32, 8), 0, st>>>(
                                      n, in, out, stride, stride, dev + off)));
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) { helm_set_error("bcr: transpose", e); return HELM_ECUDA; }
        return HELM_OK;
    });
    return HELM_OK;
}

}  // namespace

bool bcr_supported(const GridGeom &g) { return (g.nz % 2) == 0 && g.nz >= 16 && g.nx >= 4; }

// ------------------------------------------------------------------ factor

helm_status bcr_factor(helm_factor_t *f) {
    helm_op *op = f->op;
    const GridGeom &g = op->g;
    const int nx = g.nx, nz = g.nz, ns = op->n_omega;
    const long long nz2 = (long long)nz * nz;
    const int half = nx / 2 + 1;
    const cudaStream_t st = op->st;
    BcrData &b = f->bcr;
    b.half = half;
    helm_status s;
    const size_t blk = (size_t)nz2 * sizeof(float2);
    if ((s = dev_alloc((void **)&b.Dinv, (size_t)ns * nx * blk, "bcr: inverses", st)) != HELM_OK ||
        (s = dev_alloc((void **)&b.P, (size_t)ns * half * blk, "bcr: P", st)) != HELM_OK ||
        (s = dev_alloc((void **)&b.Q, (size_t)ns * half * blk, "bcr: Q", st)) != HELM_OK ||
        (s = dev_alloc((void **)&b.W, (size_t)ns * half * blk, "bcr: W", st)) != HELM_OK ||
        (s = dev_alloc((void **)&b.V, (size_t)ns * half * blk, "bcr: V", st)) != HELM_OK)
        return s;
    // working blocks of the reduction: current diagonal blocks and couplings (ping-pong)
    float2 *Dc = nullptr, *Lc = nullptr, *Ln = nullptr, *Uc = nullptr, *Un = nullptr;
    struct Work {
        float2 **p[5];
        cudaStream_t st;
        ~Work() { for (auto q : p) dev_free(*q, st); }
    } work{{&Dc, &Lc, &Ln, &Uc, &Un}, st};
    if ((s = dev_alloc((void **)&Dc, (size_t)ns * nx * blk, "bcr: work", st)) != HELM_OK ||
        (s = dev_alloc((void **)&Lc, (size_t)ns * half * blk, "bcr: work", st)) != HELM_OK ||
        (s = dev_alloc((void **)&Ln, (size_t)ns * half * blk, "bcr: work", st)) != HELM_OK ||
        (s = dev_alloc((void **)&Uc, (size_t)ns * half * blk, "bcr: work", st)) != HELM_OK ||
        (s = dev_alloc((void **)&Un, (size_t)ns * half * blk, "bcr: work", st)) != HELM_OK)
        return s;
    if ((s = dev_alloc((void **)&b.split, kSolveSplitElems * sizeof(float2), "bcr: split-K tiles", st)) != HELM_OK)
        return s;
    b.split_cap = kSolveSplitElems;
    cudaError_t e;
    Plan pl(st);
    if ((s = pl.with_split(kFactorSplitElems)) != HELM_OK) return s;
    const int per = (int)std::min<long long>(64, (nz2 + 255) / 256);
    // n_z <= 256: no line block is formed in memory before level 0, which inverts the odd lines'
    // tridiagonal blocks and updates the even lines' straight from A's diagonal and couplings
    const bool tri_level0 = nz <= 2 * INV_MAX;
    const double2 *tri_diag = tri_level0 ? op->diag : nullptr;
    TriIn tri;
    tri.diag = op->diag;
    tri.nz = nz;
    tri.nx = nx;
    tri.cz_in = coup_of(g).cz_in;
    tri.cz_edge = coup_of(g).cz_edge;
    {
        const double2 *diag = op->diag;
        float2 *D0 = Dc;
        const Coup cp = coup_of(g);
        const int perq = (int)std::min<long long>(64, (nz2 / 2 + 255) / 256);
        if (!tri_level0) pl.ops.push_back([=](const int *) -> helm_status {
            HELM_TRACED(K_BCR_FORM, st, (bcr_form_kernel<<<dim3(perq, nx, ns), 256, 0, st>>>(g, cp, diag, D0)));
            const cudaError_t e2 = cudaGetLastError();
            if (e2 != cudaSuccess) { helm_set_error("bcr: form blocks", e2); return HELM_ECUDA; }
            return HELM_OK;
        });
    }
    const Fam fD{Dc, nz2, nz}, fDinv{b.Dinv, nz2, nz};
    int levels = 0;
    for (int sp = 1; sp < nx; sp *= 2, ++levels) {
        std::vector<int> inv_pairs, tv, tw, tp, tq, td, tl, tu;
        for (int sy = 0; sy < ns; ++sy)
            for (int j = sp; j < nx; j += 2 * sp) inv_pairs.insert(inv_pairs.end(), {sy * nx + j, sy * nx + j});
        // level 0: the line blocks are still tridiagonal
        s = (sp == 1 && tri_level0) ? invert_tridiag_blocks(nz, fD, fDinv, inv_pairs, op->status, pl, tri)
                                    : invert_blocks(nz, fD, fDinv, inv_pairs, op->status, pl);
        if (s != HELM_OK) return s;
        if (sp == 1) {
            float2 *D0 = Dc, *Di = b.Dinv, *L1 = Ln, *U1 = Un;
            const Coup cp = coup_of(g);
            pl.ops.push_back([=](const int *) -> helm_status {
                HELM_TRACED(K_BCR_L0, st, (bcr_level0_kernel<<<dim3(per, (nx + 1) / 2, ns), 256, 0, st>>>(
                                              g, cp, D0, Di, L1, U1, half, tri_diag)));
                const cudaError_t e2 = cudaGetLastError();
                if (e2 != cudaSuccess) { helm_set_error("bcr: level 0", e2); return HELM_ECUDA; }
                return HELM_OK;
            });
        } else {
            std::vector<int> vpairs, wpairs;
            for (int sy = 0; sy < ns; ++sy) {
                const int hb = sy * half, lb = sy * nx;
                for (int j = sp; j < nx; j += 2 * sp) {
                    // V_j = U_{j-s} Dinv_j;  W_j = L_{j+s} Dinv_j
                    auto v = task8(hb + (j - sp) / 2, lb + j, 0, hb + j / 2);
                    tv.insert(tv.end(), v.begin(), v.end());
                    vpairs.insert(vpairs.end(), {hb + j / 2, hb + j / 2});
                    if (j + sp < nx) {
                        auto w = task8(hb + (j + sp) / 2, lb + j, 0, hb + j / 2);
                        tw.insert(tw.end(), w.begin(), w.end());
                        wpairs.insert(wpairs.end(), {hb + j / 2, hb + j / 2});
                    }
                }
                for (int k = 0; k < nx; k += 2 * sp) {
                    const bool ha = k >= sp, hc = k + sp < nx;
                    if (!ha && !hc) continue;
                    // D_k -= L_k W_a^T + U_k V_c^T
                    auto d = task8(ha ? hb + k / 2 : -1, ha ? hb + (k - sp) / 2 : 0, lb + k, lb + k,
                                   hc ? hb + k / 2 : -1, hc ? hb + (k + sp) / 2 : 0);
                    td.insert(td.end(), d.begin(), d.end());
                    if (k >= 2 * sp) {   // L_k <- -L_k V_a^T
                        auto l = task8(hb + k / 2, hb + (k - sp) / 2, 0, hb + k / 2);
                        tl.insert(tl.end(), l.begin(), l.end());
                    }
                    if (k + 2 * sp < nx) {   // U_k <- -U_k W_c^T
                        auto u = task8(hb + k / 2, hb + (k + sp) / 2, 0, hb + k / 2);
                        tu.insert(tu.end(), u.begin(), u.end());
                    }
                }
            }
            ZGemmArgs ga;
            ga.M = ga.N = ga.K = nz;
            ga.status = op->status;
            ga.nterms = 1;
            ga.B[0] = zop(b.Dinv, nz2, nz);
            ga.C = b.V; ga.c_stride = nz2; ga.ldc = nz;
            ga.A[0] = zop(Uc, nz2, nz);
            if ((s = gemm(ga, tv, pl)) != HELM_OK) return s;
            ga.C = b.W;
            ga.A[0] = zop(Lc, nz2, nz);
            if ((s = gemm(ga, tw, pl)) != HELM_OK) return s;
            if ((s = transpose_blocks(nz, b.V, b.P, nz2, vpairs, pl)) != HELM_OK) return s;
            if ((s = transpose_blocks(nz, b.W, b.Q, nz2, wpairs, pl)) != HELM_OK) return s;
            ZGemmArgs gd;
            gd.M = gd.N = gd.K = nz;
            gd.status = op->status;
            gd.nterms = 2;
            gd.A[0] = zop(Lc, nz2, nz); gd.B[0] = zop(b.W, nz2, nz); gd.sign[0] = -1.f;
            gd.A[1] = zop(Uc, nz2, nz); gd.B[1] = zop(b.V, nz2, nz); gd.sign[1] = -1.f;
            gd.C0 = zop(Dc, nz2, nz);
            gd.C = Dc; gd.c_stride = nz2; gd.ldc = nz;
            if ((s = gemm(gd, td, pl)) != HELM_OK) return s;
            ZGemmArgs gl;
            gl.M = gl.N = gl.K = nz;
            gl.status = op->status;
            gl.nterms = 1;
            gl.sign[0] = -1.f;
            gl.A[0] = zop(Lc, nz2, nz); gl.B[0] = zop(b.V, nz2, nz);
            gl.C = Ln; gl.c_stride = nz2; gl.ldc = nz;
            if ((s = gemm(gl, tl, pl)) != HELM_OK) return s;
            gl.A[0] = zop(Uc, nz2, nz); gl.B[0] = zop(b.W, nz2, nz);
            gl.C = Un;
            if ((s = gemm(gl, tu, pl)) != HELM_OK) return s;
        }
        std::swap(Lc, Ln);
        std::swap(Uc, Un);
    }
    // the last line left: line 0
    {
        std::vector<int> last;
        for (int sy = 0; sy < ns; ++sy) last.insert(last.end(), {sy * nx, sy * nx});
        if ((s = invert_blocks(nz, fD, fDinv, last, op->status, pl)) != HELM_OK) return s;
    }
    if ((s = pl.run()) != HELM_OK) return s;
    b.levels = levels;
    // the solve's task lists, built once: forward levels 1 .. L-1, last line, backward L-1 .. 1,
    // level 0 both ways (vector operands indexed system * nx + line)
    std::vector<int> all;
    b.fwd.assign(levels, BcrData::List());
    b.bwd.assign(levels, BcrData::List());
    auto list_of = [&](int off, int nt) {
        BcrData::List L;
        L.first = off;
        L.count = (int)all.size() / 8 - off;
        L.terms = count_terms(all.data() + 8 * (size_t)off, (size_t)L.count, nt);
        return L;
    };
    auto add = [&](std::vector<int> &&v) { all.insert(all.end(), v.begin(), v.end()); };
    for (int l = 0, sp = 1; l < levels; ++l, sp *= 2) {
        const int off = (int)all.size() / 8;
        for (int sy = 0; sy < ns; ++sy) {
            const int hb = sy * half, lb = sy * nx;
            if (l == 0) {
                for (int j = 1; j < nx; j += 2) add(task8(lb + j, lb + j, 0, lb + j));   // y_j = Dinv_j b_j
            } else {
                for (int k = 0; k < nx; k += 2 * sp) {
                    const bool ha = k >= sp, hc = k + sp < nx;
                    if (!ha && !hc) continue;
                    add(task8(ha ? hb + (k - sp) / 2 : -1, ha ? lb + k - sp : 0, lb + k, lb + k,
                              hc ? hb + (k + sp) / 2 : -1, hc ? lb + k + sp : 0));
                }
            }
        }
        b.fwd[l] = list_of(off, l == 0 ? 1 : 2);
    }
    {
        const int off = (int)all.size() / 8;
        for (int sy = 0; sy < ns; ++sy) add(task8(sy * nx, sy * nx, 0, sy * nx));
        b.last = list_of(off, 1);
    }
    for (int l = 0, sp = 1; l < levels; ++l, sp *= 2) {
        const int off = (int)all.size() / 8;
        for (int sy = 0; sy < ns; ++sy) {
            const int hb = sy * half, lb = sy * nx;
            for (int j = sp; j < nx; j += 2 * sp) {
                if (l == 0) {
                    add(task8(lb + j, lb + j, lb + j, lb + j));   // x_j = y_j - Dinv_j t_j
                } else {
                    const bool hc = j + sp < nx;
                    add(task8(lb + j, lb + j, 0, lb + j, hb + j / 2, lb + j - sp, hc ? hb + j / 2 : -1,
                              hc ? lb + j + sp : 0));
                }
            }
        }
        b.bwd[l] = list_of(off, l == 0 ? 1 : 3);
    }
    if ((s = dev_alloc((void **)&b.tasks, all.size() * sizeof(int), "bcr: solve plan", st)) != HELM_OK) return s;
    if ((e = cudaMemcpyAsync(b.tasks, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice, st)) != cudaSuccess) {
        helm_set_error("bcr: solve plan", e);
        return HELM_ECUDA;
    }
    // the work blocks are released on the stream after the last kernel that reads them
    return HELM_OK;
}

void bcr_free(helm_factor_t *f) {
    const cudaStream_t st = f->op ? f->op->st : nullptr;
    BcrData &b = f->bcr;
    dev_free(b.Dinv, st);
    dev_free(b.P, st);
    dev_free(b.Q, st);
    dev_free(b.W, st);
    dev_free(b.V, st);
    dev_free(b.tasks, st);
    dev_free(b.split, st);
    b = BcrData();
}

// ------------------------------------------------------------------- solve

// x = A~^{-1} r for every system and right-hand side, complex FP32: r [n_sys][nrhs][N] is the
// working vector (overwritten), x [n_sys][nrhs][N] the result.  skip: launches do nothing
// while it is set (refinement finished).
helm_status bcr_solve(const helm_factor_t *f, int nrhs, float2 *r, float2 *x, const int *skip, const int *frozen) {
    const helm_op *op = f->op;
    const GridGeom &g = op->g;
    const int nx = g.nx, nz = g.nz, ns = op->n_omega, N = nx * nz;
    const long long nz2 = (long long)nz * nz;
    const BcrData &b = f->bcr;
    const cudaStream_t st = op->st;
    const long long vhi = (long long)nrhs * N;   // vectors: index system * nx + line
    auto vec = [&](const float2 *base) {   // ns groups of nx line vectors
        ZOperand o = zop(base, nz, N, nx, vhi);
        o.count = ns;
        return o;
    };
    const long long n_lines = (long long)ns * nx, n_half = (long long)ns * b.half;
    auto blocks = [&](const float2 *base, long long count) {
        ZOperand o = zop(base, nz2, nz);
        o.count = count;
        return o;
    };
    ZGemmArgs ga;
    ga.M = nz; ga.N = nrhs; ga.K = nz;
    ga.c_col = 1;
    ga.status = op->status;
    ga.skip = skip;
    ga.tries = wait_tries();
    ga.part = b.split;
    ga.part_cap = b.split_cap;
    ga.sys_frozen = frozen;   // C index = system * nx + line
    ga.sys_div = nx;
    ga.c_stride = nz; ga.c_div = nx; ga.c_stride_hi = vhi; ga.ldc = N;
    cudaError_t e;
    auto launch = [&](ZGemmArgs a, const BcrData::List &lst) -> helm_status {
        a.tasks = b.tasks + 8 * (size_t)lst.first;
        a.flops = 8.0 * a.M * a.N * a.K * (double)lst.terms;
        e = launch_zgemm(a, lst.count, st);
        if (e != cudaSuccess) { helm_set_error("bcr solve: tensor-core GEMM", e); return HELM_ECUDA; }
        return HELM_OK;
    };
    helm_status s;
    const int nodd = nx / 2, neven = (nx + 1) / 2;
    const Coup cp = coup_of(g);
    const int cols = ns * nrhs, thr = std::min(128, nz / 2), per = (nz / 2 + thr - 1) / thr;
    const int colb = (cols + L0_COLS - 1) / L0_COLS;
    // forward, level 0: y_j = Dinv_j b_j into x, then b_k -= C (y_{k-1} + y_{k+1})
    {
        ZGemmArgs a = ga;
        a.nterms = 1;
        a.A[0] = blocks(b.Dinv, n_lines);
        a.B[0] = vec(r);
        a.C = x;
        if ((s = launch(a, b.fwd[0])) != HELM_OK) return s;
        HELM_TRACED(K_BCR_SOLVE_L0, st, (bcr_solve_l0_fwd_kernel<<<dim3(per, neven, colb), thr, 0, st>>>(
                                            g, cp, cols, r, x, skip, frozen, nrhs)));
        if ((e = cudaGetLastError()) != cudaSuccess) { helm_set_error("bcr solve: level 0", e); return HELM_ECUDA; }
    }
    for (int l = 1; l < b.levels; ++l) {   // b_k -= W_a b_a + V_c b_c
        ZGemmArgs a = ga;
        a.nterms = 2;
        a.A[0] = blocks(b.W, n_half); a.B[0] = vec(r); a.sign[0] = -1.f;
        a.A[1] = blocks(b.V, n_half); a.B[1] = vec(r); a.sign[1] = -1.f;
        a.C0 = vec(r);
        a.C = r;
        if ((s = launch(a, b.fwd[l])) != HELM_OK) return s;
    }
    {   // x_0 = Dinv_0 b_0
        ZGemmArgs a = ga;
        a.nterms = 1;
        a.A[0] = blocks(b.Dinv, n_lines);
        a.B[0] = vec(r);
        a.C = x;
        if ((s = launch(a, b.last)) != HELM_OK) return s;
    }
    for (int l = b.levels - 1; l >= 1; --l) {   // x_j = Dinv_j b_j - P_j x_{j-s} - Q_j x_{j+s}
        ZGemmArgs a = ga;
        a.nterms = 3;
        a.A[0] = blocks(b.Dinv, n_lines); a.B[0] = vec(r);
        a.A[1] = blocks(b.P, n_half); a.B[1] = vec(x); a.sign[1] = -1.f;
        a.A[2] = blocks(b.Q, n_half); a.B[2] = vec(x); a.sign[2] = -1.f;
        a.C = x;
        if ((s = launch(a, b.bwd[l])) != HELM_OK) return s;
    }
    {   // backward, level 0: t_j = C (x_{j-1} + x_{j+1}) into b_j, x_j = y_j - Dinv_j t_j
        if (nodd > 0) {
            HELM_TRACED(K_BCR_SOLVE_L0, st, (bcr_solve_l0_bwd_kernel<<<dim3(per, nodd, colb), thr, 0, st>>>(
                                                g, cp, cols, r, x, skip, frozen, nrhs)));
            if ((e = cudaGetLastError()) != cudaSuccess) { helm_set_error("bcr solve: level 0", e); return HELM_ECUDA; }
        }
        ZGemmArgs a = ga;
        a.nterms = 1;
        a.A[0] = blocks(b.Dinv, n_lines); a.B[0] = vec(r); a.sign[0] = -1.f;
        a.C0 = vec(x);
        a.C = x;
        if ((s = launch(a, b.bwd[0])) != HELM_OK) return s;
    }
    return HELM_OK;
}

// ------------------------------------------------ building blocks at the ABI (helm_blas.h)

helm_status blas_zgemm(int batch, int M, int N, int K, const float2 *A, long long sa, int lda, const float2 *Bt,
                       long long sb, int ldb, float sign, const float2 *C0, float2 *C, long long sc, int ldc,
                       cudaStream_t st, int *status) {
    ZGemmArgs a;
    a.M = M; a.N = N; a.K = K;
    a.nterms = 1;
    a.A[0] = zop(A, sa, lda);
    a.B[0] = zop(Bt, sb, ldb);
    a.sign[0] = sign;
    if (C0) a.C0 = zop(C0, sc, ldc);
    a.C = C; a.c_stride = sc; a.ldc = ldc;
    a.status = status;
    std::vector<int> tasks;
    for (int t = 0; t < batch; ++t) {
        auto v = task8(t, t, t, t);
        tasks.insert(tasks.end(), v.begin(), v.end());
    }
    Plan pl(st);
    helm_status s = pl.with_split(kFactorSplitElems);
    if (s == HELM_OK) s = gemm(a, tasks, pl);
    return s == HELM_OK ? pl.run() : s;
}

helm_status blas_zinv(int batch, int n, const float2 *A, long long sa, int lda, float2 *X, long long sx, int ldx,
                      cudaStream_t st, int *status) {
    std::vector<int> pairs;
    for (int t = 0; t < batch; ++t) pairs.insert(pairs.end(), {t, t});
    if (A != X) {   // copy into X first: the recursion works in place on the output blocks
        // blocks stacked without gaps on both sides are one 2D copy of batch * n rows
        const bool stacked = sa == (long long)n * lda && sx == (long long)n * ldx;
        cudaError_t e = cudaMemcpy2DAsync(X, (size_t)ldx * sizeof(float2), A, (size_t)lda * sizeof(float2),
                                          (size_t)n * sizeof(float2), (size_t)n * (stacked ? batch : 1),
                                          cudaMemcpyDeviceToDevice, st);
        for (int t = 1; !stacked && t < batch && e == cudaSuccess; ++t)
            e = cudaMemcpy2DAsync(X + (long long)t * sx, (size_t)ldx * sizeof(float2), A + (long long)t * sa,
                                  (size_t)lda * sizeof(float2), (size_t)n * sizeof(float2), (size_t)n,
                                  cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) { helm_set_error("helm_zinv_batched: copy", e); return HELM_ECUDA; }
    }
    const Fam f{X, sx, ldx};
    Plan pl(st);
    helm_status s = pl.with_split(kFactorSplitElems);
    if (s == HELM_OK) s = invert_blocks(n, f, f, pairs, status, pl);
    return s == HELM_OK ? pl.run() : s;
}

}  // namespace helm

// ------------------------------------------------------------------ C ABI (helm_blas.h)

#include "helm_blas.h"

namespace {
struct DevStatus {   // a device status word for the building-block calls
    int *p = nullptr;
    cudaStream_t st;
    explicit DevStatus(cudaStream_t s) : st(s) {}
    ~DevStatus() { ::dev_free(p, st); }
};
}  // namespace

extern "C" helm_status helm_zgemm_batched(int32_t batch, int32_t M, int32_t N, int32_t K, const helm_c64 *A, int64_t sa,
                                          int32_t lda, const helm_c64 *Bt, int64_t sb, int32_t ldb, float sign,
                                          const helm_c64 *C0, helm_c64 *C, int64_t sc, int32_t ldc, void *stream) {
    if (batch < 0 || batch > 65535 || M < 1 || N < 1 || K < 1 || (K & 1) || !A || !Bt || !C || lda < K || ldb < K ||
        ldc < N || (lda & 1) || (ldb & 1) || (sa & 1) || (sb & 1) || (sign != 1.f && sign != -1.f) ||
        ((uintptr_t)A & 15) || ((uintptr_t)Bt & 15)) {
        helm_set_msg("helm_zgemm_batched: bad sizes, strides, alignment or sign");
        return HELM_EINVAL;
    }
    if (batch == 0) return HELM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    DevStatus ds(st);
    helm_status s = dev_alloc((void **)&ds.p, sizeof(int), "helm_zgemm_batched: status", st);
    if (s != HELM_OK) return s;
    cudaError_t e = cudaMemsetAsync(ds.p, 0, sizeof(int), st);
    if (e != cudaSuccess) { helm_set_error("helm_zgemm_batched", e); return HELM_ECUDA; }
    return helm::blas_zgemm(batch, M, N, K, (const float2 *)A, sa, lda, (const float2 *)Bt, sb, ldb, sign,
                            (const float2 *)C0, (float2 *)C, sc, ldc, st, ds.p);
}

extern "C" helm_status helm_zinv_batched(int32_t batch, int32_t n, const helm_c64 *A, int64_t sa, int32_t lda,
                                         helm_c64 *X, int64_t sx, int32_t ldx, void *stream) {
    if (batch < 0 || batch > 65535 || n < 2 || (n & 1) || !A || !X || lda < n || ldx < n || (lda & 1) || (ldx & 1) ||
        (sa & 1) || (sx & 1) || ((uintptr_t)A & 15) || ((uintptr_t)X & 15)) {
        helm_set_msg("helm_zinv_batched: bad sizes, strides or alignment");
        return HELM_EINVAL;
    }
    if (batch == 0) return HELM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    DevStatus ds(st);
    helm_status s = dev_alloc((void **)&ds.p, sizeof(int), "helm_zinv_batched: status", st);
    if (s != HELM_OK) return s;
    cudaError_t e = cudaMemsetAsync(ds.p, 0, sizeof(int), st);
    if (e != cudaSuccess) { helm_set_error("helm_zinv_batched", e); return HELM_ECUDA; }
    if ((s = helm::blas_zinv(batch, n, (const float2 *)A, sa, lda, (float2 *)X, sx, ldx, st, ds.p)) != HELM_OK) return s;
    int h = 0;
    e = cudaMemcpyAsync(&h, ds.p, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { helm_set_error("helm_zinv_batched", e); return HELM_ECUDA; }
    if (h & helm::ST_SINGULAR) { helm_set_msg("helm_zinv_batched: zero or non-finite pivot"); return HELM_ESINGULAR; }
    return HELM_OK;
}
