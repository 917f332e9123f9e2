// Block forward/backward sweeps with the stored line inverses, and the FP64 residual.
//
// With G_i = S_i^{-1} from the line factorisation (factor.cu), A x = b is solved by
//   forward   y_0 = G_0 b_0,            y_i = G_i (b_i - C_i y_{i-1}),
//   backward  x_{nx-1} = y_{nx-1},      x_i = y_i - G_i C_{i+1} x_{i+1},
// two dense (n_z x n_z) x (n_z x R) products per line with all right-hand sides of a
// chunk as the product's N dimension (the twisted variant runs both halves at once, see
// line_sweep_kernel).  The adjoint solve of A^H uses the same factor: A is complex
// symmetric, so (A^H)^{-1} b = conj(A^{-1} conj(b)).
//
// One thread-block cluster handles one (system, right-hand-side chunk); CTA r of a team owns
// a slab of rows of every line and pushes its new rows, scaled by the line coupling, into the
// shared memory of every CTA of the team (st.async with mbarrier completion).
//
// TG = float is the correction solve of the mixed-precision refinement (refine.cu): complex
// FP32 factor, right-hand side and result.  TG = double is the plain FP64 path (Y aliases X).
#include <algorithm>
#include <map>
#include <tuple>
#include <mutex>
#include <stdlib.h>
#include "kernels.h"
#include "mma_tf32.cuh"
#include "trace.h"

namespace helm {

constexpr int SW_THREADS = 256;
constexpr int SW_KC = 64;      // K chunk of the streamed (non-prefetched) G path
constexpr int SW_MAXOPT = 2;   // outputs per thread (rows_per_cta * R <= 2 * 256)
constexpr size_t SW_SMEM_MAX = 200 * 1024;
constexpr int FM_MAX_RHS = 4;   // right-hand sides per cluster up to which the FMA product is taken

template <typename TG> struct SweepArgs {
    GridGeom g;
    int nrhs, R, cs, n_chunks, prefetch, tpo;   // tpo: threads per output (K split), power of 2
    int mid, teams;                             // twisted middle line and team count (factor layout)
    const cx_t<TG> *G;   // [n_sys][nx][nz][nz]
    const cx_t<TG> *B;   // [n_sys][nrhs][N] right-hand sides in the working precision
    double2 *X;          // [n_sys][nrhs][N]
    cx_t<TG> *Y;         // forward vectors y_i, [n_sys][nrhs][N] (== X for TG = double)
    int conj;            // FP64 path: B and X conjugated (adjoint solve)
    int *status;
    const int *skip;     // optional: nonzero -> the launch does nothing (refinement finished)
    const int *frozen;   // optional: frozen[2*sys] nonzero -> system sys is left alone (converged)
    uint32_t tries;      // polls of a bounded mbarrier wait before it gives up
};

// Padded row stride (in complex elements) of the shared-memory operands of the sweep product.
// A quarter-warp (the unit of a 16-byte shared load) reads 8/tpo rows x tpo adjacent 16-byte
// K words; the stride is chosen so that those eight words fall on distinct banks:
// 2*stride = 4*tpo (mod 32) words for complex FP32 (even stride keeps 16-byte alignment), and
// 4*stride = 4*tpo (mod 32) words for complex FP64.
template <typename TG> __host__ __device__ __forceinline__ int padded(int n, int tpo) {
    if (sizeof(TG) == 4) {
        int p = (n + 1) & ~1;
        while (p % 16 != (2 * tpo) % 16) p += 2;
        return p;
    }
    int p = n;
    while (p % 8 != tpo % 8) ++p;
    return p;
}

// sum_b g[b] t[b] over n complex entries (both 16-byte aligned), four independent chains
__device__ __forceinline__ float2 dot_row(const float2 *g, const float2 *t, int n) {
    float2 a0 = make_float2(0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
    int b = 0;
    for (; b + 4 <= n; b += 4) {
        const float4 gA = *reinterpret_cast<const float4 *>(g + b);
        const float4 gB = *reinterpret_cast<const float4 *>(g + b + 2);
        const float4 tA = *reinterpret_cast<const float4 *>(t + b);
        const float4 tB = *reinterpret_cast<const float4 *>(t + b + 2);
        cfma(a0, make_float2(gA.x, gA.y), make_float2(tA.x, tA.y));
        cfma(a1, make_float2(gA.z, gA.w), make_float2(tA.z, tA.w));
        cfma(a2, make_float2(gB.x, gB.y), make_float2(tB.x, tB.y));
        cfma(a3, make_float2(gB.z, gB.w), make_float2(tB.z, tB.w));
    }
    for (; b < n; ++b) cfma(a0, g[b], t[b]);
    return make_float2((a0.x + a1.x) + (a2.x + a3.x), (a0.y + a1.y) + (a2.y + a3.y));
}
__device__ __forceinline__ double2 dot_row(const double2 *g, const double2 *t, int n) {
    double2 a0 = make_double2(0.0, 0.0), a1 = a0, a2 = a0, a3 = a0;
    int b = 0;
    for (; b + 4 <= n; b += 4) {
        cfma(a0, g[b], t[b]);
        cfma(a1, g[b + 1], t[b + 1]);
        cfma(a2, g[b + 2], t[b + 2]);
        cfma(a3, g[b + 3], t[b + 3]);
    }
    for (; b < n; ++b) cfma(a0, g[b], t[b]);
    return make_double2((a0.x + a1.x) + (a2.x + a3.x), (a0.y + a1.y) + (a2.y + a3.y));
}

// sum over the pairs p = part, part + tpo, ... of g[2p..2p+1] t[2p..2p+1] (complex FP32, both
// operands 16-byte aligned; consecutive parts read adjacent 16-byte words, so the threads that
// share an output never collide on a bank), plus the odd tail element for part 0
__device__ __forceinline__ float2 dot_row_il(const float2 *g, const float2 *t, int n, int part, int tpo) {
    const float4 *g4 = reinterpret_cast<const float4 *>(g);
    const float4 *t4 = reinterpret_cast<const float4 *>(t);
    const int np = n >> 1;
    float2 a0 = make_float2(0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
    int p = part;
    for (; p + tpo < np; p += 2 * tpo) {
        const float4 gA = g4[p], tA = t4[p], gB = g4[p + tpo], tB = t4[p + tpo];
        cfma(a0, make_float2(gA.x, gA.y), make_float2(tA.x, tA.y));
        cfma(a1, make_float2(gA.z, gA.w), make_float2(tA.z, tA.w));
        cfma(a2, make_float2(gB.x, gB.y), make_float2(tB.x, tB.y));
        cfma(a3, make_float2(gB.z, gB.w), make_float2(tB.z, tB.w));
    }
    if (p < np) {
        const float4 gA = g4[p], tA = t4[p];
        cfma(a0, make_float2(gA.x, gA.y), make_float2(tA.x, tA.y));
        cfma(a1, make_float2(gA.z, gA.w), make_float2(tA.z, tA.w));
    }
    if ((n & 1) && part == 0) cfma(a2, g[n - 1], t[n - 1]);
    return make_float2((a0.x + a1.x) + (a2.x + a3.x), (a0.y + a1.y) + (a2.y + a3.y));
}
__device__ __forceinline__ double2 dot_row_il(const double2 *g, const double2 *t, int n, int part, int tpo) {
    double2 a0 = make_double2(0.0, 0.0), a1 = a0;
    int b = part;
    for (; b + tpo < n; b += 2 * tpo) {
        cfma(a0, g[b], t[b]);
        cfma(a1, g[b + tpo], t[b + tpo]);
    }
    if (b < n) cfma(a0, g[b], t[b]);
    return make_double2(a0.x + a1.x, a0.y + a1.y);
}

// line handled by global step s: forward s = 0..nx-1 -> line s; backward s = nx..2nx-2 -> line 2nx-2-s
__device__ __forceinline__ int step_line(int s, int nx) { return s < nx ? s : 2 * nx - 2 - s; }

// Pre-pass: Y_i = G_i b_i for every line i of every system at once (the half of the
// forward sweep that does not depend on the recurrence), a batched complex GEMM over
// (system, line, row tile, right-hand-side chunk).  b is the input in the working precision
// (conjugated for the adjoint FP64 solve).  The CUDA-core sweep uses it; the tensor-path sweep
// takes b_i into its own product instead.
constexpr int PP_ROWS = 64;    // rows of G_i per CTA
constexpr int PP_RHS = 16;     // right-hand sides per CTA
constexpr int PP_KC = 32;      // K chunk
// Register-blocked batched product: each thread computes 2 rows x 4 right-hand sides (64 rows
// x 16 right-hand sides per CTA of 128 threads), so every two shared loads of G feed eight
// complex MACs.  A warp shares its right-hand sides (broadcast reads) and takes rows tr and
// tr + 32, whose padded stride keeps the G reads free of bank conflicts.
template <typename TG>
__global__ void __launch_bounds__(128) line_gb_prepass_kernel(GridGeom g, int nrhs, const cx_t<TG> *G,
                                                             const cx_t<TG> *B, cx_t<TG> *Y, int conj,
                                                             const int *skip, const int *frozen) {
    using V = cx_t<TG>;
    if (skip && *skip) return;
    const int nx = g.nx, nz = g.nz, N = nx * nz;
    const int n_rt = (nz + PP_ROWS - 1) / PP_ROWS;
    const int n_ch = (nrhs + PP_RHS - 1) / PP_RHS;
    int bid = blockIdx.x;
    const int ch = bid % n_ch; bid /= n_ch;
    const int rt = bid % n_rt; bid /= n_rt;
    const int i = bid % nx;
    const int sys = bid / nx;
    if (frozen && frozen[2 * sys]) return;
    const int q0 = ch * PP_RHS, Rc = min(PP_RHS, nrhs - q0);
    const int r0 = rt * PP_ROWS, nrows = min(PP_ROWS, nz - r0);
    constexpr int KP = PP_KC + 1;   // padded row stride (complex elements)
    __shared__ V sg[PP_ROWS][KP];    // G_i rows x K chunk
    __shared__ V sb[PP_RHS][KP];     // right-hand sides x K chunk
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int tr = tid & 31, tq = tid >> 5;    // rows tr, tr + 32; right-hand sides 4 tq .. 4 tq + 3
    const V *Bs = B + ((size_t)sys * nrhs + q0) * N + (size_t)i * nz;
    const V *Gi = G + ((size_t)sys * nx + i) * nz * nz + (size_t)r0 * nz;
    V acc[2][4];
#pragma unroll
    for (int a2 = 0; a2 < 2; ++a2)
#pragma unroll
        for (int b2 = 0; b2 < 4; ++b2) acc[a2][b2] = mkc<TG>(TG(0), TG(0));
    for (int kc = 0; kc < nz; kc += PP_KC) {
        const int kw = min(PP_KC, nz - kc);
        for (int q = wid; q < PP_RHS; q += 4)
            for (int j = lane; j < PP_KC; j += 32) {
                V v = mkc<TG>(TG(0), TG(0));
                if (q < Rc && j < kw) {
                    v = Bs[(size_t)q * N + kc + j];
                    if (conj) v.y = -v.y;
                }
                sb[q][j] = v;
            }
        for (int r = wid; r < PP_ROWS; r += 4)
            for (int j = lane; j < PP_KC; j += 32)
                sg[r][j] = (r < nrows && j < kw) ? Gi[(size_t)r * nz + kc + j] : mkc<TG>(TG(0), TG(0));
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < PP_KC; ++k) {
            const V g0 = sg[tr][k], g1 = sg[tr + 32][k];
#pragma unroll
            for (int b2 = 0; b2 < 4; ++b2) {
                const V bb = sb[4 * tq + b2][k];
                cfma(acc[0][b2], g0, bb);
                cfma(acc[1][b2], g1, bb);
            }
        }
        __syncthreads();
    }
    V *Ys = Y + ((size_t)sys * nrhs + q0) * N + (size_t)i * nz + r0;
#pragma unroll
    for (int a2 = 0; a2 < 2; ++a2)
#pragma unroll
        for (int b2 = 0; b2 < 4; ++b2) {
            const int r = tr + 32 * a2, q = 4 * tq + b2;
            if (r < nrows && q < Rc) Ys[(size_t)q * N + r] = acc[a2][b2];
        }
}

// ------------------------------------------------- tensor-pipe line product (complex FP32)
// The product G t of a CTA's slab of G_i (rows x n_z, interleaved complex) with up to eight
// right-hand sides is one real product on the tensor pipe: with k running over the
// interleaved (re, im) columns of G,
//     [Re(G t) | Im(G t)] = [G_re G_im ...] x [[Re t, Im t], [-Im t, Re t]] (row pairs),
// an m16 x n8 tile for the real parts and one for the imaginary parts (mma.sync m16n8k8, TF32).
// Each FP32 operand x is split as x = hi + lo with hi = tf32(x), lo = tf32(x - hi); the three
// products hi*hi + hi*lo + lo*hi, accumulated in FP32, carry about 22 bits of each operand.
// Thread (g, t) of a warp (g = lane / 4, t = lane % 4) holds the k columns 2t and 2t + 1 of an
// 8-column block of complex entries as its two fragment slots, so A and B fragments come
// from one 16-byte load each (any permutation of k shared by A and B leaves the product).
constexpr int MMA_RHS = 8;   // right-hand sides per cluster on the tensor path (one n tile)
// row stride of the shared-memory line vectors on the tensor path: the 16-byte B loads of a
// quarter-warp (rows g, g + 1 at four 16-byte columns) fall on distinct banks
__host__ __device__ __forceinline__ int padded_mma(int n) {
    int p = (n + 1) & ~1;
    while (p % 16 != 8) p += 2;
    return p;
}
// FMA product of one lane: facc[q] += sum_p G(row, c_p) t_q(c_p) over its 4*KP complex columns
// c_p = c0 .. c0 + 4*KP - 1 (held in g, two per float4), for the first NQ right-hand sides of
// the line buffer tv ([rhs][nzp], complex FP32); rhs >= nq and columns >= nz read as zero.  The
// loads of one column pair for every right-hand side are issued together, then 2*NQ
// independent FMA chains.
template <int NQ, int KP>
__device__ __forceinline__ void fma_product(const float2 *tv, int nzp, int c0, int nz, int nq,
                                            const float4 (&g)[2 * KP], float2 (&facc)[MMA_RHS]) {
#pragma unroll
    for (int p = 0; p < 2 * KP; ++p) {
        const int c = c0 + 2 * p;
        float4 t2[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            t2[q] = (c < nz && q < nq) ? *reinterpret_cast<const float4 *>(tv + (size_t)q * nzp + c)
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 g2 = g[p];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            float2 f = facc[q];
            f.x = fmaf(g2.x, t2[q].x, f.x);
            f.y = fmaf(g2.x, t2[q].y, f.y);
            f.x = fmaf(-g2.y, t2[q].y, f.x);
            f.y = fmaf(g2.y, t2[q].x, f.y);
            f.x = fmaf(g2.z, t2[q].z, f.x);
            f.y = fmaf(g2.z, t2[q].w, f.y);
            f.x = fmaf(-g2.w, t2[q].w, f.x);
            f.y = fmaf(g2.w, t2[q].z, f.y);
            facc[q] = f;
        }
    }
}

// Persistent twisted sweep, after the pre-pass has stored G_i b_i in Y.  The cluster holds
// `teams` teams of `cs` CTAs; CTA rank%cs of a team owns a slab of rows of every line.
//   left team:   y_i = G_i b_i - G_i C y_{i-1},  i = 0 .. m-1            (forward)
//                x_m = G_m b_m - G_m (C y_{m-1} + C y_{m+1})              (middle)
//                x_i = y_i - G_i C x_{i+1},      i = m-1 .. 0            (backward)
//   right team:  y_i = G_i b_i - G_i C y_{i+1},  i = nx-1 .. m+1         (forward)
//                x_i = y_i - G_i C x_{i-1},      i = m+1 .. nx-1         (backward)
// with G_i the left inverses for i < m, the right ones for i > m and G_m the middle one
// (factor.cu).  One team with m = nx - 1 is the plain one-sided block substitution.
// Per step: wait (bounded mbarrier) until every CTA of the team has pushed its rows of the
// previous line vector, already multiplied by the line coupling C, into this CTA's shared
// memory (st.async with transaction-count completion); the (rows x n_z) x (n_z x R) product
// with the G_i slab that cp.async brought in during the previous step; subtract from the
// own rows (also prefetched); push the new rows.  The last forward rows of both teams go to
// the left team's middle buffers, and the left team pushes C x_m to every CTA.  Exchange
// buffers alternate; no CTA overwrites a buffer before every consumer is done with it,
// because producing the data of step s+2 needs the data of step s+1 from every CTA of the
// team, which each CTA sends only after it has finished step s (its pushes follow the CTA
// barrier of the reduction, which follows every thread's reads of the step's input).
// MT > 0: every thread waits on the mbarrier itself and there is no CTA barrier between the
// arrival of the inputs and the product; the own rows of a backward step come from a register
// loaded one step ahead, and the partial sums alternate between two buffers.
// MT > 0 selects the tensor-pipe product (complex FP32 only): MT m16 tiles of rows per CTA,
// KP 8-column blocks of K per warp (the eight warps split K and meet in shared memory), the
// G_i slab read from L2 straight into fragment registers one step ahead.  MT = 0 is the
// CUDA-core product (FP64, or shapes the tensor tiles do not cover).
// FM (with MT = 1) keeps the register-held G_i slab of the tensor path but forms the product
// with FP32 FMAs: lane (row, half) of a warp holds 4*KP complex entries of one row and reads
// the matching entries of every right-hand side from shared memory as a broadcast over the
// sixteen lanes of its half.  The 16 x 8 x 8 tile of the legacy mma.sync needs three TF32
// passes for FP32 accuracy and always eight right-hand sides; the FMA product does R of them
// at full FP32 precision.  The producer folds the right-hand side into its push,
// C y - b_{i+1}, so that the consumer's product is G_i t with no per-lane b.
template <typename TG, int MT, int KP, bool FM>
__global__ void __launch_bounds__(SW_THREADS) line_sweep_kernel(SweepArgs<TG> a) {
    using V = cx_t<TG>;
    const GridGeom g = a.g;
    const int nx = g.nx, nz = g.nz, N = nx * nz;
    const int tid = threadIdx.x;
    const int cs = a.cs, R = a.R, teams = a.teams;
    const int crank = (int)cluster_ctarank();
    const int team = crank / cs, rank = crank % cs;
    const int cid = (int)cluster_id_x();
    const int sys = cid / a.n_chunks, chunk = cid % a.n_chunks;
    const int q0 = chunk * R;
    const int Rc = min(R, a.nrhs - q0);
    const int rpc = (nz + cs - 1) / cs;
    const int r0 = min(nz, rank * rpc), r1 = min(nz, r0 + rpc);
    const int nrows = r1 - r0;
    const int nout = nrows * Rc;
    const bool pf = a.prefetch != 0;
    const int nzp = MT > 0 ? padded_mma(nz) : padded<TG>(nz, a.tpo);
    const int kcp = padded<TG>(SW_KC, a.tpo);
    const int m = a.mid;
    const int len = (team == 0) ? m : nx - 1 - m;      // forward lines of this team
    const int nsteps = 2 * len + (team == 0 ? 1 : 0);   // forward, [middle], backward

    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw);           // [0,1] team ping-pong, [2] middle, [3] x_m
    V *sY = reinterpret_cast<V *>(smem_raw + 32);                       // [2][R][nzp]  C * (line vector)
    V *sMid = sY + 2 * (size_t)R * nzp;                                 // [2][R][nzp]  C y_{m-1}, C y_{m+1}
    V *sX = sMid + 2 * (size_t)R * nzp;                                 // [R][nzp]     C x_m
    V *sG = sX + (size_t)R * nzp;                                       // pf: [2][rpc][nzp]; else [rpc][kcp]
    V *sOwn = sG + (MT > 0 ? 0 : (pf ? 2 * (size_t)rpc * nzp : (size_t)rpc * kcp));   // [2][R][rpc]: own rows
    constexpr int RP = 16 * (MT > 0 ? MT : 1) + 2;   // tensor path: padded row count of the partials
    // tensor / FMA partial sums: [step parity][8 warps (FM: 16 lane halves)][MMA_RHS][RP]
    float2 *red = reinterpret_cast<float2 *>(sOwn + 2 * (size_t)R * rpc);
    __shared__ int s_abort;

    const V *Gs = a.G + (size_t)sys * nx * nz * nz;
    double2 *Xs = a.X + ((size_t)sys * a.nrhs + q0) * N;
    V *Ys = a.Y + ((size_t)sys * a.nrhs + q0) * N;
    const uint32_t vec_bytes = (uint32_t)(nz * Rc * sizeof(V));
    const TG c_in = (TG)coup_x(g, 1), c_edge = (TG)coup_x(g, 0);
    const int lane = tid & 31, wid = tid >> 5;
    const int tpo = a.tpo, ngrp = SW_THREADS / tpo;
    const int pr = tid / tpo, part = tid % tpo;        // output group, K part
    const bool fp32 = sizeof(TG) == 4;

    // step kinds: 0 forward, 1 middle (left team), 2 backward
    auto kind_of = [&](int s) { return s < len ? 0 : ((team == 0 && s == len) ? 1 : 2); };
    auto line_of = [&](int s) {
        if (s < len) return team == 0 ? s : nx - 1 - s;
        if (team == 0) return s == len ? m : m - (s - len);
        return m + 1 + (s - len);
    };
    auto bwd_index = [&](int s) { return team == 0 ? s - len - 1 : s - len; };   // 0 for the first backward step

    // a refinement that has already finished leaves the rest of its enqueued sweeps empty; every
    // CTA reads the same flag (written by an earlier launch) and leaves before any cluster sync
    if (a.skip && *a.skip) return;
    // a converged system: every CTA of the cluster works on the same system and leaves together
    if (a.frozen && a.frozen[2 * sys]) return;
    if (tid == 0) {
        for (int b = 0; b < 4; ++b) mbar_init(&bars[b], 1);
        fence_mbar_init_cluster();
        s_abort = 0;
    }
    __syncthreads();
    cluster_sync_all();   // every mbarrier of the cluster is initialised before any push
    uint32_t ph0 = 0, ph1 = 0;

    auto prefetch = [&](int s) {
        if (s >= nsteps) return;
        const int i = line_of(s);
        if (MT == 0 || kind_of(s) == 2) {   // own rows of line i: G_i b_i (forward, middle) or y_i (backward)
            V *dst = sOwn + (size_t)(s & 1) * R * rpc;
            for (int q = wid; q < Rc; q += SW_THREADS / 32)
                for (int r = lane; r < nrows; r += 32)
                    cp_async_elem(dst + (size_t)q * rpc + r, Ys + (size_t)q * N + (size_t)i * nz + r0 + r);
        }
        if (MT > 0 || !pf || s == 0) return;   // the first forward line needs no product
        const V *src = Gs + (size_t)i * nz * nz + (size_t)r0 * nz;
        V *dst = sG + (size_t)(s & 1) * rpc * nzp;
        if (sizeof(TG) == 4 && (nz & 1) == 0) {
            for (int r = wid; r < nrows; r += SW_THREADS / 32)
                for (int b = 2 * lane; b < nz; b += 64) cp_async16(dst + (size_t)r * nzp + b, src + (size_t)r * nz + b);
        } else {
            for (int r = wid; r < nrows; r += SW_THREADS / 32)
                for (int b = lane; b < nz; b += 32) cp_async_elem(dst + (size_t)r * nzp + b, src + (size_t)r * nz + b);
        }
    };

    // tensor path: this warp's fragments of the G_i slab, rows g and g + 8 of each m tile,
    // complex columns 8j + 2t, 8j + 2t + 1 of the blocks j = wid, wid + 8, ...
    const int fg = lane >> 2, ft = lane & 3;
    const int NP = (nz + 7) >> 3;
    float4 gfr[MT > 0 ? MT : 1][2][KP > 0 ? KP : 1];
    float4 bfr[KP > 0 ? KP : 1];   // b_i (forward and middle lines): rhs fg, columns 8j + 2t, 8j + 2t + 1
    const V *Bs = a.B + ((size_t)sys * a.nrhs + q0) * N;
    // FMA product: lane (frow, fh) holds row frow, complex columns fc0 .. fc0 + 4*KP - 1
    const int frow = lane & 15, fh = lane >> 4;
    const int fc0 = KP == 2 ? 8 * (wid + 8 * fh) : 8 * wid + 4 * fh;
    float4 gq[FM ? 2 * KP : 1], gcur[FM ? 2 * KP : 1];
    auto load_g = [&](int s1) {
        if constexpr (FM) {
            if (s1 >= nsteps) return;
            const float2 *Gl = reinterpret_cast<const float2 *>(Gs) + ((size_t)line_of(s1) * nz + r0) * nz;
#pragma unroll
            for (int p = 0; p < 2 * KP; ++p) {
                const int c = fc0 + 2 * p;
                gq[p] = (frow < nrows && c < nz) ? __ldg(reinterpret_cast<const float4 *>(Gl + (size_t)frow * nz + c))
                                                 : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        } else if constexpr (MT > 0) {
            if (s1 >= nsteps) return;
            const int i1 = line_of(s1);
            const bool fwd1 = kind_of(s1) != 2;
            const float2 *Gl = reinterpret_cast<const float2 *>(Gs) + ((size_t)i1 * nz + r0) * nz;
            const float2 *Bl = reinterpret_cast<const float2 *>(Bs) + (size_t)fg * N + (size_t)i1 * nz;
#pragma unroll
            for (int jj = 0; jj < KP; ++jj) {
                const int j = wid + 8 * jj, kc = 8 * j + 2 * ft;
#pragma unroll
                for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int row = 16 * mt + fg + 8 * h;
                        gfr[mt][h][jj] = (j < NP && kc < nz && row < nrows)
                                             ? __ldg(reinterpret_cast<const float4 *>(Gl + (size_t)row * nz + kc))
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                bfr[jj] = (fwd1 && j < NP && kc < nz && fg < Rc) ? __ldg(reinterpret_cast<const float4 *>(Bl + kc))
                                                               : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    };

    // this thread's outputs, fixed for the whole sweep: right-hand side oq and slab row orow of
    // output o = pr + u * ngrp, the row's coupling to the next line, and its offsets
    constexpr int NOPT = MT > 0 ? 1 : SW_MAXOPT;
    bool ov[NOPT];
    int oq[NOPT], orow[NOPT];
    TG ocoef[NOPT];
    uint32_t obyte[NOPT];   // byte offset of the output in a [R][nzp] line buffer
    size_t ogl[NOPT];       // element offset of the output in Y / X, less i * nz
#pragma unroll
    for (int u = 0; u < NOPT; ++u) {
        const int o = pr + u * ngrp;
        ov[u] = o < nout;
        oq[u] = ov[u] ? o / nrows : 0;
        orow[u] = ov[u] ? o % nrows : 0;
        const int j = r0 + orow[u];
        ocoef[u] = (j == 0 || j == nz - 1) ? c_edge : c_in;
        obyte[u] = (uint32_t)(((size_t)oq[u] * nzp + j) * sizeof(V));
        ogl[u] = (size_t)oq[u] * N + j;
    }
    // rows computed in the previous step: the right team's first backward line is the line
    // of its last forward step, whose values the prefetch (issued before they were stored)
    // cannot see
    V vlast[NOPT];
#pragma unroll
    for (int u = 0; u < NOPT; ++u) vlast[u] = mkc<TG>(TG(0), TG(0));
    // tensor path with few fragments: the TF32 splits of this step's G_i fragments and the
    // loads of the next step's are made at the top of the step, while the team's pushes are
    // still in flight; larger tiles split inside the product (register budget)
    constexpr bool kPreSplit = !FM && MT > 0 && MT * KP <= 2;
    uint32_t ahs[kPreSplit ? MT : 1][kPreSplit ? KP : 1][2][4], als[kPreSplit ? MT : 1][kPreSplit ? KP : 1][2][4];
    float4 bcur[KP > 0 ? KP : 1];
    if constexpr (FM) {   // input of the first forward line: -b (no predecessor pushes to it)
        const int i0 = line_of(0);
        for (int e = tid; e < Rc * nz; e += SW_THREADS) {
            const int q = e / nz, k = e % nz;
            const V b = Bs[(size_t)q * N + (size_t)i0 * nz + k];
            sY[(size_t)q * nzp + k] = mkc<TG>(-b.x, -b.y);
        }
        __syncthreads();
    }
    V bpush = mkc<TG>(TG(0), TG(0));   // FM: b of the line the push of this step feeds
    // MT > 0: own rows y_i of this and of the next backward step, loaded a step ahead by the
    // K part 0 of each output (the thread that stored them on the forward pass)
    V ycur = mkc<TG>(TG(0), TG(0)), ypre = ycur;
    prefetch(0);
    cp_async_commit();
    load_g(0);
    for (int s = 0; s < nsteps; ++s) {
        const int kind = kind_of(s);
        const int i = line_of(s);
        const int bi = (kind == 2) ? bwd_index(s) : -1;
        if constexpr (kPreSplit) {
#pragma unroll
            for (int jj = 0; jj < KP; ++jj) {
#pragma unroll
                for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const float4 ga = gfr[mt][0][jj], gb = gfr[mt][1][jj];
                        split_tf32(c ? ga.z : ga.x, ahs[mt][jj][c][0], als[mt][jj][c][0]);
                        split_tf32(c ? gb.z : gb.x, ahs[mt][jj][c][1], als[mt][jj][c][1]);
                        split_tf32(c ? ga.w : ga.y, ahs[mt][jj][c][2], als[mt][jj][c][2]);
                        split_tf32(c ? gb.w : gb.y, ahs[mt][jj][c][3], als[mt][jj][c][3]);
                    }
                bcur[jj] = bfr[jj];
            }
            load_g(s + 1);
        }
        if constexpr (FM) {   // a forward or middle consumer takes C y - b of its line
#pragma unroll
            for (int p = 0; p < 2 * KP; ++p) gcur[p] = gq[p];
            load_g(s + 1);   // next line's slab: in flight for a whole step
            bpush = mkc<TG>(TG(0), TG(0));
            if (ov[0] && s + 1 < nsteps && kind_of(s + 1) != 2)
                bpush = Bs[(size_t)oq[0] * N + (size_t)line_of(s + 1) * nz + r0 + orow[0]];
        }
        if constexpr (MT > 0) {
            ycur = ypre;
            ypre = mkc<TG>(TG(0), TG(0));
            if (part == 0 && ov[0] && s + 1 < nsteps && kind_of(s + 1) == 2 && !(team == 1 && bwd_index(s + 1) == 0))
                ypre = Ys[ogl[0] + (size_t)line_of(s + 1) * nz];
        }
        // input vector of the product: none (first forward line), the middle buffers, the
        // x_m buffer (first backward line) or the team ping-pong buffer
        const V *tin = nullptr;
        const V *tin2 = nullptr;
        if (!(kind == 0 && s == 0)) {
            uint64_t *bar;
            uint32_t bytes = vec_bytes, par;
            if (kind == 1) { bar = &bars[2]; bytes = vec_bytes * (uint32_t)teams; par = 0; }
            else if (kind == 2 && bi == 0) { bar = &bars[3]; par = 0; }
            else { bar = &bars[s & 1]; par = (s & 1) ? ph1 : ph0; }
            if (tid == 0) mbar_arrive_expect_tx(bar, bytes);
            // tensor and FMA products: every thread waits for the inputs itself, with no CTA
            // barrier at the top of the step (the own rows come from registers); the CUDA-core
            // product also needs the slab its threads prefetched, behind the barrier below
            if (MT > 0 || tid == 0) {
                if (!mbar_wait_or_abort(bar, par, a.tries, &s_abort)) {
                    atomicOr(a.status, ST_TIMEOUT);
                    // the first thread of the CTA to give up stops the whole cluster
                    if (atomicExch(&s_abort, 1) == 0) cluster_abort_broadcast(&s_abort, (unsigned)(teams * cs));
                }
            }
        }
        if (!(kind == 0 && s == 0) && kind != 1 && !(kind == 2 && bi == 0)) {
            if (s & 1) ph1 ^= 1u; else ph0 ^= 1u;
        }
        if (kind == 1) { tin = sMid; tin2 = (teams == 2) ? sMid + (size_t)R * nzp : nullptr; }
        else if (kind == 2 && bi == 0) tin = sX;
        else if (FM || !(kind == 0 && s == 0)) tin = sY + (size_t)(s & 1) * R * nzp;
        const bool final_line = (kind != 0);
        if constexpr (MT == 0) {
            cp_async_wait<0>();
            // step s operands landed; every thread is done with step s - 1; the abort word
            // (which another CTA may set at any time) is read once for the whole CTA
            if (__syncthreads_or(*(volatile int *)&s_abort)) break;
            prefetch(s + 1);   // into the staging buffers that step s - 1 used
            cp_async_commit();
        }
        if (tin2) {
            // middle line: t = C y_{m-1} + C y_{m+1}
            V *tsum = const_cast<V *>(tin);
            for (int q = wid; q < Rc; q += SW_THREADS / 32)
                for (int j = lane; j < nz; j += 32) {
                    const V u1 = tin2[(size_t)q * nzp + j];
                    V &u0 = tsum[(size_t)q * nzp + j];
                    u0.x += u1.x;
                    u0.y += u1.y;
                }
            __syncthreads();
        }
        V yown[NOPT], acc[NOPT];
        const bool same_line = (team == 1 && kind == 2 && bi == 0);
#pragma unroll
        for (int u = 0; u < NOPT; ++u) {
            // the tensor path folds b_i into its forward product: v = 0 - G_i (t - b_i)
            if constexpr (MT > 0) {
                V yb = ycur;   // from the output's K part 0 (adjacent lanes)
                yb.x = __shfl_sync(0xffffffffu, yb.x, lane & ~(tpo - 1));
                yb.y = __shfl_sync(0xffffffffu, yb.y, lane & ~(tpo - 1));
                yown[u] = (ov[u] && kind == 2) ? (same_line ? vlast[u] : yb) : mkc<TG>(TG(0), TG(0));
            } else {
                yown[u] = ov[u] ? (same_line ? vlast[u] : sOwn[(size_t)(s & 1) * R * rpc + oq[u] * rpc + orow[u]])
                                : mkc<TG>(TG(0), TG(0));
            }
            acc[u] = mkc<TG>(TG(0), TG(0));
        }
        // partial sums of this step: alternate buffers, so that a warp that starts step s + 1
        // early cannot overwrite partials another warp is still summing
        float2 *redb = red + (size_t)(s & 1) * (FM ? 16 : 8) * MMA_RHS * RP;
        if constexpr (FM) {
            float2 facc[MMA_RHS];
#pragma unroll
            for (int q = 0; q < MMA_RHS; ++q) facc[q] = make_float2(0.f, 0.f);
            const float2 *tv = reinterpret_cast<const float2 *>(tin);
            if (Rc > 4) fma_product<8, KP>(tv, nzp, fc0, nz, Rc, gcur, facc);
            else if (Rc > 2) fma_product<4, KP>(tv, nzp, fc0, nz, Rc, gcur, facc);
            else if (Rc > 1) fma_product<2, KP>(tv, nzp, fc0, nz, Rc, gcur, facc);
            else fma_product<1, KP>(tv, nzp, fc0, nz, Rc, gcur, facc);
            // partial products of this lane's K part -> red[2 * wid + fh][rhs][row]
#pragma unroll
            for (int q = 0; q < MMA_RHS; ++q)
                if (q < Rc) redb[((size_t)(2 * wid + fh) * MMA_RHS + q) * RP + frow] = facc[q];
            if (__syncthreads_or(*(volatile int *)&s_abort)) break;   // a wait of the cluster gave up
            if (ov[0]) {
                const int q = oq[0], r = orow[0], wpp = 16 / tpo;
                float2 sum = make_float2(0.f, 0.f);
                for (int w = part * wpp; w < (part + 1) * wpp; ++w) {
                    const float2 v = redb[((size_t)w * MMA_RHS + q) * RP + r];
                    sum.x += v.x;
                    sum.y += v.y;
                }
                acc[0].x = sum.x;
                acc[0].y = sum.y;
            }
        } else if constexpr (MT > 0) {
            {
                const bool fwd = kind != 2;
                float accB[MT][2][4], accS[MT][2][4];   // hi*hi and the two cross terms
#pragma unroll
                for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                    for (int n = 0; n < 2; ++n)
#pragma unroll
                        for (int e = 0; e < 4; ++e) accB[mt][n][e] = accS[mt][n][e] = 0.f;
                const float2 *tv = reinterpret_cast<const float2 *>(tin);
#pragma unroll
                for (int jj = 0; jj < KP; ++jj) {
                    const int j = wid + 8 * jj, kc = 8 * j + 2 * ft;
                    if (j >= NP) break;   // warp-uniform
                    float4 xv = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (tin && fg < Rc && kc < nz) xv = *reinterpret_cast<const float4 *>(tv + (size_t)fg * nzp + kc);
                    if (fwd) {   // product input t - b_i
                        const float4 bv = kPreSplit ? bcur[jj] : bfr[jj];
                        xv.x -= bv.x; xv.y -= bv.y; xv.z -= bv.z; xv.w -= bv.w;
                    }
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        uint32_t xr_h, xr_l, xi_h, xi_l;
                        split_tf32(c ? xv.z : xv.x, xr_h, xr_l);
                        split_tf32(c ? xv.w : xv.y, xi_h, xi_l);
                        const uint32_t nxi_h = xi_h ^ 0x80000000u, nxi_l = xi_l ^ 0x80000000u;
#pragma unroll
                        for (int mt = 0; mt < MT; ++mt) {
                            uint32_t ah[4], al[4];
                            if constexpr (kPreSplit) {
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    ah[e] = ahs[mt][jj][c][e];
                                    al[e] = als[mt][jj][c][e];
                                }
                            } else {
                                const float4 ga = gfr[mt][0][jj], gb = gfr[mt][1][jj];
                                split_tf32(c ? ga.z : ga.x, ah[0], al[0]);   // row g,     Re G
                                split_tf32(c ? gb.z : gb.x, ah[1], al[1]);   // row g + 8, Re G
                                split_tf32(c ? ga.w : ga.y, ah[2], al[2]);   // row g,     Im G
                                split_tf32(c ? gb.w : gb.y, ah[3], al[3]);   // row g + 8, Im G
                            }
                            mma_tf32(accB[mt][0], ah, xr_h, nxi_h);      // Re: Re G Re t - Im G Im t
                            mma_tf32(accS[mt][0], ah, xr_l, nxi_l);
                            mma_tf32(accS[mt][0], al, xr_h, nxi_h);
                            mma_tf32(accB[mt][1], ah, xi_h, xr_h);       // Im: Re G Im t + Im G Re t
                            mma_tf32(accS[mt][1], ah, xi_l, xr_l);
                            mma_tf32(accS[mt][1], al, xi_h, xr_h);
                        }
                    }
                }
                // this warp's partial products (its K blocks) -> red[wid][rhs][row]
#pragma unroll
                for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int row = 16 * mt + fg + 8 * (e >> 1), q = 2 * ft + (e & 1);
                        redb[((size_t)wid * MMA_RHS + q) * RP + row] =
                            make_float2(accB[mt][0][e] + accS[mt][0][e], accB[mt][1][e] + accS[mt][1][e]);
                    }
            }
            if constexpr (!kPreSplit) load_g(s + 1);   // next line's fragments, in flight during the exchange
            {
                if (__syncthreads_or(*(volatile int *)&s_abort)) break;   // a wait of the cluster gave up
                if (ov[0]) {
                    const int q = oq[0], r = orow[0], wpp = 8 / tpo;
                    float2 sum = make_float2(0.f, 0.f);
                    for (int w = part * wpp; w < (part + 1) * wpp; ++w) {
                        const float2 v = redb[((size_t)w * MMA_RHS + q) * RP + r];
                        sum.x += v.x;
                        sum.y += v.y;
                    }
                    acc[0].x = sum.x;
                    acc[0].y = sum.y;
                }
            }
        } else if (tin) {
            if (pf) {
                const V *Gb = sG + (size_t)(s & 1) * rpc * nzp;
#pragma unroll
                for (int u = 0; u < NOPT; ++u) {
                    if (ov[u])
                        acc[u] = dot_row_il(Gb + (size_t)orow[u] * nzp, tin + (size_t)oq[u] * nzp, nz, part, tpo);
                }
            } else {
                const V *Gi = Gs + (size_t)i * nz * nz;
                for (int kc = 0; kc < nz; kc += SW_KC) {
                    const int kw = min(SW_KC, nz - kc);
                    for (int r = wid; r < nrows; r += SW_THREADS / 32)
                        for (int b = lane; b < kw; b += 32) sG[(size_t)r * kcp + b] = Gi[(size_t)(r0 + r) * nz + kc + b];
                    __syncthreads();
#pragma unroll
                    for (int u = 0; u < NOPT; ++u) {
                        if (ov[u]) {
                            const V d = dot_row_il(sG + (size_t)orow[u] * kcp, tin + (size_t)oq[u] * nzp + kc,
                                                   kw, part, tpo);
                            acc[u].x += d.x;
                            acc[u].y += d.y;
                        }
                    }
                    __syncthreads();
                }
            }
        }
        // the K parts of every output meet in adjacent lanes
        for (int mm = 1; mm < tpo; mm <<= 1) {
#pragma unroll
            for (int u = 0; u < NOPT; ++u) {
                acc[u].x += __shfl_xor_sync(0xffffffffu, acc[u].x, mm);
                acc[u].y += __shfl_xor_sync(0xffffffffu, acc[u].y, mm);
            }
        }
        // where the new rows go: the team's next buffer, the middle buffers of the left team
        // (last forward line), or the x_m buffer of every CTA (middle line)
        V *dstbuf = nullptr;
        uint64_t *dstbar = nullptr;
        int t_lo = team * cs, t_hi = team * cs + cs;
        if (kind == 0 && s == len - 1) {
            dstbuf = sMid + (size_t)team * R * nzp; dstbar = &bars[2]; t_lo = 0; t_hi = cs;
        } else if (kind == 1) {
            dstbuf = sX; dstbar = &bars[3]; t_lo = 0; t_hi = teams * cs;
        } else if (s + 1 < nsteps) {
            dstbuf = sY + (size_t)((s + 1) & 1) * R * nzp; dstbar = &bars[(s + 1) & 1];
        }
        const uint32_t lbar = dstbar ? smem_u32(dstbar) : 0u;
        const uint32_t lbuf = dstbuf ? smem_u32(dstbuf) : 0u;
#pragma unroll
        for (int u = 0; u < NOPT; ++u) {
            if (ov[u]) {
                const V v = mkc<TG>(yown[u].x - acc[u].x, yown[u].y - acc[u].y);
                vlast[u] = v;
                if (dstbuf) {
                    const V cv = FM ? mkc<TG>(ocoef[u] * v.x - bpush.x, ocoef[u] * v.y - bpush.y)
                                    : mkc<TG>(ocoef[u] * v.x, ocoef[u] * v.y);
                    const uint32_t la = lbuf + obyte[u];
                    for (int t = t_lo + part; t < t_hi; t += tpo)
                        st_async(mapa_u32(la, (uint32_t)t), cv, mapa_u32(lbar, (uint32_t)t));
                }
                if (part == 0) {
                    const size_t off = ogl[u] + (size_t)i * nz;
                    if (fp32 || !final_line) {
                        Ys[off] = v;   // complex FP32: the correction of the refinement
                    } else {
                        double2 d = make_double2((double)v.x, (double)v.y);
                        if (a.conj) d.y = -d.y;
                        Xs[off] = d;
                    }
                }
            }
        }
    }
    cp_async_wait<0>();
    // no CTA leaves while another can still push into it; after a give-up, pushes issued
    // before the abort word was seen are drained first
    __syncthreads();
    cluster_arrive();
    cluster_wait();
    if (*(volatile int *)&s_abort) abort_drain();
}

// Number of co-resident clusters of `cs` CTAs (0 if the size cannot be scheduled).
// Kernel attributes and occupancy queries are made once per (device, kernel, shape) and cached,
// so that host threads launching the same kernels do not keep changing their attributes.
cudaError_t ensure_nonportable_clusters(const void *fn) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, bool> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    bool &d = done[{dev, fn}];
    if (d) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) d = true;
    return e;
}

int max_active_clusters(const void *fn, int csz, int threads, size_t smem) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, int, int, size_t>, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return 0; }
    if (csz > 8 && ensure_nonportable_clusters(fn) != cudaSuccess) { cudaGetLastError(); return 0; }
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_tuple(dev, fn, csz, threads, smem);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csz, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csz;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    cache[key] = n;
    return n;
}

cudaError_t ensure_dyn_smem(const void *fn, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, size_t> limit;   // (device, kernel) -> bytes set
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    size_t &cur = limit[{dev, fn}];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

template <typename TG> using SweepFn = void (*)(SweepArgs<TG>);

// kernel of the tensor-pipe product with MT m tiles and KP K blocks per warp (null if none)
template <typename TG> SweepFn<TG> sweep_mma_fn(int MT, int KP, bool fm) {
    if constexpr (sizeof(TG) == 4) {
        if (fm && MT == 1 && KP == 1) return line_sweep_kernel<TG, 1, 1, true>;
        if (fm && MT == 1 && KP == 2) return line_sweep_kernel<TG, 1, 2, true>;
        if (MT == 1 && KP == 1) return line_sweep_kernel<TG, 1, 1, false>;
        if (MT == 1 && KP == 2) return line_sweep_kernel<TG, 1, 2, false>;
        if (MT == 2 && KP == 4) return line_sweep_kernel<TG, 2, 4, false>;
    }
    return nullptr;
}

template <typename TG>
cudaError_t launch_line_sweep(const GridGeom &g, int n_sys, int nrhs, const cx_t<TG> *G, const cx_t<TG> *B,
                              double2 *X, cx_t<TG> *Y, int conj, int rchunk, int *status, cudaStream_t st, int mid,
                              const int *skip, const int *frozen) {
    const int nz = g.nz;
    const size_t vsz = sizeof(cx_t<TG>);
    const int teams = (mid < g.nx - 1) ? 2 : 1;
    int cs = nz / 16;
    cs = cs < 1 ? 1 : (cs > 16 / teams ? 16 / teams : cs);
    // tuning overrides: CTAs per team and right-hand sides per cluster
    const char *env_cs = getenv("HELM_SWEEP_CS"), *env_r = getenv("HELM_SWEEP_R");
    if (env_cs && atoi(env_cs) > 0) cs = std::min(atoi(env_cs), 16 / teams);
    // HELM_SWEEP_CUDA_CORES=1 keeps complex-FP32 sweeps on the CUDA-core product
    const char *env_cc = getenv("HELM_SWEEP_CUDA_CORES");
    const bool allow_mma = !(env_cc && atoi(env_cc) > 0);
    // HELM_SWEEP_MMA=1 / =0 forces the tensor-pipe / FMA product where both cover the shape
    const char *env_mma = getenv("HELM_SWEEP_MMA");
    const int force_mma = (env_mma && *env_mma) ? (atoi(env_mma) > 0 ? 1 : 0) : -1;
    cudaError_t e;
    for (;;) {
        const int rpc = (nz + cs - 1) / cs;
        // threads per output (K split): as many as fit the CTA's 256 threads twice over
        auto tpo_of = [&](int R) {
            int t = 1;
            while (t < 8 && rpc * R * t * 2 <= SW_THREADS) t *= 2;
            return t;
        };
        auto smem_of = [&](int R, int pf) {
            const size_t nzp = (size_t)padded<TG>(nz, tpo_of(R)), kcp = (size_t)padded<TG>(SW_KC, tpo_of(R));
            return (size_t)32 + vsz * 5 * (size_t)R * nzp + (pf ? vsz * 2 * (size_t)rpc * nzp : vsz * (size_t)rpc * kcp) +
                   vsz * 2 * (size_t)R * rpc;
        };
        // right-hand sides per cluster (the chain is latency bound and the GPU otherwise
        // idle, so more clusters with fewer outputs each; 128 outputs per CTA measured best)
        int R = 1;
        while (R * 2 <= 16 && rpc * R * 2 <= 128) R *= 2;
        if (rchunk > 0 && R > rchunk) R = rchunk;
        if (env_r && atoi(env_r) > 0) R = atoi(env_r);
        if (R > nrhs) R = nrhs;
        if (R < 1) R = 1;
        while (R > 1 && rpc * R > SW_MAXOPT * SW_THREADS) R = (R + 1) / 2;
        int pf = 1;
        while (smem_of(R, pf) > SW_SMEM_MAX) {
            if (pf && R <= 4) pf = 0;
            else if (R > 1) R = (R + 1) / 2;
            else if (pf) pf = 0;
            else return cudaErrorInvalidConfiguration;
        }
        size_t smem = smem_of(R, pf);
        int tpo = tpo_of(R);
        SweepFn<TG> kfn = line_sweep_kernel<TG, 0, 0, false>;
        bool mma = false;
        // tensor-pipe product: complex FP32, even n_z (16-byte fragment loads), at most two m
        // tiles of rows per CTA and K blocks that the kernels below cover; one n tile of eight
        // right-hand sides per cluster
        {
            const int np = (nz + 7) / 8;
            int MT = 0, KP = 0;
            if (sizeof(TG) == 4 && allow_mma && (nz & 1) == 0) {
                if (rpc <= 16 && np <= 8) { MT = 1; KP = 1; }
                else if (rpc <= 16 && np <= 16) { MT = 1; KP = 2; }
                else if (rpc <= 32 && np <= 32) { MT = 2; KP = 4; }
            }
            int Rm = std::min(nrhs, MMA_RHS);
            if (rchunk > 0 && Rm > rchunk) Rm = rchunk;
            if (env_r && atoi(env_r) > 0) Rm = std::min(atoi(env_r), MMA_RHS);
            // one m tile of rows and few right-hand sides: the FMA product on the same
            // register-held slab (its cost grows with R; the tensor tile always pays for eight)
            const bool fm = MT == 1 && (force_mma < 0 ? Rm <= FM_MAX_RHS : force_mma == 0);
            SweepFn<TG> mfn = MT > 0 ? sweep_mma_fn<TG>(MT, KP, fm) : nullptr;
            if (mfn) {
                const size_t nzp = (size_t)padded_mma(nz);
                const size_t sm = (size_t)32 + vsz * 5 * (size_t)Rm * nzp + vsz * 2 * (size_t)Rm * rpc +
                                  2 * sizeof(float2) * (fm ? 16 : 8) * MMA_RHS * (size_t)(16 * MT + 2);
                if (sm <= SW_SMEM_MAX) {
                    kfn = mfn;
                    mma = true;
                    R = Rm;
                    smem = sm;
                    tpo = MT == 1 ? 2 : 1;   // outputs of the K halves (warps 0-3, 4-7) meet by shuffle
                    pf = 1;
                }
            }
        }
        const void *fn = (const void *)kfn;
        e = ensure_dyn_smem(fn, smem);
        if (e != cudaSuccess) return e;
        const int csz = teams * cs;
        if (csz > 8) {
            if (max_active_clusters(fn, csz, SW_THREADS, smem) == 0) {
                cudaGetLastError();
                cs = 8 / teams;
                continue;
            }
        }
        if (!mma) {   // CUDA-core sweep: Y_i = G_i b_i for all lines first
            const long blocks = (long)n_sys * g.nx * ((nz + PP_ROWS - 1) / PP_ROWS) * ((nrhs + PP_RHS - 1) / PP_RHS);
            HELM_TRACED(K_GBPRE, st, (line_gb_prepass_kernel<TG><<<(unsigned)blocks, 128, 0, st>>>(g, nrhs, G, B, Y, conj, skip, frozen)));
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        const int n_chunks = (nrhs + R - 1) / R;
        SweepArgs<TG> a{g, nrhs, R, cs, n_chunks, pf, tpo, mid, teams, G, B, X, Y, conj, status, skip, frozen, wait_tries()};
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(n_sys * n_chunks * csz, 1, 1);
        cfg.blockDim = dim3(SW_THREADS, 1, 1);
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
        HELM_TRACED(sizeof(TG) == 8 ? K_SWEEP64 : K_SWEEP32, st, (le = cudaLaunchKernelEx(&cfg, kfn, a)));
        return le;
    }
}

template cudaError_t launch_line_sweep<double>(const GridGeom &, int, int, const double2 *, const double2 *,
                                               double2 *, double2 *, int, int, int *, cudaStream_t, int,
                                               const int *, const int *);
template cudaError_t launch_line_sweep<float>(const GridGeom &, int, int, const float2 *, const float2 *,
                                              double2 *, float2 *, int, int, int *, cudaStream_t, int, const int *,
                                              const int *);


// ------------------------------------------------------------------ FP64 residual
// R = B - A X (A^H X for conj = 1) with the five-point operator, and per column the
// squared norms ||R||^2 and ||B||^2 accumulated into norms[col][0..1] (pre-zeroed).
// R32 (optional) receives conj?(R) in complex FP32: the right-hand side of the correction
// solve A delta = conj?(R) of the FP64 refinement tail (refine.cu).
constexpr int RES_THREADS = 256;

__global__ void __launch_bounds__(RES_THREADS) residual_kernel(GridGeom g, int nrhs, const double2 *diag,
                                                               const double2 *B, const double2 *X, float2 *R32,
                                                               double *norms, int conj, double cx_in, double cx_edge,
                                                               double cz_in, double cz_edge) {
    const int nx = g.nx, nz = g.nz, N = nx * nz;
    const int k = blockIdx.x * RES_THREADS + threadIdx.x;
    const int q = blockIdx.y, s = blockIdx.z;
    const size_t col = (size_t)s * nrhs + q;
    double rr = 0.0, bb = 0.0;
    if (k < N) {
        const int i = k / nz, j = k % nz;
        const double2 *x = X + col * N;
        double2 d = diag[(size_t)s * N + k];
        if (conj) d.y = -d.y;
        double2 xv = x[k];
        double2 ax = cmul(d, xv);
        const double cxj = (j == 0 || j == nz - 1) ? cx_edge : cx_in;   // grid couplings, precomputed
        const double czi = (i == 0 || i == nx - 1) ? cz_edge : cz_in;
        if (i > 0) { double2 v = x[k - nz]; ax.x += cxj * v.x; ax.y += cxj * v.y; }
        if (i < nx - 1) { double2 v = x[k + nz]; ax.x += cxj * v.x; ax.y += cxj * v.y; }
        if (j > 0) { double2 v = x[k - 1]; ax.x += czi * v.x; ax.y += czi * v.y; }
        if (j < nz - 1) { double2 v = x[k + 1]; ax.x += czi * v.x; ax.y += czi * v.y; }
        double2 b = B[col * N + k];
        double2 r = make_double2(b.x - ax.x, b.y - ax.y);
        if (R32) R32[col * N + k] = make_float2((float)r.x, conj ? -(float)r.y : (float)r.y);
        rr = r.x * r.x + r.y * r.y;
        bb = b.x * b.x + b.y * b.y;
    }
    for (int off = 16; off > 0; off >>= 1) {
        rr += __shfl_down_sync(0xffffffffu, rr, off);
        bb += __shfl_down_sync(0xffffffffu, bb, off);
    }
    __shared__ double s_r[RES_THREADS / 32], s_b[RES_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { s_r[wid] = rr; s_b[wid] = bb; }
    __syncthreads();
    if (wid == 0) {
        rr = lane < RES_THREADS / 32 ? s_r[lane] : 0.0;
        bb = lane < RES_THREADS / 32 ? s_b[lane] : 0.0;
        for (int off = 16; off > 0; off >>= 1) {
            rr += __shfl_down_sync(0xffffffffu, rr, off);
            bb += __shfl_down_sync(0xffffffffu, bb, off);
        }
        if (lane == 0 && norms) {
            atomicAdd(norms + 2 * col, rr);
            atomicAdd(norms + 2 * col + 1, bb);
        }
    }
}

cudaError_t launch_residual(const GridGeom &g, int n_sys, int nrhs, const double2 *diag, const double2 *B,
                            const double2 *X, float2 *R32, double *norms, int conj, cudaStream_t st) {
    const int N = g.nx * g.nz;
    dim3 grid((N + RES_THREADS - 1) / RES_THREADS, nrhs, n_sys);
    HELM_TRACED(K_RESIDUAL, st, (residual_kernel<<<grid, RES_THREADS, 0, st>>>(g, nrhs, diag, B, X, R32, norms, conj, coup_x(g, 1), coup_x(g, 0), coup_z(g, 1), coup_z(g, 0))));
    return cudaGetLastError();
}

}  // namespace helm
