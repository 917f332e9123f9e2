// Block forward/backward sweeps with the stored line inverses, and the FP64 residual.
//
// With G_i = S_i^{-1} from the line factorisation (factor.cu), A x = b is solved by
//   forward   y_0 = G_0 b_0,            y_i = G_i (b_i - C_i y_{i-1}),
//   backward  x_{nx-1} = y_{nx-1},      x_i = y_i - G_i C_{i+1} x_{i+1},
// two dense (n_z x n_z) x (n_z x R) products per line with all right-hand sides of a
// chunk as the product's N dimension.  The adjoint solve of A^H uses the same factor:
// A is complex symmetric, so (A^H)^{-1} b = conj(A^{-1} conj(b)).
//
// One thread-block cluster handles one (system, right-hand-side chunk); CTA r of the
// cluster owns a slab of rows of every line.  Line i+1 needs all rows of line i, so
// every line step ends with one hardware cluster barrier; the vector y_{i-1} (or
// x_{i+1}) is read back from global memory (L2) by every CTA of the cluster.
//
// Mixed precision: TG = float keeps the factor and the working vector in complex FP32;
// the input is an FP64 residual and the result is added to the FP64 iterate in the
// final pass (x += A~^{-1} r).  TG = double is the plain FP64 path (Y aliases X).
#include "kernels.h"

namespace helm {

constexpr int SW_THREADS = 256;
constexpr int SW_KC = 32;      // K chunk (columns of G_i / rows of t) staged in shared memory
constexpr int SW_MAXOPT = 4;   // outputs per thread (rows_per_cta * R <= 4 * 256)

template <typename TG> struct SweepArgs {
    GridGeom g;
    int nrhs, R, cs, n_chunks;
    const cx_t<TG> *G;   // [n_sys][nx][nz][nz]
    const double2 *B;    // [n_sys][nrhs][N]
    double2 *X;          // [n_sys][nrhs][N]
    cx_t<TG> *Y;         // working vector, [n_sys][nrhs][N] (== X for TG = double)
    int conj, accumulate;
};

template <typename TG> __device__ __forceinline__ cx_t<TG> in_cast(double2 a);
template <> __device__ __forceinline__ double2 in_cast<double>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 in_cast<float>(double2 a) { return to_c64(a); }

template <typename TG>
__global__ void __launch_bounds__(SW_THREADS) line_sweep_kernel(SweepArgs<TG> a) {
    using V = cx_t<TG>;
    const GridGeom g = a.g;
    const int nx = g.nx, nz = g.nz, N = nx * nz;
    const int tid = threadIdx.x;
    const int rank = (int)cluster_ctarank();
    const int cid = (int)cluster_id_x();
    const int sys = cid / a.n_chunks, chunk = cid % a.n_chunks;
    const int q0 = chunk * a.R;
    const int Rc = min(a.R, a.nrhs - q0);
    const int rpc = (nz + a.cs - 1) / a.cs;
    const int r0 = min(nz, rank * rpc), r1 = min(nz, r0 + rpc);
    const int nrows = r1 - r0;
    const int nout = nrows * Rc;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *sG = reinterpret_cast<V *>(smem_raw);        // rpc x SW_KC
    V *sT = sG + (size_t)rpc * SW_KC;               // SW_KC x R

    const V *Gs = a.G + (size_t)sys * nx * nz * nz;
    const double2 *Bs = a.B + ((size_t)sys * a.nrhs + q0) * N;
    double2 *Xs = a.X + ((size_t)sys * a.nrhs + q0) * N;
    V *Ys = a.Y + ((size_t)sys * a.nrhs + q0) * N;

    for (int pass = 0; pass < 2; ++pass) {
        const int i_lo = (pass == 0) ? 0 : nx - 2;
        const int i_hi = (pass == 0) ? nx : -1;
        const int di = (pass == 0) ? 1 : -1;
        for (int i = i_lo; i != i_hi; i += di) {
            const V *Gi = Gs + (size_t)i * nz * nz;
            V acc[SW_MAXOPT];
#pragma unroll
            for (int u = 0; u < SW_MAXOPT; ++u) acc[u] = mkc<TG>(TG(0), TG(0));
            for (int kc = 0; kc < nz; kc += SW_KC) {
                const int kw = min(SW_KC, nz - kc);
                for (int e = tid; e < nrows * kw; e += SW_THREADS) {
                    const int r = e / kw, b = e % kw;
                    sG[r * SW_KC + b] = Gi[(size_t)(r0 + r) * nz + kc + b];
                }
                for (int e = tid; e < kw * Rc; e += SW_THREADS) {
                    const int b = e / Rc, q = e % Rc;
                    const int j = kc + b;
                    V t;
                    if (pass == 0) {
                        double2 bv = Bs[(size_t)q * N + (size_t)i * nz + j];
                        if (a.conj) bv.y = -bv.y;
                        t = in_cast<TG>(bv);
                        if (i > 0) {
                            const TG c = (TG)coup_x(g, j);
                            V yp = ldcg(Ys + (size_t)q * N + (size_t)(i - 1) * nz + j);
                            t.x -= c * yp.x;
                            t.y -= c * yp.y;
                        }
                    } else {
                        const TG c = (TG)coup_x(g, j);
                        V xn = ldcg(Ys + (size_t)q * N + (size_t)(i + 1) * nz + j);
                        t = mkc<TG>(c * xn.x, c * xn.y);
                    }
                    sT[b * a.R + q] = t;
                }
                __syncthreads();
#pragma unroll
                for (int u = 0; u < SW_MAXOPT; ++u) {
                    const int o = tid + u * SW_THREADS;
                    if (o < nout) {
                        const int r = o / Rc, q = o % Rc;
                        V s = acc[u];
                        for (int b = 0; b < kw; ++b) cfma(s, sG[r * SW_KC + b], sT[b * a.R + q]);
                        acc[u] = s;
                    }
                }
                __syncthreads();
            }
#pragma unroll
            for (int u = 0; u < SW_MAXOPT; ++u) {
                const int o = tid + u * SW_THREADS;
                if (o < nout) {
                    const int r = o / Rc, q = o % Rc;
                    V *dst = Ys + (size_t)q * N + (size_t)i * nz + r0 + r;
                    if (pass == 0) {
                        *dst = acc[u];
                    } else {
                        V y = *dst;
                        *dst = mkc<TG>(y.x - acc[u].x, y.y - acc[u].y);
                    }
                }
            }
            cluster_sync_all();
        }
    }
    // final pass over this CTA's rows: conjugate (adjoint) and, for the mixed path,
    // promote to FP64 and add to the iterate
    for (int e = tid; e < nx * nrows * Rc; e += SW_THREADS) {
        const int q = e / (nx * nrows);
        const int rem = e % (nx * nrows);
        const int i = rem / nrows, r = rem % nrows;
        const size_t off = (size_t)q * N + (size_t)i * nz + r0 + r;
        V y = Ys[off];
        double2 d = make_double2((double)y.x, (double)y.y);
        if (a.conj) d.y = -d.y;
        if (a.accumulate) {
            double2 x = Xs[off];
            d.x += x.x;
            d.y += x.y;
        }
        Xs[off] = d;
    }
}

template <typename TG>
cudaError_t launch_line_sweep(const GridGeom &g, int n_sys, int nrhs, const cx_t<TG> *G, const double2 *B,
                              double2 *X, cx_t<TG> *Y, int conj, int accumulate, int cs, int rchunk,
                              cudaStream_t st) {
    const int rpc = (g.nz + cs - 1) / cs;
    int R = rchunk;
    while (R > 1 && rpc * R > SW_MAXOPT * SW_THREADS) R /= 2;
    if (R > nrhs) R = nrhs;
    const int n_chunks = (nrhs + R - 1) / R;
    SweepArgs<TG> a{g, nrhs, R, cs, n_chunks, G, B, X, Y, conj, accumulate};
    const size_t smem = sizeof(cx_t<TG>) * ((size_t)rpc * SW_KC + (size_t)SW_KC * R);
    cudaError_t e = cudaFuncSetAttribute(line_sweep_kernel<TG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_sys * n_chunks * cs, 1, 1);
    cfg.blockDim = dim3(SW_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, line_sweep_kernel<TG>, a);
}

template cudaError_t launch_line_sweep<double>(const GridGeom &, int, int, const double2 *, const double2 *,
                                               double2 *, double2 *, int, int, int, int, cudaStream_t);
template cudaError_t launch_line_sweep<float>(const GridGeom &, int, int, const float2 *, const double2 *,
                                              double2 *, float2 *, int, int, int, int, cudaStream_t);

// ------------------------------------------------------------------ FP64 residual
// R = B - A X (A^H X for conj = 1) with the five-point operator, and per column the
// squared norms ||R||^2 and ||B||^2 accumulated into norms[col][0..1] (pre-zeroed).
constexpr int RES_THREADS = 256;

__global__ void __launch_bounds__(RES_THREADS) residual_kernel(GridGeom g, int nrhs, const double2 *diag,
                                                               const double2 *B, const double2 *X, double2 *R,
                                                               double *norms, int conj) {
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
        const double cxj = coup_x(g, j), czi = coup_z(g, i);
        if (i > 0) { double2 v = x[k - nz]; ax.x += cxj * v.x; ax.y += cxj * v.y; }
        if (i < nx - 1) { double2 v = x[k + nz]; ax.x += cxj * v.x; ax.y += cxj * v.y; }
        if (j > 0) { double2 v = x[k - 1]; ax.x += czi * v.x; ax.y += czi * v.y; }
        if (j < nz - 1) { double2 v = x[k + 1]; ax.x += czi * v.x; ax.y += czi * v.y; }
        double2 b = B[col * N + k];
        double2 r = make_double2(b.x - ax.x, b.y - ax.y);
        if (R) R[col * N + k] = r;
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
                            const double2 *X, double2 *R, double *norms, int conj, cudaStream_t st) {
    const int N = g.nx * g.nz;
    dim3 grid((N + RES_THREADS - 1) / RES_THREADS, nrhs, n_sys);
    residual_kernel<<<grid, RES_THREADS, 0, st>>>(g, nrhs, diag, B, X, R, norms, conj);
    return cudaGetLastError();
}

}  // namespace helm
