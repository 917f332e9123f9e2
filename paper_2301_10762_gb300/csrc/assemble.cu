// Operator assembly, point-source right-hand sides and the sliding bicubic restriction.
#include <math.h>
#include "kernels.h"
#include "trace.h"

namespace helm {

// A(m, w) = S - w^2 diag(d m) - i w diag(b sqrt(m)) (Appendix "Numerical forward model",
// nodal quadrature).  Only the diagonal depends on (m, w); the off-diagonal couplings
// are the grid constants coup_x / coup_z.  For node (i, j):
//   S_kk = (hz/hx) w_z(j) [#x-neighbours] + (hx/hz) w_x(i) [#z-neighbours],
//   d_k  = hx hz q(i) q(j)                      (tensor trapezoid, q = 1/2 at ends; or the
//          triangles' vertex quadrature, lumped_mass),
//   b_k  = hx q(i) [j on top/bottom] + hz q(j) [i on left/right]  (boundary length).
__global__ void assemble_kernel(GridGeom g, const double *m, const double *omega, int n_omega, double2 *diag) {
    const int N = g.nx * g.nz;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int i = k / g.nz, j = k % g.nz;
    const double qx = edge_w(i, g.nx), qz = edge_w(j, g.nz);
    const double skk = (g.hz / g.hx) * qz * ((i > 0) + (i < g.nx - 1)) +
                       (g.hx / g.hz) * qx * ((j > 0) + (j < g.nz - 1));
    const double d = lumped_mass(g, i, j);
    double b = 0.0;
    if (j == 0 || j == g.nz - 1) b += g.hx * qx;
    if (i == 0 || i == g.nx - 1) b += g.hz * qz;
    const double mk = m[k];
    const double sq = sqrt(mk);
    for (int w = 0; w < n_omega; ++w) {
        const double om = omega[w];
        diag[(size_t)w * N + k] = make_double2(skk - om * om * d * mk, -om * b * sq);
    }
}

cudaError_t launch_assemble(const GridGeom &g, const double *m, const double *omega_dev, int n_omega,
                            double2 *diag, cudaStream_t st) {
    const int N = g.nx * g.nz;
    HELM_TRACED(K_ASSEMBLE, st, (assemble_kernel<<<(N + 255) / 256, 256, 0, st>>>(g, m, omega_dev, n_omega, diag)));
    return cudaGetLastError();
}

// g_k(w) = w^2 d_k + i w b_k / (2 sqrt(m_k)) and g'_k(w) = dg_k/dm_k = -i w b_k / (4 m_k^{3/2})
// per frequency and node (-dA/dm_k = g_k e_k e_k^T), once per operator: the FWI kernels use them
// for every right-hand side
__global__ void gcoef_kernel(GridGeom g, const double *m, const double *omega, int n_omega, double2 *gk,
                             double2 *gpk) {
    const int N = g.nx * g.nz;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int i = k / g.nz, j = k % g.nz;
    const double qx = edge_w(i, g.nx), qz = edge_w(j, g.nz);
    const double d = lumped_mass(g, i, j);
    double b = 0.0;
    if (j == 0 || j == g.nz - 1) b += g.hx * qx;
    if (i == 0 || i == g.nx - 1) b += g.hz * qz;
    const double mk = m[k], sq = sqrt(mk);
    for (int w = 0; w < n_omega; ++w) {
        const double om = omega[w];
        gk[(size_t)w * N + k] = make_double2(om * om * d, om * b / (2.0 * sq));
        gpk[(size_t)w * N + k] = make_double2(0.0, -om * b / (4.0 * mk * sq));
    }
}

cudaError_t launch_gcoef(const GridGeom &g, const double *m, const double *omega_dev, int n_omega, double2 *gk,
                         double2 *gpk, cudaStream_t st) {
    const int N = g.nx * g.nz;
    HELM_TRACED(K_GCOEF, st, (gcoef_kernel<<<(N + 255) / 256, 256, 0, st>>>(g, m, omega_dev, n_omega, gk, gpk)));
    return cudaGetLastError();
}

// e_s: value src_amp at a source on a node; off a node, bilinear weights of the four
// nodes of the containing cell.  B [n_omega][n_src][N] must be zeroed beforehand.
__global__ void sources_kernel(GridGeom g, int n_omega, int n_src, const double *src_xz, const double *amp,
                               double2 *B) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_src) return;
    const int N = g.nx * g.nz;
    const double tx = src_xz[2 * s] / g.hx, tz = src_xz[2 * s + 1] / g.hz;
    const int i0 = min(max((int)floor(tx), 0), g.nx - 2);
    const int j0 = min(max((int)floor(tz), 0), g.nz - 2);
    const double fx = tx - i0, fz = tz - j0;
    const double a = amp ? amp[s] : 1.0;
    for (int w = 0; w < n_omega; ++w) {
        double2 *b = B + ((size_t)w * n_src + s) * N;
        for (int di = 0; di < 2; ++di)
            for (int dj = 0; dj < 2; ++dj) {
                const double wt = a * (di ? fx : 1.0 - fx) * (dj ? fz : 1.0 - fz);
                if (wt != 0.0) {
                    double2 *p = b + (size_t)(i0 + di) * g.nz + (j0 + dj);
                    p->x += wt;
                }
            }
    }
}

cudaError_t launch_sources(const GridGeom &g, int n_omega, int n_src, const double *src_xz_dev,
                           const double *src_amp_dev, double2 *B, cudaStream_t st) {
    const int N = g.nx * g.nz;
    cudaError_t e = cudaMemsetAsync(B, 0, sizeof(double2) * (size_t)n_omega * n_src * N, st);
    if (e != cudaSuccess) return e;
    HELM_TRACED(K_SOURCES, st, (sources_kernel<<<(n_src + 127) / 128, 128, 0, st>>>(g, n_omega, n_src, src_xz_dev, src_amp_dev, B)));
    return cudaGetLastError();
}

// Sliding cubic (Section "Numerical restriction operator", Figs. fig:Cub1, fig:Cub2):
// along each axis the window of 4 nodes starting at clamp(floor(p/h) - 1, 0, n - 4),
// Lagrange cubic weights at the local coordinate s = p/h - i0; 2D taps are the tensor
// product.  The derivative taps differentiate one axis' weights (d/ds times 1/h).
__device__ void cubic_axis(double t, int n, int &i0, double L[4], double dL[4]) {
    int w = (int)floor(t) - 1;
    w = max(0, min(w, n - 4));
    i0 = w;
    const double s = t - w;
    const double a0 = s, a1 = s - 1.0, a2 = s - 2.0, a3 = s - 3.0;
    L[0] = -a1 * a2 * a3 / 6.0;
    L[1] = a0 * a2 * a3 / 2.0;
    L[2] = -a0 * a1 * a3 / 2.0;
    L[3] = a0 * a1 * a2 / 6.0;
    dL[0] = -(a2 * a3 + a1 * a3 + a1 * a2) / 6.0;
    dL[1] = (a2 * a3 + a0 * a3 + a0 * a2) / 2.0;
    dL[2] = -(a1 * a3 + a0 * a3 + a0 * a1) / 2.0;
    dL[3] = (a1 * a2 + a0 * a2 + a0 * a1) / 6.0;
}

__global__ void taps_kernel(GridGeom g, int n_rec, const double *rec_xz, int *idx, double *w, double *wx,
                            double *wz) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rec) return;
    int i0, j0;
    double Lx[4], dLx[4], Lz[4], dLz[4];
    cubic_axis(rec_xz[2 * r] / g.hx, g.nx, i0, Lx, dLx);
    cubic_axis(rec_xz[2 * r + 1] / g.hz, g.nz, j0, Lz, dLz);
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            const int t = r * 16 + a * 4 + b;
            idx[t] = (i0 + a) * g.nz + (j0 + b);
            w[t] = Lx[a] * Lz[b];
            wx[t] = dLx[a] / g.hx * Lz[b];
            wz[t] = Lx[a] * dLz[b] / g.hz;
        }
}

cudaError_t launch_restriction_taps(const GridGeom &g, int n_rec, const double *rec_xz_dev, int *tap_idx,
                                    double *tap_w, double *tap_wx, double *tap_wz, cudaStream_t st) {
    HELM_TRACED(K_TAPS, st, (taps_kernel<<<(n_rec + 63) / 64, 64, 0, st>>>(g, n_rec, rec_xz_dev, tap_idx, tap_w, tap_wx, tap_wz)));
    return cudaGetLastError();
}

// Y[col][r] = sum_t w_t X[col][idx_t]; one warp per (col, receiver), 16 taps.
__global__ void restrict_kernel(int N, int n_cols, int n_rec, const int *idx, const double *w, const double2 *X,
                                double2 *Y) {
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= n_cols * n_rec) return;
    const int col = gw / n_rec, r = gw % n_rec;
    double2 acc = make_double2(0.0, 0.0);
    if (lane < 16) {
        const int t = r * 16 + lane;
        const double2 v = X[(size_t)col * N + idx[t]];
        acc.x = w[t] * v.x;
        acc.y = w[t] * v.y;
    }
    for (int off = 8; off > 0; off >>= 1) {
        acc.x += __shfl_down_sync(0xffffffffu, acc.x, off);
        acc.y += __shfl_down_sync(0xffffffffu, acc.y, off);
    }
    if (lane == 0) Y[(size_t)col * n_rec + r] = acc;
}

cudaError_t launch_restrict(const GridGeom &g, int n_cols, int n_rec, const int *tap_idx, const double *tap_w,
                            const double2 *X, double2 *Y, cudaStream_t st) {
    const int N = g.nx * g.nz;
    const long warps = (long)n_cols * n_rec;
    const int blocks = (int)((warps * 32 + 255) / 256);
    if (blocks == 0) return cudaSuccess;
    HELM_TRACED(K_RESTRICT, st, (restrict_kernel<<<blocks, 256, 0, st>>>(N, n_cols, n_rec, tap_idx, tap_w, X, Y)));
    return cudaGetLastError();
}

}  // namespace helm
