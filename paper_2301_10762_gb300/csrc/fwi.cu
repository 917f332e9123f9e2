// FWI misfit / gradient (Algorithm alg:box1, Theorem th:grad), Hessian-vector products
// (Lemmas thm:H1, thm:H2, Discussion disc:Hess), PCG with P2 = Gamma(alpha0, mu)
// (Eq. (P2)) and the upper-level hypergradient (Algorithm alg:box, Theorems sogradt1,
// sogradta).  Every reduction here runs in a fixed order (block per output, partials
// combined in index order), so results are bitwise reproducible run to run.
#include <math.h>
#include <algorithm>
#include <string>
#include <thread>
#include <vector>

#include "helm.h"
#include "kernels.h"
#include "trace.h"
#include "abi_internal.h"

using namespace helm;

namespace helm {

// lumped mass d_k and boundary length b_k of node k (Appendix "Numerical forward model")
__device__ __forceinline__ void node_db(const GridGeom &g, int k, double &d, double &b) {
    const int i = k / g.nz, j = k % g.nz;
    const double qx = edge_w(i, g.nx), qz = edge_w(j, g.nz);
    d = lumped_mass(g, i, j);
    b = 0.0;
    if (j == 0 || j == g.nz - 1) b += g.hx * qx;
    if (i == 0 || i == g.nx - 1) b += g.hz * qz;
}

// g_k = w^2 d_k + i w b_k / (2 sqrt(m_k))   (-dA/dm_k = g_k e_k e_k^T)
__device__ __forceinline__ double2 g_of(double om, double d, double b, double mk) {
    return make_double2(om * om * d, om * b / (2.0 * sqrt(mk)));
}

// (R m)_k of R = D_x^T D_x + D_z^T D_z, D_n = (n-1) bidiag(1, -1) (Eq. (ThisGamma))
__device__ __forceinline__ double regR(const GridGeom &g, const double *v, int k) {
    const int i = k / g.nz, j = k % g.nz;
    const double sx = (double)(g.nx - 1) * (g.nx - 1), sz = (double)(g.nz - 1) * (g.nz - 1);
    const double vk = v[k];
    double r = 0.0;
    if (i > 0) r += sx * (vk - v[k - g.nz]);
    if (i < g.nx - 1) r += sx * (vk - v[k + g.nz]);
    if (j > 0) r += sz * (vk - v[k - 1]);
    if (j < g.nz - 1) r += sz * (vk - v[k + 1]);
    return r;
}

template <int NT> __device__ double block_sum(double v, double *sh) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; ++w) t += sh[w];
    __syncthreads();
    return t;  // valid in thread 0
}

// eps[col][r] = data[col][r] - (R u)[col][r]; phi_col[col] = 1/2 sum_r w_r^2 |eps|^2.
// Block per column, warp per receiver (16 taps), fixed-order reduction.
__global__ void misfit_kernel(int N, int n_rec, const int *idx, const double *tw, const double *rec_w,
                              const double2 *U, const double2 *data, double2 *eps, double *phi_col) {
    __shared__ double s_acc[32];
    const int col = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double acc = 0.0;
    for (int r = wid; r < n_rec; r += nw) {
        double2 v = make_double2(0.0, 0.0);
        if (lane < 16) {
            const int t = r * 16 + lane;
            const double2 u = U[(size_t)col * N + idx[t]];
            v.x = tw[t] * u.x;
            v.y = tw[t] * u.y;
        }
        for (int off = 8; off > 0; off >>= 1) {
            v.x += __shfl_down_sync(0xffffffffu, v.x, off);
            v.y += __shfl_down_sync(0xffffffffu, v.y, off);
        }
        if (lane == 0) {
            const double2 d = data[(size_t)col * n_rec + r];
            const double2 e = make_double2(d.x - v.x, d.y - v.y);
            if (eps) eps[(size_t)col * n_rec + r] = e;
            const double w = rec_w[r];
            acc += 0.5 * w * w * (e.x * e.x + e.y * e.y);
        }
    }
    if (lane == 0) s_acc[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += s_acc[w];
        phi_col[col] = t;
    }
}

// out[col][idx_t] += tw_t * s_r * z[col][r] for every receiver r, sequentially over r
// (a node may be shared by the windows of two receivers); s_r = rec_w[r]^2 or 1.
// Adjoint restriction R^T of Eq. (Rstar), discretised as the transpose of R(P).
__global__ void scatter_kernel(int N, int n_rec, const int *idx, const double *tw, const double *rec_w,
                               int square_w, const double2 *z, double2 *out) {
    const int col = blockIdx.x;
    for (int r = 0; r < n_rec; ++r) {
        if (threadIdx.x < 16) {
            const int t = r * 16 + threadIdx.x;
            double s = tw[t];
            if (rec_w) s *= square_w ? rec_w[r] * rec_w[r] : rec_w[r];
            const double2 zv = z[(size_t)col * n_rec + r];
            double2 *p = out + (size_t)col * N + idx[t];
            double2 o = *p;
            o.x += s * zv.x;
            o.y += s * zv.y;
            *p = o;
        }
        __syncthreads();
    }
}

// grad_k = -Re sum_{w,s} g_k u_k conj(lambda_k) + (Gamma m)_k; reg_part[block] = sum m_k (Gamma m)_k
__global__ void grad_kernel(GridGeom g, int n_omega, int n_src, const double *omega, const double *m,
                            const double2 *U, const double2 *Lam, double alpha, double mu, double *grad,
                            double *reg_part) {
    __shared__ double sh[32];
    const int N = g.nx * g.nz;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double reg = 0.0;
    if (k < N) {
        double d, b;
        node_db(g, k, d, b);
        const double mk = m[k];
        double acc = 0.0;
        for (int w = 0; w < n_omega; ++w) {
            const double2 gk = g_of(omega[w], d, b, mk);
            for (int s = 0; s < n_src; ++s) {
                const size_t o = ((size_t)w * n_src + s) * N + k;
                const double2 gu = cmul(gk, U[o]);
                const double2 l = Lam[o];
                acc -= gu.x * l.x + gu.y * l.y;  // Re(gu conj(l))
            }
        }
        const double gm = alpha * regR(g, m, k) + mu * mk;
        grad[k] = acc + gm;
        reg = 0.5 * mk * gm;
    }
    const double t = block_sum<256>(reg, sh);
    if (threadIdx.x == 0) reg_part[blockIdx.x] = t;
}

// grad_k = Re sum_{w,q} g_k(w) U_k conj(Lam_k): the m-gradient of a real functional of the
// wavefields from its adjoint fields (helm_field_grad)
__global__ void field_grad_kernel(GridGeom g, int n_omega, int nrhs, const double *omega, const double *m,
                                  const double2 *U, const double2 *Lam, double *grad) {
    const int N = g.nx * g.nz;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    double d, b;
    node_db(g, k, d, b);
    const double mk = m[k];
    double acc = 0.0;
    for (int w = 0; w < n_omega; ++w) {
        const double2 gk = g_of(omega[w], d, b, mk);
        for (int q = 0; q < nrhs; ++q) {
            const size_t o = ((size_t)w * nrhs + q) * N + k;
            const double2 gu = cmul(gk, U[o]);
            const double2 l = Lam[o];
            acc += gu.x * l.x + gu.y * l.y;   // Re(gu conj(l))
        }
    }
    grad[k] = acc;
}

// out[w][s][k] = g_k(w) u_k p_k   (right-hand side of v, Eq. (defv), and of tau, Eq. (tau_def))
__global__ void g_u_p_kernel(int N, int n_omega, int n_src, const double2 *gk, const double2 *U, const double *p,
                             double2 *out) {
    const size_t tot = (size_t)n_omega * n_src * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(e % N);
        const int w = (int)(e / ((size_t)n_src * N));
        out[e] = cscale(cmul(gk[(size_t)w * N + k], U[e]), p[k]);
    }
}

// out[w][s][k] = -p_k conj(g_k) lambda_k  (the G^* lambda term of z, Discussion disc:Hess)
__global__ void z_base_kernel(int N, int n_omega, int n_src, const double2 *gk, const double2 *Lam, const double *p,
                              double2 *out) {
    const size_t tot = (size_t)n_omega * n_src * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(e % N);
        const int w = (int)(e / ((size_t)n_src * N));
        out[e] = cscale(cmul(cconj(gk[(size_t)w * N + k]), Lam[e]), -p[k]);
    }
}

// (H p)_k = sum_{w,s} { Re[g u conj(z)] - Re[g v conj(lambda)] - Re[g' u conj(lambda)] p_k } + (Gamma p)_k,
// in two passes: part[c][k] sums the columns of chunk c (HESS_CHUNK columns, grid.y = chunk),
// hess_finish adds the chunks in order and the regulariser (fixed order: bitwise reproducible)
constexpr int HESS_CHUNK = 8;
__global__ void hess_acc_kernel(int N, int n_src, int cols, const double2 *gk, const double2 *gpk, const double2 *U,
                                const double2 *V, const double2 *Z, const double2 *Lam, const double *p,
                                int gauss_newton, double *part) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int c0 = blockIdx.y * HESS_CHUNK, c1 = min(cols, c0 + HESS_CHUNK);
    const double pk = p[k];
    double acc = 0.0;
    for (int c = c0; c < c1; ++c) {
        const int w = c / n_src;
        const size_t o = (size_t)c * N + k;
        const double2 g = gk[(size_t)w * N + k];
        const double2 u = U[o], z = Z[o];
        const double2 gu = cmul(g, u);
        acc += gu.x * z.x + gu.y * z.y;
        if (!gauss_newton) {
            const double2 l = Lam[o];
            const double2 gv = cmul(g, V[o]), gpu = cmul(gpk[(size_t)w * N + k], u);
            acc -= gv.x * l.x + gv.y * l.y;
            acc -= (gpu.x * l.x + gpu.y * l.y) * pk;
        }
    }
    part[(size_t)blockIdx.y * N + k] = acc;
}

__global__ void hess_finish_kernel(GridGeom g, int n_chunks, const double *part, const double *p, double alpha,
                                   double mu, double *Hp) {
    const int N = g.nx * g.nz;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    double acc = 0.0;
    for (int c = 0; c < n_chunks; ++c) acc += part[(size_t)c * N + k];
    Hp[k] = acc + alpha * regR(g, p, k) + mu * p[k];
}

// Hypergradient receiver terms for one model, accumulated into dp[r][2], dw[r]:
//   dp_{r,l} += w_r^2 Re[conj(dR_l tau) R(u - u') + conj(R tau) dR_l(u - u')],
//   dw_r    += -2 w_r Re[conj(R tau) R(u' - u)],
// with R(u - u') = R u - d and dR_l(u - u') = dR_l u - d_l, where d = R' u', d_l = dR'_l u' are
// the data and their receiver derivatives on the data's own grid (R' its restriction; the
// model's grid when the data come from it);
// scaled by inv_models; block per receiver, threads over (w, s) columns, fixed order.
__global__ void hyper_terms_kernel(int N, int n_cols, int n_rec, const int *idx, const double *tw,
                                   const double *twx, const double *twz, const double *rec_w, const double2 *T,
                                   const double2 *U, const double2 *d, const double2 *dx, const double2 *dz,
                                   double inv_models, double *dp, double *dw) {
    __shared__ double sh[32];
    const int r = blockIdx.x;
    double ax = 0.0, az = 0.0, aw = 0.0;
    for (int col = threadIdx.x; col < n_cols; col += blockDim.x) {
        double2 Rt = make_double2(0, 0), Rxt = Rt, Rzt = Rt, Ru = Rt, Rxu = Rt, Rzu = Rt;
        for (int t = 0; t < 16; ++t) {
            const int ti = r * 16 + t;
            const size_t o = (size_t)col * N + idx[ti];
            const double2 tv = T[o], uv = U[o];
            Rt.x += tw[ti] * tv.x;   Rt.y += tw[ti] * tv.y;
            Rxt.x += twx[ti] * tv.x; Rxt.y += twx[ti] * tv.y;
            Rzt.x += twz[ti] * tv.x; Rzt.y += twz[ti] * tv.y;
            Ru.x += tw[ti] * uv.x;   Ru.y += tw[ti] * uv.y;
            Rxu.x += twx[ti] * uv.x; Rxu.y += twx[ti] * uv.y;
            Rzu.x += twz[ti] * uv.x; Rzu.y += twz[ti] * uv.y;
        }
        const size_t q = (size_t)col * n_rec + r;
        const double2 Rd = make_double2(Ru.x - d[q].x, Ru.y - d[q].y);      // R(u - u')
        const double2 Rxd = make_double2(Rxu.x - dx[q].x, Rxu.y - dx[q].y);  // dR_x(u - u')
        const double2 Rzd = make_double2(Rzu.x - dz[q].x, Rzu.y - dz[q].y);  // dR_z(u - u')
        ax += (Rxt.x * Rd.x + Rxt.y * Rd.y) + (Rt.x * Rxd.x + Rt.y * Rxd.y);
        az += (Rzt.x * Rd.x + Rzt.y * Rd.y) + (Rt.x * Rzd.x + Rt.y * Rzd.y);
        aw += Rt.x * Rd.x + Rt.y * Rd.y;   // Re[conj(R tau) R(u - u')]
    }
    const double w = rec_w[r];
    const double sx = block_sum<256>(ax, sh);
    const double sz = block_sum<256>(az, sh);
    const double sw = block_sum<256>(aw, sh);
    if (threadIdx.x == 0) {
        dp[2 * r] += inv_models * w * w * sx;
        dp[2 * r + 1] += inv_models * w * w * sz;
        dw[r] += inv_models * 2.0 * w * sw;
    }
}

// --------------------------------------------------------------- vector kernels
// partial[block] = sum over the block's slice of a_k * b_k (fixed order)
__global__ void dot_partial_kernel(int n, const double *a, const double *b, double *partial) {
    __shared__ double sh[32];
    double v = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) v += a[k] * b[k];
    const double t = block_sum<256>(v, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// out[j] = sum_{i < n_part} partial[j*stride + i]  (single thread per output, fixed order)
__global__ void sum_partials_kernel(int n_out, int n_part, const double *partial, double *out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_out) return;
    double t = 0.0;
    for (int i = 0; i < n_part; ++i) t += partial[(size_t)j * n_part + i];
    out[j] = t;
}

// y = a*x + b*y
__global__ void axpby_kernel(int n, double a, const double *x, double b, double *y) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) y[k] = a * x[k] + b * y[k];
}

// PCG step with the scalars on the device: a = rz / pHp (0 if pHp = 0), x += a p, r -= a Hp
__global__ void cg_step_kernel(int n, const double *rz, const double *php, const double *p, const double *hp,
                               double *x, double *r) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double den = *php, a = den != 0.0 ? *rz / den : 0.0;
    x[k] = a * p[k] + 1.0 * x[k];
    r[k] = -a * hp[k] + 1.0 * r[k];
}

// PCG direction with the scalars on the device: p = z + (rz_new / rz) p (beta 0 if rz = 0)
__global__ void cg_dir_kernel(int n, const double *z, const double *rz_new, const double *rz, double *p) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double den = *rz, beta = den != 0.0 ? *rz_new / den : 0.0;
    p[k] = 1.0 * z[k] + beta * p[k];
}

__global__ void fill_kernel(int n, double v, double *y) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) y[k] = v;
}

// out_k = a_k - b_k
__global__ void sub_kernel(int n, const double *a, const double *b, double *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = a[k] - b[k];
}

// out_k = (R v)_k  (regulariser product, for dpsi/dalpha)
__global__ void regR_kernel(GridGeom g, const double *v, double *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < g.nx * g.nz) out[k] = regR(g, v, k);
}

// ------------------------------------------------------ P2^{-1} by the 2D DCT-II
// R = (nx-1)^2 L_nx (x) I + (nz-1)^2 I (x) L_nz with L_n the path-graph Laplacian,
// which the orthonormal DCT-II C_n (C_n[a][j] = s_a cos(pi a (2j+1) / (2n))) diagonalises:
// L_n = C_n^T diag(2 - 2 cos(pi a / n)) C_n.  Hence
//   P2^{-1} r = (C_x (x) C_z)^T diag(1 / (alpha0 lam_ab + mu)) (C_x (x) C_z) r,
// i.e. with r as the nx x nz matrix of the canonical order: C_x^T ((C_x r C_z^T) ./ L) C_z.
__global__ void dct_matrix_kernel(int n, double *Cm, double *lam) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n * n) {
        const int a = e / n, j = e % n;
        const double s = (a == 0) ? sqrt(1.0 / n) : sqrt(2.0 / n);
        Cm[e] = s * cospi((double)a * (2 * j + 1) / (2.0 * n));
    }
    if (e < n) lam[e] = 2.0 - 2.0 * cospi((double)e / n);
}

__global__ void p2_scale_kernel(int nx, int nz, const double *lx, const double *lz, double alpha0, double mu,
                                double *T) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nx * nz) return;
    const int a = e / nz, b = e % nz;
    const double sx = (double)(nx - 1) * (nx - 1), sz = (double)(nz - 1) * (nz - 1);
    T[e] = T[e] / (alpha0 * (sx * lx[a] + sz * lz[b]) + mu);
}

// C[i][j] = sum_k A(i, k) B(k, j), A(i,k) = A[i*as0 + k*as1], B(k,j) = B[k*bs0 + j*bs1],
// C row-major M x N.  DT x DT tiles in shared memory, FP64, k summed in ascending order.  The
// small tiles give a 128 x 128 product 256 blocks, enough to occupy the FP64 units of every SM
// (GB300's FP64 rate per SM is low).
constexpr int DT = 8;
__global__ void dgemm_strided_kernel(int M, int Nn, int K, const double *A, int as0, int as1, const double *B,
                                     int bs0, int bs1, double *Cout) {
    __shared__ double sA[DT][DT + 1], sB[DT][DT + 1];
    const int tx = threadIdx.x % DT, ty = threadIdx.x / DT;
    const int i = blockIdx.y * DT + ty, j = blockIdx.x * DT + tx;
    double acc = 0.0;
    for (int k0 = 0; k0 < K; k0 += DT) {
        const int ka = k0 + tx, kb = k0 + ty;
        sA[ty][tx] = (i < M && ka < K) ? A[(size_t)i * as0 + (size_t)ka * as1] : 0.0;
        sB[ty][tx] = (kb < K && j < Nn) ? B[(size_t)kb * bs0 + (size_t)j * bs1] : 0.0;
        __syncthreads();
#pragma unroll
        for (int t = 0; t < DT; ++t) acc = fma(sA[ty][t], sB[t][tx], acc);
        __syncthreads();
    }
    if (i < M && j < Nn) Cout[(size_t)i * Nn + j] = acc;
}

}  // namespace helm

// ====================================================================== host side

namespace {

struct Ws {
    std::vector<void *> bufs;
    cudaStream_t st;
    explicit Ws(cudaStream_t s) : st(s) {}
    ~Ws() {
        for (void *p : bufs) cudaFreeAsync(p, st);
    }
    template <typename T> T *get(size_t n, helm_status *s) {
        void *p = nullptr;
        if (*s != HELM_OK) return nullptr;
        if (n == 0) n = 1;
        if (fault_flags() & HELM_FAULT_ALLOC) {
            helm_set_msg("workspace: allocation refused (HELM_FAULT=alloc)");
            *s = HELM_ENOMEM;
            return nullptr;
        }
        cudaError_t e = cudaMallocAsync(&p, n * sizeof(T), st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            helm_set_error("cudaMallocAsync(workspace)", e);
            *s = (e == cudaErrorMemoryAllocation) ? HELM_ENOMEM : HELM_ECUDA;
            return nullptr;
        }
        bufs.push_back(p);
        return (T *)p;
    }
};


inline int nblk(size_t n, int t = 256) { return (int)((n + t - 1) / t); }

#define HK(call)                                          \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) {                          \
            helm_set_error(#call, e_);                    \
            return HELM_ECUDA;                            \
        }                                                 \
    } while (0)
#define HL()                                              \
    do {                                                  \
        cudaError_t e_ = cudaGetLastError();              \
        if (e_ != cudaSuccess) {                          \
            helm_set_error("kernel launch", e_);          \
            return HELM_ECUDA;                            \
        }                                                 \
    } while (0)
#define HS(x)                                             \
    do {                                                  \
        helm_status s_ = (x);                             \
        if (s_ != HELM_OK) return s_;                     \
    } while (0)

// sum of n values on the device into *out (device), fixed order
helm_status reduce_sum(const double *vals, int n, double *out, cudaStream_t st) {
    HELM_TRACED(K_SUM, st, (sum_partials_kernel<<<1, 32, 0, st>>>(1, n, vals, out)));
    HL();
    return HELM_OK;
}

// device dot product -> host value (synchronises)
struct Dotter {
    double *partial = nullptr, *res = nullptr;
    double host[4] = {};
    int nb = 0;
    helm_status init(Ws &ws, int n) {
        helm_status s = HELM_OK;
        nb = std::min(nblk(n), 304);
        partial = ws.get<double>(nb, &s);
        res = ws.get<double>(4, &s);
        return s;
    }
    helm_status dot(int n, const double *a, const double *b, int slot, cudaStream_t st) {
        HELM_TRACED(K_DOT, st, (dot_partial_kernel<<<nb, 256, 0, st>>>(n, a, b, partial)));
        HL();
        HELM_TRACED(K_SUM, st, (sum_partials_kernel<<<1, 32, 0, st>>>(1, nb, partial, res + slot)));
        HL();
        return HELM_OK;
    }
    helm_status fetch(int cnt, cudaStream_t st) {
        HK(cudaMemcpyAsync(host, res, cnt * sizeof(double), cudaMemcpyDeviceToHost, st));
        HK(cudaStreamSynchronize(st));
        return HELM_OK;
    }
};

// P2^{-1} by the DCT (see dct_matrix_kernel)
struct P2Solver {
    int nx = 0, nz = 0;
    double alpha0 = 0, mu = 0;
    double *Cx = nullptr, *Cz = nullptr, *lx = nullptr, *lz = nullptr, *T1 = nullptr, *T2 = nullptr;
    helm_status init(Ws &ws, const GridGeom &g, double a0, double m0, cudaStream_t st) {
        nx = g.nx;
        nz = g.nz;
        alpha0 = a0;
        mu = m0;
        helm_status s = HELM_OK;
        Cx = ws.get<double>((size_t)nx * nx, &s);
        Cz = ws.get<double>((size_t)nz * nz, &s);
        lx = ws.get<double>(nx, &s);
        lz = ws.get<double>(nz, &s);
        T1 = ws.get<double>((size_t)nx * nz, &s);
        T2 = ws.get<double>((size_t)nx * nz, &s);
        if (s != HELM_OK) return s;
        HELM_TRACED(K_DCTMAT, st, (dct_matrix_kernel<<<nblk((size_t)nx * nx), 256, 0, st>>>(nx, Cx, lx)));
        HL();
        HELM_TRACED(K_DCTMAT, st, (dct_matrix_kernel<<<nblk((size_t)nz * nz), 256, 0, st>>>(nz, Cz, lz)));
        HL();
        return HELM_OK;
    }
    static void gemm(int M, int Nn, int K, const double *A, int as0, int as1, const double *B, int bs0, int bs1,
                     double *C, cudaStream_t st) {
        dim3 grid((Nn + DT - 1) / DT, (M + DT - 1) / DT);
        HELM_TRACED(K_DGEMM, st, (dgemm_strided_kernel<<<grid, DT * DT, 0, st>>>(M, Nn, K, A, as0, as1, B, bs0, bs1, C)));
    }
    helm_status apply(const double *r, double *out, cudaStream_t st) {
        // T1 = Cx r          (nx x nx)(nx x nz)
        gemm(nx, nz, nx, Cx, nx, 1, r, nz, 1, T1, st);
        // T2 = T1 Cz^T       (nx x nz)(nz x nz)^T
        gemm(nx, nz, nz, T1, nz, 1, Cz, 1, nz, T2, st);
        HELM_TRACED(K_P2SCALE, st, (p2_scale_kernel<<<nblk((size_t)nx * nz), 256, 0, st>>>(nx, nz, lx, lz, alpha0, mu, T2)));
        // T1 = Cx^T T2
        gemm(nx, nz, nx, Cx, 1, nx, T2, nz, 1, T1, st);
        // out = T1 Cz
        gemm(nx, nz, nz, T1, nz, 1, Cz, nz, 1, out, st);
        HL();
        return HELM_OK;
    }
};

helm_status run_solve(helm_factor_t *f, int nrhs, const double2 *B, double2 *X, double rtol, int conj,
                      int64_t *count, int *max_it) {
    helm_solve_info info;
    helm_status s = solve_impl(f, nrhs, B, X, rtol, 40, f->prec == HELM_MIXED ? &info : nullptr, conj);
    if (count) *count += (int64_t)f->op->n_omega * nrhs;
    if (f->prec == HELM_MIXED && max_it) *max_it = std::max(*max_it, info.iters);
    return s;
}

}  // namespace

// H p = (H1 + H2 + Gamma) p by the adjoint-state formulas (Lemmas thm:H1, thm:H2,
// Discussion disc:Hess): per (s, w) two new solves,
//   v = A^{-1}(g u p),  z = A^{-H}(R^T W^2 R v - p conj(g) lambda),
//   (H p)_k = sum Re[g u conj(z)] - Re[g v conj(lambda)] - Re[g' u conj(lambda)] p_k + (Gamma p)_k.
// gauss_newton != 0: H1 + Gamma only (no lambda terms).  E, V, Z: [cols][N] scratch,
// dtmp: [cols][n_rec] scratch.
static helm_status hess_apply(helm_factor_t *f, const DevAcq &da, const double2 *U, const double2 *Lam,
                              const double *pv, double *out, double2 *E, double2 *V, double2 *Z, double2 *dtmp,
                              double alpha, double mu, double rtol, int gauss_newton, int64_t *count, int *max_it) {
    const helm_op *op = f->op;
    const GridGeom &g = op->g;
    const int N = g.nx * g.nz, ns = da.n_src, nr = da.n_rec, nw = op->n_omega;
    const size_t cols = (size_t)nw * ns;
    cudaStream_t st = op->st;
    HELM_TRACED(K_GUP, st, (g_u_p_kernel<<<nblk(cols * N), 256, 0, st>>>(N, nw, ns, op->gk, U, pv, E)));
    HL();
    HS(run_solve(f, ns, E, V, rtol, 0, count, max_it));
    if (gauss_newton) {
        HK(cudaMemsetAsync(E, 0, cols * N * sizeof(double2), st));
    } else {
        HELM_TRACED(K_ZBASE, st, (z_base_kernel<<<nblk(cols * N), 256, 0, st>>>(N, nw, ns, op->gk, Lam, pv, E)));
        HL();
    }
    HK(launch_restrict(g, (int)cols, nr, da.tap_idx, da.tap_w, V, dtmp, st));
    HELM_TRACED(K_SCATTER, st, (scatter_kernel<<<(unsigned)cols, 32, 0, st>>>(N, nr, da.tap_idx, da.tap_w, da.rec_w, 1, dtmp, E)));
    HL();
    HS(run_solve(f, ns, E, Z, rtol, 1, count, max_it));
    {   // E is free after the second solve: it holds the per-chunk partial sums
        const int n_chunks = (int)((cols + HESS_CHUNK - 1) / HESS_CHUNK);
        double *part = reinterpret_cast<double *>(E);
        HELM_TRACED(K_HESS, st, (hess_acc_kernel<<<dim3(nblk(N), n_chunks), 256, 0, st>>>(
                                     N, ns, (int)cols, op->gk, op->gpk, U, V, Z, Lam, pv, gauss_newton, part)));
        HL();
        HELM_TRACED(K_HESSFIN, st, (hess_finish_kernel<<<nblk(N), 256, 0, st>>>(g, n_chunks, part, pv, alpha, mu, out)));
        HL();
    }
    return HELM_OK;
}

extern "C" helm_status helm_field_grad(const helm_op_t *op, int32_t nrhs, const helm_c128 *U_dev,
                                      const helm_c128 *Lam_dev, double *grad_dev) {
    if (!op || nrhs < 0 || !grad_dev || (nrhs > 0 && (!U_dev || !Lam_dev))) {
        helm_set_msg("helm_field_grad: bad arguments");
        return HELM_EINVAL;
    }
    const int N = op->g.nx * op->g.nz;
    HELM_TRACED(K_FIELDGRAD, op->st, (field_grad_kernel<<<(N + 255) / 256, 256, 0, op->st>>>(
                                          op->g, op->n_omega, nrhs, op->omega_dev, op->m, (const double2 *)U_dev,
                                          (const double2 *)Lam_dev, grad_dev)));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { helm_set_error("helm_field_grad", e); return HELM_ECUDA; }
    return HELM_OK;
}

extern "C" helm_status helm_restrict_adjoint(const helm_op_t *op, const helm_acq *acq, int32_t ncol,
                                             const helm_c128 *Y_dev, helm_c128 *X_dev) {
    if (!op || !acq || ncol < 0 || (ncol > 0 && (!X_dev || !Y_dev))) {
        helm_set_msg("helm_restrict_adjoint: bad arguments");
        return HELM_EINVAL;
    }
    DevAcq d;
    helm_status s = acq_upload(op, acq, &d);
    if (s != HELM_OK) return s;
    const size_t N = (size_t)op->g.nx * op->g.nz, cols = (size_t)op->n_omega * ncol;
    cudaError_t e = cudaMemsetAsync(X_dev, 0, cols * N * sizeof(double2), op->st);
    if (e == cudaSuccess && cols > 0 && d.n_rec > 0) {
        HELM_TRACED(K_SCATTER, op->st, (scatter_kernel<<<(unsigned)cols, 32, 0, op->st>>>(
                                           (int)N, d.n_rec, d.tap_idx, d.tap_w, nullptr, 0, (const double2 *)Y_dev,
                                           (double2 *)X_dev)));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(op->st);
    acq_free(&d);
    if (e != cudaSuccess) { helm_set_error("helm_restrict_adjoint", e); return HELM_ECUDA; }
    return HELM_OK;
}

extern "C" helm_status fwi_hessian_vec(helm_factor_t *f, const helm_acq *acq, const helm_c128 *u_dev,
                                       const helm_c128 *lam_dev, const double *mt_dev, double alpha, double mu,
                                       double rtol, int32_t gauss_newton, double *hv_dev) {
    if (!f || !acq || !u_dev || !mt_dev || !hv_dev || acq->n_src < 1 || (!gauss_newton && !lam_dev)) {
        helm_set_msg("fwi_hessian_vec: bad arguments");
        return HELM_EINVAL;
    }
    keep_pool_memory();
    helm_op *op = f->op;
    const int N = op->g.nx * op->g.nz;
    const size_t cols = (size_t)op->n_omega * acq->n_src;
    DevAcq da;
    HS(acq_upload(op, acq, &da));
    helm_status s = HELM_OK;
    {
        Ws ws(op->st);
        double2 *E = ws.get<double2>(cols * N, &s);
        double2 *V = ws.get<double2>(cols * N, &s);
        double2 *Z = ws.get<double2>(cols * N, &s);
        double2 *dtmp = ws.get<double2>(cols * std::max(1, acq->n_rec), &s);
        if (s == HELM_OK)
            s = hess_apply(f, da, (const double2 *)u_dev, (const double2 *)lam_dev, mt_dev, hv_dev, E, V, Z, dtmp,
                           alpha, mu, rtol, gauss_newton, nullptr, nullptr);
        if (s == HELM_OK) {
            cudaError_t e = cudaStreamSynchronize(op->st);
            if (e != cudaSuccess) { helm_set_error("fwi_hessian_vec", e); s = HELM_ECUDA; }
        }
    }
    acq_free(&da);
    return s;
}

// --------------------------------------------------------------- helm_gamma_solve

// Z = Gamma(alpha0, mu)^{-1} R column by column with the DCT solver of the PCG (P2 of Eq. (P2))
extern "C" helm_status helm_gamma_solve(const helm_grid *grid, double alpha0, double mu, int32_t ncol,
                                        const double *R_dev, double *Z_dev, void *stream) {
    if (!grid || grid->nx < 2 || grid->nz < 2 || ncol < 0 || !(alpha0 >= 0.0) || !(mu > 0.0) ||
        (ncol > 0 && (!R_dev || !Z_dev))) {
        helm_set_msg("helm_gamma_solve: bad arguments");
        return HELM_EINVAL;
    }
    if (ncol == 0) return HELM_OK;
    keep_pool_memory();
    cudaStream_t st = (cudaStream_t)stream;
    const GridGeom g{grid->nx, grid->nz, grid->lx / (grid->nx - 1), grid->lz / (grid->nz - 1), grid->lumping};
    const size_t N = (size_t)g.nx * g.nz;
    helm_status s = HELM_OK;
    {
        Ws ws(st);
        P2Solver p2;
        s = p2.init(ws, g, alpha0, mu, st);
        for (int32_t c = 0; s == HELM_OK && c < ncol; ++c) s = p2.apply(R_dev + c * N, Z_dev + c * N, st);
        if (s == HELM_OK) {
            const cudaError_t e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) { helm_set_error("helm_gamma_solve", e); s = HELM_ECUDA; }
        }
    }
    return s;
}

// --------------------------------------------------------------- fwi_misfit_grad

// forward part: u = A^{-1} E (E = point sources, scratch supplied by the caller)
static helm_status forward_fields(helm_factor_t *f, const DevAcq &da, double rtol, double2 *E, double2 *U,
                                  int64_t *count, int *max_it) {
    const helm_op *op = f->op;
    HK(launch_sources(op->g, op->n_omega, da.n_src, da.src_xz, da.src_amp, E, op->st));
    HS(run_solve(f, da.n_src, E, U, rtol, 0, count, max_it));
    return HELM_OK;
}

// adjoint part: eps = d - R u, lambda = A^{-H} R^T(W^2 eps), grad phi and phi (device)
static helm_status adjoint_grad(helm_factor_t *f, const DevAcq &da, const double2 *data, double alpha, double mu,
                                double rtol, double *phi_dev, double *grad, const double2 *U, double2 *Lam,
                                double2 *E, Ws &ws, int64_t *count, int *max_it) {
    const helm_op *op = f->op;
    const GridGeom &g = op->g;
    const int N = g.nx * g.nz, ns = da.n_src, nr = da.n_rec, nw = op->n_omega;
    const size_t cols = (size_t)nw * ns;
    cudaStream_t st = op->st;
    helm_status s = HELM_OK;
    double2 *eps = ws.get<double2>(cols * std::max(1, nr), &s);
    double *phi_col = ws.get<double>(cols + nblk(N) + 2, &s);
    if (s != HELM_OK) return s;
    HELM_TRACED(K_MISFIT, st, (misfit_kernel<<<(unsigned)cols, 256, 0, st>>>(N, nr, da.tap_idx, da.tap_w, da.rec_w, U, data, eps, phi_col)));
    HL();
    HK(cudaMemsetAsync(E, 0, cols * N * sizeof(double2), st));
    HELM_TRACED(K_SCATTER, st, (scatter_kernel<<<(unsigned)cols, 32, 0, st>>>(N, nr, da.tap_idx, da.tap_w, da.rec_w, 1, eps, E)));
    HL();
    HS(run_solve(f, ns, E, Lam, rtol, 1, count, max_it));
    double *reg_part = phi_col + cols;
    HELM_TRACED(K_GRAD, st, (grad_kernel<<<nblk(N), 256, 0, st>>>(g, nw, ns, op->omega_dev, op->m, U, Lam, alpha, mu, grad, reg_part)));
    HL();
    HS(reduce_sum(phi_col, (int)(cols + nblk(N)), phi_dev, st));
    return HELM_OK;
}

// u = A^{-1} e_s, eps = d - R u, lambda = A^{-H} R^T(W^2 eps), grad, phi
static helm_status misfit_grad_body(helm_factor_t *f, const DevAcq &da, const double2 *data, double alpha,
                                    double mu, double rtol, double *phi_dev, double *grad, double2 *U, double2 *Lam,
                                    Ws &ws, int64_t *count, int *max_it) {
    const helm_op *op = f->op;
    const size_t cols = (size_t)op->n_omega * da.n_src;
    helm_status s = HELM_OK;
    double2 *E = ws.get<double2>(cols * op->g.nx * op->g.nz, &s);
    if (s != HELM_OK) return s;
    HS(forward_fields(f, da, rtol, E, U, count, max_it));
    return adjoint_grad(f, da, data, alpha, mu, rtol, phi_dev, grad, U, Lam, E, ws, count, max_it);
}

extern "C" helm_status fwi_misfit_grad(helm_factor_t *f, const helm_acq *acq, const helm_c128 *data_dev,
                                       double alpha, double mu, double rtol, double *phi, double *grad_dev,
                                       helm_c128 *u_out, helm_c128 *lam_out) {
    if (!f || !acq || !data_dev || !phi || !grad_dev || acq->n_src < 1) {
        helm_set_msg("fwi_misfit_grad: bad arguments");
        return HELM_EINVAL;
    }
    keep_pool_memory();
    helm_op *op = f->op;
    const int N = op->g.nx * op->g.nz;
    const size_t cols = (size_t)op->n_omega * acq->n_src;
    DevAcq da;
    HS(acq_upload(op, acq, &da));
    helm_status s = HELM_OK;
    {
        Ws ws(op->st);
        double2 *U = u_out ? (double2 *)u_out : ws.get<double2>(cols * N, &s);
        double2 *Lam = lam_out ? (double2 *)lam_out : ws.get<double2>(cols * N, &s);
        double *phi_dev = ws.get<double>(1, &s);
        if (s == HELM_OK)
            s = misfit_grad_body(f, da, (const double2 *)data_dev, alpha, mu, rtol, phi_dev, grad_dev, U, Lam, ws,
                                 nullptr, nullptr);
        if (s == HELM_OK) {
            cudaError_t e = cudaMemcpyAsync(phi, phi_dev, sizeof(double), cudaMemcpyDeviceToHost, op->st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(op->st);
            if (e != cudaSuccess) { helm_set_error("fwi_misfit_grad", e); s = HELM_ECUDA; }
        }
    }
    acq_free(&da);
    return s;
}

// ------------------------------------------------------------- bilevel_hypergrad

namespace {

struct ModelState {
    helm_op_t *op_f = nullptr, *op_t = nullptr;
    helm_factor_t *fac_f = nullptr, *fac_t = nullptr;
    ~ModelState() {
        helm_factor_destroy(fac_f);
        helm_factor_destroy(fac_t);
        helm_op_destroy(op_f);
        helm_op_destroy(op_t);
    }
};

// one training model: accumulate psi, dpsi/dalpha, dp, dw (device, scaled by 1/n_models)
helm_status hyper_one_model(const helm_grid *grid, const double *m_fwi, const double *m_true,
                            const helm_grid *data_grid, const double *m_data, const helm_acq *acq,
                            const double *omega, int n_omega, double alpha, double alpha0, double mu,
                            helm_prec prec, const helm_pcg_opts *po, cudaStream_t st, double inv_models,
                            double *acc_dev /*[2]: psi, dalpha*/, double *dp_dev, double *dw_dev,
                            helm_hyper_info *info) {
    // the data branch (A(m') assembled on the data's grid, factored, u' = A(m')^{-1} e_s, the
    // data d = R' u' and their receiver derivatives dR'_x u', dR'_z u') runs on its own stream
    // from a second host thread, concurrently with A(m_fwi) and u; the stream outlives the
    // handles allocated on it (declared first, destroyed last)
    const helm_factor_opts fopts{po->factor_method};
    cudaStream_t st2 = nullptr;
    HK(cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking));
    struct StreamGuard { cudaStream_t s; ~StreamGuard() { if (s) cudaStreamDestroy(s); } } sg{st2};
    ModelState ms;
    helm_status s = HELM_OK;
    Ws ws(st);
    Ws ws2(st2);
    int64_t count = 0, dcount = 0;
    int max_it = 0, max_it2 = 0;
    DevAcq da2;
    struct AcqGuard2 { DevAcq *d; ~AcqGuard2() { acq_free(d); } } ag2{&da2};
    double2 *dtmp = nullptr, *ddx = nullptr, *ddz = nullptr;
    helm_status s2 = HELM_OK;
    std::string msg2;   // error text of the data branch (set in its own thread)
    std::thread data_branch([&]() {
        auto run = [&]() {
            s2 = helm_assemble(data_grid, m_data, omega, n_omega, st2, &ms.op_t);
            if (s2 == HELM_OK) s2 = helm_factor(ms.op_t, prec, &fopts, &ms.fac_t);
            if (s2 == HELM_OK) s2 = acq_upload(ms.op_t, acq, &da2);
            if (s2 != HELM_OK) return;
            const GridGeom &gt = ms.op_t->g;
            const size_t ct = (size_t)n_omega * da2.n_src;
            double2 *Et = ws2.get<double2>(ct * gt.nx * gt.nz, &s2);
            double2 *Ut = ws2.get<double2>(ct * gt.nx * gt.nz, &s2);
            dtmp = ws2.get<double2>(ct * std::max(1, da2.n_rec), &s2);
            ddx = ws2.get<double2>(ct * std::max(1, da2.n_rec), &s2);
            ddz = ws2.get<double2>(ct * std::max(1, da2.n_rec), &s2);
            if (s2 != HELM_OK) return;
            s2 = forward_fields(ms.fac_t, da2, po->refine_rtol, Et, Ut, &dcount, &max_it2);
            if (s2 != HELM_OK) return;
            cudaError_t e = launch_restrict(gt, (int)ct, da2.n_rec, da2.tap_idx, da2.tap_w, Ut, dtmp, st2);
            if (e == cudaSuccess) e = launch_restrict(gt, (int)ct, da2.n_rec, da2.tap_idx, da2.tap_wx, Ut, ddx, st2);
            if (e == cudaSuccess) e = launch_restrict(gt, (int)ct, da2.n_rec, da2.tap_idx, da2.tap_wz, Ut, ddz, st2);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st2);
            if (e != cudaSuccess) { helm_set_error("data branch", e); s2 = HELM_ECUDA; }
        };
        run();
        if (s2 != HELM_OK) msg2 = helm_last_error();
    });
    struct Joiner { std::thread &t; ~Joiner() { if (t.joinable()) t.join(); } } joiner{data_branch};
    s = helm_assemble(grid, m_fwi, omega, n_omega, st, &ms.op_f);
    if (s == HELM_OK) s = helm_factor(ms.op_f, prec, &fopts, &ms.fac_f);
    if (s != HELM_OK) { data_branch.join(); return s; }
    helm_op *op = ms.op_f;
    const GridGeom &g = op->g;
    const int N = g.nx * g.nz;
    DevAcq da;
    HS(acq_upload(op, acq, &da));
    struct AcqGuard { DevAcq *d; ~AcqGuard() { acq_free(d); } } ag{&da};
    const int ns = da.n_src, nr = da.n_rec;
    const size_t cols = (size_t)n_omega * ns;
    const double rtol = po->refine_rtol;
    double2 *E = ws.get<double2>(cols * N, &s);
    double2 *U = ws.get<double2>(cols * N, &s);
    double2 *Lam = ws.get<double2>(cols * N, &s);
    double2 *V = ws.get<double2>(cols * N, &s);
    double2 *Z = ws.get<double2>(cols * N, &s);
    double2 *rtmp = ws.get<double2>(cols * std::max(1, nr), &s);
    double *phi_dev = ws.get<double>(1, &s);
    double *grad = ws.get<double>(N, &s);
    double *x = ws.get<double>(N, &s), *r = ws.get<double>(N, &s), *zz = ws.get<double>(N, &s);
    double *p = ws.get<double>(N, &s), *Hp = ws.get<double>(N, &s), *rhs = ws.get<double>(N, &s);
    if (s != HELM_OK) { data_branch.join(); return s; }
    // u at m_fwi while the data branch runs
    s = forward_fields(ms.fac_f, da, rtol, E, U, &count, &max_it);
    data_branch.join();
    if (s != HELM_OK) return s;
    if (s2 != HELM_OK) { helm_set_msg(msg2.c_str()); return s2; }
    max_it = std::max(max_it, max_it2);
    // eps, lambda (and grad phi, unused here) at m_fwi
    HS(adjoint_grad(ms.fac_f, da, dtmp, alpha, mu, rtol, phi_dev, grad, U, Lam, E, ws, &count, &max_it));
    double2 *dbuf = rtmp;

    auto hess = [&](const double *pv, double *out) -> helm_status {
        return hess_apply(ms.fac_f, da, U, Lam, pv, out, E, V, Z, dbuf, alpha, mu, rtol, 0, &count, &max_it);
    };

    // PCG for H rho = m' - m_fwi with P2 = Gamma(alpha0, mu), x0 = const
    P2Solver p2;
    HS(p2.init(ws, g, alpha0, mu, st));
    Dotter dot;
    HS(dot.init(ws, N));
    HELM_TRACED(K_SUB, st, (sub_kernel<<<nblk(N), 256, 0, st>>>(N, m_true, m_fwi, rhs)));
    HELM_TRACED(K_FILL, st, (fill_kernel<<<nblk(N), 256, 0, st>>>(N, po->x0, x)));
    HL();
    HS(hess(x, Hp));
    int nmv = 1;
    HELM_TRACED(K_SUB, st, (sub_kernel<<<nblk(N), 256, 0, st>>>(N, rhs, Hp, r)));
    HL();
    HS(p2.apply(r, zz, st));
    HK(cudaMemcpyAsync(p, zz, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    HS(dot.dot(N, r, zz, 0, st));
    HS(dot.dot(N, r, r, 1, st));
    HS(dot.fetch(2, st));
    double rz = dot.host[0];
    const double r0 = sqrt(dot.host[1]);
    double rn = r0;
    const int iters = po->fixed_iters > 0 ? po->fixed_iters : po->max_iter;
    if (po->fixed_iters > 0 && r0 != 0.0) {
        // a fixed iteration count needs no stopping test: the scalars stay on the device (r.z in
        // res[0] / res[1] by iteration parity, p.Hp in res[2]) and the host does not wait on the
        // GPU inside the loop; ||r|| is read once at the end
        for (int it = 0; it < iters; ++it) {
            double *rz_cur = dot.res + (it & 1), *rz_next = dot.res + ((it + 1) & 1);
            HS(hess(p, Hp));
            ++nmv;
            HS(dot.dot(N, p, Hp, 2, st));
            HELM_TRACED(K_AXPBY, st, (cg_step_kernel<<<nblk(N), 256, 0, st>>>(N, rz_cur, dot.res + 2, p, Hp, x, r)));
            HL();
            HS(p2.apply(r, zz, st));
            HS(dot.dot(N, r, zz, (it + 1) & 1, st));
            HELM_TRACED(K_AXPBY, st, (cg_dir_kernel<<<nblk(N), 256, 0, st>>>(N, zz, rz_next, rz_cur, p)));
            HL();
        }
        HS(dot.dot(N, r, r, 3, st));
        HS(dot.fetch(4, st));
        rn = sqrt(dot.host[3]);
    }
    for (int it = 0; po->fixed_iters <= 0 && it < iters; ++it) {
        if (r0 == 0.0 || rn <= po->rtol * r0) break;
        HS(hess(p, Hp));
        ++nmv;
        HS(dot.dot(N, p, Hp, 0, st));
        HS(dot.fetch(1, st));
        const double a = rz / dot.host[0];
        HELM_TRACED(K_AXPBY, st, (axpby_kernel<<<nblk(N), 256, 0, st>>>(N, a, p, 1.0, x)));
        HELM_TRACED(K_AXPBY, st, (axpby_kernel<<<nblk(N), 256, 0, st>>>(N, -a, Hp, 1.0, r)));
        HL();
        HS(p2.apply(r, zz, st));
        HS(dot.dot(N, r, zz, 0, st));
        HS(dot.dot(N, r, r, 1, st));
        HS(dot.fetch(2, st));
        const double rz_new = dot.host[0];
        rn = sqrt(dot.host[1]);
        HELM_TRACED(K_AXPBY, st, (axpby_kernel<<<nblk(N), 256, 0, st>>>(N, 1.0, zz, rz_new / rz, p)));
        HL();
        rz = rz_new;
    }
    const double relres = r0 > 0 ? rn / r0 : 0.0;
    // tau = A^{-1}(g u rho) and the receiver terms
    HELM_TRACED(K_GUP, st, (g_u_p_kernel<<<nblk(cols * N), 256, 0, st>>>(N, n_omega, ns, op->gk, U, x, E)));
    HL();
    HS(run_solve(ms.fac_f, ns, E, V, rtol, 0, &count, &max_it));
    HELM_TRACED(K_HYPER, st, (hyper_terms_kernel<<<nr, 256, 0, st>>>(N, (int)cols, nr, da.tap_idx, da.tap_w, da.tap_wx, da.tap_wz, da.rec_w,
                                           V, U, dtmp, ddx, ddz, inv_models, dp_dev, dw_dev)));
    HL();
    // dpsi/dalpha += m_fwi^T R rho / n_models ; psi += ||m' - m_fwi||^2 / (2 n_models)
    HELM_TRACED(K_REGR, st, (regR_kernel<<<nblk(N), 256, 0, st>>>(g, x, zz)));
    HL();
    HS(dot.dot(N, m_fwi, zz, 0, st));
    HS(dot.dot(N, rhs, rhs, 1, st));
    HS(dot.fetch(2, st));
    double host_acc[2];
    HK(cudaMemcpyAsync(host_acc, acc_dev, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    HK(cudaStreamSynchronize(st));
    host_acc[0] += 0.5 * inv_models * dot.host[1];
    host_acc[1] += inv_models * dot.host[0];
    HK(cudaMemcpyAsync(acc_dev, host_acc, 2 * sizeof(double), cudaMemcpyHostToDevice, st));
    HK(cudaStreamSynchronize(st));
    if (info) {
        info->cg_matvecs = nmv;
        info->cg_relres = std::max(info->cg_relres, relres);
        info->solves += count;
        info->data_solves += dcount;
        info->max_refine_iters = std::max(info->max_refine_iters, max_it);
    }
    if (po->fixed_iters <= 0 && !(relres <= po->rtol)) {
        helm_set_msg("bilevel_hypergrad: PCG did not reach rtol");
        return HELM_ENOCONV;
    }
    return HELM_OK;
}

}  // namespace

extern "C" helm_status bilevel_hypergrad(int32_t n_models, const helm_grid *grids, const double *const *m_fwi,
                                         const double *const *m_true, const helm_acq *acq,
                                         const helm_grid *data_grids, const double *const *m_data,
                                         const double *omega, int32_t n_omega, double alpha, double alpha0,
                                         double mu, helm_prec prec, const helm_pcg_opts *pcg, void *stream,
                                         double *psi, double *dpsi_dalpha, double *dpsi_dp, double *dpsi_dw,
                                         helm_hyper_info *info) {
    if (n_models < 1 || !grids || !m_fwi || !m_true || !acq || !omega || n_omega < 1 || !psi || !dpsi_dalpha ||
        !dpsi_dp || acq[0].n_rec < 1 || (!data_grids) != (!m_data)) {
        helm_set_msg("bilevel_hypergrad: bad arguments");
        return HELM_EINVAL;
    }
    // data from another grid: of the same domain (the sources and receivers are physical points)
    for (int k = 0; data_grids && k < n_models; ++k)
        if (!m_data[k] || data_grids[k].lx != grids[k].lx || data_grids[k].lz != grids[k].lz) {
            helm_set_msg("bilevel_hypergrad: a data grid must cover its model's domain (same lx, lz)");
            return HELM_EINVAL;
        }
    // one acquisition per model: its own sources, the same receivers (the design P)
    for (int k = 0; k < n_models; ++k)
        if (acq[k].n_src < 1 || acq[k].n_rec != acq[0].n_rec) {
            helm_set_msg("bilevel_hypergrad: every model needs sources and the same number of receivers");
            return HELM_EINVAL;
        }
    keep_pool_memory();
    helm_pcg_opts po = pcg ? *pcg : helm_pcg_opts{500, 0, 1e-13, 1.0, 1e-10, 0, HELM_FACTOR_AUTO};
    cudaStream_t st = (cudaStream_t)stream;
    if (info) *info = helm_hyper_info{0, 0.0, 0, 0, 0};
    const int nr = acq[0].n_rec;
    // Independent training models run concurrently, each on its own streams from its own host
    // thread (the chain of one model is latency bound and leaves most of the GPU idle); every
    // model writes its own partial results, which are summed here in model order.
    constexpr int kDefaultConcurrent = 3;
    const int K = std::max(1, std::min<int>(n_models, po.concurrent_models > 0 ? po.concurrent_models
                                                                                : kDefaultConcurrent));
    std::vector<double> acc_h(2 * (size_t)n_models, 0.0), dp_h(2 * (size_t)nr * n_models, 0.0),
        dw_h((size_t)nr * n_models, 0.0);
    std::vector<helm_hyper_info> infos(n_models, helm_hyper_info{0, 0.0, 0, 0, 0});
    std::vector<helm_status> stat(n_models, HELM_OK);
    std::vector<std::string> msg(n_models);
    // every worker runs on a non-blocking stream of its own that first waits for the caller's
    // stream (the inputs are ready there); none of the model's work lands on the caller's stream,
    // which may be the legacy default stream (work on it made the factorisations of the two
    // branches of a model run one after the other in most steps)
    cudaEvent_t ready = nullptr;
    {
        cudaError_t e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ready, st);
        if (e != cudaSuccess) {
            if (ready) cudaEventDestroy(ready);
            helm_set_error("bilevel_hypergrad: event", e);
            return HELM_ECUDA;
        }
    }
    auto worker = [&](int w) {
        cudaStream_t sw = nullptr;
        if (cudaStreamCreateWithFlags(&sw, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamWaitEvent(sw, ready, 0) != cudaSuccess) {
            if (sw) cudaStreamDestroy(sw);
            for (int k = w; k < n_models; k += K) { stat[k] = HELM_ECUDA; msg[k] = "bilevel_hypergrad: stream"; }
            return;
        }
        for (int k = w; k < n_models; k += K) {
            helm_status s = HELM_OK;
            {
                Ws ws(sw);
                double *acc = ws.get<double>(2, &s);
                double *dp = ws.get<double>(2 * nr, &s);
                double *dw = ws.get<double>(nr, &s);
                cudaError_t e = cudaSuccess;
                if (s == HELM_OK) e = cudaMemsetAsync(acc, 0, 2 * sizeof(double), sw);
                if (s == HELM_OK && e == cudaSuccess) e = cudaMemsetAsync(dp, 0, 2 * nr * sizeof(double), sw);
                if (s == HELM_OK && e == cudaSuccess) e = cudaMemsetAsync(dw, 0, nr * sizeof(double), sw);
                if (e != cudaSuccess) { helm_set_error("bilevel_hypergrad", e); s = HELM_ECUDA; }
                if (s == HELM_OK)
                    s = hyper_one_model(&grids[k], m_fwi[k], m_true[k], data_grids ? &data_grids[k] : &grids[k],
                                        data_grids ? m_data[k] : m_true[k], &acq[k], omega, n_omega, alpha, alpha0,
                                        mu, prec, &po, sw, 1.0 / n_models, acc, dp, dw, &infos[k]);
                if (s == HELM_OK || s == HELM_ENOCONV) {
                    e = cudaMemcpyAsync(&acc_h[2 * (size_t)k], acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, sw);
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(&dp_h[2 * (size_t)nr * k], dp, 2 * nr * sizeof(double),
                                            cudaMemcpyDeviceToHost, sw);
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(&dw_h[(size_t)nr * k], dw, nr * sizeof(double), cudaMemcpyDeviceToHost, sw);
                    if (e == cudaSuccess) e = cudaStreamSynchronize(sw);
                    if (e != cudaSuccess) { helm_set_error("bilevel_hypergrad", e); s = HELM_ECUDA; }
                }
            }
            stat[k] = s;
            if (s != HELM_OK) msg[k] = helm_last_error();
        }
        cudaStreamDestroy(sw);
    };
    {
        std::vector<std::thread> pool;
        for (int w = 1; w < K; ++w) pool.emplace_back(worker, w);
        worker(0);
        for (auto &t : pool) t.join();
    }
    cudaEventDestroy(ready);
    helm_status s = HELM_OK;
    for (int k = 0; k < n_models; ++k)
        if (stat[k] != HELM_OK && stat[k] != HELM_ENOCONV) { helm_set_msg(msg[k].c_str()); return stat[k]; }
    double a0 = 0.0, a1 = 0.0;
    for (int r = 0; r < 2 * nr; ++r) dpsi_dp[r] = 0.0;
    if (dpsi_dw)
        for (int r = 0; r < nr; ++r) dpsi_dw[r] = 0.0;
    for (int k = 0; k < n_models; ++k) {   // model order
        a0 += acc_h[2 * (size_t)k];
        a1 += acc_h[2 * (size_t)k + 1];
        for (int r = 0; r < 2 * nr; ++r) dpsi_dp[r] += dp_h[2 * (size_t)nr * k + r];
        if (dpsi_dw)
            for (int r = 0; r < nr; ++r) dpsi_dw[r] += dw_h[(size_t)nr * k + r];
        if (info) {
            info->cg_matvecs = std::max(info->cg_matvecs, infos[k].cg_matvecs);
            info->cg_relres = std::max(info->cg_relres, infos[k].cg_relres);
            info->solves += infos[k].solves;
            info->data_solves += infos[k].data_solves;
            info->max_refine_iters = std::max(info->max_refine_iters, infos[k].max_refine_iters);
        }
        if (stat[k] == HELM_ENOCONV && s == HELM_OK) { s = HELM_ENOCONV; helm_set_msg(msg[k].c_str()); }
    }
    *psi = a0;
    *dpsi_dalpha = a1;
    return s;
}
