// Internal definitions of the opaque handles of include/helm.h (C++ only).
#pragma once
#include <atomic>
#include <utility>
#include <vector>
#include <cuda_runtime.h>
#include "helm.h"
#include "common.cuh"

struct helm_op {
    helm::GridGeom g;
    double lx = 0, lz = 0;
    int n_omega = 0;
    std::vector<double> omega;
    double *m = nullptr;          // [N] squared slowness (device copy)
    double *omega_dev = nullptr;  // [n_omega]
    double2 *diag = nullptr;      // [n_omega][N] diagonal of A(m, w)
    double2 *gk = nullptr;        // [n_omega][N] g_k(w) = w^2 d_k + i w b_k / (2 sqrt(m_k))
    double2 *gpk = nullptr;       // [n_omega][N] g'_k(w) = -i w b_k / (4 m_k^{3/2})
    int *status = nullptr;        // device status word
    cudaStream_t st = nullptr;
    int dev = 0;                  // device that was current at helm_assemble (owns every buffer)
};

namespace helm {
struct RefineState;   // device-side refinement control (kernels.h)
}

// Block-cyclic-reduction factor (bcr.cu): the inverse of every line's block at the level it was
// eliminated, the back-substitution blocks P_j, Q_j and the forward blocks W_j, V_j of the lines
// eliminated at levels >= 1 (slot j / 2), and the solve's GEMM task lists on the device.
struct BcrData {
    int levels = 0, half = 0;
    float2 *Dinv = nullptr, *P = nullptr, *Q = nullptr, *W = nullptr, *V = nullptr;
    int *tasks = nullptr;
    float2 *split = nullptr;     // partial tiles of the solve's split-K GEMM launches
    size_t split_cap = 0;        // (complex elements)
    struct List {
        int first = 0, count = 0;   // tasks of one GEMM launch of the solve
        long long terms = 0;        // product terms over those tasks
    };
    std::vector<List> fwd, bwd;     // per level
    List last;
};

struct helm_factor {
    helm_op *op = nullptr;
    bool use_bcr = false;  // mixed: block-cyclic-reduction factor on the tensor cores
    BcrData bcr;
    helm_prec prec = HELM_FP64;
    int cs = 1;
    int mid = 0;           // middle line of the (twisted) line factorisation
    void *G = nullptr;     // [n_omega][nx][nz][nz] complex (FP64 or FP32)
    void *xch = nullptr;   // factor exchange slots
    float4 *diag2 = nullptr;   // mixed: [n_omega][N] diagonal of A as FP32 pairs
    int fp64_blocks = 0;       // mixed: pivot blocks inverted in FP64 (flagged)
    // solve scratch, sized for `cap` right-hand sides per frequency
    int cap = 0;
    float4 *bd = nullptr, *xa = nullptr, *xb = nullptr;   // mixed: b and the iterate (ping-pong), FP32 pairs
    float2 *r32 = nullptr, *y = nullptr;                  // mixed: correction right-hand side and result
    double *norms = nullptr;
    std::vector<double> norms_host;   // host copy of the norms (pageable: no pinned allocation)
    helm::RefineState *state = nullptr;       // mixed: device-side refinement control
    mutable std::atomic<int> last_iters{3};   // correction sweeps the previous mixed solve took
};

// working memory of one mixed-precision solve of n_omega x nrhs columns
struct MixedWork {
    float4 *bd, *xa, *xb;
    float2 *r32, *y;
    double *norms;        // device [cols][2]
    double *norms_host;   // host [cols][2]
    helm::RefineState *state;   // device
};

// acquisition on the device
struct DevAcq {
    cudaStream_t st = nullptr;   // stream the arrays were allocated on (and are freed on)
    int n_src = 0, n_rec = 0;
    double *src_xz = nullptr, *src_amp = nullptr, *rec_xz = nullptr, *rec_w = nullptr;
    int *tap_idx = nullptr;
    double *tap_w = nullptr, *tap_wx = nullptr, *tap_wz = nullptr;
};

void helm_set_error(const char *what, cudaError_t e);
void helm_set_msg(const char *what);
// Device memory of the library comes from the stream-ordered allocator (cudaMallocAsync on the
// handle's stream, the pool keeping its memory): unlike cudaMalloc / cudaFree it never waits for
// work on other streams, so handles can be created and destroyed while other threads' kernels run.
helm_status dev_alloc(void **p, size_t bytes, const char *what, cudaStream_t st);
void dev_free(void *p, cudaStream_t st);
void keep_pool_memory();
helm_status factor_reserve(helm_factor_t *f, int nrhs);
// status bits of the op after its sweeps (synchronises the op's stream): HELM_ETIMEOUT if a
// bounded wait of a sweep gave up
helm_status read_sweep_status(const helm_op *op);
helm_status solve_impl(helm_factor_t *f, int nrhs, const double2 *B, double2 *X, double rtol, int max_iter,
                       helm_solve_info *info, int conj);
// mixed-precision refinement (refine.cu kernels) to ||b - A x|| / ||b|| <= rtol per column
helm_status mixed_refine(const helm_factor_t *f, int nrhs, const double2 *B, double2 *X, int conj, double rtol,
                         int max_iter, const MixedWork &w, int *iters, double *relres);
// max over columns of ||r|| / ||b|| from a device norms buffer (synchronises the op's stream)
helm_status max_relres(const helm_op *op, size_t cols, const double *norms_dev, double *norms_host, double *out);
helm_status acq_upload(const helm_op *op, const helm_acq *acq, DevAcq *d);
// block cyclic reduction (bcr.cu)
namespace helm {
bool bcr_supported(const GridGeom &g);
// whether helm_factor builds a block-cyclic-reduction factor for this grid and precision
// (method: a helm_factor_method; HELM_FACTOR_AUTO follows HELM_FACTOR and the line length)
bool factor_picks_bcr(const GridGeom &g, helm_prec prec, int method);
helm_status bcr_factor(helm_factor_t *f);
void bcr_free(helm_factor_t *f);
// frozen: NULL, or the refinement's per-system flags (stride 2): columns of a set flag are skipped
helm_status bcr_solve(const helm_factor_t *f, int nrhs, float2 *r, float2 *x, const int *skip,
                      const int *frozen = nullptr);
helm_status blas_zgemm(int batch, int M, int N, int K, const float2 *A, long long sa, int lda, const float2 *Bt,
                       long long sb, int ldb, float sign, const float2 *C0, float2 *C, long long sc, int ldc,
                       cudaStream_t st, int *status);
helm_status blas_zinv(int batch, int n, const float2 *A, long long sa, int lda, float2 *X, long long sx, int ldx,
                      cudaStream_t st, int *status);
}  // namespace helm
void acq_free(DevAcq *d);
