// Host-side launch wrappers of the libhelm kernels (internal, C++ only).
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"

namespace helm {

constexpr int NB = 16;   // diagonal-block size of the line inversions

// ---- assemble.cu
cudaError_t launch_assemble(const GridGeom &g, const double *m, const double *omega_dev, int n_omega,
                            double2 *diag, cudaStream_t st);
// gk, gpk [n_omega][N]: g_k(w) and g'_k(w) of the model derivative of A
cudaError_t launch_gcoef(const GridGeom &g, const double *m, const double *omega_dev, int n_omega, double2 *gk,
                         double2 *gpk, cudaStream_t st);
cudaError_t launch_sources(const GridGeom &g, int n_omega, int n_src, const double *src_xz_dev,
                           const double *src_amp_dev, double2 *B, cudaStream_t st);
// taps: [n_rec][16] node index, weight, d/dx weight, d/dz weight
cudaError_t launch_restriction_taps(const GridGeom &g, int n_rec, const double *rec_xz_dev, int *tap_idx,
                                    double *tap_w, double *tap_wx, double *tap_wz, cudaStream_t st);
cudaError_t launch_restrict(const GridGeom &g, int n_cols, int n_rec, const int *tap_idx, const double *tap_w,
                            const double2 *X, double2 *Y, cudaStream_t st);

// ---- factor.cu
__host__ __device__ size_t factor_xch_elems(int nz);   // exchange-slot elements per system (both slots)
template <typename T>
cudaError_t launch_line_factor(const GridGeom &g, int n_sys, const double2 *diag, cx_t<T> *G, cx_t<T> *xch,
                               int *status, int cs, cudaStream_t st, int *mid_out);

// ---- sweep.cu
// B in the working precision; TG = double writes X (conjugated if conj), TG = float writes Y.
// skip (optional, device): nonzero when the launch runs makes it do nothing.
// frozen (optional, device): frozen[2*sys] nonzero leaves system sys untouched (Y not written).
template <typename TG>
cudaError_t launch_line_sweep(const GridGeom &g, int n_sys, int nrhs, const cx_t<TG> *G, const cx_t<TG> *B,
                              double2 *X, cx_t<TG> *Y, int conj, int rchunk, int *status, cudaStream_t st, int mid,
                              const int *skip = nullptr, const int *frozen = nullptr);
// FP64 residual B - A X (A^H X for conj), norms[col] += (||R||^2, ||B||^2); R32 = conj?(R) in FP32 if given
cudaError_t launch_residual(const GridGeom &g, int n_sys, int nrhs, const double2 *diag, const double2 *B,
                            const double2 *X, float2 *R32, double *norms, int conj, cudaStream_t st);

int pick_cluster_size(int nz);

// Raise the kernel's dynamic shared-memory limit to at least `bytes` (never lowers it), so
// that host threads launching the same kernel with different sizes do not undo each other.
cudaError_t ensure_dyn_smem(const void *fn, size_t bytes);
// Allow cluster sizes above 8 for the kernel (set once per device and kernel).
cudaError_t ensure_nonportable_clusters(const void *fn);
// Co-resident clusters of csz CTAs of the kernel (0: cannot be scheduled); cached per shape.
int max_active_clusters(const void *fn, int csz, int threads, size_t smem);

// ---- refine.cu (mixed-precision refinement in FP32-pair arithmetic)
// diag2[s][k] = (hi.re, hi.im, lo.re, lo.im) of the FP64 diagonal
cudaError_t launch_split_diag(size_t n, const double2 *diag, float4 *diag2, cudaStream_t st);
// bd = pair form of conj?(B), r32 = its leading part; norms[col][1] = ||B||^2, norms[col][0] = 0
cudaError_t launch_refine_start(const GridGeom &g, int cols, const double2 *B, int conj, float4 *bd, float2 *r32,
                                double *norms, cudaStream_t st);
// Device-side control of the refinement loop: after each update pass, the stopping test computes
// rel = max_col ||r|| / ||b|| from the norms, decides whether the pair iteration is done and
// zeroes norms[col][0] for the next pass.
struct RefineState {
    int done;        // 1: converged (rel <= rtol), 2: stopped (floor, stagnation, max_iter, not finite)
    int iters;       // correction sweeps applied
    double rel;      // latest max relative residual
    double prev;     // the one before
    unsigned blocks; // update blocks finished in the current pass (the last one runs the test)
};
// The state is followed in memory by int sys[n_sys][2]: per system (frequency) the sweeps applied
// to it and a frozen flag, set once all its columns are at rtol; later updates (and, on the
// block-cyclic-reduction path, the solve's products) skip a frozen system, whose newest iterate
// then stays in the buffer of its own last sweep.
__host__ __device__ inline size_t refine_state_bytes(int n_sys) {
    return ((sizeof(RefineState) + 15) / 16) * 16 + 2 * sizeof(int) * (size_t)(n_sys > 0 ? n_sys : 1);
}
__host__ __device__ inline int *refine_sys(RefineState *st) {
    return reinterpret_cast<int *>(reinterpret_cast<char *>(st) + ((sizeof(RefineState) + 15) / 16) * 16);
}
__host__ __device__ inline const int *refine_sys(const RefineState *st) {
    return reinterpret_cast<const int *>(reinterpret_cast<const char *>(st) + ((sizeof(RefineState) + 15) / 16) * 16);
}
struct RefineStop {  // stopping rule of the pair phase, applied on the device
    double rtol, floor_rel;
    int max_iter;
};
// x_out = x_in (none: 0) + delta; r32 = leading part of bd - A x_out; norms[col][0] += ||r||^2
// (zero on entry: refine_start and the stopping test leave it so).  With state, the last block to
// finish applies the stopping test, and state->done makes later launches do
// nothing.
cudaError_t launch_refine_update(const GridGeom &g, int n_sys, int nrhs, const float4 *diag2, const float4 *bd,
                                 const float4 *x_in, const float2 *delta, float4 *x_out, float2 *r32, double *norms,
                                 cudaStream_t st, RefineState *state = nullptr, RefineStop stop = {});

// X = conj?(hi + lo) in FP64 of each system's newest iterate: xa after an odd number of sweeps of
// that system, else xb (columns of N nodes, nrhs columns per system)
cudaError_t launch_refine_finish(size_t n, int N, int nrhs, const float4 *xa, const float4 *xb,
                                 const RefineState *state, int conj, double2 *X, cudaStream_t st);
// X += conj?(delta) in FP64 (refinement tail with FP64 residuals)
cudaError_t launch_refine_accumulate(size_t n, const float2 *delta, int conj, double2 *X, cudaStream_t st);

// ---- zgemm_tc.cu (batched complex GEMM on tcgen05, 3xTF32)
// A family of complex FP32 matrices: matrix idx starts at base + (idx / div) * stride_hi +
// (idx % div) * stride (div <= 0: base + idx * stride); rows are ld elements apart.
struct ZOperand {
    const float2 *base = nullptr;
    long long stride = 0, stride_hi = 0;
    int div = 0;
    int ld = 0;
    // matrices of the family (div <= 0) or groups of div matrices (div > 0); 0 if not known.
    // Launches whose operands all have a count stream them with tensor copies (narrow tiles).
    long long count = 0;
};
// C_t = C0_t + sum_u sign_u A_{t,u} Bt_{t,u}^T for every task t of tasks[n_tasks][8]
// (a_idx[3], b_idx[3], c0_idx, c_idx); a term with a negative A index is absent from its task.  A: M x K, Bt: N x K (row-major); C, C0: M x N, row-major or (c_col) column-major.
struct ZGemmArgs {
    int M = 0, N = 0, K = 0;
    int nterms = 1;
    ZOperand A[3], B[3];
    float sign[3] = {1.f, 1.f, 1.f};
    ZOperand C0;          // base == nullptr: no C0
    float2 *C = nullptr;
    long long c_stride = 0, c_stride_hi = 0;
    int c_div = 0;
    int ldc = 0;
    int c_col = 0;
    const int *tasks = nullptr;
    int *status = nullptr;
    const int *skip = nullptr;
    uint32_t tries = 0;
    double flops = 0.0;   // useful flops of the launch (8 M N K per complex term of every task), for tracing
    // split-K: with part != nullptr a launch that fills less than a wave of CTAs splits each
    // task's K chunks over ksplit CTAs, which write partial tiles into part (at most part_cap
    // complex elements; laid out like C, without C0); a second kernel sums them in a fixed order
    // and adds C0.  Set by launch_zgemm.
    int ksplit = 1;
    float2 *part = nullptr;
    size_t part_cap = 0;
    // per-system skip (refinement): a task whose system (C index / sys_div) has
    // sys_frozen[2 * system] set does nothing
    const int *sys_frozen = nullptr;
    int sys_div = 1;
};
cudaError_t launch_zgemm(const ZGemmArgs &a, int n_tasks, cudaStream_t st);

}  // namespace helm
