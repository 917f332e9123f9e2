// Host-side launch wrappers of the libhelm kernels (internal, C++ only).
#pragma once
#include <cuda_runtime.h>
#include "common.cuh"

namespace helm {

constexpr int NB = 16;   // diagonal-block size of the line inversions

// ---- assemble.cu
cudaError_t launch_assemble(const GridGeom &g, const double *m, const double *omega_dev, int n_omega,
                            double2 *diag, cudaStream_t st);
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
template <typename TG>
cudaError_t launch_line_sweep(const GridGeom &g, int n_sys, int nrhs, const cx_t<TG> *G, const double2 *B,
                              double2 *X, cx_t<TG> *Y, int conj, int accumulate, int rchunk, int *status,
                              cudaStream_t st, int mid);
cudaError_t launch_residual(const GridGeom &g, int n_sys, int nrhs, const double2 *diag, const double2 *B,
                            const double2 *X, double2 *R, double *norms, int conj, cudaStream_t st);

int pick_cluster_size(int nz);

}  // namespace helm
