/*
 * helm_blas.h -- the dense building blocks of libhelm's block-cyclic-reduction factor
 * (helm_factor with HELM_FACTOR_BCR), at the C ABI.  The paper has no counterpart: it factors
 * the sparse operator with a sparse direct solver.  They are exposed so that the tensor-core
 * kernels can be used, timed and checked on their own.
 *
 * Complex FP32 matrices are interleaved (re, im) pairs (helm_c64, the layout of
 * torch.complex64).  Pointers are device pointers owned by the caller; sizes and strides
 * count complex elements.  Both calls run on the given stream (a cudaStream_t, NULL = the
 * legacy default stream) of the current device.
 */
#ifndef HELM_BLAS_H
#define HELM_BLAS_H

#include <stdint.h>
#include "helm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { float re, im; } helm_c64;

/* helm_zgemm_batched -- C_t = C0_t + sign * A_t Bt_t^T for t < batch, on the tensor cores:
 * tcgen05 MMAs with the accumulator in tensor memory, the complex product as a real TF32
 * product (A as a real M x 2K matrix, each row of Bt expanded into two real rows), every
 * operand split as hi = tf32(x) + lo and hi*hi + hi*lo + lo*hi accumulated in FP32.
 *   A:  [batch] M x K, row-major, row stride lda, matrix stride sa;
 *   Bt: [batch] N x K, row-major, row stride ldb, matrix stride sb;
 *   C0: [batch] M x N, row-major (ldc, sc), or NULL (zero); may be the same memory as C;
 *   C:  [batch] M x N, row-major, row stride ldc, matrix stride sc (may not overlap A, Bt).
 *   K, lda, ldb, sa, sb even; A and Bt 16-byte aligned; sign +1 or -1; batch <= 65535.
 * Asynchronous.  Errors: EINVAL (sizes, alignment), ENOMEM, ECUDA. */
helm_status helm_zgemm_batched(int32_t batch, int32_t M, int32_t N, int32_t K, const helm_c64 *A, int64_t sa,
                               int32_t lda, const helm_c64 *Bt, int64_t sb, int32_t ldb, float sign,
                               const helm_c64 *C0, helm_c64 *C, int64_t sc, int32_t ldc, void *stream);

/* helm_zinv_batched -- X_t = A_t^{-1} for t < batch, complex FP32, n x n complex symmetric
 * matrices (A = A^T, the line blocks of the Helmholtz operator and their Schur complements).
 * n <= 128: block Gauss-Jordan in one CTA's shared memory over 16-column blocks, each 16 x 16
 * pivot block inverted by one warp with partial pivoting; n > 128: the 2 x 2 block inverse of a
 * symmetric matrix with 128-multiple leading blocks, its products on the tensor cores
 * (helm_zgemm_batched) and its two half-size inverses recursive.  A and X row-major with row
 * strides lda, ldx and matrix strides sa, sx; X may be A (in place).  n even, lda, ldx, sa, sx
 * even, 16-byte aligned.  Synchronises the stream.
 * Errors: EINVAL, ESINGULAR (a zero or non-finite pivot), ENOMEM, ECUDA. */
helm_status helm_zinv_batched(int32_t batch, int32_t n, const helm_c64 *A, int64_t sa, int32_t lda, helm_c64 *X,
                              int64_t sx, int32_t ldx, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* HELM_BLAS_H */
