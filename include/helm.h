/*
 * helm.h -- C ABI of libhelm, batched discrete 2D Helmholtz solves and the FWI /
 * bilevel-hypergradient hot path of Downing, Gazzola, Graham, Spence, "Optimising
 * seismic imaging design parameters via bilevel learning" (arXiv:2301.10762).
 *
 * Discretisation (Appendix "Numerical forward model"): P1 finite elements on a uniform
 * nx x nz rectangular grid cut into right triangles, nodal quadrature,
 *     A(m, w) = S - w^2 diag(d m) - i w diag(b sqrt(m)),
 * S the five-point stiffness (interior edge couplings -hz/hx horizontally, -hx/hz
 * vertically, halved on boundary edges, zero row sums), d the tensor-trapezoid lumped
 * mass (hx hz, halved per boundary direction), b the lumped boundary length.
 * The adjoint operator is A^H = S - w^2 diag(d m) + i w diag(b sqrt(m)).
 *
 * Layout conventions shared by every entry point:
 *   - node (i, j) sits at (x, z) = (i hx, j hz), z = 0 the top row, hx = lx/(nx-1),
 *     hz = lz/(nz-1); canonical node index k = i*nz + j (z fastest); N = nx*nz;
 *   - complex numbers are interleaved FP64 pairs (helm_c128, the layout of
 *     torch.complex128 / numpy complex128);
 *   - right-hand-side and solution blocks are [n_omega][nrhs][N]: one contiguous
 *     length-N column per (frequency, right-hand side);
 *   - "_dev" pointers are device (HBM) pointers owned by the caller; everything else is
 *     host memory owned by the caller.  Opaque handles (helm_op_t, helm_factor_t) and
 *     the HBM behind them are owned by the library and released by helm_*_destroy.
 *   - every call is asynchronous on the stream given to helm_assemble, except where a
 *     result is returned through a host pointer (that call synchronises the stream) and
 *     helm_solve / helm_adjoint_solve, which synchronise it to report the device status.
 *     A handle must not be used from two host threads or two streams at once.
 *   - a handle belongs to the device that was current at helm_assemble; make that device
 *     current for every later call on it (helm_solve_noalloc selects it itself).
 *   - no entry point aborts, exits or throws; each returns a helm_status.
 */
#ifndef HELM_H
#define HELM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HELM_OK = 0,
    HELM_EINVAL = 1,     /* invalid argument (sizes, NULL pointers, positions outside the grid) */
    HELM_ENOMEM = 2,     /* device allocation failed */
    HELM_ECUDA = 3,      /* a CUDA runtime call failed */
    HELM_ENOCONV = 4,    /* iterative refinement or PCG did not reach its tolerance */
    HELM_ESINGULAR = 5,  /* a zero or non-finite pivot was met in a line factorisation */
    HELM_ETIMEOUT = 6    /* a bounded device-side wait gave up */
} helm_status;

typedef struct { double re, im; } helm_c128;

/* Uniform grid: nx x nz nodes (both >= 4) on [0, lx] x [0, lz].  lumping: the nodal quadrature
 * of the mass term (Appendix "Numerical forward model"; the paper does not fix how the corner
 * nodes of its triangulation are weighted): HELM_LUMP_TENSOR (0, the default of a
 * zero-initialised struct) the tensor trapezoid hx hz q(i) q(j), q = 1/2 at the ends (every
 * corner hx hz / 4); HELM_LUMP_UP / HELM_LUMP_DOWN (1 / 2) the vertex quadrature of the P1
 * triangles cut along (i,j)-(i+1,j+1) / (i+1,j)-(i,j+1), a third of each triangle's area to each
 * vertex: the same weights except at the four corners (hx hz / 3 where the diagonal ends,
 * hx hz / 6 at the other two).  The stiffness of these right triangles does not depend on the
 * orientation. */
typedef struct { int32_t nx, nz; double lx, lz; int32_t lumping; } helm_grid;
#define HELM_LUMP_TENSOR 0
#define HELM_LUMP_UP 1
#define HELM_LUMP_DOWN 2

/* Precision of the line factors.  HELM_FP64: complex FP64 factors and sweeps.
 * HELM_MIXED: complex FP32 factors and sweeps, FP64 residuals and FP64 iterative
 * refinement x += A~^{-1}(b - A x) until ||b - A x|| / ||b|| <= rtol per column. */
typedef enum { HELM_FP64 = 0, HELM_MIXED = 1 } helm_prec;

/* Acquisition (Section 2, sets S and P): physical positions, host memory.
 * Sources: on a node, the right-hand side is e_s (Appendix, "Computing the wavefield");
 * off a node, the bilinear weights of the four surrounding nodes.
 * Receivers: the sliding bicubic restriction R(P) of Section "Numerical restriction
 * operator" (4 nearest nodes per direction, window clamped inside the grid).
 * rec_w are receiver weights w_j multiplying the misfit (phi uses ||W eps||^2); NULL
 * means w = 1, which is the paper's objective exactly. */
typedef struct {
    int32_t n_src, n_rec;
    const double *src_xz;   /* [n_src][2] */
    const double *src_amp;  /* [n_src] or NULL (amplitude 1) */
    const double *rec_xz;   /* [n_rec][2] */
    const double *rec_w;    /* [n_rec] or NULL (weight 1) */
} helm_acq;

typedef struct {
    int32_t iters;        /* refinement sweeps used (1 for HELM_FP64) */
    double max_relres;    /* max over columns of ||b - A x||_2 / ||b||_2, FP64; -1 if not computed */
} helm_solve_info;

typedef struct {
    int32_t max_iter;     /* PCG iteration cap (Hessian products after the first) */
    int32_t fixed_iters;  /* > 0: run exactly this many iterations, ignore rtol */
    double rtol;          /* stop when ||r_n|| / ||r_0|| <= rtol */
    double x0;            /* constant initial guess (the paper uses 1) */
    double refine_rtol;   /* residual tolerance of every Helmholtz solve (mixed mode) */
    int32_t concurrent_models;  /* training models processed at once (own streams and host
                                   threads); <= 0: library default (up to 3).  The results are
                                   summed in model order, so they do not depend on it. */
    int32_t factor_method;      /* helm_factor_method of every factor of the pass */
} helm_pcg_opts;

typedef struct {
    int32_t cg_matvecs;   /* Hessian-vector products, max over models (incl. initial residual) */
    double cg_relres;     /* ||r|| / ||r_0|| reached, max over models */
    int64_t solves;       /* Helmholtz right-hand-side solves of the hypergradient pass */
    int64_t data_solves;  /* solves spent generating the data u(m') */
    int32_t max_refine_iters;  /* largest refinement count of any solve (mixed) */
} helm_hyper_info;

typedef struct helm_op helm_op_t;
typedef struct helm_factor helm_factor_t;

const char *helm_status_string(helm_status s);
/* Text of the last error detected on the calling thread (empty if none). */
const char *helm_last_error(void);

/* helm_assemble -- operator A(m, w) for every w in omega (Appendix "Numerical forward
 * model", Eq. (matrices) with nodal quadrature).
 *   grid:    grid description (host).
 *   m_dev:   [N] squared slowness m = 1/c^2 > 0 (device, FP64); copied into the op.
 *   omega:   [n_omega] angular frequencies (host), n_omega >= 1.
 *   stream:  cudaStream_t used by every later call on this op and its factors
 *            (NULL = the legacy default stream).
 *   out:     receives the new handle.
 * Errors: EINVAL (nx or nz < 4, n_omega < 1, NULL pointers), ENOMEM, ECUDA. */
helm_status helm_assemble(const helm_grid *grid, const double *m_dev, const double *omega,
                          int32_t n_omega, void *stream, helm_op_t **out);
void helm_op_destroy(helm_op_t *op);

/* Factor methods.  HELM_FACTOR_LINE: the line-by-line Schur recurrence below.
 * HELM_FACTOR_BCR (HELM_MIXED only, even nz >= 16): block cyclic reduction of the same
 * block-tridiagonal system -- every other line of the current system is eliminated at once,
 * level by level (log2(nx) levels), so that each level is a batch of independent dense block
 * inversions and block products over all lines and frequencies, run on the tensor cores
 * (complex products as real TF32 products with the 3xTF32 split, FP32 accumulation).  Its
 * storage is about 3 nx nz^2 complex FP32 entries per frequency.  HELM_FACTOR_AUTO (unless the
 * environment sets HELM_FACTOR=line or =bcr): BCR for HELM_MIXED on lines of nz >= 192 nodes
 * (where the line recurrence's chain of nx dependent line inversions dominates), else the line
 * recurrence. */
typedef enum { HELM_FACTOR_AUTO = 0, HELM_FACTOR_LINE = 1, HELM_FACTOR_BCR = 2 } helm_factor_method;
typedef struct {
    int32_t method;       /* helm_factor_method */
} helm_factor_opts;

/* helm_factor -- block-tridiagonal (line-by-line) factorisation of every A(m, w_q):
 * with lines of constant i, A has diagonal blocks D_i (tridiagonal n_z x n_z) and
 * diagonal couplings C_i; the factor stores G_i = S_i^{-1} with
 * S_0 = D_0, S_i = D_i - C_i S_{i-1}^{-1} C_i.  This replaces the sparse direct
 * (backslash) factorisation of the Appendix ("Computing the wavefield").
 * Each S_i is inverted by block Gauss-Jordan over 16-column blocks; a 16 x 16 pivot block
 * is inverted by Newton-Schulz iteration seeded with the same block's inverse on the
 * previous line, or by Gauss-Jordan with partial pivoting where that seed is not close
 * enough.  opts may be NULL (HELM_FACTOR_AUTO).
 * Errors: EINVAL (bad method, or HELM_FACTOR_BCR where it does not apply), ESINGULAR (zero /
 * non-finite pivot), ETIMEOUT (a bounded device-side wait gave up), ENOMEM, ECUDA.
 * The factor keeps a reference to op: destroy the factor before the op. */
helm_status helm_factor(helm_op_t *op, helm_prec prec, const helm_factor_opts *opts, helm_factor_t **out);
void helm_factor_destroy(helm_factor_t *f);

/* helm_set_wait_tries -- diagnostic setting (no counterpart in the paper): the number of
 * times a bounded device-side wait of the line factor and sweep kernels polls its barrier
 * before it gives up, for launches made after the call.  tries < 0 restores the default
 * (2^22 polls, each suspended for a hardware time limit: seconds at worst); 0 gives up at
 * the first wait that is not already complete.  A kernel that gives up stops all CTAs of its
 * cluster, leaves its outputs incomplete and the call returns HELM_ETIMEOUT; the context stays
 * usable and the next call starts clean.  Process-wide; meant for tests of that error path. */
void helm_set_wait_tries(int64_t tries);

/* helm_fault_mask -- host-side fault injection (no counterpart in the paper; for tests of the
 * failure paths).  The environment variable HELM_FAULT, read at every call that can take the
 * path, is a comma-separated list of:
 *   alloc    every device allocation of the library fails (calls return HELM_ENOMEM);
 *   pivot    helm_factor factors a copy of A's diagonal whose first entry the host set to NaN
 *            (the factor kernels meet a non-finite pivot: HELM_ESINGULAR; the op is unchanged);
 *   timeout  bounded device-side waits take a try limit of zero, as after
 *            helm_set_wait_tries(0): the first wait that is not already complete gives up
 *            (HELM_ETIMEOUT);
 *   nan_rhs  helm_solve / helm_adjoint_solve solve a copy of B whose first entry is NaN (the
 *            residual is not finite: HELM_ENOCONV).
 * Returns the bits the current value selects (HELM_FAULT_UNKNOWN for unrecognised words).
 * Nothing faults, traps or hangs the device. */
#define HELM_FAULT_ALLOC 0x1u
#define HELM_FAULT_PIVOT 0x2u
#define HELM_FAULT_TIMEOUT 0x4u
#define HELM_FAULT_NAN_RHS 0x8u
#define HELM_FAULT_UNKNOWN 0x80000000u
uint32_t helm_fault_mask(void);

/* helm_factor_get_method -- the method a factor was built with (HELM_FACTOR_LINE or
 * HELM_FACTOR_BCR); -1 for NULL. */
int32_t helm_factor_get_method(const helm_factor_t *f);

/* helm_factor_fp64_blocks -- HELM_MIXED: number of 16 x 16 pivot blocks of the factor that
 * were flagged and inverted in FP64.  A block is flagged when its FP32 Gauss-Jordan inverse X
 * leaves max |I - M X| above 1e-4 (an ill-conditioned pivot of a line); it is then inverted
 * again from the same FP32 entries by Gauss-Jordan with partial pivoting in FP64 and rounded
 * to FP32.  0 for HELM_FP64; -1 for NULL.  (The paper's solver has no counterpart: it factors
 * in FP64 throughout.) */
int32_t helm_factor_fp64_blocks(const helm_factor_t *f);

/* helm_solve -- X = A(m, w_q)^{-1} B for every frequency q and column (Eq. (defu)
 * discretised: u = A^{-1} e_s).  B_dev, X_dev: [n_omega][nrhs][N] complex (device);
 * they may not alias.  rtol / max_iter drive the refinement of HELM_MIXED (ignored by
 * HELM_FP64 except that info->max_relres is computed when info != NULL).  The call
 * synchronises the op's stream.
 * Errors: EINVAL, ENOCONV (mixed: max_iter reached above rtol, or a non-finite residual;
 * FP64 with info: a non-finite residual; X holds the last iterate), ETIMEOUT (a bounded device-side wait of a sweep gave up; X is incomplete),
 * ECUDA. */
helm_status helm_solve(helm_factor_t *f, int32_t nrhs, const helm_c128 *B_dev, helm_c128 *X_dev,
                       double rtol, int32_t max_iter, helm_solve_info *info);

/* helm_adjoint_solve -- X = (A^H)^{-1} B, the discrete adjoint solution operator
 * S*_{m,w} of Definition def:solnop (Eq. (lambda)).  Since A is complex symmetric,
 * it is computed from the same factor as conj(A^{-1} conj(B)).  Arguments as helm_solve. */
helm_status helm_adjoint_solve(helm_factor_t *f, int32_t nrhs, const helm_c128 *B_dev,
                               helm_c128 *X_dev, double rtol, int32_t max_iter,
                               helm_solve_info *info);

/* helm_solve_noalloc -- helm_solve (adjoint = 0) or helm_adjoint_solve (adjoint != 0)
 * that allocates nothing, for callers that cannot allocate device memory at solve time
 * (a serving process whose device memory was partitioned once at start-up, a host
 * framework whose caching allocator owns the free device memory, or a loop that cannot
 * take the device-wide synchronisation of cudaMalloc / cudaFree).  The paper has no
 * counterpart: this is a property of the library, not of the method.
 * The working memory of the refinement (right-hand side and iterates as FP32 pairs, FP32
 * line vectors, per-column norms, the refinement's stopping state) lives in one fixed 32 MiB array in device global memory
 * that every GPU loading the library holds until exit; the caller still passes B_dev and
 * X_dev.  Limits: n_omega * nrhs * N * 64 bytes (mixed; norms only for FP64) within 32 MiB and at most
 * 16384 columns, else HELM_EINVAL.  The call makes the op's device (the one current at
 * helm_assemble) current while it runs and restores the caller's device before returning.
 * The first call on a device resolves the array's device address with that device
 * current: make it before any stream capture.  Calls
 * share the array (each clears what must start at zero); calls that overlap on the GPU
 * race and must be serialised by the caller.  Other arguments and errors as helm_solve. */
helm_status helm_solve_noalloc(helm_factor_t *f, int32_t nrhs, const helm_c128 *B_dev, helm_c128 *X_dev,
                               double rtol, int32_t max_iter, int32_t adjoint, helm_solve_info *info);

/* helm_sources -- right-hand sides e_s (Appendix, "Computing the wavefield"),
 * B_dev [n_omega][n_src][N] (identical for every frequency), amplitudes src_amp. */
helm_status helm_sources(const helm_op_t *op, const helm_acq *acq, helm_c128 *B_dev);

/* helm_restrict -- Y = R(P) X (Eq. (Rv), sliding bicubic), X_dev [n_omega][ncol][N],
 * Y_dev [n_omega][ncol][n_rec]. */
helm_status helm_restrict(const helm_op_t *op, const helm_acq *acq, int32_t ncol,
                          const helm_c128 *X_dev, helm_c128 *Y_dev);

/* helm_restrict_adjoint -- X = R(P)^T Y, the transpose of helm_restrict (the discrete
 * realisation of R* used for the adjoint right-hand side, Theorem th:grad).  Y_dev
 * [n_omega][ncol][n_rec], X_dev [n_omega][ncol][N] (overwritten).  Sums run over the
 * receivers in a fixed order (bitwise reproducible).  Synchronises the op's stream. */
helm_status helm_restrict_adjoint(const helm_op_t *op, const helm_acq *acq, int32_t ncol,
                                  const helm_c128 *Y_dev, helm_c128 *X_dev);

/* helm_field_grad -- gradient with respect to m of a real functional L of the wavefields
 * U = A(m)^{-1} B, by the adjoint-state argument of Theorem th:grad (Eq. (I4)): for
 * dL = Re sum conj(G) dU and Lam = (A^H)^{-1} G (helm_adjoint_solve),
 *   grad_k = Re sum_{w,q} g_k(w) U_{w,q,k} conj(Lam_{w,q,k}),  g_k = w^2 d_k + i w b_k / (2 sqrt(m_k)),
 * since dU/dm_k = A^{-1}(g_k e_k U_k) (Proposition prop:elem, Eq. (oneMgrad2a)).  U_dev, Lam_dev [n_omega][nrhs][N] (device),
 * grad_dev [N] FP64 (device, overwritten; summed over frequencies and columns in a fixed
 * order).  Asynchronous on the op's stream. */
helm_status helm_field_grad(const helm_op_t *op, int32_t nrhs, const helm_c128 *U_dev, const helm_c128 *Lam_dev,
                            double *grad_dev);

/* fwi_misfit_grad -- phi and grad phi of Eq. (newphi) by the adjoint-state method
 * (Algorithm alg:box1, Theorem th:grad):
 *   u = A^{-1} e_s, eps = d - R u, lambda = (A^H)^{-1} R^T (W^2 eps),
 *   phi = 1/2 sum |W eps|^2 + 1/2 m^T Gamma m,
 *   grad_k = -Re sum_{s,w} g_k u_k conj(lambda_k) + (Gamma m)_k,
 *   g_k = w^2 d_k + i w b_k / (2 sqrt(m_k)),  Gamma = alpha R + mu I (Eq. (Gamma)).
 *   data_dev: [n_omega][n_src][n_rec] complex (device).
 *   phi: host scalar (this call synchronises).  grad_dev: [N] FP64 (device).
 *   u_out, lam_out: optional [n_omega][n_src][N] (device) or NULL. */
helm_status fwi_misfit_grad(helm_factor_t *f, const helm_acq *acq, const helm_c128 *data_dev,
                            double alpha, double mu, double rtol, double *phi, double *grad_dev,
                            helm_c128 *u_out, helm_c128 *lam_out);

/* helm_gamma_solve -- Z = Gamma(alpha0, mu)^{-1} R for ncol real vectors: the preconditioner
 * P2 = Gamma(alpha0, mu) = alpha0 R + mu I of Eq. (P2) (R the regulariser of Eq. (Gamma), with
 * the literal (n - 1) difference scaling, so Gamma depends on nx and nz only, not on lx, lz).
 * The same solver as the PCG of bilevel_hypergrad: the 2D DCT-II diagonalises R, so the
 * inverse is exact (FP64 rounding), not iterative.
 *   R_dev, Z_dev: [ncol][N] FP64 (device, canonical node order); Z_dev may alias R_dev.
 *   stream: cudaStream_t (as void *); the call synchronises it.
 * Errors: EINVAL (nx or nz < 2, ncol < 0, alpha0 < 0, mu <= 0, NULL arrays), ENOMEM, ECUDA. */
helm_status helm_gamma_solve(const helm_grid *grid, double alpha0, double mu, int32_t ncol, const double *R_dev,
                             double *Z_dev, void *stream);

/* fwi_hessian_vec -- Hessian-vector product of phi for a real direction m~ (Lemmas
 * thm:H1 and thm:H2, Discussion disc:Hess): per (s, w) two new solves
 *   v = A^{-1}(g u m~),  z = (A^H)^{-1}(R^T W^2 R v - m~ conj(g) lambda),
 *   (H m~)_k = sum_{s,w} Re[g_k u_k conj(z_k)] - Re[g_k v_k conj(lambda_k)]
 *              - Re[g'_k u_k conj(lambda_k)] m~_k + (Gamma m~)_k,   g'_k = -i w b_k / (4 m_k^{3/2}).
 * (The second term uses G^* lambda = conj(g) lambda, as in the proof of Lemma thm:H2.)
 *   u_dev, lam_dev: [n_omega][n_src][N] wavefields and adjoint fields at the factor's
 *   model, e.g. the u_out / lam_out of fwi_misfit_grad (lam_dev may be NULL when
 *   gauss_newton != 0).  mt_dev, hv_dev: [N] FP64 (device).
 *   gauss_newton != 0: the Gauss-Newton part H1 m~ + Gamma m~ only (z without the
 *   lambda term, no H2 terms). */
helm_status fwi_hessian_vec(helm_factor_t *f, const helm_acq *acq, const helm_c128 *u_dev,
                            const helm_c128 *lam_dev, const double *mt_dev, double alpha, double mu,
                            double rtol, int32_t gauss_newton, double *hv_dev);

/* bilevel_hypergrad -- upper-level objective and hypergradient (Algorithm alg:box,
 * Theorems sogradt1 and sogradta), averaged over n_models training models:
 *   per model: data u' = A(m')^{-1} e_s on the same grid; u, lambda at m_fwi;
 *   rho = H^{-1}(m' - m_fwi) by PCG with preconditioner P2 = Gamma(alpha0, mu)
 *   (Eq. (P2)), each Hessian product costing 2 solves per (s, w) (Discussion disc:Hess);
 *   tau = A^{-1}(g u rho) (Eq. (tau_def));
 *   psi = 1/(2 N_m') sum ||m' - m_fwi||^2, dpsi/dalpha = 1/N_m' sum m_fwi^T R rho,
 *   dpsi/dp_{j,l} = 1/N_m' sum_{m',s,w} w_j^2 Re[conj((dR_l tau)_j)(R(u-u'))_j
 *                                              + conj((R tau)_j)(dR_l(u-u'))_j],
 *   dpsi/dw_j = -1/N_m' sum 2 w_j Re[conj((R tau)_j)(R(u'-u))_j].
 *   grids[n_models], m_fwi[n_models], m_true[n_models], acq[n_models]: per model (device
 *   vectors of length nx*nz of that model's grid; each model's own sources, and receivers in
 *   the same number for all models, since dpsi_dp and dpsi_dw are per receiver); omega is
 *   shared by all models.
 *   data_grids[n_models], m_data[n_models]: both NULL (the data u' = A(m')^{-1} e_s on the
 *   model's grid, from m_true) or both given: the data computed on another grid of the same
 *   domain (same lx, lz; the Appendix's data generation against the inverse crime), from m'
 *   sampled on it (device, length nx*nz of that grid); then d = R' u' and the receiver
 *   derivatives dR'_l u' are that grid's and R(u - u') above reads R u - R' u' (likewise for
 *   dR_l).  m_true stays the model on the inversion grid (psi and the rho system).
 *   Outputs are host scalars / arrays (the call synchronises).  dpsi_dw may be NULL. */
helm_status bilevel_hypergrad(int32_t n_models, const helm_grid *grids, const double *const *m_fwi,
                              const double *const *m_true, const helm_acq *acq /* [n_models] */,
                              const helm_grid *data_grids /* [n_models] or NULL */,
                              const double *const *m_data /* [n_models] or NULL */,
                              const double *omega, int32_t n_omega, double alpha, double alpha0,
                              double mu, helm_prec prec, const helm_pcg_opts *pcg, void *stream,
                              double *psi, double *dpsi_dalpha, double *dpsi_dp, double *dpsi_dw,
                              helm_hyper_info *info);

#ifdef __cplusplus
}
#endif
#endif /* HELM_H */
