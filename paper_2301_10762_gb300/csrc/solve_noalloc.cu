// helm_solve_noalloc: helm_solve / helm_adjoint_solve for callers that cannot allocate
// device memory at solve time.
//
// Some callers must not call cudaMalloc when they solve: a serving process whose device
// memory was carved up once at start-up (a further allocation could fail or fragment
// it), a host framework whose caching allocator already owns the free device memory,
// and latency-critical loops that cannot afford the device-wide synchronisation that
// cudaMalloc / cudaFree imply.  helm_solve meets the working memory of the mixed path
// (FP32-pair right-hand side and iterates, FP32 line vectors, per-column norms) by growing
// buffers inside the factor handle on first use, which allocates.  This variant runs the same kernels with
// that working memory placed in one fixed array in device global memory, declared
// below, which every GPU that loads the library holds until the process exits.
//
// Consequences for the caller:
//   * the call runs with the op's device current (the device that was current at
//     helm_assemble), whichever device the caller has made current, and restores the
//     caller's device before it returns;
//   * the first call on a device resolves the device address of the array
//     (cudaGetSymbolAddress, with that device current); make that first call before
//     any stream capture;
//   * every call shares the array and it keeps the previous call's contents (the
//     norms are cleared by each call before use); calls that overlap on the GPU, from
//     any stream or host thread, race on it and must be serialised by the caller;
//   * sizes beyond the array are rejected with HELM_EINVAL.
#include <math.h>
#include <mutex>

#include "helm.h"
#include "kernels.h"
#include "abi_internal.h"

using namespace helm;

namespace {

constexpr size_t kScratchBytes = (size_t)32 << 20;   // 32 MiB per GPU
constexpr size_t kMaxCols = 16384;                    // columns (frequency x right-hand side) per call
constexpr int kMaxDevices = 64;

// the working memory of the no-allocation solve (device global memory, one per GPU)
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_dev_addr[kMaxDevices] = {};
double g_norms_host[2 * kMaxCols];

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// device address of the array on device `dev`, which must be current (resolved once per device)
helm_status scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= kMaxDevices) {
        helm_set_msg("helm_solve_noalloc: device index beyond the library's table");
        return HELM_EINVAL;
    }
    if (!g_dev_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            helm_set_error("helm_solve_noalloc: cudaGetSymbolAddress", e);
            return HELM_ECUDA;
        }
        g_dev_addr[dev] = p;
    }
    *out = g_dev_addr[dev];
    return HELM_OK;
}

// makes `dev` the current device for the lifetime of the guard and restores the caller's
struct DeviceGuard {
    int prev = -1;
    bool switched = false;
    cudaError_t enter(int dev) {
        cudaError_t e = cudaGetDevice(&prev);
        if (e != cudaSuccess) return e;
        if (prev != dev) {
            if ((e = cudaSetDevice(dev)) != cudaSuccess) return e;
            switched = true;
        }
        return cudaSuccess;
    }
    ~DeviceGuard() {
        if (switched) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" helm_status helm_solve_noalloc(helm_factor_t *f, int32_t nrhs, const helm_c128 *B_dev,
                                          helm_c128 *X_dev, double rtol, int32_t max_iter, int32_t adjoint,
                                          helm_solve_info *info) {
    if (!f || nrhs < 0 || (nrhs > 0 && (!B_dev || !X_dev)) || (const void *)B_dev == (const void *)X_dev) {
        helm_set_msg("helm_solve_noalloc: bad arguments (NULL, nrhs < 0 or B aliases X)");
        return HELM_EINVAL;
    }
    if (info) { info->iters = 0; info->max_relres = -1.0; }
    if (nrhs == 0) return HELM_OK;
    const helm_op *op = f->op;
    const GridGeom &g = op->g;
    const int n_sys = op->n_omega;
    const size_t N = (size_t)g.nx * g.nz;
    const size_t cols = (size_t)n_sys * nrhs;
    const bool mixed = f->prec == HELM_MIXED;
    const size_t p_bytes = mixed ? align256(cols * N * sizeof(float4)) : 0;   // bd, xa, xb
    const size_t v_bytes = mixed ? align256(cols * N * sizeof(float2)) : 0;   // r32, y
    const size_t n_bytes = align256(cols * 2 * sizeof(double));
    const size_t s_bytes = mixed ? align256(refine_state_bytes(n_sys)) : 0;
    if (cols > kMaxCols || 3 * p_bytes + 2 * v_bytes + n_bytes + s_bytes > kScratchBytes) {
        helm_set_msg("helm_solve_noalloc: problem larger than the fixed working array "
                     "(32 MiB: n_omega*nrhs*N*64 bytes plus norms and the refinement state, at most 16384 columns)");
        return HELM_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    // every buffer of the op, its stream and the array's address belong to the device that was
    // current at helm_assemble: the call runs with that device current, whichever is current now
    DeviceGuard dg;
    cudaError_t e = dg.enter(op->dev);
    if (e != cudaSuccess) { helm_set_error("helm_solve_noalloc: select the op's device", e); return HELM_ECUDA; }
    void *base = nullptr;
    helm_status s = scratch_address(op->dev, &base);
    if (s != HELM_OK) return s;
    unsigned char *p = (unsigned char *)base;
    const double2 *B = (const double2 *)B_dev;
    double2 *X = (double2 *)X_dev;
    const int conj = adjoint ? 1 : 0;
    const int rchunk = 16;
    double rel = -1.0;
    int it = 1;
    // the status bits report this call only
    if ((e = cudaMemsetAsync(op->status, 0, sizeof(int), op->st)) != cudaSuccess) {
        helm_set_error("helm_solve_noalloc: clear status", e);
        return HELM_ECUDA;
    }
    if (!mixed) {
        double *norms = (double *)p;
        e = launch_line_sweep<double>(g, n_sys, nrhs, (const double2 *)f->G, B, X, X, conj, rchunk, op->status, op->st,
                                      f->mid);
        if (e != cudaSuccess) { helm_set_error("helm_solve_noalloc: sweep", e); return HELM_ECUDA; }
        if (info) {
            e = cudaMemsetAsync(norms, 0, cols * 2 * sizeof(double), op->st);
            if (e == cudaSuccess) e = launch_residual(g, n_sys, nrhs, op->diag, B, X, nullptr, norms, conj, op->st);
            if (e != cudaSuccess) { helm_set_error("helm_solve_noalloc: residual", e); return HELM_ECUDA; }
            if ((s = max_relres(op, cols, norms, g_norms_host, &rel)) != HELM_OK) return s;
        }
    } else {
        MixedWork w;
        w.bd = (float4 *)p;
        w.xa = (float4 *)(p + p_bytes);
        w.xb = (float4 *)(p + 2 * p_bytes);
        w.r32 = (float2 *)(p + 3 * p_bytes);
        w.y = (float2 *)(p + 3 * p_bytes + v_bytes);
        w.norms = (double *)(p + 3 * p_bytes + 2 * v_bytes);
        w.norms_host = g_norms_host;
        w.state = (RefineState *)(p + 3 * p_bytes + 2 * v_bytes + n_bytes);
        if ((s = mixed_refine(f, nrhs, B, X, conj, rtol, max_iter, w, &it, &rel)) != HELM_OK) return s;
    }
    if (info) { info->iters = it; info->max_relres = rel; }
    if ((s = read_sweep_status(op)) != HELM_OK) return s;
    if (mixed && !(rel <= rtol)) { helm_set_msg("refinement did not reach rtol"); return HELM_ENOCONV; }
    return HELM_OK;
}
