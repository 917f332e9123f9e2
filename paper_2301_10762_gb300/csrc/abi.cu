// extern "C" entry points of libhelm (declared in include/helm.h): handle management,
// argument checks and orchestration of the kernels.  No computation of the path runs
// on the host; the host only sequences launches and reads scalars back.
#include <math.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>
#include <algorithm>
#include <string>
#include <vector>

#include <atomic>
#include <mutex>
#include "helm.h"
#include "kernels.h"
#include "abi_internal.h"

using namespace helm;

static thread_local std::string g_last_error;

void helm_set_error(const char *what, cudaError_t e) {
    char buf[512];
    snprintf(buf, sizeof buf, "%s: %s", what, e == cudaSuccess ? "ok" : cudaGetErrorString(e));
    g_last_error = buf;
}
void helm_set_msg(const char *what) { g_last_error = what; }

extern "C" const char *helm_status_string(helm_status s) {
    switch (s) {
        case HELM_OK: return "HELM_OK";
        case HELM_EINVAL: return "HELM_EINVAL: invalid argument";
        case HELM_ENOMEM: return "HELM_ENOMEM: device allocation failed";
        case HELM_ECUDA: return "HELM_ECUDA: CUDA runtime error";
        case HELM_ENOCONV: return "HELM_ENOCONV: iteration did not reach its tolerance";
        case HELM_ESINGULAR: return "HELM_ESINGULAR: zero or non-finite pivot in a line factorisation";
        case HELM_ETIMEOUT: return "HELM_ETIMEOUT: bounded device wait gave up";
    }
    return "HELM_?: unknown status";
}

extern "C" const char *helm_last_error(void) { return g_last_error.c_str(); }

static std::atomic<int64_t> g_wait_tries{-1};

// Host-side fault injection, read from the environment at every call that can take the path.
// HELM_FAULT is a comma-separated list of: alloc (every device allocation of the library
// fails: ENOMEM), pivot (helm_factor factors a copy of A's diagonal with its first entry set
// to NaN from the host, so the factor kernels meet a non-finite pivot: ESINGULAR), timeout
// (the bounded device waits take a try limit of zero and give up at the first wait that is not
// already complete: ETIMEOUT), nan_rhs (helm_solve / helm_adjoint_solve work on a copy of B whose first entry is
// NaN: the residual is not finite, ENOCONV).  Unknown words set HELM_FAULT_UNKNOWN.  Nothing
// here faults, traps or hangs the device.
uint32_t helm::fault_flags() {
    const char *env = getenv("HELM_FAULT");
    uint32_t f = 0;
    if (!env) return 0;
    const char *p = env;
    while (*p) {
        const char *q = p;
        while (*q && *q != ',') ++q;
        const size_t n = (size_t)(q - p);
        if (n == 5 && !strncmp(p, "alloc", 5)) f |= HELM_FAULT_ALLOC;
        else if (n == 5 && !strncmp(p, "pivot", 5)) f |= HELM_FAULT_PIVOT;
        else if (n == 7 && !strncmp(p, "timeout", 7)) f |= HELM_FAULT_TIMEOUT;
        else if (n == 7 && !strncmp(p, "nan_rhs", 7)) f |= HELM_FAULT_NAN_RHS;
        else if (n > 0) f |= HELM_FAULT_UNKNOWN;
        p = *q ? q + 1 : q;
    }
    return f;
}

extern "C" uint32_t helm_fault_mask(void) { return helm::fault_flags(); }

uint32_t helm::wait_tries() {
    if (fault_flags() & HELM_FAULT_TIMEOUT) return 0;
    const int64_t v = g_wait_tries.load(std::memory_order_relaxed);
    return v < 0 ? kDefaultWaitTries : (uint32_t)std::min<int64_t>(v, 0xffffffffLL);
}

extern "C" void helm_set_wait_tries(int64_t tries) { g_wait_tries.store(tries < 0 ? -1 : tries); }

void keep_pool_memory() {
    static std::once_flag once;
    std::call_once(once, []() {
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        cudaGetLastError();
    });
}

helm_status dev_alloc(void **p, size_t bytes, const char *what, cudaStream_t st) {
    *p = nullptr;
    if (bytes == 0) return HELM_OK;
    if (fault_flags() & HELM_FAULT_ALLOC) {
        helm_set_msg((std::string(what) + ": allocation refused (HELM_FAULT=alloc)").c_str());
        return HELM_ENOMEM;
    }
    keep_pool_memory();
    cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        helm_set_error(what, e);
        return e == cudaErrorMemoryAllocation ? HELM_ENOMEM : HELM_ECUDA;
    }
    return HELM_OK;
}

void dev_free(void *p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

// ---------------------------------------------------------------------- operator

extern "C" helm_status helm_assemble(const helm_grid *grid, const double *m_dev, const double *omega,
                                     int32_t n_omega, void *stream, helm_op_t **out) {
    if (!out) { helm_set_msg("helm_assemble: NULL out"); return HELM_EINVAL; }
    *out = nullptr;
    if (!grid || !m_dev || !omega || n_omega < 1) { helm_set_msg("helm_assemble: NULL argument or n_omega < 1"); return HELM_EINVAL; }
    if (grid->nx < 4 || grid->nz < 4 || !(grid->lx > 0) || !(grid->lz > 0) || grid->lumping < HELM_LUMP_TENSOR ||
        grid->lumping > HELM_LUMP_DOWN) {
        helm_set_msg("helm_assemble: need nx, nz >= 4, positive lengths and a known lumping");
        return HELM_EINVAL;
    }
    for (int w = 0; w < n_omega; ++w)
        if (!isfinite(omega[w])) { helm_set_msg("helm_assemble: non-finite omega"); return HELM_EINVAL; }
    helm_op *op = new (std::nothrow) helm_op();
    if (!op) return HELM_ENOMEM;
    op->g = GridGeom{grid->nx, grid->nz, grid->lx / (grid->nx - 1), grid->lz / (grid->nz - 1), grid->lumping};
    op->lx = grid->lx;
    op->lz = grid->lz;
    op->n_omega = n_omega;
    op->omega.assign(omega, omega + n_omega);
    op->st = (cudaStream_t)stream;
    if (cudaGetDevice(&op->dev) != cudaSuccess) {
        cudaGetLastError();
        helm_set_msg("helm_assemble: cudaGetDevice failed");
        delete op;
        return HELM_ECUDA;
    }
    const size_t N = (size_t)grid->nx * grid->nz;
    helm_status s;
    if ((s = dev_alloc((void **)&op->m, N * sizeof(double), "allocate(m)", op->st)) != HELM_OK ||
        (s = dev_alloc((void **)&op->omega_dev, n_omega * sizeof(double), "allocate(omega)", op->st)) != HELM_OK ||
        (s = dev_alloc((void **)&op->diag, (size_t)n_omega * N * sizeof(double2), "allocate(diag)", op->st)) != HELM_OK ||
        (s = dev_alloc((void **)&op->status, 2 * sizeof(int), "allocate(status)", op->st)) != HELM_OK ||
        (s = dev_alloc((void **)&op->gk, (size_t)n_omega * N * sizeof(double2), "allocate(g)", op->st)) != HELM_OK ||
        (s = dev_alloc((void **)&op->gpk, (size_t)n_omega * N * sizeof(double2), "allocate(g')", op->st)) != HELM_OK) {
        helm_op_destroy(op);
        return s;
    }
    cudaError_t e;
    if ((e = cudaMemcpyAsync(op->m, m_dev, N * sizeof(double), cudaMemcpyDeviceToDevice, op->st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(op->omega_dev, omega, n_omega * sizeof(double), cudaMemcpyHostToDevice, op->st)) !=
            cudaSuccess ||
        (e = cudaMemsetAsync(op->status, 0, 2 * sizeof(int), op->st)) != cudaSuccess ||
        (e = launch_assemble(op->g, op->m, op->omega_dev, n_omega, op->diag, op->st)) != cudaSuccess ||
        (e = launch_gcoef(op->g, op->m, op->omega_dev, n_omega, op->gk, op->gpk, op->st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(op->st)) != cudaSuccess) {
        helm_set_error("helm_assemble", e);
        helm_op_destroy(op);
        return HELM_ECUDA;
    }
    *out = op;
    return HELM_OK;
}

extern "C" void helm_op_destroy(helm_op_t *op) {
    if (!op) return;
    dev_free(op->m, op->st);
    dev_free(op->omega_dev, op->st);
    dev_free(op->diag, op->st);
    dev_free(op->status, op->st);
    dev_free(op->gk, op->st);
    dev_free(op->gpk, op->st);
    delete op;
}

// ------------------------------------------------------------------------ factor

// Factor method of a mixed factor: the options, else HELM_FACTOR=line|bcr, else BCR on lines of
// at least kBcrMinNz nodes and the line recurrence below.  The line recurrence's dependent chain
// (n_x line inversions, n_x line steps per solve) is what BCR removes; on short lines its
// per-step cost is small and BCR's extra arithmetic and launches do not pay (measured: 128 x 128
// with 16 right-hand sides per frequency favours the line factor, 256 x 256 with 64 favours BCR
// by 2.5x).  FP64 factors are line factors (the tensor cores have no FP64 path).
static constexpr int kBcrMinNz = 192;
bool helm::factor_picks_bcr(const GridGeom &g, helm_prec prec, int method) {
    if (prec != HELM_MIXED || !bcr_supported(g)) return false;
    int m = method;
    if (m == HELM_FACTOR_AUTO) {
        const char *env = getenv("HELM_FACTOR");
        if (env && !strcmp(env, "line")) m = HELM_FACTOR_LINE;
        else if (env && !strcmp(env, "bcr")) m = HELM_FACTOR_BCR;
        else m = g.nz >= kBcrMinNz ? HELM_FACTOR_BCR : HELM_FACTOR_LINE;
    }
    return m == HELM_FACTOR_BCR;
}
static bool pick_bcr(const helm_op *op, helm_prec prec, const helm_factor_opts *opts) {
    return factor_picks_bcr(op->g, prec, opts ? opts->method : HELM_FACTOR_AUTO);
}

extern "C" helm_status helm_factor(helm_op_t *op, helm_prec prec, const helm_factor_opts *opts, helm_factor_t **out) {
    if (!out) { helm_set_msg("helm_factor: NULL out"); return HELM_EINVAL; }
    *out = nullptr;
    if (!op || (prec != HELM_FP64 && prec != HELM_MIXED) ||
        (opts && (opts->method < HELM_FACTOR_AUTO || opts->method > HELM_FACTOR_BCR))) {
        helm_set_msg("helm_factor: bad op, precision or method");
        return HELM_EINVAL;
    }
    if (opts && opts->method == HELM_FACTOR_BCR && (prec != HELM_MIXED || !bcr_supported(op->g))) {
        helm_set_msg("helm_factor: block cyclic reduction needs HELM_MIXED and an even nz >= 16");
        return HELM_EINVAL;
    }
    helm_factor_t *f = new (std::nothrow) struct helm_factor();
    if (!f) return HELM_ENOMEM;
    f->op = op;
    f->prec = prec;
    f->use_bcr = pick_bcr(op, prec, opts);
    const GridGeom &g = op->g;
    f->cs = pick_cluster_size(g.nz);
    const size_t esz = prec == HELM_FP64 ? sizeof(double2) : sizeof(float2);
    const size_t gelems = (size_t)op->n_omega * g.nx * g.nz * g.nz;
    helm_status s;
    cudaError_t e;
    if ((e = cudaMemsetAsync(op->status, 0, 2 * sizeof(int), op->st)) != cudaSuccess) {
        helm_set_error("helm_factor", e);
        helm_factor_destroy(f);
        return HELM_ECUDA;
    }
    // HELM_FAULT=pivot: the factor kernels read a copy of the diagonal whose first entry the host
    // set to NaN; op keeps its own diagonal (restored below, before anything else reads it)
    double2 *diag_saved = nullptr, *diag_bad = nullptr;
    if (fault_flags() & HELM_FAULT_PIVOT) {
        const size_t nd = (size_t)op->n_omega * g.nx * g.nz;
        const double2 bad = make_double2(NAN, 0.0);
        if ((s = dev_alloc((void **)&diag_bad, nd * sizeof(double2), "allocate(diag copy)", op->st)) != HELM_OK) {
            helm_factor_destroy(f);
            return s;
        }
        e = cudaMemcpyAsync(diag_bad, op->diag, nd * sizeof(double2), cudaMemcpyDeviceToDevice, op->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(diag_bad, &bad, sizeof(bad), cudaMemcpyHostToDevice, op->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(op->st);   // the host value is on the stack
        if (e != cudaSuccess) {
            helm_set_error("helm_factor: inject a NaN pivot", e);
            dev_free(diag_bad, op->st);
            helm_factor_destroy(f);
            return HELM_ECUDA;
        }
        diag_saved = op->diag;
        op->diag = diag_bad;
    }
    auto restore_diag = [&]() {
        if (diag_bad) {
            op->diag = diag_saved;
            dev_free(diag_bad, op->st);
            diag_bad = nullptr;
        }
    };
    if (f->use_bcr) {
        if ((s = bcr_factor(f)) != HELM_OK) {
            cudaStreamSynchronize(op->st);
            restore_diag();
            helm_factor_destroy(f);
            return s;
        }
        e = cudaSuccess;
    } else {
        if ((s = dev_alloc(&f->G, gelems * esz, "allocate(factor)", op->st)) != HELM_OK ||
            (s = dev_alloc(&f->xch, (size_t)op->n_omega * factor_xch_elems(g.nz) * esz, "allocate(exchange)",
                           op->st)) != HELM_OK) {
            restore_diag();
            helm_factor_destroy(f);
            return s;
        }
        if (prec == HELM_FP64)
            e = launch_line_factor<double>(g, op->n_omega, op->diag, (double2 *)f->G, (double2 *)f->xch, op->status,
                                           f->cs, op->st, &f->mid);
        else
            e = launch_line_factor<float>(g, op->n_omega, op->diag, (float2 *)f->G, (float2 *)f->xch, op->status,
                                          f->cs, op->st, &f->mid);
    }
    int st_host[2] = {0, 0};   // status bits, pivot blocks inverted in FP64
    if (e == cudaSuccess) e = cudaMemcpyAsync(st_host, op->status, 2 * sizeof(int), cudaMemcpyDeviceToHost, op->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(op->st);
    restore_diag();
    f->fp64_blocks = st_host[1];
    if (e != cudaSuccess) {
        helm_set_error("helm_factor: launch", e);
        helm_factor_destroy(f);
        return HELM_ECUDA;
    }
    if (st_host[0] & ST_TIMEOUT) {
        helm_set_msg("helm_factor: a factor kernel gave up waiting for its cluster");
        helm_factor_destroy(f);
        return HELM_ETIMEOUT;
    }
    if (st_host[0] & ST_SINGULAR) {
        helm_set_msg("helm_factor: zero or non-finite pivot");
        helm_factor_destroy(f);
        return HELM_ESINGULAR;
    }
    if (prec == HELM_MIXED) {   // diagonal of A as FP32 pairs for the refinement residual
        const size_t n = (size_t)op->n_omega * g.nx * g.nz;
        if ((s = dev_alloc((void **)&f->diag2, n * sizeof(float4), "allocate(diag pairs)", op->st)) != HELM_OK) {
            helm_factor_destroy(f);
            return s;
        }
        if ((e = launch_split_diag(n, op->diag, f->diag2, op->st)) != cudaSuccess) {
            helm_set_error("helm_factor: split diagonal", e);
            helm_factor_destroy(f);
            return HELM_ECUDA;
        }
    }
    *out = f;
    return HELM_OK;
}

extern "C" int32_t helm_factor_fp64_blocks(const helm_factor_t *f) { return f ? f->fp64_blocks : -1; }

extern "C" int32_t helm_factor_get_method(const helm_factor_t *f) {
    return f ? (f->use_bcr ? HELM_FACTOR_BCR : HELM_FACTOR_LINE) : -1;
}

extern "C" void helm_factor_destroy(helm_factor_t *f) {
    if (!f) return;
    cudaStream_t st = f->op ? f->op->st : nullptr;
    dev_free(f->G, st);
    dev_free(f->xch, st);
    dev_free(f->diag2, st);
    dev_free(f->bd, st);
    dev_free(f->xa, st);
    dev_free(f->xb, st);
    dev_free(f->r32, st);
    dev_free(f->y, st);
    dev_free(f->norms, st);
    dev_free(f->state, st);
    bcr_free(f);
    delete f;
}

helm_status factor_reserve(helm_factor_t *f, int nrhs) {
    if (nrhs <= f->cap) return HELM_OK;
    const helm_op *op = f->op;
    const size_t cols = (size_t)op->n_omega * nrhs;
    const size_t N = (size_t)op->g.nx * op->g.nz;
    const cudaStream_t st = op->st;
    dev_free(f->bd, st);
    dev_free(f->xa, st);
    dev_free(f->xb, st);
    dev_free(f->r32, st);
    dev_free(f->y, st);
    dev_free(f->norms, st);
    dev_free(f->state, st);
    f->bd = f->xa = f->xb = nullptr;
    f->r32 = f->y = nullptr;
    f->norms = nullptr;
    f->state = nullptr;
    f->cap = 0;
    helm_status s;
    if (f->prec == HELM_MIXED &&
        ((s = dev_alloc((void **)&f->bd, cols * N * sizeof(float4), "allocate(rhs pairs)", st)) != HELM_OK ||
         (s = dev_alloc((void **)&f->xa, cols * N * sizeof(float4), "allocate(iterate)", st)) != HELM_OK ||
         (s = dev_alloc((void **)&f->xb, cols * N * sizeof(float4), "allocate(iterate)", st)) != HELM_OK ||
         (s = dev_alloc((void **)&f->r32, cols * N * sizeof(float2), "allocate(residual)", st)) != HELM_OK ||
         (s = dev_alloc((void **)&f->y, cols * N * sizeof(float2), "allocate(work)", st)) != HELM_OK ||
         (s = dev_alloc((void **)&f->state, refine_state_bytes(op->n_omega), "allocate(refinement state)", st)) !=
             HELM_OK))
        return s;
    if ((s = dev_alloc((void **)&f->norms, cols * 2 * sizeof(double), "allocate(norms)", st)) != HELM_OK) return s;
    f->norms_host.assign(cols * 2, 0.0);
    f->cap = nrhs;
    return HELM_OK;
}

helm_status max_relres(const helm_op *op, size_t cols, const double *norms_dev, double *norms_host, double *out) {
    cudaError_t e = cudaMemcpyAsync(norms_host, norms_dev, cols * 2 * sizeof(double), cudaMemcpyDeviceToHost, op->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(op->st);
    if (e != cudaSuccess) { helm_set_error("read residual norms", e); return HELM_ECUDA; }
    double mx = 0.0;
    for (size_t c = 0; c < cols; ++c) {
        const double rr = norms_host[2 * c], bb = norms_host[2 * c + 1];
        // a non-finite right-hand side (bb NaN or inf) or residual gives NaN: not converged
        const double rel = (isnan(rr) || !isfinite(bb)) ? NAN : (bb > 0 ? sqrt(rr / bb) : (rr > 0 ? INFINITY : 0.0));
        if (isnan(mx) || isnan(rel)) mx = NAN;   // a NaN column stays visible in the maximum
        else if (rel > mx) mx = rel;
    }
    *out = mx;
    return HELM_OK;
}

// Iterative refinement with the complex-FP32 factor: x_1 = A~^{-1} b, then
// x_{k+1} = x_k + A~^{-1}(b - A x_k) until ||b - A x|| / ||b|| <= rtol (every column) or max_iter
// correction solves.  The iterate and the residual are FP32 pairs (refine.cu) down to
// kPairFloor or until the pair residual stops falling; a tighter rtol continues with FP64
// residuals on the FP64 iterate.
// The stopping test of the pair phase runs on the device (the last block of every update), so
// the host enqueues several sweeps at a time and reads the state once per batch; sweeps and
// updates enqueued after the test has stopped the loop return at once.  The first batch is as
// long as the previous solve with this factor took.
helm_status mixed_refine(const helm_factor_t *f, int nrhs, const double2 *B, double2 *X, int conj, double rtol,
                         int max_iter, const MixedWork &w, int *iters, double *relres) {
    constexpr double kPairFloor = 1e-12;   // well above the pair residual's floor (about 1e-13)
    constexpr int kLaterBatch = 2;
    const helm_op *op = f->op;
    const GridGeom &g = op->g;
    const int n_sys = op->n_omega;
    const int cols = n_sys * nrhs;
    const size_t n = (size_t)cols * g.nx * g.nz;
    const int rchunk = 16;
    if (max_iter < 1) max_iter = 1;
    cudaError_t e = cudaMemsetAsync(w.state, 0, refine_state_bytes(n_sys), op->st);
    if (e == cudaSuccess) e = launch_refine_start(g, cols, B, conj, w.bd, w.r32, w.norms, op->st);
    if (e != cudaSuccess) { helm_set_error("refinement start", e); return HELM_ECUDA; }
    const int *skip = &w.state->done;
    // the correction A~^{-1} r: line sweep, or the block-cyclic-reduction solve (which works in
    // place on r, recomputed before every correction)
    // (in the pair phase a system whose columns are all at rtol is frozen: its solve products and
    // updates are skipped; the FP64 phase corrects every column)
    auto sweep = [&](const int *skip_flag) -> cudaError_t {
        const int *frozen = skip_flag ? refine_sys(w.state) + 1 : nullptr;
        if (f->use_bcr) {
            const helm_status bs = bcr_solve(f, nrhs, w.r32, w.y, skip_flag, frozen);
            return bs == HELM_OK ? cudaSuccess : cudaErrorLaunchFailure;
        }
        return launch_line_sweep<float>(g, n_sys, nrhs, (const float2 *)f->G, w.r32, nullptr, w.y, 0, rchunk,
                                        op->status, op->st, f->mid, skip_flag, frozen);
    };
    RefineState hs{};
    int enq = 0, batch = std::max(1, std::min(f->last_iters.load(std::memory_order_relaxed), max_iter));
    helm_status s;
    while (enq < max_iter) {   // FP32-pair phase
        for (const int end = std::min(enq + batch, max_iter); enq < end; ++enq) {
            // sweep k (from 0) writes xa for even k, xb for odd k and reads the other
            const float4 *x_in = enq == 0 ? nullptr : ((enq & 1) ? w.xa : w.xb);
            float4 *x_out = (enq & 1) ? w.xb : w.xa;
            if ((e = sweep(skip)) != cudaSuccess) { helm_set_error("sweep mixed", e); return HELM_ECUDA; }
            e = launch_refine_update(g, n_sys, nrhs, f->diag2, w.bd, x_in, w.y, x_out, w.r32, w.norms, op->st, w.state,
                                     RefineStop{rtol, kPairFloor, max_iter});
            if (e != cudaSuccess) { helm_set_error("refinement update", e); return HELM_ECUDA; }
        }
        e = cudaMemcpyAsync(&hs, w.state, sizeof(RefineState), cudaMemcpyDeviceToHost, op->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(op->st);
        if (e != cudaSuccess) { helm_set_error("read refinement state", e); return HELM_ECUDA; }
        if (hs.done) break;
        batch = kLaterBatch;
    }
    int it = hs.iters;
    double rel = hs.rel;
    f->last_iters.store(std::max(1, it), std::memory_order_relaxed);
    e = launch_refine_finish(n, g.nx * g.nz, nrhs, w.xa, w.xb, w.state, conj, X, op->st);
    if (e != cudaSuccess) { helm_set_error("refinement finish", e); return HELM_ECUDA; }
    if (!(rel <= rtol) && it < max_iter && isfinite(rel)) {
        // FP64 phase: r = b - A x in FP64 on the FP64 iterate, correction conj?(A~^{-1} conj?(r))
        for (;;) {
            e = cudaMemsetAsync(w.norms, 0, (size_t)cols * 2 * sizeof(double), op->st);
            if (e == cudaSuccess) e = launch_residual(g, n_sys, nrhs, op->diag, B, X, w.r32, w.norms, conj, op->st);
            if (e != cudaSuccess) { helm_set_error("residual", e); return HELM_ECUDA; }
            if ((s = max_relres(op, (size_t)cols, w.norms, w.norms_host, &rel)) != HELM_OK) return s;
            if (rel <= rtol || it >= max_iter || !isfinite(rel)) break;
            if ((e = sweep(nullptr)) != cudaSuccess) { helm_set_error("sweep mixed", e); return HELM_ECUDA; }
            e = launch_refine_accumulate(n, w.y, conj, X, op->st);
            if (e != cudaSuccess) { helm_set_error("refinement accumulate", e); return HELM_ECUDA; }
            ++it;
        }
    }
    *iters = it;
    *relres = rel;
    return HELM_OK;
}

helm_status read_sweep_status(const helm_op *op) {
    int st_host = 0;
    cudaError_t e = cudaMemcpyAsync(&st_host, op->status, sizeof(int), cudaMemcpyDeviceToHost, op->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(op->st);
    if (e != cudaSuccess) { helm_set_error("solve status", e); return HELM_ECUDA; }
    if (st_host & ST_TIMEOUT) { helm_set_msg("a sweep kernel gave up waiting for its cluster"); return HELM_ETIMEOUT; }
    return HELM_OK;
}

helm_status solve_impl(helm_factor_t *f, int nrhs, const double2 *B, double2 *X, double rtol, int max_iter,
                       helm_solve_info *info, int conj) {
    const helm_op *op = f->op;
    const GridGeom &g = op->g;
    const int n_sys = op->n_omega;
    const size_t cols = (size_t)n_sys * nrhs;
    const int rchunk = 16;
    cudaError_t e;
    helm_status s;
    if (info) { info->iters = 0; info->max_relres = -1.0; }
    // the status bits report this solve only (a give-up of an earlier call does not stick)
    if ((e = cudaMemsetAsync(op->status, 0, sizeof(int), op->st)) != cudaSuccess) {
        helm_set_error("solve: clear status", e);
        return HELM_ECUDA;
    }
    if (f->prec == HELM_FP64) {
        e = launch_line_sweep<double>(g, n_sys, nrhs, (const double2 *)f->G, B, X, X, conj, rchunk, op->status, op->st,
                                      f->mid);
        if (e != cudaSuccess) { helm_set_error("sweep fp64", e); return HELM_ECUDA; }
        if ((s = read_sweep_status(op)) != HELM_OK) return s;
        if (info) {
            info->iters = 1;
            if ((s = factor_reserve(f, nrhs)) != HELM_OK) return s;
            e = cudaMemsetAsync(f->norms, 0, cols * 2 * sizeof(double), op->st);
            if (e == cudaSuccess) e = launch_residual(g, n_sys, nrhs, op->diag, B, X, nullptr, f->norms, conj, op->st);
            if (e != cudaSuccess) { helm_set_error("residual", e); return HELM_ECUDA; }
            if ((s = max_relres(op, cols, f->norms, f->norms_host.data(), &info->max_relres)) != HELM_OK) return s;
            if (!isfinite(info->max_relres)) { helm_set_msg("non-finite residual"); return HELM_ENOCONV; }
        }
        return HELM_OK;
    }
    if ((s = factor_reserve(f, nrhs)) != HELM_OK) return s;
    const MixedWork w{f->bd, f->xa, f->xb, f->r32, f->y, f->norms, f->norms_host.data(), f->state};
    int it = 0;
    double rel = INFINITY;
    if ((s = mixed_refine(f, nrhs, B, X, conj, rtol, max_iter, w, &it, &rel)) != HELM_OK) return s;
    if (info) { info->iters = it; info->max_relres = rel; }
    if ((s = read_sweep_status(op)) != HELM_OK) return s;
    if (!(rel <= rtol)) { helm_set_msg("refinement did not reach rtol"); return HELM_ENOCONV; }
    return HELM_OK;
}

static helm_status check_solve_args(const char *who, helm_factor_t *f, int32_t nrhs, const helm_c128 *B,
                                    helm_c128 *X) {
    if (!f || nrhs < 0 || (nrhs > 0 && (!B || !X)) || (const void *)B == (const void *)X) {
        helm_set_msg((std::string(who) + ": bad arguments (NULL, nrhs < 0 or B aliases X)").c_str());
        return HELM_EINVAL;
    }
    return HELM_OK;
}

// solve_impl, or (HELM_FAULT=nan_rhs) solve_impl on a copy of B whose first entry is NaN
static helm_status solve_entry(helm_factor_t *f, int nrhs, const double2 *B, double2 *X, double rtol, int max_iter,
                               helm_solve_info *info, int conj) {
    if (!(fault_flags() & HELM_FAULT_NAN_RHS)) return solve_impl(f, nrhs, B, X, rtol, max_iter, info, conj);
    const helm_op *op = f->op;
    const size_t n = (size_t)op->n_omega * nrhs * op->g.nx * op->g.nz;
    const double2 bad = make_double2(NAN, 0.0);
    double2 *Bc = nullptr;
    helm_status s = dev_alloc((void **)&Bc, n * sizeof(double2), "allocate(rhs copy)", op->st);
    if (s != HELM_OK) return s;
    cudaError_t e = cudaMemcpyAsync(Bc, B, n * sizeof(double2), cudaMemcpyDeviceToDevice, op->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Bc, &bad, sizeof(bad), cudaMemcpyHostToDevice, op->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(op->st);   // the host value is on the stack
    if (e != cudaSuccess) {
        helm_set_error("solve: inject a NaN right-hand side", e);
        dev_free(Bc, op->st);
        return HELM_ECUDA;
    }
    s = solve_impl(f, nrhs, Bc, X, rtol, max_iter, info, conj);
    dev_free(Bc, op->st);
    return s;
}

extern "C" helm_status helm_solve(helm_factor_t *f, int32_t nrhs, const helm_c128 *B_dev, helm_c128 *X_dev,
                                  double rtol, int32_t max_iter, helm_solve_info *info) {
    helm_status s = check_solve_args("helm_solve", f, nrhs, B_dev, X_dev);
    if (s != HELM_OK || nrhs == 0) return s;
    return solve_entry(f, nrhs, (const double2 *)B_dev, (double2 *)X_dev, rtol, max_iter, info, 0);
}

extern "C" helm_status helm_adjoint_solve(helm_factor_t *f, int32_t nrhs, const helm_c128 *B_dev,
                                          helm_c128 *X_dev, double rtol, int32_t max_iter,
                                          helm_solve_info *info) {
    helm_status s = check_solve_args("helm_adjoint_solve", f, nrhs, B_dev, X_dev);
    if (s != HELM_OK || nrhs == 0) return s;
    return solve_entry(f, nrhs, (const double2 *)B_dev, (double2 *)X_dev, rtol, max_iter, info, 1);
}

// ------------------------------------------------------------ acquisition helpers

helm_status acq_upload(const helm_op *op, const helm_acq *acq, DevAcq *d) {
    *d = DevAcq();
    if (!acq || acq->n_src < 0 || acq->n_rec < 0 || (acq->n_src > 0 && !acq->src_xz) ||
        (acq->n_rec > 0 && !acq->rec_xz)) {
        helm_set_msg("acquisition: bad arguments");
        return HELM_EINVAL;
    }
    for (int s = 0; s < acq->n_src; ++s) {
        const double x = acq->src_xz[2 * s], z = acq->src_xz[2 * s + 1];
        if (!(x >= 0 && x <= op->lx && z >= 0 && z <= op->lz)) { helm_set_msg("source outside the grid"); return HELM_EINVAL; }
    }
    for (int r = 0; r < acq->n_rec; ++r) {
        const double x = acq->rec_xz[2 * r], z = acq->rec_xz[2 * r + 1];
        if (!(x >= 0 && x <= op->lx && z >= 0 && z <= op->lz)) { helm_set_msg("receiver outside the grid"); return HELM_EINVAL; }
    }
    d->st = op->st;
    d->n_src = acq->n_src;
    d->n_rec = acq->n_rec;
    const int ns = std::max(1, acq->n_src), nr = std::max(1, acq->n_rec);
    helm_status s;
    if ((s = dev_alloc((void **)&d->src_xz, ns * 2 * sizeof(double), "acq", op->st)) != HELM_OK ||
        (s = dev_alloc((void **)&d->src_amp, ns * sizeof(double), "acq", op->st)) != HELM_OK ||
        (s = dev_alloc((void **)&d->rec_xz, nr * 2 * sizeof(double), "acq", op->st)) != HELM_OK ||
        (s = dev_alloc((void **)&d->rec_w, nr * sizeof(double), "acq", op->st)) != HELM_OK ||
        (s = dev_alloc((void **)&d->tap_idx, nr * 16 * sizeof(int), "acq", op->st)) != HELM_OK ||
        (s = dev_alloc((void **)&d->tap_w, nr * 16 * sizeof(double), "acq", op->st)) != HELM_OK ||
        (s = dev_alloc((void **)&d->tap_wx, nr * 16 * sizeof(double), "acq", op->st)) != HELM_OK ||
        (s = dev_alloc((void **)&d->tap_wz, nr * 16 * sizeof(double), "acq", op->st)) != HELM_OK) {
        acq_free(d);
        return s;
    }
    std::vector<double> amp(ns, 1.0), w(nr, 1.0);
    if (acq->src_amp) std::copy(acq->src_amp, acq->src_amp + acq->n_src, amp.begin());
    if (acq->rec_w) std::copy(acq->rec_w, acq->rec_w + acq->n_rec, w.begin());
    cudaError_t e = cudaSuccess;
    if (acq->n_src > 0) e = cudaMemcpyAsync(d->src_xz, acq->src_xz, acq->n_src * 2 * sizeof(double), cudaMemcpyHostToDevice, op->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d->src_amp, amp.data(), ns * sizeof(double), cudaMemcpyHostToDevice, op->st);
    if (e == cudaSuccess && acq->n_rec > 0) e = cudaMemcpyAsync(d->rec_xz, acq->rec_xz, acq->n_rec * 2 * sizeof(double), cudaMemcpyHostToDevice, op->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d->rec_w, w.data(), nr * sizeof(double), cudaMemcpyHostToDevice, op->st);
    if (e == cudaSuccess && acq->n_rec > 0)
        e = launch_restriction_taps(op->g, acq->n_rec, d->rec_xz, d->tap_idx, d->tap_w, d->tap_wx, d->tap_wz, op->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(op->st);   // host vectors above go out of scope
    if (e != cudaSuccess) {
        helm_set_error("acquisition upload", e);
        acq_free(d);
        return HELM_ECUDA;
    }
    return HELM_OK;
}

void acq_free(DevAcq *d) {
    dev_free(d->src_xz, d->st);
    dev_free(d->src_amp, d->st);
    dev_free(d->rec_xz, d->st);
    dev_free(d->rec_w, d->st);
    dev_free(d->tap_idx, d->st);
    dev_free(d->tap_w, d->st);
    dev_free(d->tap_wx, d->st);
    dev_free(d->tap_wz, d->st);
    *d = DevAcq();
}

extern "C" helm_status helm_sources(const helm_op_t *op, const helm_acq *acq, helm_c128 *B_dev) {
    if (!op || !acq || !B_dev) { helm_set_msg("helm_sources: bad arguments"); return HELM_EINVAL; }
    DevAcq d;
    helm_status s = acq_upload(op, acq, &d);
    if (s != HELM_OK) return s;
    cudaError_t e = launch_sources(op->g, op->n_omega, d.n_src, d.src_xz, d.src_amp, (double2 *)B_dev, op->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(op->st);
    acq_free(&d);
    if (e != cudaSuccess) { helm_set_error("helm_sources", e); return HELM_ECUDA; }
    return HELM_OK;
}

extern "C" helm_status helm_restrict(const helm_op_t *op, const helm_acq *acq, int32_t ncol,
                                     const helm_c128 *X_dev, helm_c128 *Y_dev) {
    if (!op || !acq || ncol < 0 || (ncol > 0 && (!X_dev || !Y_dev))) {
        helm_set_msg("helm_restrict: bad arguments");
        return HELM_EINVAL;
    }
    DevAcq d;
    helm_status s = acq_upload(op, acq, &d);
    if (s != HELM_OK) return s;
    cudaError_t e = launch_restrict(op->g, op->n_omega * ncol, d.n_rec, d.tap_idx, d.tap_w, (const double2 *)X_dev,
                                    (double2 *)Y_dev, op->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(op->st);
    acq_free(&d);
    if (e != cudaSuccess) { helm_set_error("helm_restrict", e); return HELM_ECUDA; }
    return HELM_OK;
}
