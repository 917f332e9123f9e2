// Internal tracing hooks: construct a TraceScope around every kernel launch.
#pragma once
#include <cuda_runtime.h>

namespace helm {

enum KernelId {
    K_ASSEMBLE, K_SOURCES, K_TAPS, K_RESTRICT, K_FACTOR64, K_FACTOR32, K_SWEEP64, K_SWEEP32, K_RESIDUAL,
    K_MISFIT, K_SCATTER, K_GRAD, K_GUP, K_ZBASE, K_HESS, K_HYPER, K_DOT, K_SUM, K_AXPBY, K_FILL, K_SUB,
    K_REGR, K_DCTMAT, K_P2SCALE, K_DGEMM, K_GBPRE, K_SPLITDIAG, K_REFSTART, K_REFUPDATE, K_REFFINISH, K_REFACCUM, K_FIELDGRAD, K_GCOEF, K_HESSFIN,
    K_ZGEMM, K_ZINV, K_ZTRANS, K_BCR_FORM, K_BCR_L0, K_BCR_SOLVE_L0, K_ZSPLIT,
    K_COUNT
};

// Counts the launch and, when tracing is on, records CUDA events on `st` at
// construction and destruction (bracketing the launch made inside the scope).
class TraceScope {
  public:
    TraceScope(int id, cudaStream_t st, double flops = 0.0);
    ~TraceScope();
    TraceScope(const TraceScope &) = delete;
    TraceScope &operator=(const TraceScope &) = delete;

  private:
    int id_;
    cudaStream_t st_;
    cudaEvent_t a_;
    double flops_;
};

}  // namespace helm

#define HELM_TRACED(id, st, launch)            \
    do {                                       \
        ::helm::TraceScope ts_((id), (st));    \
        launch;                                \
    } while (0)
// the same, for a launch doing `flops` useful floating-point operations
#define HELM_TRACED_W(id, st, flops, launch)           \
    do {                                               \
        ::helm::TraceScope ts_((id), (st), (flops));   \
        launch;                                        \
    } while (0)
