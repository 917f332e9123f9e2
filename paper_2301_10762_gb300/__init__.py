"""GB300-native batched Helmholtz solves and the FWI / bilevel-hypergradient hot path
(arXiv:2301.10762).  The compute runs in libhelm.so (CUDA, sm_103a) behind the C ABI
of include/helm.h; `helm` is its thin Python binding."""
from . import helm  # noqa: F401
from .helm import (HELM_FP64, HELM_MIXED, Acq, HelmError, bilevel_hypergrad, fwi_misfit_grad,  # noqa: F401
                   helm_adjoint_solve, helm_assemble, helm_factor, helm_restrict, helm_solve, helm_sources)
