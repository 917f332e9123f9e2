// placeholder, replaced below
#include "helm.h"
extern "C" helm_status fwi_misfit_grad(helm_factor_t *, const helm_acq *, const helm_c128 *, double, double,
                                       double, double *, double *, helm_c128 *, helm_c128 *) {
    return HELM_EINVAL;
}
extern "C" helm_status bilevel_hypergrad(int32_t, const helm_grid *, const double *const *, const double *const *,
                                         const helm_acq *, const double *, int32_t, double, double, double,
                                         helm_prec, const helm_pcg_opts *, void *, double *, double *, double *,
                                         double *, helm_hyper_info *) {
    return HELM_EINVAL;
}
