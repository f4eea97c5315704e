// Block-coordinate trust-region Newton fit driver (Section IV-D).
#include "internal.cuh"

extern "C" {

void celeste_fit_options_default(celeste_fit_options* o) {
    o->max_iter = 50;
    o->grad_tol = 1e-8;
    o->pred_tol_rel = 1e-12;
    o->delta0 = 1.0;
    o->delta_max = 1e3;
    o->eta = 1e-4;
    o->f_noise_rel = 1e-13;
    o->precision = CELESTE_FP64;
    o->max_sweeps = 20;
    o->sweep_tol = 1e-8;
}

celeste_status celeste_fit_sources(celeste_problem*, double*, const int32_t*, int32_t,
                                   const celeste_fit_options*, int32_t*, int32_t*, double*) {
    return CELESTE_ERR_ARG;
}

}  // extern "C"
