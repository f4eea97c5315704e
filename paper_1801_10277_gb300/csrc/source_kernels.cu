// Per-source epilogue of the ELBO and gradient (Section IV: 44 parameters per source;
// Section IV-D: the block of one source): item partials (already mapped to the 44
// constrained parameters by k_adjoint) summed per source, the KL terms from k_prep
// subtracted, and the total folded in by the last CTA.  FP64 sums.
#include <math.h>

#include "internal.cuh"
#include "source_math.cuh"
#include "epilogue.cuh"

namespace cel {

__global__ void __launch_bounds__(FZ_THREADS)
k_finalize(int n_src, int mode, const PatchGeo* __restrict__ geo,
           const int32_t* __restrict__ patch_off, const int32_t* __restrict__ item_off,
           const double* __restrict__ part,
           const double* __restrict__ item_ll, const double* __restrict__ tile_ll, int n_tile,
           const double* __restrict__ kl, const double* __restrict__ kl_grad,
           double* __restrict__ local_out, double* __restrict__ grad_out,
           double* __restrict__ src_total, int32_t* __restrict__ done,
           double* __restrict__ total_out) {
    if ((int)blockIdx.x >= n_src) return;
    finalize_source(blockIdx.x, n_src, mode, geo, patch_off, item_off, part, item_ll, tile_ll, n_tile, kl,
                    kl_grad, local_out, grad_out, src_total, done, total_out);
}

__global__ void __launch_bounds__(TOTAL_THREADS)
k_total(const double* __restrict__ tile_ll, int n_tile, const double* __restrict__ item_ll, int n_item,
        const double* __restrict__ kl, int n_src, double* __restrict__ part, int32_t* __restrict__ done,
        double* __restrict__ out) {
    total_reduce(tile_ll, n_tile, item_ll, n_item, kl, n_src, part, done, out);
}

cudaError_t launch_finalize_hess(const DevProblem& P, const double* d_theta, double* d_local,
                                 double* d_grad, double* d_hess, cudaStream_t st);

// total = tile ll sums + item ll sums - KL (fixed order, TOTAL_CTAS slices)
cudaError_t launch_total(const DevProblem& P, double* d_total, cudaStream_t st) {
    k_total<<<TOTAL_CTAS, TOTAL_THREADS, 0, st>>>(P.tile_ll, P.n_tile, P.item_ll,
                                                  P.single ? P.n_item : 0, P.kl, P.n_src, P.tot_part,
                                                  P.tot_done, d_total);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const DevProblem& P, const double* d_theta, int precision, int mode,
                            double* d_total, double* d_local, double* d_grad, double* d_hess,
                            cudaStream_t st) {
    if (mode == MODE_HESS) {
        cudaError_t e = launch_finalize_hess(P, d_theta, d_local, d_grad, d_hess, st);
        if (e != cudaSuccess) return e;
    } else if (P.n_src > 0) {
        // the KL value and gradient come from k_prep of the same theta
        (void)precision;
        (void)d_theta;
        k_finalize<<<P.n_src, FZ_THREADS, 0, st>>>(P.n_src, mode, P.geo, P.patch_off, nullptr, P.item_part,
                                                   P.single ? P.item_ll : nullptr, P.tile_ll,
                                                   P.n_tile, P.kl, P.kl_grad, d_local, d_grad,
                                                   P.src_total, P.done, d_total);
        return cudaGetLastError();
    }
    if (d_total)
        k_total<<<TOTAL_CTAS, TOTAL_THREADS, 0, st>>>(P.tile_ll, P.n_tile, P.item_ll,
                                                      P.single ? P.n_item : 0, P.kl, P.n_src,
                                                      P.tot_part, P.tot_done, d_total);
    return cudaGetLastError();
}

}  // namespace cel
