// Per-source kernels: KL terms (value, gradient) and the chain rule from the twelve
// intermediate pixel variables y of each (source, patch) to the source's 44
// constrained parameters (Section IV: 44 parameters per source; Section IV-D: the
// block of one source).  FP64 throughout.
#include <math.h>

#include "internal.cuh"
#include "source_math.cuh"
#include "epilogue.cuh"

namespace cel {

template <class R>
__global__ void __launch_bounds__(FZ_THREADS)
k_finalize(int n_src, int mode, const double* __restrict__ theta,
           const PatchGeo* __restrict__ geo, const int32_t* __restrict__ patch_off,
           const ImgMeta* __restrict__ img, const ModelDev* __restrict__ md,
           const double* __restrict__ part, double* __restrict__ kl_out,
           double* __restrict__ local_out, double* __restrict__ grad_out,
           int32_t* __restrict__ status) {
    if ((int)blockIdx.x >= n_src) return;
    finalize_source<R>(blockIdx.x, mode, theta, geo, patch_off, img, md, part, kl_out, local_out,
                       grad_out, status);
}

__global__ void k_total(const double* __restrict__ tile_ll, int n_tile,
                        const double* __restrict__ item_ll, int n_item,
                        const double* __restrict__ kl, int n_src, double* __restrict__ out) {
    total_reduce(tile_ll, n_tile, item_ll, n_item, kl, n_src, out);
}

cudaError_t launch_finalize_hess(const DevProblem& P, const double* d_theta, double* d_local,
                                 double* d_grad, double* d_hess, cudaStream_t st);

cudaError_t launch_finalize(const DevProblem& P, const double* d_theta, int precision, int mode,
                            double* d_total, double* d_local, double* d_grad, double* d_hess,
                            cudaStream_t st) {
    if (mode == MODE_HESS) {
        cudaError_t e = launch_finalize_hess(P, d_theta, d_local, d_grad, d_hess, st);
        if (e != cudaSuccess) return e;
    } else if (P.n_src > 0) {
        if (precision == CELESTE_FP64)
            k_finalize<double><<<P.n_src, FZ_THREADS, 0, st>>>(P.n_src, mode, d_theta, P.geo,
                                                               P.patch_off, P.img, P.model,
                                                               P.item_part, P.kl, d_local, d_grad,
                                                               P.status);
        else
            k_finalize<float><<<P.n_src, FZ_THREADS, 0, st>>>(P.n_src, mode, d_theta, P.geo,
                                                              P.patch_off, P.img, P.model,
                                                              P.item_part, P.kl, d_local, d_grad,
                                                              P.status);
    }
    if (d_total)
        k_total<<<1, 512, 0, st>>>(P.tile_ll, P.n_tile, P.item_ll, P.single ? P.n_item : 0, P.kl,
                                   P.n_src, d_total);
    return cudaGetLastError();
}

}  // namespace cel
