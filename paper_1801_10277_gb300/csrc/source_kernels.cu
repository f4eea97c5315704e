// Per-source kernels: KL terms (value, gradient) and the chain rule from the twelve
// intermediate pixel variables y of each (source, patch) to the source's 44
// constrained parameters (Section IV: 44 parameters per source; Section IV-D: the
// block of one source).  FP64 throughout.
#include <math.h>

#include "internal.cuh"
#include "source_math.cuh"

namespace cel {

// grad += J^T Gy for one patch
__device__ void chain_grad(const ImgMeta& im, const double* th, const double* Gy, double* grad) {
    grad[P_A] += Gy[Y_A0];
    grad[P_A + 1] += Gy[Y_A1];
    for (int i = 0; i < 2; ++i) {
        double el, el2;
        band_moments(th, im.band, i, el, el2);
        const double gl = Gy[i == 0 ? Y_EL0 : Y_EL1] * el;
        const double gl2 = Gy[i == 0 ? Y_EL20 : Y_EL21] * el2;
        // d El = El d(m + v/2),  d El2 = El2 d(2m + 2v)
        const double dm = gl + 2.0 * gl2, dv = 0.5 * gl + 2.0 * gl2;
        grad[P_R1 + i] += dm;
        grad[P_R2 + i] += dv;
        for (int j = 0; j < 4; ++j) {
            const double b = color_beta(im.band, j);
            grad[P_C1 + 4 * i + j] += b * dm;
            grad[P_C2 + 4 * i + j] += b * b * dv;
        }
    }
    const double* A = im.A;
    grad[0] += Gy[Y_MX] * A[0] + Gy[Y_MY] * A[2];
    grad[1] += Gy[Y_MX] * A[1] + Gy[Y_MY] * A[3];
    grad[P_EDEV] += Gy[Y_EDEV];
    double dG[3][3];
    shape_jacobian(A, th, dG);
    for (int q = 0; q < 3; ++q)
        grad[P_AXIS + q] += Gy[Y_GXX] * dG[q][0] + Gy[Y_GXY] * dG[q][1] + Gy[Y_GYY] * dG[q][2];
}

// one thread per source: local objective, KL, gradient
__global__ void k_finalize(int n_src, int mode, const double* __restrict__ theta,
                           const PatchGeo* __restrict__ geo, const int32_t* __restrict__ patch_off,
                           const ImgMeta* __restrict__ img, const ModelDev* __restrict__ md,
                           const double* __restrict__ part, double* __restrict__ kl_out,
                           double* __restrict__ local_out, double* __restrict__ grad_out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_src) return;
    const double* th = theta + (size_t)NP * s;
    double grad[NP];
    double kl;
    if (mode >= MODE_GRAD) {
        kl = kl_value_grad(*md, th, grad);
        for (int i = 0; i < NP; ++i) grad[i] = -grad[i];
    } else {
        kl = kl_value_grad(*md, th, nullptr);
    }
    double loc = -kl;
    for (int p = patch_off[s]; p < patch_off[s + 1]; ++p) {
        const PatchGeo g = geo[p];
        double Gy[NY];
        for (int y = 0; y < NY; ++y) Gy[y] = 0.0;
        for (int it = g.item0; it < g.item0 + g.nitem; ++it) {
            const double* pr = part + (size_t)it * NPART;
            loc += pr[PART_LL];
            if (mode >= MODE_GRAD)
                for (int y = 0; y < NY; ++y) Gy[y] += pr[PART_G + y];
        }
        if (mode >= MODE_GRAD) chain_grad(img[g.img], th, Gy, grad);
    }
    kl_out[s] = kl;
    if (local_out) local_out[s] = loc;
    if (grad_out && mode >= MODE_GRAD)
        for (int i = 0; i < NP; ++i) grad_out[(size_t)NP * s + i] = grad[i];
}

// total = sum of tile ll sums - sum of KL, one CTA, fixed order
__global__ void k_total(const double* __restrict__ tile_ll, int n_tile,
                        const double* __restrict__ kl, int n_src, double* __restrict__ out) {
    __shared__ double red[512];
    double s = 0.0;
    for (int i = threadIdx.x; i < n_tile; i += blockDim.x) s += tile_ll[i];
    for (int i = threadIdx.x; i < n_src; i += blockDim.x) s -= kl[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

cudaError_t launch_finalize_hess(const DevProblem& P, const double* d_theta, double* d_local,
                                 double* d_grad, double* d_hess, cudaStream_t st);

cudaError_t launch_finalize(const DevProblem& P, const double* d_theta, int mode,
                            double* d_total, double* d_local, double* d_grad, double* d_hess,
                            cudaStream_t st) {
    if (mode == MODE_HESS) {
        cudaError_t e = launch_finalize_hess(P, d_theta, d_local, d_grad, d_hess, st);
        if (e != cudaSuccess) return e;
    } else if (P.n_src > 0) {
        k_finalize<<<(P.n_src + 127) / 128, 128, 0, st>>>(P.n_src, mode, d_theta, P.geo,
                                                          P.patch_off, P.img, P.model,
                                                          P.item_part, P.kl, d_local, d_grad);
    }
    if (d_total) k_total<<<1, 512, 0, st>>>(P.tile_ll, P.n_tile, P.kl, P.n_src, d_total);
    return cudaGetLastError();
}

}  // namespace cel
