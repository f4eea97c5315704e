// Per-source kernels: KL terms (value, gradient) and the chain rule from the twelve
// intermediate pixel variables y of each (source, patch) to the source's 44
// constrained parameters (Section IV: 44 parameters per source; Section IV-D: the
// block of one source).  FP64 throughout.
#include <math.h>

#include "internal.cuh"

namespace cel {

// KL(q_s || prior) and its gradient (Section III priors Phi, Upsilon, Xi; Eq. 1):
//   KL = sum_i a_i [ log(a_i / Phi_i) + KL_r,i + sum_d k_id ( log(k_id / w_id) + KL_c,id ) ]
//   KL_r,i  = (log(pv/r2) + (r2 + (r1 - pm)^2)/pv - 1) / 2
//   KL_c,id = (tr(P_d diag c2) + (c1 - mu_d)' P_d (c1 - mu_d) - 4 + log det Sigma_d
//              - sum_j log c2_j) / 2
__device__ double kl_value_grad(const ModelDev& md, const double* th, double* g) {
    double kl = 0.0;
    for (int i = 0; i < 2; ++i) {
        const double a = th[P_A + i];
        const double phi = (i == 0) ? md.prior_star : 1.0 - md.prior_star;
        const double r1 = th[P_R1 + i], r2 = th[P_R2 + i];
        const double pm = md.prior_r[i][0], pv = md.prior_r[i][1];
        double K = 0.5 * (log(pv / r2) + (r2 + (r1 - pm) * (r1 - pm)) / pv - 1.0);
        const double dr1 = (r1 - pm) / pv, dr2 = 0.5 * (1.0 / pv - 1.0 / r2);
        double dc1[4] = {0, 0, 0, 0}, dc2[4] = {0, 0, 0, 0};
        double c1[4], c2[4], slog = 0.0;
        for (int j = 0; j < 4; ++j) {
            c1[j] = th[P_C1 + 4 * i + j];
            c2[j] = th[P_C2 + 4 * i + j];
            slog += log(c2[j]);
        }
        for (int d = 0; d < NCOMP; ++d) {
            const double k = th[P_K + NCOMP * i + d];
            const double* Pm = md.prior_P[i][d];
            const double* mu = md.prior_mu[i][d];
            double diff[4], Pd[4];
            for (int j = 0; j < 4; ++j) diff[j] = c1[j] - mu[j];
            double quad = 0.0, tr = 0.0;
            for (int j = 0; j < 4; ++j) {
                double s = 0.0;
                for (int l = 0; l < 4; ++l) s += Pm[4 * j + l] * diff[l];
                Pd[j] = s;
                quad += diff[j] * s;
                tr += Pm[5 * j] * c2[j];
            }
            const double klc = 0.5 * (tr + quad - 4.0 + md.prior_logdet[i][d] - slog);
            const double lk = log(k / md.prior_w[i][d]);
            K += k * (lk + klc);
            if (g) g[P_K + NCOMP * i + d] = a * (lk + 1.0 + klc);
            for (int j = 0; j < 4; ++j) {
                dc1[j] += k * Pd[j];
                dc2[j] += 0.5 * k * (Pm[5 * j] - 1.0 / c2[j]);
            }
        }
        const double la = log(a / phi);
        kl += a * (la + K);
        if (g) {
            g[P_A + i] = la + 1.0 + K;
            g[P_R1 + i] = a * dr1;
            g[P_R2 + i] = a * dr2;
            for (int j = 0; j < 4; ++j) {
                g[P_C1 + 4 * i + j] = a * dc1[j];
                g[P_C2 + 4 * i + j] = a * dc2[j];
            }
        }
    }
    return kl;
}

// d(Gxx, Gxy, Gyy)/d(e_axis, e_angle, e_scale), G = A W A^T in the image's pixel frame.
__device__ void shape_jacobian(const double* A, const double* th, double dG[3][3]) {
    const double rho = th[P_AXIS], phi = th[P_ANGLE], sg = th[P_SCALE];
    const double bh = 0.5 * sg * sg * (1.0 - rho * rho);
    double s2, c2;
    sincos(2.0 * phi, &s2, &c2);
    double dW[3][3];
    // d/d rho: d ah = sg^2 rho, d bh = -sg^2 rho
    {
        const double da = sg * sg * rho, db = -sg * sg * rho;
        dW[0][0] = da + db * c2; dW[0][1] = db * s2; dW[0][2] = da - db * c2;
    }
    // d/d phi
    dW[1][0] = -2.0 * bh * s2; dW[1][1] = 2.0 * bh * c2; dW[1][2] = 2.0 * bh * s2;
    // d/d sigma: d ah = sg (1 + rho^2), d bh = sg (1 - rho^2)
    {
        const double da = sg * (1.0 + rho * rho), db = sg * (1.0 - rho * rho);
        dW[2][0] = da + db * c2; dW[2][1] = db * s2; dW[2][2] = da - db * c2;
    }
    for (int q = 0; q < 3; ++q) {
        const double wxx = dW[q][0], wxy = dW[q][1], wyy = dW[q][2];
        dG[q][0] = A[0] * A[0] * wxx + 2.0 * A[0] * A[1] * wxy + A[1] * A[1] * wyy;
        dG[q][1] = A[0] * A[2] * wxx + (A[0] * A[3] + A[1] * A[2]) * wxy + A[1] * A[3] * wyy;
        dG[q][2] = A[2] * A[2] * wxx + 2.0 * A[2] * A[3] * wxy + A[3] * A[3] * wyy;
    }
}

__device__ void band_moments(const double* th, int band, int i, double& el, double& el2) {
    double m = th[P_R1 + i], v = th[P_R2 + i];
    for (int j = 0; j < 4; ++j) {
        const double b = color_beta(band, j);
        m += b * th[P_C1 + 4 * i + j];
        v += b * b * th[P_C2 + 4 * i + j];
    }
    el = exp(m + 0.5 * v);
    el2 = exp(2.0 * m + 2.0 * v);
}

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
