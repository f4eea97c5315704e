// Per-source epilogue: item sums -> chain rule -> KL -> local objective and gradient;
// and the total.  FP64 sums; transcendentals of the FP32 path in FP32 where the range allows.
#pragma once

#include <math.h>

#include "internal.cuh"
#include "source_math.cuh"

namespace cel {

template <class R> __device__ __forceinline__ R band_beta(int band, int j) { return (R)color_beta(band, j); }
template <> __device__ __forceinline__ float band_beta<float>(int band, int j) {
    const int ref = 2;   // the same rule as color_beta, in FP32
    if (band < ref) return (j >= band && j < ref) ? -1.f : 0.f;
    if (band > ref) return (j >= ref && j < band) ? 1.f : 0.f;
    return 0.f;
}
template <class R> __device__ __forceinline__ const R* wcs_row(const ImgMeta& im);
template <> __device__ __forceinline__ const double* wcs_row<double>(const ImgMeta& im) { return im.A; }
template <> __device__ __forceinline__ const float* wcs_row<float>(const ImgMeta& im) { return im.A_f; }

// Column j of dy/dtheta for one patch as up to three (y, coefficient) pairs (unused
// pairs point at y = 0 with coefficient 0), El = E[l|i] = exp(m + v/2),
// El2 = E[l^2|i] = exp(2m + 2v):
//   u -> mean via A;  e_dev -> e_dev;  (e_axis, e_angle, e_scale) -> G via dG;
//   r1 -> (El, 2 El2);  r2 -> (El/2, 2 El2);  c1_j -> beta_j (El, 2 El2);
//   c2_j -> beta_j^2 (El/2, 2 El2);  a_i -> a_i;  k -> nothing.
template <class R>
__device__ __forceinline__ void chain_column(int j, int band, const R* A, const R* el,
                                             const R* el2, const R (*dG)[3], int* y0, R* c0,
                                             int* y1, R* c1, int* y2, R* c2) {
    *y0 = *y1 = *y2 = 0;
    *c0 = *c1 = *c2 = (R)0;
    if (j < 2) {
        *y0 = Y_MX; *c0 = A[j];
        *y1 = Y_MY; *c1 = A[2 + j];
    } else if (j == P_EDEV) {
        *y0 = Y_EDEV; *c0 = (R)1;
    } else if (j <= P_SCALE) {
        const int q = j - P_AXIS;
        *y0 = Y_GXX; *c0 = dG[q][0];
        *y1 = Y_GXY; *c1 = dG[q][1];
        *y2 = Y_GYY; *c2 = dG[q][2];
    } else if (j < P_A) {
        int i, c = 0;
        R fm, fv;   // weights of El and El2
        if (j < P_R2) { i = j - P_R1; fm = (R)1; fv = (R)2; }
        else if (j < P_C1) { i = j - P_R2; fm = (R)0.5; fv = (R)2; }
        else if (j < P_C2) { i = (j - P_C1) / 4; c = (j - P_C1) % 4; const R b = band_beta<R>(band, c); fm = b; fv = (R)2 * b; }
        else { i = (j - P_C2) / 4; c = (j - P_C2) % 4; const R b = band_beta<R>(band, c); fm = (R)0.5 * b * b; fv = (R)2 * b * b; }
        *y0 = (i == 0) ? Y_EL0 : Y_EL1; *c0 = fm * el[i];
        *y1 = (i == 0) ? Y_EL20 : Y_EL21; *c1 = fv * el2[i];
    } else if (j < P_K) {
        *y0 = (j == P_A) ? Y_A0 : Y_A1; *c0 = (R)1;
    }
}

// one CTA per source: the KL in warp 0 (kl_warp), the shape derivative in lane 32,
// then per patch the item sums (lanes 0..12), the band's brightness moments (lanes
// 32..35) and the image-frame shape Jacobian (lanes 40..48), and the chain rule with
// one lane per parameter.  Transcendentals and the small per-source algebra run in the
// path precision R; every sum is FP64.  (A lone FP64 lane costs a whole warp slot of
// the narrow FP64 pipe, so no FP64 work is left to a single thread.)
constexpr int FZ_THREADS = 64;

__device__ __forceinline__ float exr(float x) { return expf(x); }
__device__ __forceinline__ double exr(double x) { return exp(x); }
__device__ __forceinline__ void scr(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void scr(double x, double* s, double* c) { sincos(x, s, c); }

// Called by every thread of a CTA of >= FZ_THREADS threads (it holds barriers); the
// first 64 threads do the work.
template <class R>
__device__ __forceinline__ void finalize_source(int s, int mode, const double* __restrict__ theta,
                                                const PatchGeo* __restrict__ geo,
                                                const int32_t* __restrict__ patch_off,
                                                const ImgMeta* __restrict__ img,
                                                const ModelDev* __restrict__ md,
                                                const double* __restrict__ part,
                                                double* __restrict__ kl_out,
                                                double* __restrict__ local_out,
                                                double* __restrict__ grad_out,
                                                int32_t* __restrict__ status) {
    const int t = threadIdx.x;
    __shared__ double th[NP], klg[NP];
    __shared__ double klv;
    __shared__ R thr[NP];
    for (int i = t; i < NP; i += blockDim.x) {
        const double v = theta[(size_t)NP * s + i];
        th[i] = v;
        thr[i] = (R)v;   // one conversion per parameter
    }
    if (status && t < NP) theta_domain_check(t, theta[(size_t)NP * s + t], status);
    __syncthreads();
    if (t < 32) {
        const double v = kl_warp<R>(*md, th, klg);
        if (t == 0) klv = v;
    }
    // item partials: the source's items are contiguous
    const int pa = patch_off[s], pb = patch_off[s + 1];
    double gacc = 0.0, lacc = 0.0;
    if (pb > pa) {
        const int i0 = geo[pa].item0;
        const PatchGeo gl = geo[pb - 1];
        const int i1 = gl.item0 + gl.nitem;
        // four independent FP64 accumulators so the loads overlap; fixed order
        const int col = (mode >= MODE_GRAD && t < NP) ? PART_TH + t : (t == 48 ? PART_LL : -1);
        if (col >= 0) {
            double q0 = 0.0, q1 = 0.0, q2 = 0.0, q3 = 0.0;
            int it = i0;
            for (; it + 4 <= i1; it += 4) {
                q0 += part[(size_t)it * NPART + col];
                q1 += part[(size_t)(it + 1) * NPART + col];
                q2 += part[(size_t)(it + 2) * NPART + col];
                q3 += part[(size_t)(it + 3) * NPART + col];
            }
            for (; it < i1; ++it) q0 += part[(size_t)it * NPART + col];
            const double sum = (q0 + q1) + (q2 + q3);
            if (t == 48) lacc = sum;
            else gacc = sum;
        }
    }
    __shared__ double lsum;
    if (t == 48) lsum = lacc;
    __syncthreads();
    if (t == 0) {
        kl_out[s] = klv;
        if (local_out) local_out[s] = lsum - klv;
    }
    if (mode >= MODE_GRAD && grad_out && t < NP) grad_out[(size_t)NP * s + t] = gacc - klg[t];
    __syncthreads();   // shared scratch is reused by the caller
}

// total = sum of tile and item ll sums - sum of KL, fixed order; every thread of a CTA
// of <= 512 threads calls it
__device__ __forceinline__ void total_reduce(const double* __restrict__ tile_ll, int n_tile,
                                             const double* __restrict__ item_ll, int n_item,
                                             const double* __restrict__ kl, int n_src,
                                             double* __restrict__ out) {
    __shared__ double red[512];
    double s = 0.0;
    for (int i = threadIdx.x; i < n_tile; i += blockDim.x) s += tile_ll[i];
    for (int i = threadIdx.x; i < n_item; i += blockDim.x) s += item_ll[i];
    for (int i = threadIdx.x; i < n_src; i += blockDim.x) s -= kl[i];
    red[threadIdx.x] = s;
    __syncthreads();
    int n = blockDim.x;
    while (n > 1) {
        const int h = (n + 1) / 2;
        if ((int)threadIdx.x < n - h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
        n = h;
    }
    if (threadIdx.x == 0) *out = red[0];
    __syncthreads();
}

}  // namespace cel
