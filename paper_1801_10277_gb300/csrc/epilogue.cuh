// Per-source epilogue shared by the standalone finalize kernel and the tail of the
// adjoint kernel: item sums -> chain rule -> KL -> local objective and gradient; and
// the total.  FP64 sums; transcendentals of the FP32 path in FP32 where the range allows.
#pragma once

#include <math.h>

#include "internal.cuh"
#include "source_math.cuh"

namespace cel {

// d ELBO / d theta_j contributed by one patch through the intermediate variables y:
// sum_y Gy[y] dy/dtheta_j (El = E[l|i] = exp(m + v/2), El2 = E[l^2|i] = exp(2m + 2v)).
__device__ __forceinline__ double chain_entry(int j, int band, const double* A, const double* Gy,
                                              const double* el, const double* el2,
                                              const double (*dG)[3]) {
    if (j == 0) return Gy[Y_MX] * A[0] + Gy[Y_MY] * A[2];
    if (j == 1) return Gy[Y_MX] * A[1] + Gy[Y_MY] * A[3];
    if (j == P_EDEV) return Gy[Y_EDEV];
    if (j >= P_AXIS && j <= P_SCALE) {
        const int q = j - P_AXIS;
        return Gy[Y_GXX] * dG[q][0] + Gy[Y_GXY] * dG[q][1] + Gy[Y_GYY] * dG[q][2];
    }
    if (j >= P_A) return (j < P_K) ? Gy[j == P_A ? Y_A0 : Y_A1] : 0.0;
    int i, kind, c = 0;   // kind: 0 r1, 1 r2, 2 c1, 3 c2
    if (j < P_R2) { i = j - P_R1; kind = 0; }
    else if (j < P_C1) { i = j - P_R2; kind = 1; }
    else if (j < P_C2) { i = (j - P_C1) / 4; c = (j - P_C1) % 4; kind = 2; }
    else { i = (j - P_C2) / 4; c = (j - P_C2) % 4; kind = 3; }
    const double gl = Gy[i == 0 ? Y_EL0 : Y_EL1] * el[i];
    const double gl2 = Gy[i == 0 ? Y_EL20 : Y_EL21] * el2[i];
    const double dm = gl + 2.0 * gl2, dv = 0.5 * gl + 2.0 * gl2;
    if (kind == 0) return dm;
    if (kind == 1) return dv;
    const double b = color_beta(band, c);
    return kind == 2 ? b * dm : b * b * dv;
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
    __shared__ double th[NP], klg[NP], Gy[NY + 1];
    __shared__ double el[2], el2[2], dG[3][3], klv;
    __shared__ R dW[3][3];
    for (int i = t; i < NP; i += blockDim.x) th[i] = theta[(size_t)NP * s + i];
    if (status && t < NP) theta_domain_check(t, theta[(size_t)NP * s + t], status);
    __syncthreads();
    if (t < 32) {
        const double v = kl_warp<R>(*md, th, klg);
        if (t == 0) klv = v;
    } else if (t == 32 && mode >= MODE_GRAD) {
        // world-frame d(Wxx, Wxy, Wyy)/d(e_axis, e_angle, e_scale)
        const R rho = (R)th[P_AXIS], phi = (R)th[P_ANGLE], sg = (R)th[P_SCALE];
        const R bh = (R)0.5 * sg * sg * ((R)1 - rho * rho);
        R s2, c2;
        scr((R)2 * phi, &s2, &c2);
        R da = sg * sg * rho, db = -sg * sg * rho;
        dW[0][0] = da + db * c2; dW[0][1] = db * s2; dW[0][2] = da - db * c2;
        dW[1][0] = (R)-2 * bh * s2; dW[1][1] = (R)2 * bh * c2; dW[1][2] = (R)2 * bh * s2;
        da = sg * ((R)1 + rho * rho); db = sg * ((R)1 - rho * rho);
        dW[2][0] = da + db * c2; dW[2][1] = db * s2; dW[2][2] = da - db * c2;
    }
    __syncthreads();
    double gacc = 0.0, lacc = 0.0;
    const int nv = (mode >= MODE_GRAD) ? 1 + NY : 1;
    for (int p = patch_off[s]; p < patch_off[s + 1]; ++p) {
        const PatchGeo g = geo[p];
        const ImgMeta& im = img[g.img];
        if (t < nv) {
            double v = 0.0;
            for (int it = g.item0; it < g.item0 + g.nitem; ++it) v += part[(size_t)it * NPART + t];
            Gy[t] = v;
        } else if (mode >= MODE_GRAD && t >= 32 && t < 36) {
            const int i = (t - 32) >> 1, second = (t - 32) & 1;
            R m = (R)th[P_R1 + i], v = (R)th[P_R2 + i];
            for (int j = 0; j < 4; ++j) {
                const R b = (R)color_beta(im.band, j);
                m += b * (R)th[P_C1 + 4 * i + j];
                v += b * b * (R)th[P_C2 + 4 * i + j];
            }
            if (second) el2[i] = (double)exr((R)2 * m + (R)2 * v);
            else el[i] = (double)exr(m + (R)0.5 * v);
        } else if (mode >= MODE_GRAD && t >= 40 && t < 49) {
            const int q = (t - 40) / 3, c = (t - 40) % 3;
            const R a0 = (R)im.A[0], a1 = (R)im.A[1], a2 = (R)im.A[2], a3 = (R)im.A[3];
            const R wxx = dW[q][0], wxy = dW[q][1], wyy = dW[q][2];
            R v;
            if (c == 0) v = a0 * a0 * wxx + (R)2 * a0 * a1 * wxy + a1 * a1 * wyy;
            else if (c == 1) v = a0 * a2 * wxx + (a0 * a3 + a1 * a2) * wxy + a1 * a3 * wyy;
            else v = a2 * a2 * wxx + (R)2 * a2 * a3 * wxy + a3 * a3 * wyy;
            dG[q][c] = (double)v;
        }
        __syncthreads();
        if (t == 0) lacc += Gy[0];
        if (mode >= MODE_GRAD && t < NP) gacc += chain_entry(t, im.band, im.A, Gy + 1, el, el2, dG);
        __syncthreads();
    }
    if (t == 0) {
        kl_out[s] = klv;
        if (local_out) local_out[s] = lacc - klv;
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

// Arguments of the epilogue fused into the adjoint's tail (the last CTA of a source
// finalises it; the last source also forms the total).
struct EpilogueArgs {
    int32_t* src_count;           // per source: work items done (reset to 0 by its finaliser)
    const int32_t* src_nitems;    // per source: work items in total
    int32_t* done;                // sources finalised (reset by the last one)
    int32_t n_with_items;         // sources owning at least one work item
    const int32_t* idle_src;      // sources without work items (finalised by the last one)
    int32_t n_idle;
    int32_t n_src, mode;
    const double* theta;
    const int32_t* patch_off;
    const ModelDev* md;
    double* kl;
    double* local_out;
    double* grad_out;
    double* total_out;
    int32_t* status;
    const double* tile_ll;
    int32_t n_tile;
    const double* item_ll;
    int32_t n_item_ll;
};

// The fused tail: call from every thread after the CTA wrote its item partials.
template <class R>
__device__ __forceinline__ void adjoint_tail(const EpilogueArgs& ep, int src,
                                             const PatchGeo* __restrict__ geo,
                                             const ImgMeta* __restrict__ img,
                                             const double* __restrict__ part) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&ep.src_count[src], 1) == ep.src_nitems[src] - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    finalize_source<R>(src, ep.mode, ep.theta, geo, ep.patch_off, img, ep.md, part, ep.kl,
                       ep.local_out, ep.grad_out, ep.status);
    if (threadIdx.x == 0) ep.src_count[src] = 0;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(ep.done, 1) == ep.n_with_items - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int k = 0; k < ep.n_idle; ++k)
        finalize_source<R>(ep.idle_src[k], ep.mode, ep.theta, geo, ep.patch_off, img, ep.md, part,
                           ep.kl, ep.local_out, ep.grad_out, ep.status);
    if (ep.total_out)
        total_reduce(ep.tile_ll, ep.n_tile, ep.item_ll, ep.n_item_ll, ep.kl, ep.n_src, ep.total_out);
    if (threadIdx.x == 0) *ep.done = 0;
}

}  // namespace cel
