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

// One CTA per source: FZ_SLICES slices of FZ_LANES column lanes (lanes 0..43 one
// parameter each, 48 the ll column, 49 the ll of the singly covered pixels, 50 the
// tiles) each sum every FZ_SLICES-th item of the source (items are contiguous per
// source), so a source with hundreds of items is not one long chain of loads; the
// slices are then added in slice order (FP64 throughout, fixed order).  The KL value
// and gradient come from k_prep.  The total's share of the source (ll of its singly
// covered pixels + a strided slice of the tile sums - its KL) goes to src_total; the
// last CTA to finish adds the shares in index order and resets the counter.
constexpr int FZ_LANES = 64;
constexpr int FZ_SLICES = 8;
constexpr int FZ_THREADS = FZ_LANES * FZ_SLICES;

// sum of a[i * stride] for i = i0, i0 + step, ... < i1; four independent accumulators
// so the loads overlap; fixed order
__device__ __forceinline__ double sum_strided4(const double* __restrict__ a, int i0, int i1, int step,
                                               int stride = 1) {
    double q0 = 0.0, q1 = 0.0, q2 = 0.0, q3 = 0.0;
    int i = i0;
    for (; i + 3 * step < i1; i += 4 * step) {
        q0 += a[(size_t)i * stride];
        q1 += a[(size_t)(i + step) * stride];
        q2 += a[(size_t)(i + 2 * step) * stride];
        q3 += a[(size_t)(i + 3 * step) * stride];
    }
    for (; i < i1; i += step) q0 += a[(size_t)i * stride];
    return (q0 + q1) + (q2 + q3);
}

__device__ __forceinline__ void finalize_source(int s, int n_src, int mode,
                                                const PatchGeo* __restrict__ geo,
                                                const int32_t* __restrict__ patch_off,
                                                const int32_t* __restrict__ item_off,
                                                const double* __restrict__ part,
                                                const double* __restrict__ item_ll,
                                                const double* __restrict__ tile_ll, int n_tile,
                                                const double* __restrict__ kl,
                                                const double* __restrict__ kl_grad,
                                                double* __restrict__ local_out,
                                                double* __restrict__ grad_out,
                                                double* __restrict__ src_total,
                                                int32_t* __restrict__ done,
                                                double* __restrict__ total_out) {
    const int t = threadIdx.x, c = t % FZ_LANES, sl = t / FZ_LANES;
    __shared__ double red[FZ_SLICES][FZ_LANES];
    // the source's items: item_off (the split item set) or its patches' items
    int i0 = 0, i1 = 0;
    if (item_off) {
        i0 = item_off[s];
        i1 = item_off[s + 1];
    } else {
        const int pa = patch_off[s], pb = patch_off[s + 1];
        if (pb > pa) {
            i0 = geo[pa].item0;
            const PatchGeo gl = geo[pb - 1];
            i1 = gl.item0 + gl.nitem;
        }
    }
    double acc = 0.0;
    if (i1 > i0) {
        const int col = (mode >= MODE_GRAD && c < NP) ? PART_TH + c : (c == 48 ? PART_LL : -1);
        if (col >= 0) acc = sum_strided4(part + col, i0 + sl, i1, FZ_SLICES, NPART);
        else if (c == 49 && total_out && item_ll) acc = sum_strided4(item_ll, i0 + sl, i1, FZ_SLICES);
    }
    if (c == 50 && total_out) acc = sum_strided4(tile_ll, s + n_src * sl, n_tile, n_src * FZ_SLICES);
    red[sl][c] = acc;
    __syncthreads();
    if (sl == 0) {
        double v = red[0][c];
        for (int q = 1; q < FZ_SLICES; ++q) v += red[q][c];
        red[0][c] = v;
    }
    __syncthreads();
    const double klv = kl[s];
    if (t == 0 && local_out) local_out[s] = red[0][48] - klv;
    if (mode >= MODE_GRAD && grad_out && t < NP) grad_out[(size_t)NP * s + t] = red[0][t] - kl_grad[(size_t)NP * s + t];
    if (!total_out) return;
    __shared__ int last;
    if (t == 0) {
        src_total[s] = (red[0][49] + red[0][50]) - klv;
        __threadfence();
        last = atomicAdd(done, 1) == n_src - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v = 0.0;
    for (int i = t; i < n_src; i += FZ_THREADS) v += __ldcg(src_total + i);
    double* r = &red[0][0];   // FZ_THREADS doubles
    r[t] = v;
    __syncthreads();
    for (int h = FZ_THREADS / 2; h > 0; h >>= 1) {
        if (t < h) r[t] += r[t + h];
        __syncthreads();
    }
    if (t == 0) {
        *total_out = r[0];
        *done = 0;
    }
}

// total = sum of tile and item ll sums - sum of KL, over the concatenated index space
// [tile_ll | item_ll | kl], split into gridDim.x contiguous slices: each CTA of
// TOTAL_THREADS sums its slice (fixed order), the last CTA to finish adds the slice sums
// in order and resets the counter.  Spread over many SMs because GB300's FP64 adds are
// slow on any one SM.
constexpr int TOTAL_THREADS = 256;
constexpr int TOTAL_CTAS = 64;

__device__ __forceinline__ double total_term(const double* __restrict__ tile_ll, int n_tile,
                                             const double* __restrict__ item_ll, int n_item,
                                             const double* __restrict__ kl, int i) {
    if (i < n_tile) return tile_ll[i];
    i -= n_tile;
    if (i < n_item) return item_ll[i];
    return -kl[i - n_item];
}

__device__ __forceinline__ void total_reduce(const double* __restrict__ tile_ll, int n_tile,
                                             const double* __restrict__ item_ll, int n_item,
                                             const double* __restrict__ kl, int n_src,
                                             double* __restrict__ part, int32_t* __restrict__ done,
                                             double* __restrict__ out) {
    __shared__ double red[TOTAL_THREADS];
    __shared__ int last;
    const int t = threadIdx.x;
    const int n = n_tile + n_item + n_src;
    const int per = (n + (int)gridDim.x - 1) / (int)gridDim.x;
    const int i0 = (int)blockIdx.x * per, i1 = min(n, i0 + per);
    double v = 0.0;
    for (int i = i0 + t; i < i1; i += TOTAL_THREADS) v += total_term(tile_ll, n_tile, item_ll, n_item, kl, i);
    red[t] = v;
    __syncthreads();
    for (int h = TOTAL_THREADS / 2; h > 0; h >>= 1) {
        if (t < h) red[t] += red[t + h];
        __syncthreads();
    }
    if (t == 0) {
        part[blockIdx.x] = red[0];
        __threadfence();
        last = atomicAdd(done, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    red[t] = t < (int)gridDim.x ? __ldcg(part + t) : 0.0;
    __syncthreads();
    for (int h = TOTAL_THREADS / 2; h > 0; h >>= 1) {
        if (t < h) red[t] += red[t + h];
        __syncthreads();
    }
    if (t == 0) {
        *out = red[0];
        *done = 0;
    }
}

}  // namespace cel
