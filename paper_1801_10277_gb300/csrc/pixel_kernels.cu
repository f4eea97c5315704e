// Pixel-level kernels of the Celeste ELBO hot path (Section III model, Section VI-B:
// the cost is proportional to active pixel visits).
//
//   k_prep     per (source, patch): brightness moments and the PSF x profile
//              mixture table (FP64 arithmetic, stored in the pixel precision)
//   k_contrib  per work item (<= CHUNK pixels of one patch): each source's own
//              E_s and Var_s at its patch pixels
//   k_gather   per 16x16 tile of an image: E and Var summed over the sources
//              whose patches cover the pixel, in ascending source order (no
//              atomics, deterministic), and the pixel's expected log-likelihood
//   k_adjoint  per work item: recomputes the mixture terms (nothing stored from
//              k_contrib but E_s) and accumulates the gradient of the pixel terms
//              wrt the twelve intermediate variables y of the (source, patch)
//
// R = float: mixture and likelihood arithmetic in FP32, warp sums in FP32, every
// sum across warps in FP64.  R = double: FP64 throughout.
#include <math.h>

#include <map>
#include <mutex>
#include <tuple>

#include "internal.cuh"
#include "async_copy.cuh"
#include "epilogue.cuh"

namespace cel {

namespace {

constexpr double LOG2E = 1.4426950408889634073599246810019;


// 2^x on the SFU in one instruction (flush-to-zero: results below 2^-126 become 0)
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double ex2(double x) { return exp2(x); }
__device__ __forceinline__ float lg(float x) { return logf(x); }
__device__ __forceinline__ double lg(double x) { return log(x); }

template <class R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum NV per-thread values over the CTA: FP32/FP64 within a warp, FP64 across warps
// in warp order.  Thread i < NV returns the CTA total of value i.
template <class R, int NV>
__device__ __forceinline__ void cta_sum(const R (&v)[NV], double* out) {
    // warp sums in R (a fixed tree over <= 32 threads' pixels), then FP64 across the
    // warps in warp order
    __shared__ R red[32][NV > 0 ? NV : 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    R ws[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) ws[i] = warp_sum(v[i]);
    __syncthreads();   // a previous call with the same NV may still be reading red
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) red[warp][i] = ws[i];
    __syncthreads();
    if (threadIdx.x < NV) {
        // across warps in FP64 (so no FP32 sum runs over more than one warp's pixels)
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += (double)red[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
}

template <class R>
__device__ __forceinline__ void load_table(R* sT, const R* gT, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) sT[i] = gT[i];
    __syncthreads();
}

}  // namespace

// ---------------------------------------------------------------------------------
// k_prep: one CTA per source; groups of 8 lanes build the patch headers, then the
// threads build the mixture components of all its patches.
//   star component k:        weight alpha_k, mean mu + xi_k, covariance Sigma_k
//   galaxy component (k, j): weight alpha_k w_j (1 - e_dev) [exp] or alpha_k w_j e_dev [dev],
//                            covariance Sigma_k + nu_j G,  G = A W A^T,
//                            W = sigma^2 R(phi) diag(1, rho^2) R(phi)^T
// Positions are formed in FP64 and stored relative to the patch origin (so FP32
// differences stay exact); the galaxy covariance, the brightness moments and the
// per-component algebra run in the table's precision R, spread over lanes (a lone
// FP64 lane costs a whole warp slot of the narrow FP64 pipe).

__device__ __forceinline__ float lg2(float x) { return log2f(x); }
__device__ __forceinline__ double lg2(double x) { return log2(x); }

// Per-pixel FP32 quantities with every rounding written out (no contraction left to the
// compiler), so that every kernel that forms them -- the value-only and the gradient
// variants, the fused pass and the gather / adjoint passes -- gets the same bits.
//   f_i = iota E[l_i] g_i,  E_s = a0 f0 + a1 f1,
//   Var_s = a0 f0^2 em0 + a1 f1^2 em1 + a0 (1 - a0) f0^2 + a1 (1 - a1) f1^2 - 2 a0 a1 f0 f1
//   (em_i = E[l_i^2] / E[l_i]^2 - 1)
__device__ __forceinline__ void pixel_ev(float iota, float a0, float a1, float el0, float el1,
                                         float em0, float em1, float G0, float G1, float& f0,
                                         float& f1, float& es, float& vs) {
    f0 = __fmul_rn(__fmul_rn(iota, el0), G0);
    f1 = __fmul_rn(__fmul_rn(iota, el1), G1);
    es = __fadd_rn(__fmul_rn(a0, f0), __fmul_rn(a1, f1));
    const float f00 = __fmul_rn(f0, f0), f11 = __fmul_rn(f1, f1);
    float v = __fmul_rn(__fmul_rn(a0, f00), em0);
    v = __fadd_rn(v, __fmul_rn(__fmul_rn(a1, f11), em1));
    v = __fadd_rn(v, __fmul_rn(__fmul_rn(a0, __fsub_rn(1.f, a0)), f00));
    v = __fadd_rn(v, __fmul_rn(__fmul_rn(a1, __fsub_rn(1.f, a1)), f11));
    vs = __fsub_rn(v, __fmul_rn(__fmul_rn(2.f, __fmul_rn(a0, a1)), __fmul_rn(f0, f1)));
}
// ll = x (log E - Var / (2 E^2)) - E and its weights c_E = x (1/E + Var/E^3) - 1,
// c_V = -x / (2 E^2)
__device__ __forceinline__ float pixel_ll(float x, float E, float V) {
    const float iE = __fdiv_rn(1.f, E), iE2 = __fmul_rn(iE, iE);
    return __fsub_rn(__fmul_rn(x, __fsub_rn(lg(E), __fmul_rn(__fmul_rn(0.5f, V), iE2))), E);
}
__device__ __forceinline__ void pixel_weights(float x, float E, float V, float& cE, float& cV) {
    const float iE = __fdiv_rn(1.f, E), iE2 = __fmul_rn(iE, iE);
    cE = __fsub_rn(__fmul_rn(x, __fadd_rn(iE, __fmul_rn(V, __fmul_rn(iE2, iE)))), 1.f);
    cV = __fmul_rn(__fmul_rn(-0.5f, x), iE2);
}
__device__ __forceinline__ float ex(float x) { return expf(x); }
__device__ __forceinline__ double ex(double x) { return exp(x); }
__device__ __forceinline__ void sc(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sc(double x, double* s, double* c) { sincos(x, s, c); }

constexpr int PREP_THREADS = 256;
constexpr int PREP_HDR = 8;   // lanes per patch header

// The KL of source s (value, gradient; Section III priors) and the domain check of its
// parameters, by warp PREP_KL_WARP of the source's block while the other warps build
// the patch headers: the KL depends on theta alone, so it costs no step of its own.
constexpr int PREP_KL_WARP = PREP_THREADS / 32 - 1;

template <class R>
__device__ __forceinline__ void prep_kl(int s, const double* th, const R* thr,
                                        const ModelDev* __restrict__ md, double* __restrict__ kl_out,
                                        double* __restrict__ klg_out, int32_t* __restrict__ status,
                                        double* kg /* shared, NP */) {
    const int lane = threadIdx.x & 31;
    if (status)
        for (int i = lane; i < NP; i += 32) theta_domain_check(i, th[i], status);
    const double v = kl_warp<R>(*md, th, thr, kg);
    __syncwarp();
    if (lane == 0) kl_out[s] = v;
    for (int i = lane; i < NP; i += 32) klg_out[(size_t)NP * s + i] = kg[i];
}

template <class R>
__global__ void __launch_bounds__(PREP_THREADS)
k_prep(const double* __restrict__ theta, const PatchGeo* __restrict__ geo,
       const int32_t* __restrict__ patch_off, const ImgMeta* __restrict__ img,
       const ModelDev* __restrict__ md, int n_src, int nprof, R* __restrict__ tbl,
       double* __restrict__ kl_out, double* __restrict__ klg_out, int32_t* __restrict__ status,
       const int32_t* __restrict__ src_active) {
    pdl_trigger();   // the map pass may be scheduled; it waits for the tables
    const int s = blockIdx.x;
    if (s >= n_src || (src_active && !src_active[s])) return;
    const int p0 = patch_off[s], np = patch_off[s + 1] - p0;
    // blockIdx.y picks the rounds of PREP_THREADS / PREP_HDR patches this CTA builds (a
    // source seen in hundreds of images spreads over several CTAs); the KL is y = 0's
    if (blockIdx.y > 0 && (int)blockIdx.y * (PREP_THREADS / PREP_HDR) >= np) return;
    __shared__ double th[NP];
    __shared__ R thr[NP];
    __shared__ R gsh[PREP_THREADS / PREP_HDR][4];   // gxx gxy gyy e_dev per patch of a round
    const int t = threadIdx.x;
    if (t < NP) {
        const double v = theta[(size_t)NP * s + t];
        th[t] = v;
        thr[t] = (R)v;   // the parameters converted once per source
    }
    __syncthreads();
    const bool kl_here = klg_out && (t >> 5) == PREP_KL_WARP && blockIdx.y == 0;
    __shared__ double kg[NP];
    if (np == 0) {
        if (kl_here) prep_kl<R>(s, th, thr, md, kl_out, klg_out, status, kg);
        return;
    }
    const int per_k = 1 + nprof;
    // patches in rounds of PREP_THREADS / PREP_HDR
    for (int r0 = blockIdx.y * (PREP_THREADS / PREP_HDR); r0 < np; r0 += gridDim.y * (PREP_THREADS / PREP_HDR)) {
        const int pi = r0 + t / PREP_HDR, role = t % PREP_HDR;
        if (pi < np) {
            const PatchGeo g = geo[p0 + pi];
            const ImgMeta& im = img[g.img];
            R* T = tbl + (size_t)(p0 + pi) * TBL_STRIDE;
            const int npsf = im.npsf;
            if (role == 0) {
                // position relative to the patch origin in FP64 (the pixel frame spans 2048 px)
                const double* A = im.A;
                const R mux = (R)(A[0] * th[0] + A[1] * th[1] + im.t[0] - g.x0);
                const R muy = (R)(A[2] * th[0] + A[3] * th[1] + im.t[1] - g.y0);
                for (int k = 0; k < MAXPSF; ++k) {
                    const R* ps = psf_row(im, k, R());
                    T[T_MEAN + 2 * k] = k < npsf ? mux + ps[1] : (R)0;
                    T[T_MEAN + 2 * k + 1] = k < npsf ? muy + ps[2] : (R)0;
                }
            } else if (role == 1) {
                // world-frame ellipse W = ah I + bh (cos 2phi, sin 2phi; sin 2phi, -cos 2phi),
                // G = A W A^T, and the chain-rule block dG = A dW A^T over (axis, angle, scale)
                const R rho = thr[P_AXIS], phi = thr[P_ANGLE], sg = thr[P_SCALE];
                const R ah = (R)0.5 * sg * sg * ((R)1 + rho * rho), bh = (R)0.5 * sg * sg * ((R)1 - rho * rho);
                R s2, c2;
                sc(2 * phi, &s2, &c2);
                const R wxx = ah + bh * c2, wxy = bh * s2, wyy = ah - bh * c2;
                const R a0 = wcs_of(im, 0, R()), a1 = wcs_of(im, 1, R()), a2 = wcs_of(im, 2, R()),
                        a3 = wcs_of(im, 3, R());
                R* G = gsh[t / PREP_HDR];
                G[0] = a0 * a0 * wxx + (R)2 * a0 * a1 * wxy + a1 * a1 * wyy;
                G[1] = a0 * a2 * wxx + (a0 * a3 + a1 * a2) * wxy + a1 * a3 * wyy;
                G[2] = a2 * a2 * wxx + (R)2 * a2 * a3 * wxy + a3 * a3 * wyy;
                G[3] = thr[P_EDEV];
                T[T_G + 0] = G[0];
                T[T_G + 1] = G[1];
                T[T_G + 2] = G[2];
                R dW[3][3];
                R da = sg * sg * rho, db = -sg * sg * rho;
                dW[0][0] = da + db * c2; dW[0][1] = db * s2; dW[0][2] = da - db * c2;
                dW[1][0] = (R)-2 * bh * s2; dW[1][1] = (R)2 * bh * c2; dW[1][2] = (R)2 * bh * s2;
                da = sg * ((R)1 + rho * rho); db = sg * ((R)1 - rho * rho);
                dW[2][0] = da + db * c2; dW[2][1] = db * s2; dW[2][2] = da - db * c2;
                for (int q = 0; q < 3; ++q) {
                    const R ux = dW[q][0], uxy = dW[q][1], uy = dW[q][2];
                    T[T_DG + 3 * q + 0] = a0 * a0 * ux + (R)2 * a0 * a1 * uxy + a1 * a1 * uy;
                    T[T_DG + 3 * q + 1] = a0 * a2 * ux + (a0 * a3 + a1 * a2) * uxy + a1 * a3 * uy;
                    T[T_DG + 3 * q + 2] = a2 * a2 * ux + (R)2 * a2 * a3 * uxy + a3 * a3 * uy;
                }
            } else if (role < 6) {
                // brightness moments in this band: log l | type i ~ N(m, v);
                // E[l] = e^{m+v/2}, E[l^2] = e^{2m+2v}
                const int i = (role - 2) >> 1, second = (role - 2) & 1;
                R m = thr[P_R1 + i], v = thr[P_R2 + i];
                for (int j = 0; j < 4; ++j) {
                    const R b = band_beta<R>(im.band, j);
                    m += b * thr[P_C1 + 4 * i + j];
                    v += b * b * thr[P_C2 + 4 * i + j];
                }
                const R arg = second ? (R)2 * m + (R)2 * v : m + (R)0.5 * v;
                T[(i == 0) ? (second ? H_EL20 : H_EL0) : (second ? H_EL21 : H_EL1)] = ex(arg);
            } else if (role == 6) {
                T[H_A0] = thr[P_A];
                T[H_A1] = thr[P_A + 1];
                T[H_IOTA] = (R)im.iota;
                T[7] = (R)0;
            }
        }
        if (r0 == 0 && kl_here) {
            __syncwarp();
            prep_kl<R>(s, th, thr, md, kl_out, klg_out, status, kg);
        }
        __syncthreads();
        // components of the patches of this round
        const int nr = min(np - r0, PREP_THREADS / PREP_HDR);
        const R log2e = (R)LOG2E, log2_2pi = (R)2.6514961294723187;   // log2(2 pi)
        for (int idx = t; ; idx += blockDim.x) {
            // component idx of the round: patch pj = first patch whose running count exceeds idx
            int pj = 0, base_c = idx;
            int npsf_j = 0;
            const ImgMeta* imj = nullptr;
            while (pj < nr) {
                imj = &img[geo[p0 + r0 + pj].img];
                npsf_j = imj->npsf;
                if (base_c < npsf_j * per_k) break;
                base_c -= npsf_j * per_k;
                ++pj;
            }
            if (pj >= nr) break;
            const ImgMeta& im = *imj;
            R* T = tbl + (size_t)(p0 + r0 + pj) * TBL_STRIDE;
            const R* Gp = gsh[pj];
            const R gxx = Gp[0], gxy = Gp[1], gyy = Gp[2], edev = Gp[3];
            const int k = base_c / per_k, j = base_c % per_k - 1;
            const R* ps = psf_row(im, k, R());
            R cxx = ps[3], cxy = ps[4], cyy = ps[5], w = ps[0], dw = 0, nu = 0;
            if (j >= 0) {
                nu = prof_nu_of(*md, j, R());
                const bool dev = j >= md->n_exp;
                cxx += nu * gxx;
                cxy += nu * gxy;
                cyy += nu * gyy;
                const R aw = ps[0] * prof_w_of(*md, j, R());
                w = aw * (dev ? edev : (R)1 - edev);
                dw = dev ? aw : -aw;
            }
            const R det = cxx * cyy - cxy * cxy;
            const R idet = (R)1 / det;
            const R pxx = cyy * idet, pxy = -cxy * idet, pyy = cxx * idet;
            const int base = (j < 0) ? T_STAR + k * STAR_STRIDE : T_GAL + (k * nprof + j) * GAL_STRIDE;
            T[base + 0] = (R)-0.5 * log2e * pxx;
            T[base + 1] = -log2e * pxy;
            T[base + 2] = (R)-0.5 * log2e * pyy;
            T[base + 3] = -log2_2pi - (R)0.5 * lg2(det);
            T[base + 4] = pxx;
            T[base + 5] = pxy;
            T[base + 6] = pyy;
            T[base + 7] = w;
            if (j >= 0) {
                T[base + 8] = dw;
                T[base + 9] = nu;
                T[base + 10] = 0;
                T[base + 11] = 0;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------
// k_contrib: E_s and Var_s of the item's source at each of its pixels.
//   E_s   = a0 f0 + a1 f1,  f_i = iota E[l_i] g_i
//   Var_s = sum_i a_i iota^2 E[l_i^2] g_i^2 - E_s^2, evaluated as
//           sum_i a_i f_i^2 (E[l_i^2]/E[l_i]^2 - 1) + a0 (1-a0) f0^2 + a1 (1-a1) f1^2 - 2 a0 a1 f0 f1
//   (the same polynomial, rearranged so FP32 does not cancel two large squares).
// A pixel no other patch covers is finished here: E = sky + E_s, Var = Var_s and its
// expected log-likelihood go straight to the maps and to the item's ll sum; only
// pixels covered by several patches keep E_s / Var_s for k_gather.

template <class R, int PPT>
__global__ void __launch_bounds__(CHUNK / PPT) k_contrib(const WorkItem* __restrict__ items,
                                                         const int32_t* __restrict__ idx,
                                                         const PatchGeo* __restrict__ geo,
                                                         const ImgMeta* __restrict__ img, int nprof,
                                                         const R* __restrict__ tbl, R* __restrict__ spE,
                                                         R* __restrict__ spV,
                                                         const uint8_t* __restrict__ single,
                                                         const float* __restrict__ pixels,
                                                         const float* __restrict__ sky_map,
                                                         R* __restrict__ emap, R* __restrict__ vmap,
                                                         double* __restrict__ item_ll,
                                                         const int32_t* __restrict__ src_active) {
    __shared__ R sT[TBL_STRIDE];
    const int item = idx ? idx[blockIdx.x] : (int)blockIdx.x;
    const WorkItem it = items[item];
    const PatchGeo g = geo[it.patch];
    if (src_active && !src_active[g.src]) return;
    const ImgMeta& im = img[g.img];
    const int npsf = im.npsf;
    load_table(sT, tbl + (size_t)it.patch * TBL_STRIDE, T_GAL + npsf * nprof * GAL_STRIDE);
    const int t = threadIdx.x;
    // each thread evaluates PPT pixels with every component load shared between them
    int xs[PPT], ys[PPT];
    bool ok[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int l = t + p * (CHUNK / PPT);
        ok[p] = l < it.n;
        const int q = it.q0 + (ok[p] ? l : 0);
        ys[p] = q / g.w;
        xs[p] = q - ys[p] * g.w;
    }
    R g0[PPT], g1[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) g0[p] = g1[p] = 0;
    for (int k = 0; k < npsf; ++k) {
        const R mx = sT[T_MEAN + 2 * k], my = sT[T_MEAN + 2 * k + 1];
        R dxx[PPT], dxy[PPT], dyy[PPT];
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const R dx = (R)xs[p] - mx, dy = (R)ys[p] - my;
            dxx[p] = dx * dx;
            dxy[p] = dx * dy;
            dyy[p] = dy * dy;
        }
        const R* S = sT + T_STAR + k * STAR_STRIDE;
        const R s0 = S[0], s1 = S[1], s2 = S[2], s3 = S[3], s7 = S[7];
#pragma unroll
        for (int p = 0; p < PPT; ++p) g0[p] += s7 * ex2(s0 * dxx[p] + s1 * dxy[p] + s2 * dyy[p] + s3);
        const R* G = sT + T_GAL + k * nprof * GAL_STRIDE;
        for (int j = 0; j < nprof; ++j, G += GAL_STRIDE) {
            const R c0 = G[0], c1 = G[1], c2 = G[2], c3 = G[3], c7 = G[7];
#pragma unroll
            for (int p = 0; p < PPT; ++p) g1[p] += c7 * ex2(c0 * dxx[p] + c1 * dxy[p] + c2 * dyy[p] + c3);
        }
    }
    const R iota = sT[H_IOTA], a0 = sT[H_A0], a1 = sT[H_A1];
    const R el0 = sT[H_EL0], el1 = sT[H_EL1];
    const R em0 = sT[H_EL20] / (el0 * el0) - (R)1, em1 = sT[H_EL21] / (el1 * el1) - (R)1;
    R ll[1] = {0};
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        if (!ok[p]) continue;
        const R f0 = iota * el0 * g0[p], f1 = iota * el1 * g1[p];
        const R e = a0 * f0 + a1 * f1;
        const R v = a0 * f0 * f0 * em0 + a1 * f1 * f1 * em1 + a0 * ((R)1 - a0) * f0 * f0 +
                    a1 * ((R)1 - a1) * f1 * f1 - (R)2 * a0 * a1 * f0 * f1;
        const int q = it.q0 + t + p * (CHUNK / PPT);
        const int64_t sp = g.sp_off + q;
        if (single && single[sp]) {
            const int64_t m = im.px_off + (int64_t)(g.y0 + ys[p]) * im.W + (g.x0 + xs[p]);
            const R E = (im.has_sky_map ? (R)sky_map[m] : (R)im.sky) + e;
            const R x = (R)pixels[m];
            const R iE = (R)1 / E;
            ll[0] += x * (lg(E) - (R)0.5 * v * iE * iE) - E;
            emap[m] = E;
            vmap[m] = v;
        } else {
            spE[sp] = e;
            spV[sp] = v;
        }
    }
    if (single) {
        double tot[1];
        cta_sum<R, 1>(ll, tot);
        if (threadIdx.x == 0) item_ll[item] = tot[0];
    }
}

// ---------------------------------------------------------------------------------
// k_gather: E = sky + sum_s E_s, Var = sum_s Var_s over the sources covering each
// pixel of a tile (ascending source order), and the expected log-likelihood
//   ll = x (log E - Var / (2 E^2)) - E      (delta-method reading of E_q[log F])
// at pixels covered by at least min_cover patches (2 when k_contrib finished the
// singly covered ones, else 1).  One ll sum per tile.

template <class R>
__global__ void __launch_bounds__(TILE* TILE) k_gather(const Tile* __restrict__ tiles,
                                                       const int32_t* __restrict__ tile_list,
                                                       const PatchGeo* __restrict__ geo,
                                                       const ImgMeta* __restrict__ img,
                                                       const float* __restrict__ pixels,
                                                       const float* __restrict__ sky_map,
                                                       const R* __restrict__ spE,
                                                       const R* __restrict__ spV,
                                                       R* __restrict__ emap, R* __restrict__ vmap,
                                                       double* __restrict__ tile_ll,
                                                       int min_cover, CsrBounds cb) {
    const Tile tl = tiles[blockIdx.x];
    const ImgMeta& im = img[tl.img];
    const int gx = tl.x0 + (int)(threadIdx.x % TILE), gy = tl.y0 + (int)(threadIdx.x / TILE);
    const bool list_ok = CEL_IN_BOUNDS(
        tl.list_off >= 0 && tl.list_n >= 0 && (int64_t)tl.list_off + tl.list_n <= cb.n_tile_list, cb.status);
    R ll[1] = {0};
    if (gx < im.W && gy < im.H && list_ok) {
        const int64_t m = im.px_off + (int64_t)gy * im.W + gx;
        R E = im.has_sky_map ? (R)sky_map[m] : (R)im.sky;
        R V = 0;
        int cov = 0;
        for (int e = 0; e < tl.list_n; ++e) {
            const int pe = tile_list[tl.list_off + e];
            if (!CEL_IN_BOUNDS(pe >= 0 && pe < cb.n_patch, cb.status)) continue;
            const PatchGeo g = geo[pe];
            const int xx = gx - g.x0, yy = gy - g.y0;
            if (xx >= 0 && xx < g.w && yy >= 0 && yy < g.h) {
                const int64_t q = g.sp_off + (int64_t)yy * g.w + xx;
                E += spE[q];
                V += spV[q];
                ++cov;
            }
        }
        if (cov >= min_cover) {
            const R x = (R)pixels[m];
            const R iE = (R)1 / E;
            ll[0] = x * (lg(E) - (R)0.5 * V * iE * iE) - E;
            emap[m] = E;
            vmap[m] = V;
        }
    }
    double tot[1];
    cta_sum<R, 1>(ll, tot);
    if (threadIdx.x == 0) tile_ll[blockIdx.x] = tot[0];
}

// ---------------------------------------------------------------------------------
// k_adjoint: per work item, sum over its pixels of ll and of d ll / d y.
//   c_E = d ll/dE = x (1/E + V/E^3) - 1,   c_V = d ll/dV = -x / (2 E^2)
//   d ll/dy = (c_E - 2 c_V E_s) dE_s/dy + c_V dE2_s/dy,  E2_s = sum_i a_i iota^2 E[l_i^2] g_i^2
// Mixture derivatives per component N = c exp(-d'Pd/2)/(2 pi sqrt det C), d = p - mean:
//   dN/dmean = N P d,  dN/dG_xx = nu N ((Pd)_x^2 - Pxx)/2,  dN/dG_xy = nu N ((Pd)_x (Pd)_y - Pxy),
//   dN/dG_yy = nu N ((Pd)_y^2 - Pyy)/2,  dN/de_dev = dc exp(...)/(...)

template <class R, int MODE, int PPT>
__global__ void __launch_bounds__(CHUNK / PPT) k_adjoint(const WorkItem* __restrict__ items,
                                                         const int32_t* __restrict__ idx,
                                                         const PatchGeo* __restrict__ geo,
                                                         const ImgMeta* __restrict__ img, int nprof,
                                                         const float* __restrict__ pixels,
                                                         const R* __restrict__ tbl,
                                                         const R* __restrict__ emap,
                                                         const R* __restrict__ vmap,
                                                         double* __restrict__ part) {
    constexpr int NV = (MODE == MODE_LL) ? 1 : 1 + NY;
    __shared__ R sT[TBL_STRIDE];
    const int item = idx ? idx[blockIdx.x] : (int)blockIdx.x;
    const WorkItem it = items[item];
    const PatchGeo g = geo[it.patch];
    const ImgMeta& im = img[g.img];
    const int npsf = im.npsf;
    load_table(sT, tbl + (size_t)it.patch * TBL_STRIDE, T_GAL + npsf * nprof * GAL_STRIDE);
    R v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = 0;
    const int t = threadIdx.x;
    int xs[PPT], ys[PPT];
    bool ok[PPT];
    R x[PPT], cE[PPT], cV[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int l = t + p * (CHUNK / PPT);
        ok[p] = l < it.n;
        const int q = it.q0 + (ok[p] ? l : 0);
        ys[p] = q / g.w;
        xs[p] = q - ys[p] * g.w;
        const int64_t m = im.px_off + (int64_t)(g.y0 + ys[p]) * im.W + (g.x0 + xs[p]);
        x[p] = (R)pixels[m];
        const R E = emap[m], V = vmap[m];
        const R iE = (R)1 / E;
        if (ok[p]) v[0] += x[p] * (lg(E) - (R)0.5 * V * iE * iE) - E;
        cE[p] = x[p] * (iE + V * iE * iE * iE) - (R)1;
        cV[p] = (R)-0.5 * x[p] * iE * iE;
    }
    if constexpr (MODE >= MODE_GRAD) {
        R g0[PPT], gx0[PPT], gy0[PPT], g1[PPT], gx1[PPT], gy1[PPT], de1[PPT], sxx[PPT], sxy[PPT], syy[PPT];
#pragma unroll
        for (int p = 0; p < PPT; ++p)
            g0[p] = gx0[p] = gy0[p] = g1[p] = gx1[p] = gy1[p] = de1[p] = sxx[p] = sxy[p] = syy[p] = 0;
        for (int k = 0; k < npsf; ++k) {
            const R mx = sT[T_MEAN + 2 * k], my = sT[T_MEAN + 2 * k + 1];
            R dx[PPT], dy[PPT], dxx[PPT], dxy[PPT], dyy[PPT];
#pragma unroll
            for (int p = 0; p < PPT; ++p) {
                dx[p] = (R)xs[p] - mx;
                dy[p] = (R)ys[p] - my;
                dxx[p] = dx[p] * dx[p];
                dxy[p] = dx[p] * dy[p];
                dyy[p] = dy[p] * dy[p];
            }
            {
                const R* S = sT + T_STAR + k * STAR_STRIDE;
                const R s0 = S[0], s1 = S[1], s2 = S[2], s3 = S[3];
                const R pxx = S[4], pxy = S[5], pyy = S[6], c = S[7];
#pragma unroll
                for (int p = 0; p < PPT; ++p) {
                    const R n = c * ex2(s0 * dxx[p] + s1 * dxy[p] + s2 * dyy[p] + s3);
                    const R qx = pxx * dx[p] + pxy * dy[p], qy = pxy * dx[p] + pyy * dy[p];
                    g0[p] += n;
                    gx0[p] += n * qx;
                    gy0[p] += n * qy;
                }
            }
            const R* G = sT + T_GAL + k * nprof * GAL_STRIDE;
            for (int j = 0; j < nprof; ++j, G += GAL_STRIDE) {
                const R c0 = G[0], c1 = G[1], c2 = G[2], c3 = G[3];
                const R pxx = G[4], pxy = G[5], pyy = G[6], c = G[7], dc = G[8], nu = G[9];
#pragma unroll
                for (int p = 0; p < PPT; ++p) {
                    const R e = ex2(c0 * dxx[p] + c1 * dxy[p] + c2 * dyy[p] + c3);
                    const R n = c * e;
                    const R qx = pxx * dx[p] + pxy * dy[p], qy = pxy * dx[p] + pyy * dy[p];
                    g1[p] += n;
                    gx1[p] += n * qx;
                    gy1[p] += n * qy;
                    de1[p] += dc * e;
                    const R nn = n * nu;
                    sxx[p] += nn * (qx * qx - pxx);
                    sxy[p] += nn * (qx * qy - pxy);
                    syy[p] += nn * (qy * qy - pyy);
                }
            }
        }
        const R iota = sT[H_IOTA], a0 = sT[H_A0], a1 = sT[H_A1];
        const R el0 = sT[H_EL0], el20 = sT[H_EL20], el1 = sT[H_EL1], el21 = sT[H_EL21];
        const R i2 = iota * iota;
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            if (!ok[p]) continue;
            const R f0 = iota * el0 * g0[p], f1 = iota * el1 * g1[p];
            const R Es = a0 * f0 + a1 * f1;
            const R w1 = cE[p] - (R)2 * cV[p] * Es, w2 = cV[p];
            const R s0 = i2 * g0[p] * g0[p], s1 = i2 * g1[p] * g1[p];
            v[1 + Y_A0] += w1 * f0 + w2 * el20 * s0;
            v[1 + Y_A1] += w1 * f1 + w2 * el21 * s1;
            v[1 + Y_EL0] += w1 * a0 * iota * g0[p];
            v[1 + Y_EL20] += w2 * a0 * s0;
            v[1 + Y_EL1] += w1 * a1 * iota * g1[p];
            v[1 + Y_EL21] += w2 * a1 * s1;
            const R u0 = a0 * iota * (w1 * el0 + (R)2 * w2 * iota * el20 * g0[p]);
            const R u1 = a1 * iota * (w1 * el1 + (R)2 * w2 * iota * el21 * g1[p]);
            v[1 + Y_MX] += u0 * gx0[p] + u1 * gx1[p];
            v[1 + Y_MY] += u0 * gy0[p] + u1 * gy1[p];
            v[1 + Y_EDEV] += u1 * de1[p];
            v[1 + Y_GXX] += (R)0.5 * u1 * sxx[p];
            v[1 + Y_GXY] += u1 * sxy[p];
            v[1 + Y_GYY] += (R)0.5 * u1 * syy[p];
        }
    }
    __shared__ double tot[NV];
    cta_sum<R, NV>(v, tot);
    __syncthreads();
    double* out = part + (size_t)item * NPART;
    if (threadIdx.x == 0) out[PART_LL] = tot[0];
    if constexpr (MODE >= MODE_GRAD) {
        // chain rule of this item's y-gradient: d/dtheta_j = sum_y dy/dtheta_j d/dy
        // (coefficients in R, sums in FP64), one thread per parameter
        for (int j = threadIdx.x; j < NP; j += blockDim.x) {
            const R el[2] = {sT[H_EL0], sT[H_EL1]}, el2[2] = {sT[H_EL20], sT[H_EL21]};
            int y0, y1, y2;
            R c0, c1, c2;
            chain_column<R>(j, im.band, wcs_row<R>(im), el, el2, (const R(*)[3])(sT + T_DG), &y0,
                            &c0, &y1, &c1, &y2, &c2);
            out[PART_TH + j] = (double)c0 * tot[1 + y0] + (double)c1 * tot[1 + y1] +
                               (double)c2 * tot[1 + y2];
        }
    }
}

// ---------------------------------------------------------------------------------
// Packed FP32x2 variants (tuning code 3): two pixels per thread carried in float2
// registers, every per-component operation one fma/mul/add.rn.f32x2 instruction (half
// the issue slots of the scalar pair).  The table is staged in shared memory with each
// coefficient duplicated, so a coefficient pair is one 64-bit load.

// compile-time knobs of the packed kernels (defaults measured best on GB300)
#ifndef CEL_GAL_UNROLL
#define CEL_GAL_UNROLL 1
#endif
#ifndef CEL_FUSED_MINB
#define CEL_FUSED_MINB 8
#endif
constexpr int GAL_UNROLL = CEL_GAL_UNROLL;

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 ex2x2(float2 a) { return make_float2(ex2(a.x), ex2(a.y)); }

// The PSF-shifted means and the precision entries (Pxx, Pxy, Pyy) are staged negated, so
// d = p - mean is one add and (Pd)_x^2 - Pxx one fma; the kernels then carry -(Pd) and
// flip the sign of its sums once per pixel.
__device__ __forceinline__ bool staged_negated(int i) {
    if (i >= T_MEAN && i < T_STAR) return true;
    if (i >= T_STAR && i < T_STAR + MAXPSF * STAR_STRIDE) {
        const int r = (i - T_STAR) % STAR_STRIDE;
        return r >= 4 && r <= 6;
    }
    if (i >= T_GAL) {
        const int r = (i - T_GAL) % GAL_STRIDE;
        return r >= 4 && r <= 6;
    }
    return false;
}

__device__ __forceinline__ void load_table_x2(float2* sT2, const float* gT, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float v = gT[i];
        sT2[i] = f2(staged_negated(i) ? -v : v);
    }
    __syncthreads();
}

// two coefficient pairs in one 128-bit shared load (p at an even index of the table)
__device__ __forceinline__ void ld2(const float2* p, float2& a, float2& b) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
}

// Work of one item on a staged table, NPAIR pixel pairs per thread (CHUNK / (2 NPAIR)
// threads; every thread of the CTA calls it, it holds barriers).

template <int NPAIR>
__device__ __forceinline__ void contrib_x2_item(int item, const WorkItem& it, const PatchGeo& g,
                                                const ImgMeta& im, int nprof, const float2* sT2,
                                                float* __restrict__ spE, float* __restrict__ spV,
                                                const uint8_t* __restrict__ single,
                                                const float* __restrict__ pixels,
                                                const float* __restrict__ sky_map,
                                                float* __restrict__ emap, float* __restrict__ vmap,
                                                double* __restrict__ item_ll) {
    constexpr int NT = CHUNK / (2 * NPAIR);
    constexpr int PPT = 2 * NPAIR;
    const int npsf = im.npsf;
    const int t = threadIdx.x;
    int xs[PPT], ys[PPT], qs[PPT];
    bool ok[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int l = t + p * NT;
        ok[p] = l < it.n;
        const int q = it.q0 + (ok[p] ? l : 0);
        qs[p] = q;
        ys[p] = q / g.w;
        xs[p] = q - ys[p] * g.w;
    }
    float2 X[NPAIR], Y[NPAIR], g0[NPAIR], g1[NPAIR];
#pragma unroll
    for (int r = 0; r < NPAIR; ++r) {
        X[r] = make_float2((float)xs[2 * r], (float)xs[2 * r + 1]);
        Y[r] = make_float2((float)ys[2 * r], (float)ys[2 * r + 1]);
        g0[r] = g1[r] = f2(0.f);
    }
    for (int k = 0; k < npsf; ++k) {
        float2 nmx, nmy;
        ld2(sT2 + T_MEAN + 2 * k, nmx, nmy);
        float2 dxx[NPAIR], dxy[NPAIR], dyy[NPAIR];
#pragma unroll
        for (int r = 0; r < NPAIR; ++r) {
            const float2 dx = __fadd2_rn(X[r], nmx), dy = __fadd2_rn(Y[r], nmy);
            dxx[r] = __fmul2_rn(dx, dx);
            dxy[r] = __fmul2_rn(dx, dy);
            dyy[r] = __fmul2_rn(dy, dy);
        }
        const float2* S = sT2 + T_STAR + k * STAR_STRIDE;
        float2 s0, s1, s2, s3;
        ld2(S, s0, s1);
        ld2(S + 2, s2, s3);
        const float2 s7 = S[7];
#pragma unroll
        for (int r = 0; r < NPAIR; ++r) {
            float2 a = __ffma2_rn(s2, dyy[r], s3);
            a = __ffma2_rn(s1, dxy[r], a);
            a = __ffma2_rn(s0, dxx[r], a);
            g0[r] = __ffma2_rn(s7, ex2x2(a), g0[r]);
        }
        const float2* G = sT2 + T_GAL + k * nprof * GAL_STRIDE;
        for (int j = 0; j < nprof; ++j, G += GAL_STRIDE) {
            float2 c0, c1, c2, c3;
            ld2(G, c0, c1);
            ld2(G + 2, c2, c3);
            const float2 c7 = G[7];
#pragma unroll
            for (int r = 0; r < NPAIR; ++r) {
                float2 b = __ffma2_rn(c2, dyy[r], c3);
                b = __ffma2_rn(c1, dxy[r], b);
                b = __ffma2_rn(c0, dxx[r], b);
                g1[r] = __ffma2_rn(c7, ex2x2(b), g1[r]);
            }
        }
    }
    const float iota = sT2[H_IOTA].x, a0 = sT2[H_A0].x, a1 = sT2[H_A1].x;
    const float el0 = sT2[H_EL0].x, el1 = sT2[H_EL1].x;
    const float em0 = sT2[H_EL20].x / (el0 * el0) - 1.f, em1 = sT2[H_EL21].x / (el1 * el1) - 1.f;
    float ll[1] = {0.f};
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        if (!ok[p]) continue;
        const int r = p >> 1;
        const float G0 = (p & 1) ? g0[r].y : g0[r].x, G1 = (p & 1) ? g1[r].y : g1[r].x;
        const float f0 = iota * el0 * G0, f1 = iota * el1 * G1;
        const float e = a0 * f0 + a1 * f1;
        const float v = a0 * f0 * f0 * em0 + a1 * f1 * f1 * em1 + a0 * (1.f - a0) * f0 * f0 +
                        a1 * (1.f - a1) * f1 * f1 - 2.f * a0 * a1 * f0 * f1;
        const int64_t sp = g.sp_off + qs[p];
        if (single && single[sp]) {
            const int64_t m = im.px_off + (int64_t)(g.y0 + ys[p]) * im.W + (g.x0 + xs[p]);
            const float E = (im.has_sky_map ? sky_map[m] : (float)im.sky) + e;
            const float x = pixels[m];
            const float iE = 1.f / E;
            ll[0] += x * (lg(E) - 0.5f * v * iE * iE) - E;
            emap[m] = E;
            vmap[m] = v;
        } else {
            spE[sp] = e;
            spV[sp] = v;
        }
    }
    if (single) {
        double tot[1];
        cta_sum<float, 1>(ll, tot);
        if (threadIdx.x == 0) item_ll[item] = tot[0];
    }
}

// The adjoint of one item from the maps (k_contrib / k_gather wrote E and Var).
template <int MODE, int NPAIR>
__device__ __forceinline__ void adjoint_x2_item(int item, const WorkItem& it, const PatchGeo& g,
                                                const ImgMeta& im, int nprof, const float2* sT2,
                                                const float* __restrict__ pixels,
                                                const float* __restrict__ emap,
                                                const float* __restrict__ vmap,
                                                double* __restrict__ part) {
    constexpr int NV = (MODE == MODE_LL) ? 1 : 1 + NY;
    constexpr int NT = CHUNK / (2 * NPAIR);
    constexpr int PPT = 2 * NPAIR;
    const int npsf = im.npsf;
    float v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = 0.f;
    const int t = threadIdx.x;
    // pixel p of this thread: t + p * NT; pair r holds pixels 2r, 2r + 1
    int xs[PPT], ys[PPT];
    bool ok[PPT];
    float cE[PPT], cV[PPT];
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int l = t + p * NT;
        ok[p] = l < it.n;
        const int q = it.q0 + (ok[p] ? l : 0);
        ys[p] = q / g.w;
        xs[p] = q - ys[p] * g.w;
        const int64_t m = im.px_off + (int64_t)(g.y0 + ys[p]) * im.W + (g.x0 + xs[p]);
        const float x = pixels[m];
        const float E = emap[m], V = vmap[m];
        const float ll = pixel_ll(x, E, V);
        if (ok[p]) v[0] += ll;
        pixel_weights(x, E, V, cE[p], cV[p]);
    }
    if constexpr (MODE >= MODE_GRAD) {
        float2 X[NPAIR], Y[NPAIR];
        float2 g0[NPAIR], gx0[NPAIR], gy0[NPAIR], g1[NPAIR], gx1[NPAIR], gy1[NPAIR], de1[NPAIR],
            sxx[NPAIR], sxy[NPAIR], syy[NPAIR];
#pragma unroll
        for (int r = 0; r < NPAIR; ++r) {
            X[r] = make_float2((float)xs[2 * r], (float)xs[2 * r + 1]);
            Y[r] = make_float2((float)ys[2 * r], (float)ys[2 * r + 1]);
            g0[r] = gx0[r] = gy0[r] = g1[r] = gx1[r] = gy1[r] = de1[r] = sxx[r] = sxy[r] = syy[r] = f2(0.f);
        }
        for (int k = 0; k < npsf; ++k) {
            float2 nmx, nmy;
            ld2(sT2 + T_MEAN + 2 * k, nmx, nmy);
            float2 dx[NPAIR], dy[NPAIR], dxx[NPAIR], dxy[NPAIR], dyy[NPAIR];
#pragma unroll
            for (int r = 0; r < NPAIR; ++r) {
                dx[r] = __fadd2_rn(X[r], nmx);
                dy[r] = __fadd2_rn(Y[r], nmy);
                dxx[r] = __fmul2_rn(dx[r], dx[r]);
                dxy[r] = __fmul2_rn(dx[r], dy[r]);
                dyy[r] = __fmul2_rn(dy[r], dy[r]);
            }
            {
                const float2* S = sT2 + T_STAR + k * STAR_STRIDE;
                float2 s0, s1, s2, s3, npxx, npxy, npyy, c;
                ld2(S, s0, s1);
                ld2(S + 2, s2, s3);
                ld2(S + 4, npxx, npxy);
                ld2(S + 6, npyy, c);
#pragma unroll
                for (int r = 0; r < NPAIR; ++r) {
                    float2 a = __ffma2_rn(s2, dyy[r], s3);
                    a = __ffma2_rn(s1, dxy[r], a);
                    a = __ffma2_rn(s0, dxx[r], a);
                    const float2 ea = ex2x2(a);
                    const float2 n = __fmul2_rn(c, ea);
                    const float2 qx = __ffma2_rn(npxx, dx[r], __fmul2_rn(npxy, dy[r]));   // -(Pd)_x
                    const float2 qy = __ffma2_rn(npxy, dx[r], __fmul2_rn(npyy, dy[r]));   // -(Pd)_y
                    // g as one fused multiply-add (the value-only pass forms it the same way)
                    g0[r] = __ffma2_rn(c, ea, g0[r]);
                    gx0[r] = __ffma2_rn(n, qx, gx0[r]);
                    gy0[r] = __ffma2_rn(n, qy, gy0[r]);
                }
            }
            const float2* G = sT2 + T_GAL + k * nprof * GAL_STRIDE;
#pragma unroll (GAL_UNROLL)
            for (int j = 0; j < nprof; ++j, G += GAL_STRIDE) {
                float2 c0, c1, c2, c3, npxx, npxy, npyy, c, dc, nu;
                ld2(G, c0, c1);
                ld2(G + 2, c2, c3);
                ld2(G + 4, npxx, npxy);
                ld2(G + 6, npyy, c);
                ld2(G + 8, dc, nu);
#pragma unroll
                for (int r = 0; r < NPAIR; ++r) {
                    float2 b = __ffma2_rn(c2, dyy[r], c3);
                    b = __ffma2_rn(c1, dxy[r], b);
                    b = __ffma2_rn(c0, dxx[r], b);
                    const float2 e = ex2x2(b);
                    const float2 n = __fmul2_rn(c, e);
                    const float2 qx = __ffma2_rn(npxx, dx[r], __fmul2_rn(npxy, dy[r]));
                    const float2 qy = __ffma2_rn(npxy, dx[r], __fmul2_rn(npyy, dy[r]));
                    g1[r] = __ffma2_rn(c, e, g1[r]);
                    gx1[r] = __ffma2_rn(n, qx, gx1[r]);
                    gy1[r] = __ffma2_rn(n, qy, gy1[r]);
                    de1[r] = __ffma2_rn(dc, e, de1[r]);
                    const float2 nn = __fmul2_rn(n, nu);
                    sxx[r] = __ffma2_rn(nn, __ffma2_rn(qx, qx, npxx), sxx[r]);
                    sxy[r] = __ffma2_rn(nn, __ffma2_rn(qx, qy, npxy), sxy[r]);
                    syy[r] = __ffma2_rn(nn, __ffma2_rn(qy, qy, npyy), syy[r]);
                }
            }
        }
        const float iota = sT2[H_IOTA].x, a0 = sT2[H_A0].x, a1 = sT2[H_A1].x;
        const float el0 = sT2[H_EL0].x, el20 = sT2[H_EL20].x, el1 = sT2[H_EL1].x, el21 = sT2[H_EL21].x;
        const float i2 = iota * iota;
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            if (!ok[p]) continue;
            const int r = p >> 1;
            const bool hi = p & 1;
            // gx, gy were accumulated with -(Pd): flip them here
            const float G0 = hi ? g0[r].y : g0[r].x, G1 = hi ? g1[r].y : g1[r].x;
            const float GX0 = -(hi ? gx0[r].y : gx0[r].x), GY0 = -(hi ? gy0[r].y : gy0[r].x);
            const float GX1 = -(hi ? gx1[r].y : gx1[r].x), GY1 = -(hi ? gy1[r].y : gy1[r].x);
            const float DE = hi ? de1[r].y : de1[r].x;
            const float SXX = hi ? sxx[r].y : sxx[r].x, SXY = hi ? sxy[r].y : sxy[r].x,
                        SYY = hi ? syy[r].y : syy[r].x;
            const float f0 = __fmul_rn(__fmul_rn(iota, el0), G0);   // as pixel_ev forms them
            const float f1 = __fmul_rn(__fmul_rn(iota, el1), G1);
            const float Es = __fadd_rn(__fmul_rn(a0, f0), __fmul_rn(a1, f1));
            const float w1 = cE[p] - 2.f * cV[p] * Es, w2 = cV[p];
            const float s0 = i2 * G0 * G0, s1 = i2 * G1 * G1;
            v[1 + Y_A0] += w1 * f0 + w2 * el20 * s0;
            v[1 + Y_A1] += w1 * f1 + w2 * el21 * s1;
            v[1 + Y_EL0] += w1 * a0 * iota * G0;
            v[1 + Y_EL20] += w2 * a0 * s0;
            v[1 + Y_EL1] += w1 * a1 * iota * G1;
            v[1 + Y_EL21] += w2 * a1 * s1;
            const float u0 = a0 * iota * (w1 * el0 + 2.f * w2 * iota * el20 * G0);
            const float u1 = a1 * iota * (w1 * el1 + 2.f * w2 * iota * el21 * G1);
            v[1 + Y_MX] += u0 * GX0 + u1 * GX1;
            v[1 + Y_MY] += u0 * GY0 + u1 * GY1;
            v[1 + Y_EDEV] += u1 * DE;
            v[1 + Y_GXX] += 0.5f * u1 * SXX;
            v[1 + Y_GXY] += u1 * SXY;
            v[1 + Y_GYY] += 0.5f * u1 * SYY;
        }
    }
    __shared__ double tot[NV];
    cta_sum<float, NV>(v, tot);
    __syncthreads();
    double* out = part + (size_t)item * NPART;
    if (threadIdx.x == 0) out[PART_LL] = tot[0];
    if constexpr (MODE >= MODE_GRAD) {
        for (int j = threadIdx.x; j < NP; j += blockDim.x) {
            const float el[2] = {sT2[H_EL0].x, sT2[H_EL1].x}, el2[2] = {sT2[H_EL20].x, sT2[H_EL21].x};
            float dG[3][3];
            for (int q = 0; q < 9; ++q) dG[q / 3][q % 3] = sT2[T_DG + q].x;
            int y0, y1, y2;
            float c0, c1, c2;
            chain_column<float>(j, im.band, wcs_row<float>(im), el, el2, dG, &y0, &c0, &y1, &c1, &y2, &c2);
            out[PART_TH + j] = (double)c0 * tot[1 + y0] + (double)c1 * tot[1 + y1] +
                               (double)c2 * tot[1 + y2];
        }
    }
}

// ---- one CTA per item (tuning codes 3, 5): the table staged with plain loads

template <int NPAIR>
__global__ void __launch_bounds__(CHUNK / (2 * NPAIR)) k_contrib_x2(const WorkItem* __restrict__ items,
                                                                  const int32_t* __restrict__ idx,
                                                                  const PatchGeo* __restrict__ geo,
                                                                  const ImgMeta* __restrict__ img, int nprof,
                                                                  const float* __restrict__ tbl,
                                                                  float* __restrict__ spE,
                                                                  float* __restrict__ spV,
                                                                  const uint8_t* __restrict__ single,
                                                                  const float* __restrict__ pixels,
                                                                  const float* __restrict__ sky_map,
                                                                  float* __restrict__ emap,
                                                                  float* __restrict__ vmap,
                                                                  double* __restrict__ item_ll,
                                                                  const int32_t* __restrict__ src_active) {
    __shared__ __align__(16) float2 sT2[TBL_STRIDE];
    const int item = idx ? idx[blockIdx.x] : (int)blockIdx.x;
    const WorkItem it = items[item];
    const PatchGeo g = geo[it.patch];
    if (src_active && !src_active[g.src]) return;
    const ImgMeta& im = img[g.img];
    load_table_x2(sT2, tbl + (size_t)it.patch * TBL_STRIDE, T_GAL + im.npsf * nprof * GAL_STRIDE);
    contrib_x2_item<NPAIR>(item, it, g, im, nprof, sT2, spE, spV, single, pixels, sky_map, emap,
                           vmap, item_ll);
}

template <int MODE, int NPAIR>
__global__ void __launch_bounds__(CHUNK / (2 * NPAIR)) k_adjoint_x2(const WorkItem* __restrict__ items,
                                                                  const int32_t* __restrict__ idx,
                                                                  const PatchGeo* __restrict__ geo,
                                                                  const ImgMeta* __restrict__ img, int nprof,
                                                                  const float* __restrict__ pixels,
                                                                  const float* __restrict__ tbl,
                                                                  const float* __restrict__ emap,
                                                                  const float* __restrict__ vmap,
                                                                  double* __restrict__ part) {
    __shared__ __align__(16) float2 sT2[TBL_STRIDE];
    const int item = idx ? idx[blockIdx.x] : (int)blockIdx.x;
    const WorkItem it = items[item];
    const PatchGeo g = geo[it.patch];
    const ImgMeta& im = img[g.img];
    load_table_x2(sT2, tbl + (size_t)it.patch * TBL_STRIDE, T_GAL + im.npsf * nprof * GAL_STRIDE);
    adjoint_x2_item<MODE, NPAIR>(item, it, g, im, nprof, sT2, pixels, emap, vmap, part);
}

// ---- persistent CTAs with a work queue (tuning codes 6, 7)
//
// A grid of (resident CTAs per SM) x (SMs) CTAs takes items from a global counter.
// Thread 0 runs the queue ahead of the CTA so that no global latency sits on an item's
// critical path: the queue slot of item i + 2 is taken during item i - 1... i, its
// WorkItem is loaded during item i, and at the top of item i + 1's predecessor the
// bulk asynchronous copy of its mixture table is issued (landing in shared memory and
// completing an mbarrier while the current item is computed) together with the load of
// its PatchGeo.  The raw table is double-buffered; each CTA expands it into the
// duplicated / negated FP32x2 layout before use.  The last CTA to finish resets the
// counters for the next launch.

struct PersistentQueue {
    int32_t* queue;    // [0] next item, [1] finished CTAs
    int32_t* status;   // CELESTE_ERR_TIMEOUT when a bounded wait gives up (nullable)
};

// queue slot q -> item index (through the optional list)
__device__ __forceinline__ int queue_item(const int32_t* __restrict__ idx, int q) { return idx ? idx[q] : q; }

template <class Body>
__device__ __forceinline__ void run_items_persistent(const WorkItem* __restrict__ items,
                                                     const int32_t* __restrict__ idx,
                                                     const PatchGeo* __restrict__ geo,
                                                     const ImgMeta* __restrict__ img, int n_item,
                                                     const float* __restrict__ tbl, int tbl_floats,
                                                     PersistentQueue Q, Body& body) {
    __shared__ __align__(16) float raw[2][TBL_STRIDE];
    __shared__ __align__(16) float2 sT2[TBL_STRIDE];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_item[2];
    __shared__ WorkItem s_it[2];
    __shared__ PatchGeo s_g[2];
    const int t = threadIdx.x;
    const unsigned bytes = (unsigned)tbl_floats * 4u;
    // thread 0's look-ahead: n1 / w1 = the item after the current one and its WorkItem,
    // n2 = the one after that (queue slot taken), g_next = the PatchGeo of the item whose
    // table was issued last (stored to shared memory at the top of the next item)
    int n1 = 0, n2 = 0;
    WorkItem w1{};
    PatchGeo g_next{};
    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init_fence();
        fence_proxy_async_smem();
        const int n0 = atomicAdd(Q.queue, 1);
        s_item[0] = n0;
        if (n0 < n_item) {
            const WorkItem w0 = items[queue_item(idx, n0)];
            s_it[0] = w0;
            s_g[0] = geo[w0.patch];
            bulk_copy_g2s(raw[0], tbl + (size_t)w0.patch * TBL_STRIDE, bytes, &bar[0]);
        }
        n1 = atomicAdd(Q.queue, 1);
        if (n1 < n_item) w1 = items[queue_item(idx, n1)];
        n2 = atomicAdd(Q.queue, 1);
    }
    __syncthreads();
    unsigned parity[2] = {0u, 0u};
    int b = 0;
    bool failed = false, first = true;
    for (;;) {
        if (t == 0) {
            if (!first) s_g[b] = g_next;
            first = false;
        }
        const int cur = s_item[b];
        if (cur >= n_item) break;
        if (t == 0) {
            s_item[b ^ 1] = n1;
            if (n1 < n_item) {
                s_it[b ^ 1] = w1;
                g_next = geo[w1.patch];
                fence_proxy_async_smem();   // raw[b ^ 1] was last read by the generic proxy
                bulk_copy_g2s(raw[b ^ 1], tbl + (size_t)w1.patch * TBL_STRIDE, bytes, &bar[b ^ 1]);
            }
            n1 = n2;
            if (n1 < n_item) w1 = items[queue_item(idx, n1)];
            n2 = atomicAdd(Q.queue, 1);
        }
        const bool ok = mbar_wait_bounded(&bar[b], parity[b]);
        parity[b] ^= 1u;
        if (__syncthreads_or(!ok)) {   // also publishes s_g[b]
            failed = true;
            break;
        }
        for (int i = t; i < tbl_floats; i += blockDim.x) {
            const float v = raw[b][i];
            sT2[i] = f2(staged_negated(i) ? -v : v);
        }
        const WorkItem it = s_it[b];
        const PatchGeo g = s_g[b];
        const ImgMeta& im = img[g.img];
        const int item = queue_item(idx, cur);
        __syncthreads();
        body(item, it, g, im, sT2);
        __syncthreads();   // sT2 and the shared item records are rewritten by the next item
        b ^= 1;
    }
    if (failed && t == 0) {
        if (Q.status) atomicExch(Q.status, (int32_t)CELESTE_ERR_TIMEOUT);
        // a copy into the other buffer may still be in flight: let it land (bounded)
        if (s_item[b ^ 1] < n_item) mbar_wait_bounded(&bar[b ^ 1], parity[b ^ 1]);
    }
    if (t == 0) {
        __threadfence();
        if (atomicAdd(Q.queue + 1, 1) == (int)gridDim.x - 1) {
            Q.queue[0] = 0;
            Q.queue[1] = 0;
            __threadfence();
        }
    }
}

template <int NPAIR>
struct ContribBody {
    const int32_t* src_active;
    int nprof;
    float* spE;
    float* spV;
    const uint8_t* single;
    const float* pixels;
    const float* sky_map;
    float* emap;
    float* vmap;
    double* item_ll;
    __device__ void operator()(int item, const WorkItem& it, const PatchGeo& g, const ImgMeta& im,
                               const float2* sT2) const {
        if (src_active && !src_active[g.src]) return;   // uniform over the CTA
        contrib_x2_item<NPAIR>(item, it, g, im, nprof, sT2, spE, spV, single, pixels, sky_map, emap,
                               vmap, item_ll);
    }
};

template <int MODE, int NPAIR>
struct AdjointBody {
    int nprof;
    const float* pixels;
    const float* emap;
    const float* vmap;
    double* part;
    __device__ void operator()(int item, const WorkItem& it, const PatchGeo& g, const ImgMeta& im,
                               const float2* sT2) const {
        adjoint_x2_item<MODE, NPAIR>(item, it, g, im, nprof, sT2, pixels, emap, vmap, part);
    }
};

// at most 64 registers for one pixel pair per thread, so that 8 CTAs fit on an SM
template <int NPAIR>
__global__ void __launch_bounds__(CHUNK / (2 * NPAIR), 8 / NPAIR) k_contrib_pq(const WorkItem* __restrict__ items,
                                                                  const int32_t* __restrict__ idx,
                                                                  const PatchGeo* __restrict__ geo,
                                                                  const ImgMeta* __restrict__ img,
                                                                  int n_item, const float* __restrict__ tbl,
                                                                  int tbl_floats, PersistentQueue Q,
                                                                  ContribBody<NPAIR> body) {
    run_items_persistent(items, idx, geo, img, n_item, tbl, tbl_floats, Q, body);
}

template <int MODE, int NPAIR>
__global__ void __launch_bounds__(CHUNK / (2 * NPAIR), 8 / NPAIR) k_adjoint_pq(const WorkItem* __restrict__ items,
                                                                  const int32_t* __restrict__ idx,
                                                                  const PatchGeo* __restrict__ geo,
                                                                  const ImgMeta* __restrict__ img,
                                                                  int n_item, const float* __restrict__ tbl,
                                                                  int tbl_floats, PersistentQueue Q,
                                                                  AdjointBody<MODE, NPAIR> body) {
    run_items_persistent(items, idx, geo, img, n_item, tbl, tbl_floats, Q, body);
}

// table floats a persistent CTA copies per item: header .. galaxy components of the
// problem's largest PSF (a multiple of 4 floats, so the copy is a multiple of 16 bytes)
static inline int table_floats(const DevProblem& P) { return T_GAL + P.npsf_max * P.nprof * GAL_STRIDE; }

// resident CTAs of a kernel x SMs of the current device, cached per (kernel, device)
static int persistent_grid(const void* kernel, int threads, int n_item) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    int grid = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto f = cache.find({kernel, dev});
        if (f != cache.end()) grid = f->second;
    }
    if (grid == 0) {
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
        grid = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
        std::lock_guard<std::mutex> lk(mu);
        cache[{kernel, dev}] = grid;
    }
    return grid < n_item ? grid : n_item;
}

// The item set of one launch: the items listed in idx[0 .. n) (idx null: items 0 .. n).
struct ItemSet {
    const int32_t* idx;
    int n;
};

template <int NPAIR>
static void contrib_x2(const DevProblem& P, ItemSet S, cudaStream_t st) {
    k_contrib_x2<NPAIR><<<S.n, CHUNK / (2 * NPAIR), 0, st>>>(
        P.items, S.idx, P.geo, P.img, P.nprof, P.tbl32, (float*)P.spE, (float*)P.spE2, P.single,
        P.pixels, P.sky_map, (float*)P.emap, (float*)P.vmap, P.item_ll, P.src_active);
}

template <int NPAIR>
static void contrib_pq(const DevProblem& P, ItemSet S, cudaStream_t st) {
    constexpr int NT = CHUNK / (2 * NPAIR);
    const ContribBody<NPAIR> body{P.src_active, P.nprof, (float*)P.spE, (float*)P.spE2, P.single, P.pixels,
                                  P.sky_map, (float*)P.emap, (float*)P.vmap, P.item_ll};
    const int grid = persistent_grid((const void*)k_contrib_pq<NPAIR>, NT, S.n);
    k_contrib_pq<NPAIR><<<grid, NT, 0, st>>>(P.items, S.idx, P.geo, P.img, S.n, P.tbl32,
                                             table_floats(P), PersistentQueue{P.queue, P.status}, body);
}

template <int NPAIR>
static void adjoint_x2(const DevProblem& P, int mode, ItemSet S, cudaStream_t st) {
    constexpr int NT = CHUNK / (2 * NPAIR);
    if (mode == MODE_LL)
        k_adjoint_x2<MODE_LL, NPAIR><<<S.n, NT, 0, st>>>(P.items, S.idx, P.geo, P.img, P.nprof, P.pixels,
                                                        P.tbl32, (const float*)P.emap,
                                                        (const float*)P.vmap, P.item_part);
    else
        k_adjoint_x2<MODE_GRAD, NPAIR><<<S.n, NT, 0, st>>>(P.items, S.idx, P.geo, P.img, P.nprof, P.pixels,
                                                          P.tbl32, (const float*)P.emap,
                                                          (const float*)P.vmap, P.item_part);
}

template <int MODE, int NPAIR>
static void adjoint_pq_mode(const DevProblem& P, ItemSet S, cudaStream_t st) {
    constexpr int NT = CHUNK / (2 * NPAIR);
    const AdjointBody<MODE, NPAIR> body{P.nprof, P.pixels, (const float*)P.emap, (const float*)P.vmap,
                                        P.item_part};
    const int grid = persistent_grid((const void*)k_adjoint_pq<MODE, NPAIR>, NT, S.n);
    k_adjoint_pq<MODE, NPAIR><<<grid, NT, 0, st>>>(P.items, S.idx, P.geo, P.img, S.n, P.tbl32,
                                                   table_floats(P), PersistentQueue{P.queue, P.status},
                                                   body);
}

template <int NPAIR>
static void adjoint_pq(const DevProblem& P, int mode, ItemSet S, cudaStream_t st) {
    if (mode == MODE_LL) adjoint_pq_mode<MODE_LL, NPAIR>(P, S, st);
    else adjoint_pq_mode<MODE_GRAD, NPAIR>(P, S, st);
}

// Occupancy queries of the persistent kernels, made once on the current device outside
// any stream capture (a CUDA graph of the fit may launch them later).
void prime_persistent_grids() {
    persistent_grid((const void*)k_contrib_pq<1>, CHUNK / 2, 1);
    persistent_grid((const void*)k_contrib_pq<2>, CHUNK / 4, 1);
    persistent_grid((const void*)k_adjoint_pq<MODE_LL, 1>, CHUNK / 2, 1);
    persistent_grid((const void*)k_adjoint_pq<MODE_GRAD, 1>, CHUNK / 2, 1);
    persistent_grid((const void*)k_adjoint_pq<MODE_LL, 2>, CHUNK / 4, 1);
    persistent_grid((const void*)k_adjoint_pq<MODE_GRAD, 2>, CHUNK / 4, 1);
}

// ---------------------------------------------------------------------------------
// launchers

// pixels per thread of the FP32 contrib / adjoint kernels: P.tune (autotuned per
// problem, celeste_autotune), 2 when untuned
static inline int ppt_contrib(const DevProblem& P) { return P.tune_contrib > 0 ? P.tune_contrib : 2; }
static inline int ppt_adjoint(const DevProblem& P) { return P.tune_adjoint > 0 ? P.tune_adjoint : 2; }

cudaError_t launch_prep(const DevProblem& P, const double* d_theta, int precision,
                        cudaStream_t st, bool with_kl) {
    double* klg = with_kl ? P.kl_grad : nullptr;
    if (P.n_src == 0 || (P.n_patch == 0 && !klg)) return cudaSuccess;
    const int per_cta = PREP_THREADS / PREP_HDR;
    const dim3 grid(P.n_src, std::max(1, std::min(64, (P.max_src_patches + per_cta - 1) / per_cta)));
    if (precision == CELESTE_FP64)
        k_prep<double><<<grid, PREP_THREADS, 0, st>>>(d_theta, P.geo, P.patch_off, P.img, P.model,
                                                      P.n_src, P.nprof, P.tbl64, P.kl, klg, P.status,
                                                      P.src_active);
    else
        k_prep<float><<<grid, PREP_THREADS, 0, st>>>(d_theta, P.geo, P.patch_off, P.img, P.model,
                                                     P.n_src, P.nprof, P.tbl32, P.kl, klg, P.status,
                                                     P.src_active);
    return cudaGetLastError();
}

static ItemSet item_set(const DevProblem& P, const int32_t* idx, int n) {
    return ItemSet{idx, n < 0 ? P.n_item : n};
}

cudaError_t launch_contrib(const DevProblem& P, int precision, cudaStream_t st, const int32_t* idx, int n) {
    const ItemSet S = item_set(P, idx, n);
    if (S.n == 0) return cudaSuccess;
    if (precision == CELESTE_FP64)
        k_contrib<double, 1><<<S.n, CHUNK, 0, st>>>(P.items, S.idx, P.geo, P.img, P.nprof, P.tbl64,
                                                    (double*)P.spE, (double*)P.spE2, P.single,
                                                    P.pixels, P.sky_map, (double*)P.emap,
                                                    (double*)P.vmap, P.item_ll, P.src_active);
    else
        switch (ppt_contrib(P)) {
#define CEL_CONTRIB32(N)                                                                          \
    case N:                                                                                       \
        k_contrib<float, N><<<S.n, CHUNK / N, 0, st>>>(P.items, S.idx, P.geo, P.img, P.nprof,       \
                                                       P.tbl32, (float*)P.spE, (float*)P.spE2,      \
                                                       P.single, P.pixels, P.sky_map,              \
                                                       (float*)P.emap, (float*)P.vmap, P.item_ll,  \
                                                       P.src_active);                              \
        break;
            CEL_CONTRIB32(1)
            CEL_CONTRIB32(2)
            CEL_CONTRIB32(4)
#undef CEL_CONTRIB32
            case 3: contrib_x2<1>(P, S, st); break;
            case 5: contrib_x2<2>(P, S, st); break;
            case 6: if (P.queue) contrib_pq<1>(P, S, st); else contrib_x2<1>(P, S, st); break;
            case 7: if (P.queue) contrib_pq<2>(P, S, st); else contrib_x2<2>(P, S, st); break;
            default: return cudaErrorInvalidValue;
        }
    return cudaGetLastError();
}

cudaError_t launch_gather(const DevProblem& P, int precision, cudaStream_t st) {
    if (P.n_tile == 0) return cudaSuccess;
    if (precision == CELESTE_FP64)
        k_gather<double><<<P.n_tile, TILE * TILE, 0, st>>>(
            P.tiles, P.tile_list, P.geo, P.img, P.pixels, P.sky_map, (const double*)P.spE,
            (const double*)P.spE2, (double*)P.emap, (double*)P.vmap, P.tile_ll, P.single ? 2 : 1, csr_bounds(P));
    else
        k_gather<float><<<P.n_tile, TILE * TILE, 0, st>>>(
            P.tiles, P.tile_list, P.geo, P.img, P.pixels, P.sky_map, (const float*)P.spE,
            (const float*)P.spE2, (float*)P.emap, (float*)P.vmap, P.tile_ll, P.single ? 2 : 1, csr_bounds(P));
    return cudaGetLastError();
}

template <class R, int PPT>
static void adjoint_impl(const DevProblem& P, const R* tbl, int mode, ItemSet S, cudaStream_t st) {
    const R* em = (const R*)P.emap;
    const R* vm = (const R*)P.vmap;
    if (mode == MODE_LL)
        k_adjoint<R, MODE_LL, PPT><<<S.n, CHUNK / PPT, 0, st>>>(
            P.items, S.idx, P.geo, P.img, P.nprof, P.pixels, tbl, em, vm, P.item_part);
    else
        k_adjoint<R, MODE_GRAD, PPT><<<S.n, CHUNK / PPT, 0, st>>>(
            P.items, S.idx, P.geo, P.img, P.nprof, P.pixels, tbl, em, vm, P.item_part);
}

cudaError_t launch_adjoint(const DevProblem& P, int precision, int mode, cudaStream_t st,
                           const int32_t* idx, int n) {
    const ItemSet S = item_set(P, idx, n);
    if (S.n == 0) return cudaSuccess;
    if (precision == CELESTE_FP64) {
        adjoint_impl<double, 1>(P, P.tbl64, mode, S, st);
    } else {
        switch (ppt_adjoint(P)) {
            case 1: adjoint_impl<float, 1>(P, P.tbl32, mode, S, st); break;
            case 2: adjoint_impl<float, 2>(P, P.tbl32, mode, S, st); break;
            case 4: adjoint_impl<float, 4>(P, P.tbl32, mode, S, st); break;
            case 3: adjoint_x2<1>(P, mode, S, st); break;
            case 5: adjoint_x2<2>(P, mode, S, st); break;
            case 6: if (P.queue) adjoint_pq<1>(P, mode, S, st); else adjoint_x2<1>(P, mode, S, st); break;
            case 7: if (P.queue) adjoint_pq<2>(P, mode, S, st); else adjoint_x2<2>(P, mode, S, st); break;
            default: return cudaErrorInvalidValue;
        }
    }
    return cudaGetLastError();
}

}  // namespace cel
