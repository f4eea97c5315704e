// Per-source FP64 helpers shared by the gradient and Hessian epilogues: KL terms,
// band brightness moments and the galaxy-shape Jacobian.
#pragma once

#include <math.h>

#include "internal.cuh"

namespace cel {

// KL(q_s || prior) and its gradient (Section III priors Phi, Upsilon, Xi; Eq. 1):
//   KL = sum_i a_i [ log(a_i / Phi_i) + KL_r,i + sum_d k_id ( log(k_id / w_id) + KL_c,id ) ]
//   KL_r,i  = (log(pv/r2) + (r2 + (r1 - pm)^2)/pv - 1) / 2
//   KL_c,id = (tr(P_d diag c2) + (c1 - mu_d)' P_d (c1 - mu_d) - 4 + log det Sigma_d
//              - sum_j log c2_j) / 2
// g (nullable) receives all 44 entries; position and shape entries are zero.
__device__ inline double kl_value_grad(const ModelDev& md, const double* th, double* g) {
    double kl = 0.0;
    if (g)
        for (int i = 0; i < NP; ++i) g[i] = 0.0;
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

__device__ inline void band_moments(const double* th, int band, int i, double& el, double& el2) {
    double m = th[P_R1 + i], v = th[P_R2 + i];
    for (int j = 0; j < 4; ++j) {
        const double b = color_beta(band, j);
        m += b * th[P_C1 + 4 * i + j];
        v += b * b * th[P_C2 + 4 * i + j];
    }
    el = exp(m + 0.5 * v);
    el2 = exp(2.0 * m + 2.0 * v);
}

__device__ inline const double* prior_P_of(const ModelDev& m, int i, int d, double) { return m.prior_P[i][d]; }
__device__ inline const float* prior_P_of(const ModelDev& m, int i, int d, float) { return m.prior_P_f[i][d]; }
__device__ inline const double* prior_mu_of(const ModelDev& m, int i, int d, double) { return m.prior_mu[i][d]; }
__device__ inline const float* prior_mu_of(const ModelDev& m, int i, int d, float) { return m.prior_mu_f[i][d]; }
__device__ inline double prior_ld_of(const ModelDev& m, int i, int d, double) { return m.prior_logdet[i][d]; }
__device__ inline float prior_ld_of(const ModelDev& m, int i, int d, float) { return m.prior_logdet_f[i][d]; }
__device__ inline double prior_w_of(const ModelDev& m, int i, int d, double) { return m.prior_w[i][d]; }
__device__ inline float prior_w_of(const ModelDev& m, int i, int d, float) { return m.prior_w_f[i][d]; }
__device__ __forceinline__ float lgr(float x) { return logf(x); }
__device__ __forceinline__ double lgr(double x) { return log(x); }

// log and reciprocal of a positive normal double for the FP32 path: x = m 2^e split
// with integer operations, the mantissa's log / reciprocal in FP32 (relative error
// ~1e-7), the exponent applied in FP64 -- three FP64-pipe instructions instead of the
// ~40 of a full FP64 log, with FP64's range (k or c2 can fall below FP32's).
__device__ __forceinline__ void split_pos(double x, float* mant, int* ex) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    *ex = (int)((b >> 52) & 0x7FF) - 1023;                    // x = 1.f * 2^ex
    *mant = __uint_as_float(0x3F800000u | (unsigned)((b >> 29) & 0x7FFFFFu));   // 1.f in [1, 2)
}
__device__ __forceinline__ double log_fast(double x) {
    float m;
    int e;
    split_pos(x, &m, &e);
    return (double)logf(m) + (double)e * 0.69314718055994530942;
}
__device__ __forceinline__ double rcp_fast(double x) {
    float m;
    int e;
    split_pos(x, &m, &e);
    return (double)(1.0f / m) * __longlong_as_double((long long)(1023 - e) << 52);
}
template <class R> __device__ __forceinline__ double logp(double x) { return log_fast(x); }
template <> __device__ __forceinline__ double logp<double>(double x) { return log(x); }
template <class R> __device__ __forceinline__ double rcpp(double x) { return rcp_fast(x); }
template <> __device__ __forceinline__ double rcpp<double>(double x) { return 1.0 / x; }

// The KL and its gradient (closed forms of kl_value_grad) computed by one warp; every
// lane must call it.  th: the 44 parameters (FP64), thr: the same in R (shared).
//   phase one (FP64 range, one logarithm / reciprocal per lane): lanes 0..15 log(k_id /
//     w_id), 16..23 log c2 and 1/c2, 24..25 log(a_i / Phi_i), 26..27 log(pv_i / r2_i) and
//     1/r2_i;
//   phase two (lanes 0..15, lane = 8 i + d: type i, colour-prior component d): the 4 x 4
//     algebra of component d in R, then sums over the eight components in R of
//     k_d (log k_d/w_d + KL_d), k_d P_d (c1 - mu_d), k_d diag P_d and k_d;
//   outputs: lanes 8 i + j (j < 4) the c1 / c2 entries of colour j, lanes 8 i + 4..6 the
//     a, r1, r2 entries, in FP64 where a reciprocal can exceed FP32's range.
// The c2 derivative is (sum_d k_d diag P_d - (sum_d k_d) / c2) / 2, the 1/c2 term taken
// out of the component sum.  Writes all 44 entries of g (shared; zero for position and
// shape) and returns the KL on every lane.
template <class R>
__device__ inline double kl_warp(const ModelDev& md, const double* th, const R* thr, double* g) {
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    double lv = 0.0, rv = 0.0;
    if (lane < 16) {
        const int i = lane >> 3, d = lane & 7;
        lv = logp<R>(th[P_K + NCOMP * i + d]) - md.prior_logw[i][d];
    } else if (lane < 24) {
        const double c = th[P_C2 + (lane - 16)];
        lv = logp<R>(c);
        rv = rcpp<R>(c);
    } else if (lane < 26) {
        const int i = lane - 24;
        lv = logp<R>(th[P_A + i]) - md.prior_logphi[i];
    } else if (lane < 28) {
        const int i = lane - 26;
        lv = md.prior_logpv[i] - logp<R>(th[P_R2 + i]);
        rv = rcpp<R>(th[P_R2 + i]);
    }
    const int i = (lane >> 3) & 1, d = lane & 7;
    // log det of q's colour covariance: sum of the four log c2 of type i
    R slog = 0;
    for (int j = 0; j < 4; ++j) slog += (R)__shfl_sync(full, lv, 16 + 4 * i + j);
    // phase two
    R term = 0, ks = 0, kP[4] = {0, 0, 0, 0}, kD[4] = {0, 0, 0, 0};
    if (lane < 16) {
        const R k = thr[P_K + NCOMP * i + d];
        const R* Pm = prior_P_of(md, i, d, R());
        const R* mu = prior_mu_of(md, i, d, R());
        R diff[4], quad = 0, tr = 0;
        for (int j = 0; j < 4; ++j) diff[j] = thr[P_C1 + 4 * i + j] - mu[j];
        for (int j = 0; j < 4; ++j) {
            R sj = 0;
            for (int l = 0; l < 4; ++l) sj += Pm[4 * j + l] * diff[l];
            kP[j] = k * sj;
            kD[j] = k * Pm[5 * j];
            quad += diff[j] * sj;
            tr += Pm[5 * j] * thr[P_C2 + 4 * i + j];
        }
        const R klc = (R)0.5 * (tr + quad - (R)4 + prior_ld_of(md, i, d, R()) - slog);
        term = k * ((R)lv + klc);
        ks = k;
        g[P_K + NCOMP * i + d] = th[P_A + i] * (lv + 1.0 + (double)klc);
    }
    for (int o = 1; o < 8; o <<= 1) {
        term += __shfl_xor_sync(full, term, o);
        ks += __shfl_xor_sync(full, ks, o);
        for (int j = 0; j < 4; ++j) {
            kP[j] += __shfl_xor_sync(full, kP[j], o);
            kD[j] += __shfl_xor_sync(full, kD[j], o);
        }
    }
    // every lane of the group 8 i .. 8 i + 7 holds the type's sums
    const double la = __shfl_sync(full, lv, 24 + i);
    const double lpr = __shfl_sync(full, lv, 26 + i);
    const double ir2 = __shfl_sync(full, rv, 26 + i);
    const double icd = __shfl_sync(full, rv, 16 + 4 * i + (d & 3));   // 1 / c2 of colour d (d < 4)
    double klv = 0.0;
    if (lane < 16) {
        const double ad = th[P_A + i];
        if (d < 4) {
            R kp = kP[0], kd = kD[0];
            for (int j = 1; j < 4; ++j)
                if (j == d) { kp = kP[j]; kd = kD[j]; }
            g[P_C1 + 4 * i + d] = (double)((R)ad * kp);
            g[P_C2 + 4 * i + d] = 0.5 * ad * ((double)kd - icd * (double)ks);
        } else {
            const double r1 = th[P_R1 + i], r2 = th[P_R2 + i];
            const double pm = md.prior_r[i][0];
            const double ipv = md.prior_inv_pv[i];
            if (d == 4) {
                const double K = 0.5 * (lpr + (r2 + (r1 - pm) * (r1 - pm)) * ipv - 1.0) + (double)term;
                klv = ad * (la + K);
                g[P_A + i] = la + 1.0 + K;
            } else if (d == 5) {
                g[P_R1 + i] = ad * (r1 - pm) * ipv;
            } else if (d == 6) {
                g[P_R2 + i] = ad * 0.5 * (ipv - ir2);
            }
        }
    }
    if (lane < 6) g[lane] = 0.0;   // position and shape carry no prior
    klv += __shfl_xor_sync(full, klv, 8);
    return __shfl_sync(full, klv, 4);
}

// Domain of parameter j (celeste.h): every entry finite; e_dev in [0,1]; e_axis in
// (0,1]; e_scale, r2, c2, k > 0; a in (0,1).  A violation sets the status word
// (CELESTE_ERR_NONFINITE or CELESTE_ERR_ARG); nothing traps.
// The comparisons run on the bit pattern (integer operations): for a finite double the
// signed 64-bit pattern orders like the value when the value is >= +0, every negative
// value has a negative pattern and -0 is the pattern's minimum (GB300's FP64 pipe is
// narrow, and these checks run for every parameter of every source in every evaluation).
__device__ inline void theta_domain_check(int j, double x, int32_t* status) {
    const long long b = __double_as_longlong(x);
    constexpr long long ONE = 0x3FF0000000000000LL, NEG_ZERO = (long long)0x8000000000000000ULL;
    if (((b >> 52) & 0x7FF) == 0x7FF) {   // Inf or NaN
        atomicExch(status, (int32_t)CELESTE_ERR_NONFINITE);
        return;
    }
    bool ok;
    if (j == P_EDEV) ok = (b >= 0 && b <= ONE) || b == NEG_ZERO;   // [0, 1]
    else if (j == P_AXIS) ok = b > 0 && b <= ONE;                   // (0, 1]
    else if (j == P_SCALE || (j >= P_R2 && j < P_C1) || (j >= P_C2 && j < P_A) || j >= P_K) ok = b > 0;   // > 0
    else if (j == P_A || j == P_A + 1) ok = b > 0 && b < ONE;       // (0, 1)
    else ok = true;
    if (!ok) atomicExch(status, (int32_t)CELESTE_ERR_ARG);
}

// world-frame d(Wxx, Wxy, Wyy)/d(e_axis, e_angle, e_scale)
__device__ inline void shape_dW(const double* th, double dW[3][3]) {
    const double rho = th[P_AXIS], phi = th[P_ANGLE], sg = th[P_SCALE];
    const double bh = 0.5 * sg * sg * (1.0 - rho * rho);
    double s2, c2;
    sincos(2.0 * phi, &s2, &c2);
    double da = sg * sg * rho, db = -sg * sg * rho;
    dW[0][0] = da + db * c2; dW[0][1] = db * s2; dW[0][2] = da - db * c2;
    dW[1][0] = -2.0 * bh * s2; dW[1][1] = 2.0 * bh * c2; dW[1][2] = 2.0 * bh * s2;
    da = sg * (1.0 + rho * rho); db = sg * (1.0 - rho * rho);
    dW[2][0] = da + db * c2; dW[2][1] = db * s2; dW[2][2] = da - db * c2;
}

// one entry (q, c) of dG = A dW A^T, c = 0 xx, 1 xy, 2 yy
__device__ inline double shape_dG_entry(const double* A, const double dW[3][3], int q, int c) {
    const double wxx = dW[q][0], wxy = dW[q][1], wyy = dW[q][2];
    if (c == 0) return A[0] * A[0] * wxx + 2.0 * A[0] * A[1] * wxy + A[1] * A[1] * wyy;
    if (c == 1) return A[0] * A[2] * wxx + (A[0] * A[3] + A[1] * A[2]) * wxy + A[1] * A[3] * wyy;
    return A[2] * A[2] * wxx + 2.0 * A[2] * A[3] * wxy + A[3] * A[3] * wyy;
}

}  // namespace cel
