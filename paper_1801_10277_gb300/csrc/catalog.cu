// Catalog rows with posterior uncertainty (Section VIII: the variational posterior
// gives type probabilities and brightness / colour uncertainties besides the point
// estimates), the fit-quality summary of Table II against a known truth, and the sky
// fill of the model's expected images.
//
// Under q (Section III) a source's type is Bernoulli(a_star); given type t,
// log l_r ~ N(r1_t, r2_t) and the four adjacent-band log colours c_j ~ N(c1_tj, c2_tj)
// independently, so log l_b = log l_r + beta_b . c is Gaussian, and so is the
// magnitude m_b = 22.5 - (2.5 / ln 10) log l_b (nanomaggy zero point 22.5).
#include <math.h>

#include "internal.cuh"

namespace cel {

namespace {

constexpr int CAT_NF = CELESTE_CAT_NFIELD;
constexpr int CAT_BLOCK = 64;           // sources per CTA: rows staged in shared memory
constexpr int SCORE_THREADS = 256;
constexpr int SCORE_NACC = 14;          // 12 error sums + 2 type counts
constexpr double KMAG = 2.5 / 2.302585092994045684;   // 2.5 / ln 10

// log l_b = log l_r + sum_j BETA[b][j] c_j: colours are log(l_{j+1} / l_j) over u g r i z
__constant__ double BETA[5][4] = {{-1, -1, 0, 0}, {0, -1, 0, 0}, {0, 0, 0, 0}, {0, 0, 1, 0}, {0, 0, 1, 1}};

__device__ void catalog_row(const double* __restrict__ th, double* __restrict__ o, int32_t* status) {
    bool ok = true;
    for (int i = 0; i < NP; ++i) ok = ok && isfinite(th[i]);
    for (int t = 0; t < 2; ++t) {
        ok = ok && th[P_R2 + t] > 0;
        for (int j = 0; j < 4; ++j) ok = ok && th[P_C2 + 4 * t + j] > 0;
    }
    if (!ok && status) atomicCAS(status, 0, (int32_t)CELESTE_ERR_ARG);
    o[CELESTE_CAT_U0] = th[0];
    o[CELESTE_CAT_U1] = th[1];
    o[CELESTE_CAT_PSTAR] = th[P_A];
    o[CELESTE_CAT_IS_STAR] = th[P_A] >= 0.5 ? 1.0 : 0.0;
    double mt[2], vt[2];   // E[l_r | t], Var[l_r | t]
    for (int t = 0; t < 2; ++t) {
        double* b = o + (t == 0 ? CELESTE_CAT_STAR : CELESTE_CAT_GAL);
        const double r1 = th[P_R1 + t], r2 = th[P_R2 + t];
        b[CELESTE_CAT_RMAG] = 22.5 - KMAG * r1;
        b[CELESTE_CAT_RMAG_SD] = KMAG * sqrt(r2);
        const double mean = exp(r1 + 0.5 * r2);
        b[CELESTE_CAT_RFLUX] = mean;
        const double sd = mean * sqrt(expm1(r2));
        b[CELESTE_CAT_RFLUX_SD] = sd;
        mt[t] = mean;
        vt[t] = sd * sd;
        for (int j = 0; j < 4; ++j) {
            b[CELESTE_CAT_COLOR + j] = KMAG * th[P_C1 + 4 * t + j];
            b[CELESTE_CAT_COLOR_SD + j] = KMAG * sqrt(th[P_C2 + 4 * t + j]);
        }
        for (int band = 0; band < 5; ++band) {
            double mu = r1, var = r2;
            for (int j = 0; j < 4; ++j) {
                mu += BETA[band][j] * th[P_C1 + 4 * t + j];
                var += BETA[band][j] * BETA[band][j] * th[P_C2 + 4 * t + j];
            }
            b[CELESTE_CAT_MAG + band] = 22.5 - KMAG * mu;
            b[CELESTE_CAT_MAG_SD + band] = KMAG * sqrt(var);
        }
    }
    // two-component mixture over types with weights a_star + a_gal = 1: the variance
    // a0 v0 + a1 v1 + a0 a1 (m0 - m1)^2 has no cancellation (E[l^2] - E[l]^2 loses
    // digits when r2 is small)
    const double a0 = th[P_A], a1 = th[P_A + 1], dm = mt[0] - mt[1];
    o[CELESTE_CAT_RFLUX_MIX] = a0 * mt[0] + a1 * mt[1];
    o[CELESTE_CAT_RFLUX_MIX_SD] = sqrt(a0 * vt[0] + a1 * vt[1] + a0 * a1 * dm * dm);
    o[CELESTE_CAT_EDEV] = th[P_EDEV];
    o[CELESTE_CAT_AXIS] = th[P_AXIS];
    // the orientation has period pi: report it in [0, 180) degrees
    double phi = fmod(th[P_ANGLE], M_PI);
    if (phi < 0) phi += M_PI;
    double deg = phi * (180.0 / M_PI);
    if (deg >= 180.0) deg -= 180.0;
    o[CELESTE_CAT_ANGLE_DEG] = deg;
    o[CELESTE_CAT_SCALE] = th[P_SCALE];
}

// one thread per source; the CTA's 64 rows are staged in shared memory and written out
// as one contiguous, coalesced span
__global__ void __launch_bounds__(CAT_BLOCK) k_catalog(int n, const double* __restrict__ theta,
                                                       double* __restrict__ cat, int32_t* status) {
    __shared__ double rows[CAT_BLOCK * CAT_NF];
    const int s0 = blockIdx.x * CAT_BLOCK;
    const int s = s0 + threadIdx.x;
    if (s < n) catalog_row(theta + (size_t)NP * s, rows + threadIdx.x * CAT_NF, status);
    __syncthreads();
    const int cnt = min(CAT_BLOCK, n - s0) * CAT_NF;
    double* dst = cat + (size_t)s0 * CAT_NF;
    for (int i = threadIdx.x; i < cnt; i += CAT_BLOCK) dst[i] = rows[i];
}

// Table II's error summary: per-thread FP64 partial sums over a strided subset of the
// sources, then a fixed-order tree over the CTA, so the result is reproducible
__global__ void __launch_bounds__(SCORE_THREADS) k_score(int n, const double* __restrict__ est,
                                                         const double* __restrict__ tru,
                                                         double* __restrict__ score) {
    __shared__ double red[SCORE_NACC][SCORE_THREADS];
    double acc[SCORE_NACC];
    for (int k = 0; k < SCORE_NACC; ++k) acc[k] = 0.0;
    for (int i = threadIdx.x; i < n; i += SCORE_THREADS) {
        const double* e = est + (size_t)CAT_NF * i;
        const double* t = tru + (size_t)CAT_NF * i;
        const bool e_star = e[CELESTE_CAT_IS_STAR] != 0.0, t_star = t[CELESTE_CAT_IS_STAR] != 0.0;
        acc[0] += hypot(e[CELESTE_CAT_U0] - t[CELESTE_CAT_U0], e[CELESTE_CAT_U1] - t[CELESTE_CAT_U1]);
        const double* be = e + (e_star ? CELESTE_CAT_STAR : CELESTE_CAT_GAL);
        const double* bt = t + (t_star ? CELESTE_CAT_STAR : CELESTE_CAT_GAL);
        acc[1] += fabs(be[CELESTE_CAT_RMAG] - bt[CELESTE_CAT_RMAG]);
        for (int j = 0; j < 4; ++j) acc[2 + j] += fabs(be[CELESTE_CAT_COLOR + j] - bt[CELESTE_CAT_COLOR + j]);
        if (t_star) {
            acc[6] += 1.0;
            acc[7] += e_star ? 0.0 : 1.0;
        } else {
            acc[8] += 1.0;
            acc[9] += e_star ? 1.0 : 0.0;
            acc[10] += fabs(e[CELESTE_CAT_EDEV] - t[CELESTE_CAT_EDEV]);
            acc[11] += fabs(e[CELESTE_CAT_AXIS] - t[CELESTE_CAT_AXIS]);
            acc[12] += fabs(e[CELESTE_CAT_SCALE] - t[CELESTE_CAT_SCALE]);
            const double d = fabs(e[CELESTE_CAT_ANGLE_DEG] - t[CELESTE_CAT_ANGLE_DEG]);
            acc[13] += fmin(d, 180.0 - d);
        }
    }
    for (int k = 0; k < SCORE_NACC; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = SCORE_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < SCORE_NACC; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double N = (double)n, ns = red[6][0], ng = red[8][0];
        auto mean = [](double s, double c) { return c > 0 ? s / c : 0.0; };
        score[CELESTE_SCORE_POSITION] = mean(red[0][0], N);
        score[CELESTE_SCORE_MISSED_GAL] = mean(red[9][0], ng);
        score[CELESTE_SCORE_MISSED_STAR] = mean(red[7][0], ns);
        score[CELESTE_SCORE_BRIGHTNESS] = mean(red[1][0], N);
        for (int j = 0; j < 4; ++j) score[CELESTE_SCORE_COLOR + j] = mean(red[2 + j][0], N);
        score[CELESTE_SCORE_PROFILE] = mean(red[10][0], ng);
        score[CELESTE_SCORE_AXIS] = mean(red[11][0], ng);
        score[CELESTE_SCORE_SCALE] = mean(red[12][0], ng);
        score[CELESTE_SCORE_ANGLE_DEG] = mean(red[13][0], ng);
        score[CELESTE_SCORE_N_GAL] = ng;
        score[CELESTE_SCORE_N_STAR] = ns;
    }
}

// E = sky, Var = 0 over every pixel of every image (blockIdx.y = image); the covered
// pixels are then overwritten by the gather
__global__ void k_fill_sky(const ImgMeta* __restrict__ img, const float* __restrict__ sky_map,
                           double* __restrict__ e, double* __restrict__ v) {
    const ImgMeta& im = img[blockIdx.y];
    const int64_t npx = (int64_t)im.H * im.W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npx; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = im.px_off + i;
        e[m] = im.has_sky_map ? (double)sky_map[m] : im.sky;
        v[m] = 0.0;
    }
}

}  // namespace

cudaError_t launch_fill_sky(const DevProblem& P, double* d_e, double* d_v, cudaStream_t st) {
    if (P.n_img <= 0) return cudaSuccess;
    k_fill_sky<<<dim3(2 * 152, P.n_img), 256, 0, st>>>(P.img, P.sky_map, d_e, d_v);
    return cudaGetLastError();
}

cudaError_t launch_catalog(int n, const double* d_theta, double* d_cat, int32_t* d_status, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_catalog<<<(n + CAT_BLOCK - 1) / CAT_BLOCK, CAT_BLOCK, 0, st>>>(n, d_theta, d_cat, d_status);
    return cudaGetLastError();
}

cudaError_t launch_score(int n, const double* d_est, const double* d_true, double* d_score, cudaStream_t st) {
    k_score<<<1, SCORE_THREADS, 0, st>>>(n, d_est, d_true, d_score);
    return cudaGetLastError();
}

}  // namespace cel
