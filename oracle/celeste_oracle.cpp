// Celeste ELBO oracle: a plain, slow, FP64 CPU implementation of the variational
// objective, its exact gradient and Hessian, and the per-source trust-region Newton
// fit that consumes them.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load
// this file; it exists so the CUDA path can be checked against an independent
// statement of the method.  It shares no code, header, table or constant with the
// CUDA library: the only common inputs are the arrays the seeded generator draws.
//
// Method (Regier et al., "Cataloging the Visible Universe through Bayesian
// Inference at Petascale", Section III and Section IV-D):
//   * pixel x_nm ~ Poisson(F_nm), F a deterministic function of the catalog and the
//     image metadata (Section III);
//   * per source: Bernoulli type a (star/galaxy), log-normal reference-band
//     brightness r, Gaussian colours c (log ratios of adjacent bands), position mu
//     and galaxy shape phi (Section III);
//   * the ELBO  L = E_q[log p(x, z) - log q(z)]  (Eq. 1);
//   * 44 parameters per source (Section IV), block coordinate ascent with one
//     source per block, Newton steps with exact Hessians inside a trust region
//     (Section IV-D).
// The paper defers the full form of q and of the expected log-likelihood to its
// reference [regier2015celeste], which is not available; every formula below past
// those statements is the reading recorded in the design notes:
//   E_q[log F] ~= log E[F] - Var[F] / (2 E[F]^2)     (second-order delta method)
//   ll(x; E, V) = x (log E - V / (2 E^2)) - E          (log x! dropped)
//
// Derivatives are not hand-derived here.  The value code is written once, as a
// template over its number type, and evaluated on truncated second-order Taylor
// numbers ("jets": value, gradient, Hessian).  Each jet operation applies the
// textbook sum/product/chain rule, so gradient and Hessian are the exact
// derivatives of the value code up to rounding.  Sums over pixels use Neumaier
// compensation.  Compiled without fast-math and with -ffp-contract=off.
//
// Parity status: every function here is pinned by the tests in tests/test_oracle_*.py
// (closed forms, quadrature, finite differences, limits, brute force).

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int NP = 44;
constexpr double BOX_LO_ = 0.01, BOX_HI_ = 0.99, A_LO_ = 0.005, A_HI_ = 0.995;
constexpr double TWO_PI = 6.283185307179586476925286766559;

// ------------------------------------------------------------------------------
// Jets: truncated Taylor polynomials of order 1 (H = false) or 2 (H = true) in N
// variables.

template <int N, bool H>
struct Jet {
    double v;
    double g[N];
    double h[H ? N : 1][H ? N : 1];
};

template <int N, bool H>
inline Jet<N, H> jconst(double c) {
    Jet<N, H> r;
    std::memset(&r, 0, sizeof(r));
    r.v = c;
    return r;
}

template <int N, bool H>
inline Jet<N, H> jvar(double c, int i) {
    Jet<N, H> r = jconst<N, H>(c);
    r.g[i] = 1.0;
    return r;
}

// value-only arithmetic keeps the same spelling as the jet arithmetic
inline double val(double x) { return x; }
template <int N, bool H>
inline double val(const Jet<N, H>& x) { return x.v; }

template <int N, bool H>
inline Jet<N, H> operator+(const Jet<N, H>& a, const Jet<N, H>& b) {
    Jet<N, H> r;
    r.v = a.v + b.v;
    for (int i = 0; i < N; ++i) r.g[i] = a.g[i] + b.g[i];
    if constexpr (H)
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) r.h[i][j] = a.h[i][j] + b.h[i][j];
    return r;
}
template <int N, bool H>
inline Jet<N, H> operator-(const Jet<N, H>& a, const Jet<N, H>& b) {
    Jet<N, H> r;
    r.v = a.v - b.v;
    for (int i = 0; i < N; ++i) r.g[i] = a.g[i] - b.g[i];
    if constexpr (H)
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) r.h[i][j] = a.h[i][j] - b.h[i][j];
    return r;
}
template <int N, bool H>
inline Jet<N, H> operator-(const Jet<N, H>& a) {
    Jet<N, H> r;
    r.v = -a.v;
    for (int i = 0; i < N; ++i) r.g[i] = -a.g[i];
    if constexpr (H)
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) r.h[i][j] = -a.h[i][j];
    return r;
}
template <int N, bool H>
inline Jet<N, H> operator+(const Jet<N, H>& a, double c) {
    Jet<N, H> r = a;
    r.v += c;
    return r;
}
template <int N, bool H>
inline Jet<N, H> operator+(double c, const Jet<N, H>& a) { return a + c; }
template <int N, bool H>
inline Jet<N, H> operator-(const Jet<N, H>& a, double c) { return a + (-c); }
template <int N, bool H>
inline Jet<N, H> operator-(double c, const Jet<N, H>& a) { return (-a) + c; }
template <int N, bool H>
inline Jet<N, H> operator*(const Jet<N, H>& a, double c) {
    Jet<N, H> r;
    r.v = a.v * c;
    for (int i = 0; i < N; ++i) r.g[i] = a.g[i] * c;
    if constexpr (H)
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) r.h[i][j] = a.h[i][j] * c;
    return r;
}
template <int N, bool H>
inline Jet<N, H> operator*(double c, const Jet<N, H>& a) { return a * c; }
// product rule
template <int N, bool H>
inline Jet<N, H> operator*(const Jet<N, H>& a, const Jet<N, H>& b) {
    Jet<N, H> r;
    r.v = a.v * b.v;
    for (int i = 0; i < N; ++i) r.g[i] = a.v * b.g[i] + b.v * a.g[i];
    if constexpr (H)
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j)
                r.h[i][j] = a.v * b.h[i][j] + b.v * a.h[i][j] + a.g[i] * b.g[j] + b.g[i] * a.g[j];
    return r;
}
// chain rule for a scalar function with value f0, first derivative f1, second f2
template <int N, bool H>
inline Jet<N, H> chain(const Jet<N, H>& a, double f0, double f1, double f2) {
    Jet<N, H> r;
    r.v = f0;
    for (int i = 0; i < N; ++i) r.g[i] = f1 * a.g[i];
    if constexpr (H)
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) r.h[i][j] = f1 * a.h[i][j] + f2 * a.g[i] * a.g[j];
    return r;
}
template <int N, bool H>
inline Jet<N, H> recip(const Jet<N, H>& a) {
    double x = a.v;
    return chain(a, 1.0 / x, -1.0 / (x * x), 2.0 / (x * x * x));
}
template <int N, bool H>
inline Jet<N, H> operator/(const Jet<N, H>& a, const Jet<N, H>& b) { return a * recip(b); }
template <int N, bool H>
inline Jet<N, H> operator/(const Jet<N, H>& a, double c) { return a * (1.0 / c); }
template <int N, bool H>
inline Jet<N, H> operator/(double c, const Jet<N, H>& a) { return recip(a) * c; }

inline double jexp(double x) { return std::exp(x); }
inline double jlog(double x) { return std::log(x); }
inline double jsin(double x) { return std::sin(x); }
inline double jcos(double x) { return std::cos(x); }
inline double jsqrt(double x) { return std::sqrt(x); }
template <int N, bool H>
inline Jet<N, H> jexp(const Jet<N, H>& a) {
    double e = std::exp(a.v);
    return chain(a, e, e, e);
}
template <int N, bool H>
inline Jet<N, H> jlog(const Jet<N, H>& a) {
    double x = a.v;
    return chain(a, std::log(x), 1.0 / x, -1.0 / (x * x));
}
template <int N, bool H>
inline Jet<N, H> jsin(const Jet<N, H>& a) {
    return chain(a, std::sin(a.v), std::cos(a.v), -std::sin(a.v));
}
template <int N, bool H>
inline Jet<N, H> jcos(const Jet<N, H>& a) {
    return chain(a, std::cos(a.v), -std::sin(a.v), -std::cos(a.v));
}
template <int N, bool H>
inline Jet<N, H> jsqrt(const Jet<N, H>& a) {
    double s = std::sqrt(a.v);
    return chain(a, s, 0.5 / s, -0.25 / (s * a.v));
}

// Place a jet in M variables into a jet in N variables; slot[i] is the position of
// variable i among the N.  The variables are the same parameters, so this is an
// embedding (no chain rule).
template <int M, int N, bool H>
inline Jet<N, H> embed(const Jet<M, H>& a, const int* slot) {
    Jet<N, H> r = jconst<N, H>(a.v);
    for (int i = 0; i < M; ++i) r.g[slot[i]] = a.g[i];
    if constexpr (H)
        for (int i = 0; i < M; ++i)
            for (int j = 0; j < M; ++j) r.h[slot[i]][slot[j]] = a.h[i][j];
    return r;
}

// Neumaier-compensated accumulator over scalars
struct Acc {
    double s = 0, c = 0;
    void add(double x) {
        double t = s + x;
        if (std::fabs(s) >= std::fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    double sum() const { return s + c; }
};

// ------------------------------------------------------------------------------
// Problem description (flat C layout filled from Python through ctypes)

struct OImage {
    int32_t band, height, width, npsf;
    const float* pixels;     // [H][W] counts
    const float* sky_map;    // [H][W] or null
    double sky;              // counts per pixel when sky_map is null
    double calib;            // nanomaggies per count; iota = 1 / calib
    double wcs[6];           // pixel = A u + t, A row-major
    const double* psf;       // [npsf][6]: alpha, xi_x, xi_y, Sxx, Sxy, Syy
};

struct OProblem {
    int32_t n_img;
    const OImage* imgs;
    int32_t n_exp, n_dev;
    const double* exp_mix;   // [n_exp][2]: weight, variance (unit half-light radius)
    const double* dev_mix;   // [n_dev][2]
    double prior_star;       // Phi: prior probability of a star
    const double* prior_r;   // [2][2]: mean, variance of log r per type
    int32_t n_comp;          // D colour-prior components per type
    const double* prior_c;   // [2][D][21]: weight, mean[4], cov[4][4]
    int32_t n_src;
    const int32_t* patch_off;  // [n_src + 1]
    const int32_t* patches;    // [P][5]: image, x0, y0, w, h
    const int32_t* nbr_off;    // [n_src + 1]
    const int32_t* nbrs;
    // per patch, the image's world -> pixel map linearised at the source ([P][6], same
    // layout as OImage::wcs); null: every patch uses its image's affine wcs
    const double* patch_wcs;
};

// the affine world -> pixel map a patch's source is drawn with
inline const double* patch_map(const OProblem& P, int p) {
    return P.patch_wcs ? P.patch_wcs + 6 * (size_t)p : P.imgs[P.patches[5 * p]].wcs;
}

// parameter indices (constrained layout)
constexpr int IU = 0, IEDEV = 2, IAXIS = 3, IANGLE = 4, ISCALE = 5;
constexpr int IR1 = 6, IR2 = 8, IC1 = 10, IC2 = 18, IA = 26, IK = 28;

// colours are log ratios of adjacent bands (Section III); log l_b = log r + beta_b . c
// with r the reference (r) band brightness and c = (u-g, g-r, r-i, i-z) log ratios
constexpr double BETA[5][4] = {
    {-1, -1, 0, 0}, {0, -1, 0, 0}, {0, 0, 0, 0}, {0, 0, 1, 0}, {0, 0, 1, 1}};

// ------------------------------------------------------------------------------
// The model, written once over a number type T.

// Bivariate normal density at offset (dx, dy) with covariance [[cxx, cxy], [cxy, cyy]].
template <class T>
inline T normal2(const T& dx, const T& dy, const T& cxx, const T& cxy, const T& cyy) {
    T det = cxx * cyy - cxy * cxy;
    T q = (cyy * dx * dx - 2.0 * cxy * dx * dy + cxx * dy * dy) / det;
    return jexp(-0.5 * q - 0.5 * jlog(det)) * (1.0 / TWO_PI);
}
// same with a constant covariance (star: only the mean depends on the parameters)
template <class T>
inline T normal2c(const T& dx, const T& dy, double cxx, double cxy, double cyy) {
    double det = cxx * cyy - cxy * cxy;
    T q = (cyy * dx * dx - 2.0 * cxy * dx * dy + cxx * dy * dy) * (1.0 / det);
    return jexp(-0.5 * q) * (1.0 / (TWO_PI * std::sqrt(det)));
}

// Spatial profile shape part of one source in one image, as a function of the six
// position/shape parameters (u0, u1, e_dev, e_axis, e_angle, e_scale).
template <class T>
struct Shape {
    T mux, muy;          // pixel position  mu = A u + t
    T gxx, gxy, gyy;     // galaxy covariance (unit mixture variance) in pixel coords
    T edev;
};

template <class T>
inline Shape<T> make_shape(const double* A, const T& u0, const T& u1, const T& edev,
                           const T& rho, const T& phi, const T& sigma) {
    Shape<T> s;
    s.mux = A[0] * u0 + A[1] * u1 + A[4];
    s.muy = A[2] * u0 + A[3] * u1 + A[5];
    // world-frame galaxy covariance: sigma^2 R(phi) diag(1, rho^2) R(phi)^T
    T c = jcos(phi), sn = jsin(phi);
    T s2 = sigma * sigma, r2 = rho * rho;
    T wxx = s2 * (c * c + r2 * sn * sn);
    T wxy = s2 * (1.0 - r2) * c * sn;
    T wyy = s2 * (sn * sn + r2 * c * c);
    // pixel frame: A W A^T
    s.gxx = A[0] * A[0] * wxx + 2.0 * A[0] * A[1] * wxy + A[1] * A[1] * wyy;
    s.gxy = A[0] * A[2] * wxx + (A[0] * A[3] + A[1] * A[2]) * wxy + A[1] * A[3] * wyy;
    s.gyy = A[2] * A[2] * wxx + 2.0 * A[2] * A[3] * wxy + A[3] * A[3] * wyy;
    s.edev = edev;
    return s;
}

// Star profile g_star(p) = sum_k alpha_k N(p; mu + xi_k, Sigma_k) and galaxy profile
// g_gal(p) = sum_k alpha_k sum_j [(1 - e_dev) w^e_j N(p; mu + xi_k, Sigma_k + nu^e_j G)
//                                 + e_dev w^d_j N(p; mu + xi_k, Sigma_k + nu^d_j G)]
// at the pixel centre p = (px, py).
template <class T>
inline void profiles(const OProblem& P, const OImage& im, const Shape<T>& s, double px,
                     double py, T& gstar, T& ggal) {
    bool first = true;
    T one_minus = 1.0 - s.edev;
    for (int k = 0; k < im.npsf; ++k) {
        const double* ps = im.psf + 6 * k;
        T dx = px - (s.mux + ps[1]);
        T dy = py - (s.muy + ps[2]);
        T st = normal2c(dx, dy, ps[3], ps[4], ps[5]) * ps[0];
        T ge = st * 0.0, gd = st * 0.0;
        for (int j = 0; j < P.n_exp; ++j) {
            double w = P.exp_mix[2 * j], nu = P.exp_mix[2 * j + 1];
            ge = ge + normal2(dx, dy, ps[3] + nu * s.gxx, ps[4] + nu * s.gxy,
                              ps[5] + nu * s.gyy) * w;
        }
        for (int j = 0; j < P.n_dev; ++j) {
            double w = P.dev_mix[2 * j], nu = P.dev_mix[2 * j + 1];
            gd = gd + normal2(dx, dy, ps[3] + nu * s.gxx, ps[4] + nu * s.gxy,
                              ps[5] + nu * s.gyy) * w;
        }
        T gg = (one_minus * ge + s.edev * gd) * ps[0];
        if (first) {
            gstar = st;
            ggal = gg;
            first = false;
        } else {
            gstar = gstar + st;
            ggal = ggal + gg;
        }
    }
}

// Brightness moments in band b under q given type i: log l ~ N(m, v) with
// m = r1_i + beta_b . c1_i, v = r2_i + (beta_b^2) . c2_i;  E[l] = exp(m + v/2),
// E[l^2] = exp(2m + 2v).
template <class T>
inline void brightness(const T* th, int band, int i, T& El, T& El2) {
    T m = th[IR1 + i], v = th[IR2 + i];
    for (int j = 0; j < 4; ++j) {
        double b = BETA[band][j];
        if (b != 0.0) {
            m = m + b * th[IC1 + 4 * i + j];
            v = v + (b * b) * th[IC2 + 4 * i + j];
        }
    }
    El = jexp(m + 0.5 * v);
    El2 = jexp(2.0 * m + 2.0 * v);
}

// Expected log-likelihood of one pixel with count x under the delta-method reading
// of E_q[log F]:  x (log E - V / (2 E^2)) - E.
template <class T>
inline T pixel_ll(double x, const T& E, const T& V) {
    return x * (jlog(E) - V / (2.0 * E * E)) - E;
}

// KL(q || p) of one source (Eq. 1's  E_q[log q(z) - log p(z)]):
//   sum_i a_i log(a_i / Phi_i)
// + sum_i a_i [ KL(N(r1_i, r2_i) || N(Upsilon_i))
//             + sum_d k_id log(k_id / w_id)
//             + sum_d k_id KL(N(c1_i, diag c2_i) || N(Xi_id)) ]
template <class T>
inline T source_kl(const OProblem& P, const T* th, const double* cinv, const double* cld) {
    const int D = P.n_comp;
    double phi[2] = {P.prior_star, 1.0 - P.prior_star};
    T kl = th[IA] * 0.0;
    for (int i = 0; i < 2; ++i) {
        const T& a = th[IA + i];
        kl = kl + a * jlog(a * (1.0 / phi[i]));
        double pm = P.prior_r[2 * i], pv = P.prior_r[2 * i + 1];
        T r1 = th[IR1 + i], r2 = th[IR2 + i];
        T klr = 0.5 * (std::log(pv) - jlog(r2) + (r2 + (r1 - pm) * (r1 - pm)) * (1.0 / pv) - 1.0);
        T inner = klr;
        for (int d = 0; d < D; ++d) {
            const double* pc = P.prior_c + (size_t)(i * D + d) * 21;
            const double* Pi = cinv + (size_t)(i * D + d) * 16;
            const T& k = th[IK + 8 * i + d];
            T klc = th[IA] * 0.0 + (-4.0 + cld[i * D + d]);
            for (int j = 0; j < 4; ++j) {
                klc = klc + Pi[5 * j] * th[IC2 + 4 * i + j] - jlog(th[IC2 + 4 * i + j]);
            }
            for (int j = 0; j < 4; ++j)
                for (int l = 0; l < 4; ++l) {
                    T dj = th[IC1 + 4 * i + j] - pc[1 + j];
                    T dl = th[IC1 + 4 * i + l] - pc[1 + l];
                    klc = klc + Pi[4 * j + l] * dj * dl;
                }
            klc = 0.5 * klc;
            inner = inner + k * jlog(k * (1.0 / pc[0])) + k * klc;
        }
        kl = kl + a * inner;
    }
    return kl;
}

// inverse and log-determinant of the colour-prior covariances (Cholesky, 4x4)
bool prior_inverses(const OProblem& P, std::vector<double>& inv, std::vector<double>& ld) {
    const int D = P.n_comp;
    inv.assign((size_t)2 * D * 16, 0.0);
    ld.assign((size_t)2 * D, 0.0);
    for (int c = 0; c < 2 * D; ++c) {
        const double* S = P.prior_c + (size_t)c * 21 + 5;
        double L[4][4] = {{0}};
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j <= i; ++j) {
                double s = S[4 * i + j];
                for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
                if (i == j) {
                    if (s <= 0) return false;
                    L[i][i] = std::sqrt(s);
                } else {
                    L[i][j] = s / L[j][j];
                }
            }
        double logdet = 0;
        for (int i = 0; i < 4; ++i) logdet += 2 * std::log(L[i][i]);
        ld[c] = logdet;
        // columns of S^{-1} by forward/back substitution
        for (int col = 0; col < 4; ++col) {
            double y[4], x[4];
            for (int i = 0; i < 4; ++i) {
                double s = (i == col) ? 1.0 : 0.0;
                for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
                y[i] = s / L[i][i];
            }
            for (int i = 3; i >= 0; --i) {
                double s = y[i];
                for (int k = i + 1; k < 4; ++k) s -= L[k][i] * x[k];
                x[i] = s / L[i][i];
            }
            for (int i = 0; i < 4; ++i) inv[(size_t)c * 16 + 4 * i + col] = x[i];
        }
    }
    return true;
}

// the trust region's unconstrained map needs these open intervals
bool theta_in_box(const double* th) {
    return th[IEDEV] > BOX_LO_ && th[IEDEV] < BOX_HI_ && th[IAXIS] > BOX_LO_ &&
           th[IAXIS] < BOX_HI_ && th[IA] > A_LO_ && th[IA] < A_HI_;
}

bool theta_valid(const double* th) {
    for (int i = 0; i < NP; ++i)
        if (!std::isfinite(th[i])) return false;
    if (th[IEDEV] < 0 || th[IEDEV] > 1) return false;
    if (th[IAXIS] <= 0 || th[IAXIS] > 1) return false;
    if (th[ISCALE] <= 0) return false;
    for (int i = 0; i < 2; ++i) {
        if (th[IR2 + i] <= 0) return false;
        if (th[IA + i] <= 0 || th[IA + i] >= 1) return false;
        for (int j = 0; j < 4; ++j)
            if (th[IC2 + 4 * i + j] <= 0) return false;
        for (int d = 0; d < 8; ++d)
            if (th[IK + 8 * i + d] <= 0) return false;
    }
    return true;
}

// ------------------------------------------------------------------------------
// Per-(source, patch) value arrays: E_s and E[F_s^2] over the patch pixels.

struct PatchVals {
    std::vector<double> e, e2;   // row-major over the patch
};

void source_patch_values(const OProblem& P, const double* th, int p, PatchVals& out) {
    const int32_t* pt = P.patches + 5 * p;
    const OImage& im = P.imgs[pt[0]];
    int x0 = pt[1], y0 = pt[2], w = pt[3], h = pt[4];
    double iota = 1.0 / im.calib;
    Shape<double> sh = make_shape<double>(patch_map(P, p), th[IU], th[IU + 1], th[IEDEV], th[IAXIS],
                                          th[IANGLE], th[ISCALE]);
    double El[2], El2[2];
    for (int i = 0; i < 2; ++i) brightness<double>(th, im.band, i, El[i], El2[i]);
    out.e.assign((size_t)w * h, 0.0);
    out.e2.assign((size_t)w * h, 0.0);
    for (int yy = 0; yy < h; ++yy)
        for (int xx = 0; xx < w; ++xx) {
            double g0, g1;
            profiles<double>(P, im, sh, x0 + xx, y0 + yy, g0, g1);
            double a0 = th[IA], a1 = th[IA + 1];
            double f0 = iota * El[0] * g0, f1 = iota * El[1] * g1;
            out.e[(size_t)yy * w + xx] = a0 * f0 + a1 * f1;
            out.e2[(size_t)yy * w + xx] = a0 * iota * iota * El2[0] * g0 * g0 +
                                          a1 * iota * iota * El2[1] * g1 * g1;
        }
}

struct Maps {
    // per image: compensated E and V over all pixels, and a coverage count
    std::vector<std::vector<Acc>> E, V;
    std::vector<std::vector<int32_t>> cover;
};

void build_patch_values(const OProblem& P, const double* theta, std::vector<PatchVals>& pv) {
    int np = P.patch_off[P.n_src];
    pv.assign(np, PatchVals());
#pragma omp parallel for schedule(dynamic, 1)
    for (int s = 0; s < P.n_src; ++s)
        for (int p = P.patch_off[s]; p < P.patch_off[s + 1]; ++p)
            source_patch_values(P, theta + (size_t)NP * s, p, pv[p]);
}

void build_maps(const OProblem& P, const std::vector<PatchVals>& pv, Maps& M) {
    M.E.assign(P.n_img, {});
    M.V.assign(P.n_img, {});
    M.cover.assign(P.n_img, {});
    for (int n = 0; n < P.n_img; ++n) {
        size_t npx = (size_t)P.imgs[n].height * P.imgs[n].width;
        M.E[n].assign(npx, Acc());
        M.V[n].assign(npx, Acc());
        M.cover[n].assign(npx, 0);
    }
    // sources in ascending id
    for (int s = 0; s < P.n_src; ++s)
        for (int p = P.patch_off[s]; p < P.patch_off[s + 1]; ++p) {
            const int32_t* pt = P.patches + 5 * p;
            const OImage& im = P.imgs[pt[0]];
            for (int yy = 0; yy < pt[4]; ++yy)
                for (int xx = 0; xx < pt[3]; ++xx) {
                    size_t m = (size_t)(pt[2] + yy) * im.width + (pt[1] + xx);
                    size_t q = (size_t)yy * pt[3] + xx;
                    double e = pv[p].e[q], e2 = pv[p].e2[q];
                    M.E[pt[0]][m].add(e);
                    M.V[pt[0]][m].add(e2 - e * e);
                    M.cover[pt[0]][m] += 1;
                }
        }
}

inline double sky_at(const OImage& im, size_t m) {
    return im.sky_map ? (double)im.sky_map[m] : im.sky;
}

// E and V at pixel (gx, gy) of the patch's image from every source except `self`
// that covers it (neighbours only can), plus sky: summed directly, no subtraction.
inline void others_at(const OProblem& P, const std::vector<PatchVals>& pv, int self,
                      int img, int gx, int gy, double& E, double& V) {
    const OImage& im = P.imgs[img];
    Acc ae, av;
    ae.add(sky_at(im, (size_t)gy * im.width + gx));
    for (int e = P.nbr_off[self]; e < P.nbr_off[self + 1]; ++e) {
        int o = P.nbrs[e];
        for (int p = P.patch_off[o]; p < P.patch_off[o + 1]; ++p) {
            const int32_t* pt = P.patches + 5 * p;
            if (pt[0] != img) continue;
            int xx = gx - pt[1], yy = gy - pt[2];
            if (xx < 0 || yy < 0 || xx >= pt[3] || yy >= pt[4]) continue;
            size_t q = (size_t)yy * pt[3] + xx;
            ae.add(pv[p].e[q]);
            av.add(pv[p].e2[q] - pv[p].e[q] * pv[p].e[q]);
        }
    }
    E = ae.sum();
    V = av.sum();
}

// ------------------------------------------------------------------------------
// Local objective of one source and its derivatives wrt the 44 constrained params.
//   ELBO_s = sum_{m in P_s} ll_m - KL_s     (neighbours fixed)

constexpr int NA = 20;   // parameters one band can touch

template <bool H>
void local_derivs(const OProblem& P, const std::vector<PatchVals>& pv, const double* cinv,
                  const double* cld, int s, const double* th, double* f_out, double* g_out,
                  double* h_out) {
    std::vector<Acc> G(NP), Hs(H ? NP * NP : 0);
    Acc F;
    for (int p = P.patch_off[s]; p < P.patch_off[s + 1]; ++p) {
        const int32_t* pt = P.patches + 5 * p;
        const OImage& im = P.imgs[pt[0]];
        const double iota = 1.0 / im.calib;
        // active parameters of this band
        int idx[NA], n = 0;
        for (int i = 0; i < 6; ++i) idx[n++] = i;            // u0 u1 e_dev axis angle scale
        for (int i = 0; i < 2; ++i) idx[n++] = IR1 + i;
        for (int i = 0; i < 2; ++i) idx[n++] = IR2 + i;
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 4; ++j)
                if (BETA[im.band][j] != 0.0) {
                    idx[n++] = IC1 + 4 * i + j;
                    idx[n++] = IC2 + 4 * i + j;
                }
        idx[n++] = IA;
        idx[n++] = IA + 1;
        using J20 = Jet<NA, H>;
        using J6 = Jet<6, H>;
        J20 t[NP];
        for (int i = 0; i < NP; ++i) t[i] = jconst<NA, H>(th[i]);
        for (int k = 0; k < n; ++k) t[idx[k]] = jvar<NA, H>(th[idx[k]], k);
        J6 sv[6];
        for (int i = 0; i < 6; ++i) sv[i] = jvar<6, H>(th[i], i);
        int slot6[6] = {0, 1, 2, 3, 4, 5};
        Shape<J6> sh = make_shape<J6>(patch_map(P, p), sv[0], sv[1], sv[2], sv[3], sv[4], sv[5]);
        J20 El[2], El2[2];
        for (int i = 0; i < 2; ++i) brightness<J20>(t, im.band, i, El[i], El2[i]);
        std::vector<Acc> gl(n), hl(H ? n * n : 0);
        for (int yy = 0; yy < pt[4]; ++yy)
            for (int xx = 0; xx < pt[3]; ++xx) {
                int gx = pt[1] + xx, gy = pt[2] + yy;
                size_t m = (size_t)gy * im.width + gx;
                double Eo, Vo;
                others_at(P, pv, s, pt[0], gx, gy, Eo, Vo);
                J6 g0s = jconst<6, H>(0.0), g1s = jconst<6, H>(0.0);
                profiles<J6>(P, im, sh, gx, gy, g0s, g1s);
                J20 g0 = embed<6, NA, H>(g0s, slot6), g1 = embed<6, NA, H>(g1s, slot6);
                J20 Es = t[IA] * (iota * El[0] * g0) + t[IA + 1] * (iota * El[1] * g1);
                J20 E2s = t[IA] * (iota * iota * El2[0] * g0 * g0) +
                          t[IA + 1] * (iota * iota * El2[1] * g1 * g1);
                J20 E = Es + Eo;
                J20 V = (E2s - Es * Es) + Vo;
                J20 ll = pixel_ll((double)im.pixels[m], E, V);
                F.add(ll.v);
                for (int a = 0; a < n; ++a) gl[a].add(ll.g[a]);
                if constexpr (H)
                    for (int a = 0; a < n; ++a)
                        for (int b = 0; b < n; ++b) hl[a * n + b].add(ll.h[a][b]);
            }
        for (int a = 0; a < n; ++a) G[idx[a]].add(gl[a].sum());
        if constexpr (H)
            for (int a = 0; a < n; ++a)
                for (int b = 0; b < n; ++b) Hs[idx[a] * NP + idx[b]].add(hl[a * n + b].sum());
    }
    // KL over all 44 parameters
    using J44 = Jet<NP, H>;
    std::vector<J44> t44(NP);
    for (int i = 0; i < NP; ++i) t44[i] = jvar<NP, H>(th[i], i);
    J44 kl = source_kl<J44>(P, t44.data(), cinv, cld);
    F.add(-kl.v);
    if (f_out) *f_out = F.sum();
    if (g_out)
        for (int i = 0; i < NP; ++i) {
            G[i].add(-kl.g[i]);
            g_out[i] = G[i].sum();
        }
    if constexpr (H) {
        if (h_out)
            for (int i = 0; i < NP; ++i)
                for (int j = 0; j < NP; ++j) {
                    Hs[i * NP + j].add(-kl.h[i][j]);
                    h_out[i * NP + j] = Hs[i * NP + j].sum();
                }
    }
}

// local objective value only (for trust-region trial points)
double local_value(const OProblem& P, const std::vector<PatchVals>& pv, const double* cinv,
                   const double* cld, int s, const double* th) {
    Acc F;
    for (int p = P.patch_off[s]; p < P.patch_off[s + 1]; ++p) {
        const int32_t* pt = P.patches + 5 * p;
        const OImage& im = P.imgs[pt[0]];
        PatchVals own;
        source_patch_values(P, th, p, own);
        for (int yy = 0; yy < pt[4]; ++yy)
            for (int xx = 0; xx < pt[3]; ++xx) {
                int gx = pt[1] + xx, gy = pt[2] + yy;
                size_t m = (size_t)gy * im.width + gx;
                double Eo, Vo;
                others_at(P, pv, s, pt[0], gx, gy, Eo, Vo);
                size_t q = (size_t)yy * pt[3] + xx;
                double E = own.e[q] + Eo;
                double V = (own.e2[q] - own.e[q] * own.e[q]) + Vo;
                F.add(pixel_ll((double)im.pixels[m], E, V));
            }
    }
    F.add(-source_kl<double>(P, th, cinv, cld));
    return F.sum();
}

// ------------------------------------------------------------------------------
// Unconstrained coordinates t (41) -> constrained theta (44) for the trust region:
//   u, angle, r1, c1: identity; scale, r2, c2: exp;
//   e_dev, e_axis: 0.01 + 0.98 sigmoid;  a_star = 0.005 + 0.99 sigmoid, a_gal = 1 - a_star;
//   k_i: softmax with the last component's logit fixed at 0 (7 free per type), plus
//   K_LO = 1e-120: a weight whose softmax underflows keeps 1 / k and 1 / k^2 (the KL's
//   derivatives in k) finite in FP64; for every weight above ~1e-104 the sum is the
//   softmax itself, bit for bit.

constexpr int NT = 41;
constexpr double BOX_LO = BOX_LO_, BOX_HI = BOX_HI_, A_LO = A_LO_, A_HI = A_HI_, K_LO = 1e-120;

inline double sigm(double x) { return 1.0 / (1.0 + std::exp(-x)); }
inline double logit(double p) { return std::log(p / (1.0 - p)); }

void to_free(const double* th, double* t) {
    int n = 0;
    t[n++] = th[0];
    t[n++] = th[1];
    t[n++] = logit((th[IEDEV] - BOX_LO) / (BOX_HI - BOX_LO));
    t[n++] = logit((th[IAXIS] - BOX_LO) / (BOX_HI - BOX_LO));
    t[n++] = th[IANGLE];
    t[n++] = std::log(th[ISCALE]);
    for (int i = 0; i < 2; ++i) t[n++] = th[IR1 + i];
    for (int i = 0; i < 2; ++i) t[n++] = std::log(th[IR2 + i]);
    for (int j = 0; j < 8; ++j) t[n++] = th[IC1 + j];
    for (int j = 0; j < 8; ++j) t[n++] = std::log(th[IC2 + j]);
    t[n++] = logit((th[IA] - A_LO) / (A_HI - A_LO));
    for (int i = 0; i < 2; ++i)
        for (int d = 0; d < 7; ++d)
            t[n++] = std::log(th[IK + 8 * i + d] / th[IK + 8 * i + 7]);
}

// theta(t) as jets in the 41 free variables
template <bool H>
void from_free(const double* t, Jet<NT, H>* th) {
    using J = Jet<NT, H>;
    J v[NT];
    for (int i = 0; i < NT; ++i) v[i] = jvar<NT, H>(t[i], i);
    int n = 0;
    auto sg = [](const J& x) { return 1.0 / (1.0 + jexp(-x)); };
    th[0] = v[n++];
    th[1] = v[n++];
    th[IEDEV] = BOX_LO + (BOX_HI - BOX_LO) * sg(v[n++]);
    th[IAXIS] = BOX_LO + (BOX_HI - BOX_LO) * sg(v[n++]);
    th[IANGLE] = v[n++];
    th[ISCALE] = jexp(v[n++]);
    for (int i = 0; i < 2; ++i) th[IR1 + i] = v[n++];
    for (int i = 0; i < 2; ++i) th[IR2 + i] = jexp(v[n++]);
    for (int j = 0; j < 8; ++j) th[IC1 + j] = v[n++];
    for (int j = 0; j < 8; ++j) th[IC2 + j] = jexp(v[n++]);
    th[IA] = A_LO + (A_HI - A_LO) * sg(v[n++]);
    th[IA + 1] = 1.0 - th[IA];
    for (int i = 0; i < 2; ++i) {
        J e[8];
        J den = jconst<NT, H>(1.0);
        for (int d = 0; d < 7; ++d) {
            e[d] = jexp(v[n++]);
            den = den + e[d];
        }
        e[7] = jconst<NT, H>(1.0);
        for (int d = 0; d < 8; ++d) th[IK + 8 * i + d] = jconst<NT, H>(K_LO) + e[d] / den;
    }
}

// f(theta(t)): compose the 44-variable derivatives with the map's jets (chain rule
// for second-order Taylor polynomials)
void compose(const double* g44, const double* h44, const Jet<NT, true>* th, double* gt,
             double* ht) {
    for (int a = 0; a < NT; ++a) {
        double s = 0;
        for (int j = 0; j < NP; ++j) s += g44[j] * th[j].g[a];
        gt[a] = s;
    }
    for (int a = 0; a < NT; ++a)
        for (int b = 0; b < NT; ++b) {
            double s = 0;
            for (int j = 0; j < NP; ++j) {
                s += g44[j] * th[j].h[a][b];
                for (int k = 0; k < NP; ++k) s += h44[j * NP + k] * th[j].g[a] * th[k].g[b];
            }
            ht[a * NT + b] = s;
        }
}

// ------------------------------------------------------------------------------
// Trust-region subproblem  min  m(p) = c.p + 1/2 p.B p,  |p| <= Delta  (Nocedal & Wright
// Ch. 4: exact solution characterised by (B + lambda I) p = -c, lambda >= 0,
// lambda (Delta - |p|) = 0, B + lambda I positive semidefinite).  Solved through a
// cyclic Jacobi eigendecomposition of B.

void jacobi_eigen(int n, std::vector<double> A, std::vector<double>& w, std::vector<double>& Q) {
    Q.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
    double fro = 0;
    for (double x : A) fro += x * x;
    fro = std::sqrt(fro);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += 2 * A[(size_t)i * n + j] * A[(size_t)i * n + j];
        if (std::sqrt(off) <= 1e-15 * fro || fro == 0) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                double tau = (aqq - app) / (2 * apq);
                double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1 + tau * tau));
                double c = 1 / std::sqrt(1 + t * t), s = t * c;
                for (int k = 0; k < n; ++k) {
                    double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double qkp = Q[(size_t)k * n + p], qkq = Q[(size_t)k * n + q];
                    Q[(size_t)k * n + p] = c * qkp - s * qkq;
                    Q[(size_t)k * n + q] = s * qkp + c * qkq;
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

// returns |p|; hard case handled by adding the multiple of the lowest eigenvector
double tr_solve(int n, const double* c, const double* B, double Delta, double* p) {
    std::vector<double> A(B, B + (size_t)n * n), w, Q;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j) {
            double m = 0.5 * (A[(size_t)i * n + j] + A[(size_t)j * n + i]);
            A[(size_t)i * n + j] = A[(size_t)j * n + i] = m;
        }
    jacobi_eigen(n, A, w, Q);
    std::vector<double> ch(n);
    double cn = 0;
    for (int i = 0; i < n; ++i) {
        double s = 0;
        for (int k = 0; k < n; ++k) s += Q[(size_t)k * n + i] * c[k];
        ch[i] = s;
        cn += s * s;
    }
    cn = std::sqrt(cn);
    int imin = 0;
    for (int i = 1; i < n; ++i)
        if (w[i] < w[imin]) imin = i;
    double lmin = w[imin];
    auto pnorm2 = [&](double lam) {
        double s = 0;
        for (int i = 0; i < n; ++i) {
            double d = w[i] + lam;
            s += ch[i] * ch[i] / (d * d);
        }
        return s;
    };
    auto build = [&](double lam, int skip, double tau) {
        for (int k = 0; k < n; ++k) p[k] = 0;
        for (int i = 0; i < n; ++i) {
            if (i == skip) continue;
            double coef = -ch[i] / (w[i] + lam);
            for (int k = 0; k < n; ++k) p[k] += coef * Q[(size_t)k * n + i];
        }
        if (skip >= 0)
            for (int k = 0; k < n; ++k) p[k] += tau * Q[(size_t)k * n + skip];
    };
    // interior Newton step
    if (lmin > 0 && pnorm2(0.0) <= Delta * Delta) {
        build(0.0, -1, 0);
        return std::sqrt(pnorm2(0.0));
    }
    double lo = std::max(0.0, -lmin);
    // hard case: c has (numerically) no component along the lowest eigenvector
    if (std::fabs(ch[imin]) <= 1e-12 * (cn + 1e-300)) {
        double s = 0;
        for (int i = 0; i < n; ++i) {
            if (i == imin) continue;
            double d = w[i] + lo;
            s += ch[i] * ch[i] / (d * d);
        }
        if (s <= Delta * Delta) {
            double tau = std::sqrt(Delta * Delta - s);
            build(lo, imin, tau);
            return Delta;
        }
    }
    // bracket lambda in (lo, hi) with |p(lo+)| > Delta >= |p(hi)|
    double hi = lo + cn / Delta + 1.0;
    while (pnorm2(hi) > Delta * Delta) hi *= 2;
    double lam = hi;
    for (int it = 0; it < 200; ++it) {
        // Newton on 1/|p(lambda)| - 1/Delta (More & Sorensen), safeguarded by bisection
        double s2 = pnorm2(lam), s = std::sqrt(s2);
        double d3 = 0;
        for (int i = 0; i < n; ++i) {
            double d = w[i] + lam;
            d3 += ch[i] * ch[i] / (d * d * d);
        }
        if (s > Delta) lo = lam;
        else hi = lam;
        if (std::fabs(s - Delta) <= 1e-13 * Delta) break;
        // phi(l) = 1/s - 1/Delta;  phi'(l) = d3 / s^3
        double step = (1.0 / s - 1.0 / Delta) / (d3 / (s2 * s));
        double nl = lam - step;
        if (!(nl > lo && nl < hi)) nl = 0.5 * (lo + hi);
        if (hi - lo <= 1e-15 * std::max(1.0, hi)) {
            lam = hi;
            break;
        }
        lam = nl;
    }
    build(lam, -1, 0);
    return std::sqrt(pnorm2(lam));
}

// ------------------------------------------------------------------------------
// Per-source trust-region Newton (maximising ELBO_s with neighbours fixed)

struct FitOpts {
    int32_t max_iter;
    double grad_tol;       // stop when max |d ELBO_s / d t| <= grad_tol
    double pred_tol_rel;   // stop when the model's predicted gain <= pred_tol_rel (1 + |f|)
    double delta0, delta_max, eta;
    double f_noise_rel;    // gains below f_noise_rel (1 + |f|) skip the ratio test
};

enum { ST_CONVERGED = 0, ST_MAXITER = 1, ST_NONFINITE = 2 };

int fit_one(const OProblem& P, const std::vector<PatchVals>& pv, const double* cinv,
            const double* cld, int s, double* th, const FitOpts& o, int* iters) {
    double t[NT];
    to_free(th, t);
    double Delta = o.delta0;
    double thc[NP];
    std::memcpy(thc, th, sizeof(thc));
    std::vector<double> g44(NP), h44(NP * NP), gt(NT), ht(NT * NT), B(NT * NT), c(NT), p(NT);
    int status = ST_MAXITER;
    int it = 0;
    for (; it < o.max_iter; ++it) {
        double f;
        local_derivs<true>(P, pv, cinv, cld, s, thc, &f, g44.data(), h44.data());
        std::vector<Jet<NT, true>> tj(NP);
        from_free<true>(t, tj.data());
        compose(g44.data(), h44.data(), tj.data(), gt.data(), ht.data());
        double gmax = 0;
        bool finite = std::isfinite(f);
        for (int a = 0; a < NT; ++a) {
            gmax = std::max(gmax, std::fabs(gt[a]));
            finite = finite && std::isfinite(gt[a]);
        }
        if (!finite) {
            status = ST_NONFINITE;
            break;
        }
        if (gmax <= o.grad_tol) {
            status = ST_CONVERGED;
            break;
        }
        // maximise f  <=>  minimise -f:  c = -g, B = -H
        for (int a = 0; a < NT; ++a) c[a] = -gt[a];
        for (int a = 0; a < NT * NT; ++a) B[a] = -ht[a];
        double pn = tr_solve(NT, c.data(), B.data(), Delta, p.data());
        double pred = 0;   // predicted gain g.p + 1/2 p.H p
        for (int a = 0; a < NT; ++a) {
            double hp = 0;
            for (int b = 0; b < NT; ++b) hp += ht[a * NT + b] * p[b];
            pred += gt[a] * p[a] + 0.5 * p[a] * hp;
        }
        double scale = 1.0 + std::fabs(f);
        if (pred <= o.pred_tol_rel * scale) {
            status = ST_CONVERGED;
            break;
        }
        double tn[NT];
        for (int a = 0; a < NT; ++a) tn[a] = t[a] + p[a];
        std::vector<Jet<NT, false>> tnj(NP);
        from_free<false>(tn, tnj.data());
        double thn[NP];
        for (int j = 0; j < NP; ++j) thn[j] = tnj[j].v;
        double fn = local_value(P, pv, cinv, cld, s, thn);
        double rho = (pred <= o.f_noise_rel * scale) ? 1.0 : (fn - f) / pred;
        if (!std::isfinite(fn)) rho = -1.0;
        if (rho < 0.25) Delta = 0.25 * Delta;
        else if (rho > 0.75 && pn >= (1.0 - 1e-9) * Delta) Delta = std::min(2.0 * Delta, o.delta_max);
        if (rho > o.eta) {
            std::memcpy(t, tn, sizeof(t));
            std::memcpy(thc, thn, sizeof(thc));
        }
    }
    std::memcpy(th, thc, sizeof(thc));
    if (iters) *iters = it;
    return status;
}

}  // namespace

// ------------------------------------------------------------------------------
// C entry points used by the Python test harness

extern "C" {

int oracle_abi_version() { return 1; }

int oracle_num_threads() {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

// Pixel moments of one source on its own: E_s and E[F_s^2] over a patch.
int oracle_patch_values(const OProblem* P, const double* theta, int p, double* e, double* e2) {
    int s = 0;
    while (!(P->patch_off[s] <= p && p < P->patch_off[s + 1])) ++s;
    PatchVals v;
    source_patch_values(*P, theta + (size_t)NP * s, p, v);
    std::memcpy(e, v.e.data(), v.e.size() * sizeof(double));
    std::memcpy(e2, v.e2.data(), v.e2.size() * sizeof(double));
    return 0;
}

// Star and galaxy profiles of a source at arbitrary pixel centres of image n.
int oracle_profiles(const OProblem* P, const double* th, int n, int npts, const double* px,
                    const double* py, double* gstar, double* ggal) {
    const OImage& im = P->imgs[n];
    Shape<double> sh = make_shape<double>(im.wcs, th[IU], th[IU + 1], th[IEDEV], th[IAXIS],
                                          th[IANGLE], th[ISCALE]);
    for (int i = 0; i < npts; ++i) profiles<double>(*P, im, sh, px[i], py[i], gstar[i], ggal[i]);
    return 0;
}

// Brightness moments E[l], E[l^2] for type i in band b.
int oracle_brightness(const double* th, int band, int i, double* El, double* El2) {
    brightness<double>(th, band, i, *El, *El2);
    return 0;
}

int oracle_kl(const OProblem* P, const double* theta, double* kl) {
    std::vector<double> inv, ld;
    if (!prior_inverses(*P, inv, ld)) return -2;
    for (int s = 0; s < P->n_src; ++s)
        kl[s] = source_kl<double>(*P, theta + (size_t)NP * s, inv.data(), ld.data());
    return 0;
}

// ELBO total over the union of patches and the local ELBO_s of every source;
// optionally the E and V maps (concatenated images, row-major).
int oracle_elbo(const OProblem* P, const double* theta, double* total, double* local,
                double* emap, double* vmap) {
    for (int s = 0; s < P->n_src; ++s)
        if (!theta_valid(theta + (size_t)NP * s)) return -1;
    std::vector<double> inv, ld;
    if (!prior_inverses(*P, inv, ld)) return -2;
    std::vector<PatchVals> pv;
    build_patch_values(*P, theta, pv);
    Maps M;
    build_maps(*P, pv, M);
    Acc tot;
    size_t off = 0;
    std::vector<std::vector<double>> llmap(P->n_img);
    for (int n = 0; n < P->n_img; ++n) {
        const OImage& im = P->imgs[n];
        size_t npx = (size_t)im.height * im.width;
        llmap[n].assign(npx, 0.0);
        for (size_t m = 0; m < npx; ++m) {
            double E = M.E[n][m].sum() + sky_at(im, m);
            double V = M.V[n][m].sum();
            if (emap) emap[off + m] = E;
            if (vmap) vmap[off + m] = V;
            if (M.cover[n][m] == 0) continue;
            double ll = pixel_ll((double)im.pixels[m], E, V);
            llmap[n][m] = ll;
            tot.add(ll);
        }
        off += npx;
    }
    for (int s = 0; s < P->n_src; ++s) {
        double kl = source_kl<double>(*P, theta + (size_t)NP * s, inv.data(), ld.data());
        tot.add(-kl);
        if (local) {
            Acc a;
            for (int p = P->patch_off[s]; p < P->patch_off[s + 1]; ++p) {
                const int32_t* pt = P->patches + 5 * p;
                const OImage& im = P->imgs[pt[0]];
                for (int yy = 0; yy < pt[4]; ++yy)
                    for (int xx = 0; xx < pt[3]; ++xx)
                        a.add(llmap[pt[0]][(size_t)(pt[2] + yy) * im.width + pt[1] + xx]);
            }
            a.add(-kl);
            local[s] = a.sum();
        }
    }
    *total = tot.sum();
    return 0;
}

// Gradient (and optionally Hessian) of ELBO_s wrt source s's 44 constrained
// parameters for each s in `which` (null: all).  grad [n][44], hess [n][44][44].
int oracle_derivs(const OProblem* P, const double* theta, const int32_t* which, int n_which,
                  int want_hess, double* local, double* grad, double* hess) {
    for (int s = 0; s < P->n_src; ++s)
        if (!theta_valid(theta + (size_t)NP * s)) return -1;
    std::vector<double> inv, ld;
    if (!prior_inverses(*P, inv, ld)) return -2;
    std::vector<PatchVals> pv;
    build_patch_values(*P, theta, pv);
    int n = which ? n_which : P->n_src;
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < n; ++k) {
        int s = which ? which[k] : k;
        double f;
        if (want_hess)
            local_derivs<true>(*P, pv, inv.data(), ld.data(), s, theta + (size_t)NP * s, &f,
                               grad ? grad + (size_t)NP * k : nullptr,
                               hess ? hess + (size_t)NP * NP * k : nullptr);
        else
            local_derivs<false>(*P, pv, inv.data(), ld.data(), s, theta + (size_t)NP * s, &f,
                                grad ? grad + (size_t)NP * k : nullptr, nullptr);
        if (local) local[k] = f;
    }
    return 0;
}

// Unconstrained <-> constrained maps and the chain rule, exposed for tests.
int oracle_to_free(const double* th, double* t) {
    to_free(th, t);
    return 0;
}
int oracle_from_free(const double* t, double* th, double* jac /*[44][41] or null*/) {
    std::vector<Jet<NT, false>> tj(NP);
    from_free<false>(t, tj.data());
    for (int j = 0; j < NP; ++j) {
        th[j] = tj[j].v;
        if (jac)
            for (int a = 0; a < NT; ++a) jac[j * NT + a] = tj[j].g[a];
    }
    return 0;
}
int oracle_free_derivs(const double* t, const double* g44, const double* h44, double* gt,
                       double* ht) {
    std::vector<Jet<NT, true>> tj(NP);
    from_free<true>(t, tj.data());
    compose(g44, h44, tj.data(), gt, ht);
    return 0;
}

int oracle_tr_solve(int n, const double* c, const double* B, double Delta, double* p,
                    double* pnorm) {
    *pnorm = tr_solve(n, c, B, Delta, p);
    return 0;
}

// Greedy colouring of the neighbour graph in ascending source id.
int oracle_colouring(const OProblem* P, int32_t* colour) {
    int maxc = 0;
    for (int s = 0; s < P->n_src; ++s) {
        std::vector<char> used(P->n_src + 1, 0);
        for (int e = P->nbr_off[s]; e < P->nbr_off[s + 1]; ++e) {
            int o = P->nbrs[e];
            if (o < s) used[colour[o]] = 1;
        }
        int c = 0;
        while (used[c]) ++c;
        colour[s] = c;
        maxc = std::max(maxc, c + 1);
    }
    return maxc;
}

// Cyclades schedule (Section IV-D; Pan et al., "Cyclades"): positions [k B, (k+1) B)
// of the order form sample k; the neighbour graph restricted to the sample splits into
// connected components (breadth-first search from each unlabelled member in order, so
// a component is labelled with the order position of its first member); the members
// of one component are updated one after another in order and different components
// side by side, i.e. the r-th member of every component forms the sample's r-th batch.
// Samples take consecutive batch numbers.  Returns the number of batches.
int oracle_cyclades_batches(const OProblem* P, const int32_t* order, int m, int B,
                            int32_t* comp_of, int32_t* batch_of) {
    int base = 0;
    for (int k0 = 0; k0 < m; k0 += B) {
        const int k1 = std::min(m, k0 + B);
        std::vector<int> at(P->n_src, -1);   // order position of a sampled source
        for (int i = k0; i < k1; ++i) at[order[i]] = i;
        for (int i = k0; i < k1; ++i) comp_of[i] = -1;
        for (int i = k0; i < k1; ++i) {
            if (comp_of[i] >= 0) continue;
            std::vector<int> queue{i};
            comp_of[i] = i;
            for (size_t q = 0; q < queue.size(); ++q) {
                const int s = order[queue[q]];
                for (int e = P->nbr_off[s]; e < P->nbr_off[s + 1]; ++e) {
                    const int j = at[P->nbrs[e]];
                    if (j >= 0 && comp_of[j] < 0) {
                        comp_of[j] = i;
                        queue.push_back(j);
                    }
                }
            }
        }
        int rounds = 0;
        for (int i = k0; i < k1; ++i) {
            int r = 0;   // earlier members of the same component
            for (int j = k0; j < i; ++j) r += comp_of[j] == comp_of[i];
            batch_of[i] = base + r;
            rounds = std::max(rounds, r + 1);
        }
        base += rounds;
    }
    return base;
}

// Block-coordinate fit: colour classes in order; every source of a class is fitted
// by trust-region Newton with all other sources fixed; E and V are refreshed after
// each class; sweeps repeat until the total ELBO changes by < sweep_tol relative.
// `which` (null: all) restricts the sources that move.  With schedule 1 the batches of
// sweep g are the Cyclades batches of order row g mod max_sweeps ([max_sweeps][n_moving],
// each row a permutation of the moving sources) with samples of sample_size.
int oracle_fit(const OProblem* P, double* theta, const int32_t* which, int n_which,
               int max_iter, double grad_tol, double pred_tol_rel, double delta0,
               double delta_max, double eta, double f_noise_rel, int max_sweeps,
               double sweep_tol, int32_t* iters_out, int32_t* status_out, double* elbo_out,
               int32_t* sweeps_out, int schedule, int sample_size, const int32_t* order) {
    for (int s = 0; s < P->n_src; ++s)
        if (!theta_valid(theta + (size_t)NP * s) || !theta_in_box(theta + (size_t)NP * s))
            return -1;
    std::vector<double> inv, ld;
    if (!prior_inverses(*P, inv, ld)) return -2;
    FitOpts o{max_iter, grad_tol, pred_tol_rel, delta0, delta_max, eta, f_noise_rel};
    std::vector<int32_t> colour(P->n_src, 0);
    int nc = oracle_colouring(P, colour.data());
    std::vector<char> moves(P->n_src, which ? 0 : 1);
    if (which)
        for (int k = 0; k < n_which; ++k) moves[which[k]] = 1;
    for (int s = 0; s < P->n_src; ++s) {
        iters_out[s] = 0;
        status_out[s] = ST_CONVERGED;
    }
    double prev;
    oracle_elbo(P, theta, &prev, nullptr, nullptr, nullptr);
    int n_moving = 0;
    for (int s = 0; s < P->n_src; ++s) n_moving += moves[s];
    int sw = 0;
    for (; sw < max_sweeps; ++sw) {
        // this sweep's batches: colour classes, or the Cyclades batches of its order row
        std::vector<std::vector<int>> batches;
        if (schedule == 1) {
            const int32_t* row = order + (size_t)sw * n_moving;
            std::vector<int32_t> comp(n_moving), bat(n_moving);
            const int nb = oracle_cyclades_batches(P, row, n_moving, sample_size, comp.data(), bat.data());
            batches.resize(nb);
            for (int i = 0; i < n_moving; ++i) batches[bat[i]].push_back(row[i]);
        } else {
            batches.resize(nc);
            for (int s = 0; s < P->n_src; ++s)
                if (moves[s]) batches[colour[s]].push_back(s);
        }
        for (size_t c = 0; c < batches.size(); ++c) {
            std::vector<PatchVals> pv;
            build_patch_values(*P, theta, pv);
            const std::vector<int>& members = batches[c];
#pragma omp parallel for schedule(dynamic, 1)
            for (int k = 0; k < (int)members.size(); ++k) {
                int s = members[k];
                int it = 0;
                status_out[s] = fit_one(*P, pv, inv.data(), ld.data(), s,
                                        theta + (size_t)NP * s, o, &it);
                iters_out[s] += it;
            }
        }
        double cur;
        oracle_elbo(P, theta, &cur, nullptr, nullptr, nullptr);
        double rel = std::fabs(cur - prev) / std::max(1.0, std::fabs(cur));
        prev = cur;
        if (rel < sweep_tol) {
            ++sw;
            break;
        }
    }
    if (elbo_out) *elbo_out = prev;
    if (sweeps_out) *sweeps_out = sw;
    return 0;
}

}  // extern "C"
