// Host check of the FP32 Hessian kernel's whitened-frame galaxy terms (k_hess<float>):
// whiten_frame, whiten_row, the per-component sums and whitened_add, run on the CPU,
// against the pixel-frame formulas of the Gaussian mixture's derivatives over the mean
// and the shape (Section IV-D needs these second derivatives) written out in FP64, on
// random PSF and galaxy covariances (including equal eigenvalues, G = 0 and a tiny G)
// and pixel offsets out to three standard deviations.  The same pixel-frame formulas in
// FP32 give the accuracy an FP32 evaluation can be held to.
//
// Output: one line per quantity "name worst_whitened worst_pixel_frame_fp32"; exit
// status 1 if any single case is off by more than 1e-3 of its scale.
#include "hess_kernels.cu"

#include <cstdio>
#include <random>

using namespace cel;

// value, mean/shape gradient, e_dev derivative, packed 5 x 5 Hessian and e_dev x
// gradient of sum_j w_j N(d; 0, Sigma + nu_j G) (dw_j for the e_dev terms): 27 numbers
template <class F>
static void pixel_frame(double dx_, double dy_, const double Sg[3], const double Gm[3], int np,
                        const double* nu, const double* w, const double* dw, double* out) {
    F g1 = 0, d1[5] = {0, 0, 0, 0, 0}, de = 0, h1[15] = {}, he[5] = {0, 0, 0, 0, 0};
    const F dx = (F)dx_, dy = (F)dy_;
    for (int j = 0; j < np; ++j) {
        const F cxx = (F)(Sg[0] + nu[j] * Gm[0]), cxy = (F)(Sg[1] + nu[j] * Gm[1]),
                cyy = (F)(Sg[2] + nu[j] * Gm[2]);
        const F det = cxx * cyy - cxy * cxy;
        const F pxx = cyy / det, pxy = -cxy / det, pyy = cxx / det;
        const F e = exp(-(F)0.5 * (pxx * dx * dx + 2 * pxy * dx * dy + pyy * dy * dy)) /
                    ((F)(2 * M_PI) * sqrt(det));
        const F n = (F)w[j] * e, ne = (F)dw[j] * e, v = (F)nu[j], v2 = v * v;
        // log-density derivatives: d/dmu = q = P d, d/dG[E] = nu (q'Eq - tr PE) / 2
        const F qx = pxx * dx + pxy * dy, qy = pxy * dx + pyy * dy;
        const F l[5] = {qx, qy, (F)0.5 * v * (qx * qx - pxx), v * (qx * qy - pxy),
                        (F)0.5 * v * (qy * qy - pyy)};
        // second log-derivatives: -P, -nu P E q, nu^2 (tr(PEPF)/2 - q'E P F q)
        const F Px = pxx * qy + pxy * qx, Py = pxy * qy + pyy * qx;
        const F L[15] = {-pxx, -pxy, -v * pxx * qx, -v * Px, -v * pxy * qy,
                         -pyy, -v * pxy * qx, -v * Py, -v * pyy * qy,
                         v2 * ((F)0.5 * pxx * pxx - pxx * qx * qx), v2 * (pxx * pxy - qx * Px),
                         v2 * ((F)0.5 * pxy * pxy - pxy * qx * qy),
                         v2 * (pxy * pxy + pxx * pyy - (qy * Px + qx * Py)), v2 * (pxy * pyy - qy * Py),
                         v2 * ((F)0.5 * pyy * pyy - pyy * qy * qy)};
        g1 += n;
        de += ne;
        int c = 0;
        for (int a = 0; a < 5; ++a) {
            d1[a] += n * l[a];
            he[a] += ne * l[a];
            for (int b = a; b < 5; ++b, ++c) h1[c] += n * (l[a] * l[b] + L[c]);
        }
    }
    out[0] = g1;
    for (int i = 0; i < 5; ++i) out[1 + i] = d1[i];
    out[6] = de;
    for (int i = 0; i < 15; ++i) out[7 + i] = h1[i];
    for (int i = 0; i < 5; ++i) out[22 + i] = he[i];
}

int main() {
    std::mt19937 rng(5);
    std::normal_distribution<double> N01;
    std::uniform_real_distribution<double> U01(0, 1);
    const char* name[5] = {"value", "gradient", "e_dev", "hessian", "e_dev_gradient"};
    const int lo[5] = {0, 1, 6, 7, 22}, hi[5] = {1, 6, 7, 22, 27};
    double worst[5] = {0, 0, 0, 0, 0}, worst32[5] = {0, 0, 0, 0, 0};
    for (int trial = 0; trial < 4000; ++trial) {
        const double a0 = N01(rng), a1 = N01(rng), a2 = N01(rng), a3 = N01(rng);
        double Sg[3] = {a0 * a0 + a1 * a1 + 0.5, a0 * a2 + a1 * a3, a2 * a2 + a3 * a3 + 0.5};
        const double sc = 0.1 + 5 * U01(rng);
        const double b0 = N01(rng) * sc, b1 = N01(rng) * sc, b2 = N01(rng) * sc, b3 = N01(rng) * sc;
        double Gm[3] = {b0 * b0 + b1 * b1, b0 * b2 + b1 * b3, b2 * b2 + b3 * b3};
        if (trial % 5 == 0) {   // round galaxy, round PSF: no preferred axes
            Gm[0] = Gm[2] = 2.0;
            Gm[1] = 0.0;
            Sg[0] = Sg[2] = 1.3;
            Sg[1] = 0.0;
        }
        if (trial % 5 == 1) Gm[0] = Gm[1] = Gm[2] = 0.0;   // a point source
        if (trial % 5 == 2)
            for (double& g : Gm) g *= 1e-6;
        const int np = 14;
        double nu[16], w[16], dw[16];
        for (int j = 0; j < np; ++j) {
            nu[j] = 0.02 + 4 * U01(rng);
            w[j] = 0.05 + U01(rng);
            dw[j] = (U01(rng) - 0.5) * 2;
        }
        // the kernel's table: the PSF component's precision, G, and per galaxy component
        // its log2 normaliser, weight, e_dev weight and variance scale
        float sT[TBL_STRIDE] = {};
        const double det = Sg[0] * Sg[2] - Sg[1] * Sg[1];
        sT[T_STAR + 4] = (float)(Sg[2] / det);
        sT[T_STAR + 5] = (float)(-Sg[1] / det);
        sT[T_STAR + 6] = (float)(Sg[0] / det);
        for (int c = 0; c < 3; ++c) sT[T_G + c] = (float)Gm[c];
        for (int j = 0; j < np; ++j) {
            float* G = sT + T_GAL + j * GAL_STRIDE;
            const double cxx = Sg[0] + nu[j] * Gm[0], cxy = Sg[1] + nu[j] * Gm[1], cyy = Sg[2] + nu[j] * Gm[2];
            G[3] = (float)(-log2(2 * M_PI) - 0.5 * log2(cxx * cyy - cxy * cxy));
            G[7] = (float)w[j];
            G[8] = (float)dw[j];
            G[9] = (float)nu[j];
        }
        float fr[WFR], rows[MAXPROF * WROW];
        whiten_frame(sT, 0, fr);
        for (int j = 0; j < np; ++j) whiten_row(sT + T_GAL + j * GAL_STRIDE, fr, rows + j * WROW);
        const double r = 3.0 * U01(rng) * sqrt(Sg[0] + Sg[2] + 4 * (Gm[0] + Gm[2]));
        const double ang = 6.283185307179586 * U01(rng);
        const float dx = (float)(r * cos(ang)), dy = (float)(r * sin(ang));
        // the kernel's per-pixel steps
        const float z1 = fr[0] * dx + fr[1] * dy, z2 = fr[2] * dx + fr[3] * dy;
        const float z1s = z1 * z1, z2s = z2 * z2;
        float sw[NWS] = {};
        for (int j = 0; j < np; ++j) {
            const float* cw = rows + j * WROW;
            const float e = exp2f(fmaf(cw[0], z1s, fmaf(cw[1], z2s, cw[2])));
            for (int m = 0; m < NWS; ++m) sw[m] = fmaf(e, cw[3 + m], sw[m]);
        }
        float g1 = 0, d1[5] = {0, 0, 0, 0, 0}, de = 0, h1[15] = {}, he[5] = {0, 0, 0, 0, 0};
        whitened_add(sw, z1, z2, fr, g1, d1, de, h1, he);
        double got[27];
        got[0] = g1;
        for (int i = 0; i < 5; ++i) got[1 + i] = d1[i];
        got[6] = de;
        for (int i = 0; i < 15; ++i) got[7 + i] = h1[i];
        for (int i = 0; i < 5; ++i) got[22 + i] = he[i];
        double ref[27], refa[27], f32[27], dwa[16];
        pixel_frame<double>(dx, dy, Sg, Gm, np, nu, w, dw, ref);
        pixel_frame<float>(dx, dy, Sg, Gm, np, nu, w, dw, f32);
        // the e_dev sums mix signs: their scale is the same sum with |dw|
        for (int j = 0; j < np; ++j) dwa[j] = fabs(dw[j]);
        pixel_frame<double>(dx, dy, Sg, Gm, np, nu, w, dwa, refa);
        for (int g = 0; g < 5; ++g) {
            double scale = 0, err = 0, err32 = 0;
            for (int i = lo[g]; i < hi[g]; ++i) {
                scale = fmax(scale, fabs(ref[i]));
                if (g == 2 || g == 4) scale = fmax(scale, fabs(refa[i]));
                err = fmax(err, fabs(got[i] - ref[i]));
                err32 = fmax(err32, fabs(f32[i] - ref[i]));
            }
            if (scale < 1e-30) continue;   // FP32 subnormal range
            worst[g] = fmax(worst[g], err / scale);
            worst32[g] = fmax(worst32[g], err32 / scale);
            if (err / scale > 1e-3) {
                printf("case %d: %s off by %.3e of its scale\n", trial, name[g], err / scale);
                return 1;
            }
        }
    }
    for (int g = 0; g < 5; ++g) printf("%s %.6e %.6e\n", name[g], worst[g], worst32[g]);
    return 0;
}
