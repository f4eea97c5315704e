// Host check of the Hessian epilogue's galaxy-shape derivatives (k_finalize_hess):
// shape_w_derivs (the world-frame ellipse's first and second derivatives over
// s = (e_axis, e_angle, e_scale), once per source) and a_transform (each patch's map
// A W A'), run on the CPU, against central differences of the pixel-frame ellipse
// G(s) = A W(s) A', W = sigma^2 R(phi) diag(1, rho^2) R(phi)' (Section III's galaxy
// shape), written out here as a rotation, on random shapes and maps.
//
// Output: "first worst_rel" and "second worst_rel"; exit status 1 if a case is off by
// more than 1e-5 of its scale.
#include "hess_kernels.cu"

#include <cstdio>
#include <random>

using namespace cel;

static void ellipse(const double* A, double rho, double phi, double sg, double G[3]) {
    const double c = cos(phi), s = sin(phi);
    // W = sigma^2 R diag(1, rho^2) R', R = [[c, -s], [s, c]]
    const double w[2][2] = {{sg * sg * (c * c + rho * rho * s * s), sg * sg * (1 - rho * rho) * c * s},
                            {sg * sg * (1 - rho * rho) * c * s, sg * sg * (s * s + rho * rho * c * c)}};
    double M[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double v = 0;
            for (int k = 0; k < 2; ++k)
                for (int l = 0; l < 2; ++l) v += A[2 * i + k] * w[k][l] * A[2 * j + l];
            M[i][j] = v;
        }
    G[0] = M[0][0];
    G[1] = M[0][1];
    G[2] = M[1][1];
}

int main() {
    std::mt19937 rng(11);
    std::uniform_real_distribution<double> U01(0, 1);
    double worst1 = 0, worst2 = 0;
    for (int trial = 0; trial < 2000; ++trial) {
        double th[NP] = {};
        const double s0[3] = {0.05 + 0.9 * U01(rng), (U01(rng) - 0.5) * 6.283185307179586, 0.2 + 5 * U01(rng)};
        th[P_AXIS] = s0[0];
        th[P_ANGLE] = s0[1];
        th[P_SCALE] = s0[2];
        double A[4];
        do {
            for (double& a : A) a = (U01(rng) - 0.5) * 2;
        } while (fabs(A[0] * A[3] - A[1] * A[2]) < 0.2);
        double dW[3][3], d2W[3][3][3], dG[3][3], d2G[3][3][3];
        shape_w_derivs(th, dW, d2W);
        for (int q = 0; q < 3; ++q)
            for (int c = 0; c < 3; ++c) {
                dG[q][c] = a_transform(A, dW[q], c);
                for (int r = 0; r < 3; ++r) d2G[q][r][c] = a_transform(A, d2W[q][r], c);
            }
        auto G_at = [&](const double* sv, double G[3]) { ellipse(A, sv[0], sv[1], sv[2], G); };
        double scale1 = 0, err1 = 0, scale2 = 0, err2 = 0;
        const double h1 = 1e-6, h2 = 1e-4;
        for (int q = 0; q < 3; ++q) {
            double sp[3] = {s0[0], s0[1], s0[2]}, sm[3] = {s0[0], s0[1], s0[2]}, Gp[3], Gm[3];
            sp[q] += h1;
            sm[q] -= h1;
            G_at(sp, Gp);
            G_at(sm, Gm);
            for (int c = 0; c < 3; ++c) {
                const double fd = (Gp[c] - Gm[c]) / (2 * h1);
                scale1 = fmax(scale1, fabs(fd));
                err1 = fmax(err1, fabs(dG[q][c] - fd));
            }
            for (int r = 0; r < 3; ++r) {
                double G4[4][3];
                for (int u = 0; u < 4; ++u) {
                    double sv[3] = {s0[0], s0[1], s0[2]};
                    sv[q] += (u & 1) ? -h2 : h2;
                    sv[r] += (u & 2) ? -h2 : h2;
                    G_at(sv, G4[u]);
                }
                for (int c = 0; c < 3; ++c) {
                    const double fd = (G4[0][c] - G4[1][c] - G4[2][c] + G4[3][c]) / (4 * h2 * h2);
                    scale2 = fmax(scale2, fabs(fd));
                    err2 = fmax(err2, fabs(d2G[q][r][c] - fd));
                }
            }
        }
        worst1 = fmax(worst1, err1 / scale1);
        worst2 = fmax(worst2, err2 / scale2);
        if (err1 / scale1 > 1e-5 || err2 / scale2 > 1e-5) {
            printf("case %d: first %.3e second %.3e of scale\n", trial, err1 / scale1, err2 / scale2);
            return 1;
        }
    }
    printf("first %.6e\nsecond %.6e\n", worst1, worst2);
    return 0;
}
