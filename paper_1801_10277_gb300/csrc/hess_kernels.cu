// Per-source exact Hessians (Section IV-D: Newton steps need the exact 44 x 44
// Hessian of each source's block).
//
//   k_hess           per work item: value, gradient and Hessian of the pixel terms
//                    wrt the twelve intermediate variables y of the (source, patch);
//                    the mixture terms are recomputed here, nothing is stored.
//   k_finalize_hess  one CTA per source: sparse chain rule y -> theta over the
//                    source's patches, plus the KL Hessian; writes the full
//                    symmetric 44 x 44 matrix, the gradient and the local objective.
//
// With e = dE_s/dy, v = dVar_s/dy = dE2_s/dy - 2 E_s e and the second derivatives
// DE = d2E_s/dy2, DE2 = d2E2_s/dy2 (E2_s = sum_i a_i iota^2 E[l_i^2] g_i^2):
//   d2 ll/dy2 = (h_EE - 2 c_V) e e' + h_EV (e v' + v e') + (c_E - 2 c_V E_s) DE + c_V DE2
//   h_EE = -x (1/E^2 + 3 Var/E^4),  h_EV = x / E^3,  h_VV = 0.
// Per Gaussian component N (log-density derivatives, q = P d, C = Sigma_psf + nu G):
//   dlogN/dmu = q,  d2logN/dmu2 = -P,
//   dlogN/dC[E] = (q'Eq - tr PE)/2,   d2logN/dmu dC[F] = -P F q,
//   d2logN/dC[E]dC[F] = -q'E P F q + tr(P E P F)/2,   d2N = N (dlogN dlogN' + d2logN).
#include <math.h>

#include <type_traits>

#include "internal.cuh"
#include "source_math.cuh"

namespace cel {

namespace {

__device__ __forceinline__ float ex2h(float x) { return exp2f(x); }
__device__ __forceinline__ double ex2h(double x) { return exp2(x); }
__device__ __forceinline__ float lgh(float x) { return logf(x); }
__device__ __forceinline__ double lgh(double x) { return log(x); }

constexpr double LOG2E_H = 1.4426950408889634;   // log2(e)

// packed index of the symmetric 12 x 12 (a <= b not required)
__device__ __forceinline__ int P2(int a, int b) { return a <= b ? yh_index(a, b) : yh_index(b, a); }

}  // namespace

constexpr int HV = 1 + NY + NYH;   // values reduced per work item
constexpr int HVP = 96;            // HV padded to three per lane
static_assert(HV <= HVP && HVP == 3 * 32, "the reduce-scatter leaves three sums per lane");

// Sums v over the warp's 32 lanes and leaves lane l holding the sums of entries
// 3 l, 3 l + 1, 3 l + 2 in v[0..2].  Five halving steps: at the step on lane bit m the
// two lanes that differ in m hold the same index range; the one with m set keeps the
// upper half and adds its partner's upper half, the other keeps and adds the lower
// half.  93 shuffles instead of 5 per entry.
template <class R>
__device__ __forceinline__ void warp_reduce_scatter(R (&v)[HVP], int lane) {
#pragma unroll
    for (int m = 16, n = HVP; m > 0; m >>= 1, n >>= 1) {
        const bool up = (lane & m) != 0;
#pragma unroll
        for (int i = 0; i < n / 2; ++i) {
            const R send = up ? v[i] : v[i + n / 2];
            const R keep = up ? v[i + n / 2] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, m);
        }
    }
}

// ---- The galaxy components in the frame that whitens PSF component k (FP32 path).
// T_k maps a pixel offset d to z = T_k d with T_k Sigma_k T_k' = I and T_k G T_k' =
// diag(g1, g2), so component j's precision is T_k' diag(lam1, lam2) T_k with
// lam_a = 1 / (1 + nu_j g_a).  With r = lam z and E~ = T_k E T_k', every derivative of
// N_kj over (mu, G) is N_kj times T_k' (a polynomial in z) T_k:
//   d/dmu: r;   d/dG[E]: (nu/2)(r' E~ r - tr(lam E~));   d2/dmu2: r r' - lam;
//   d2/dmu dG[E]: r d/dG[E] - nu lam E~ r;
//   d2/dG[E] dG[F]: d/dG[E] d/dG[F] - nu^2 r' E~ lam F~ r + (nu^2/2) tr(lam E~ lam F~).
// A pixel therefore needs, per k, 35 sums over j of N_kj (or of its e_dev derivative)
// times a monomial in (nu, lam1, lam2); the z-polynomials and the maps back to the
// pixel frame are applied once per (pixel, k) instead of once per component.
// Sums (monomial lam1^(deg - i) lam2^i at offset i):
constexpr int WS_N = 0,    // N
              WS_L = 1,    // N lam            (deg 1)
              WS_LL = 3,   // N lam lam        (deg 2)
              WS_B = 6,    // N nu lam         (deg 1)
              WS_A = 8,    // N nu lam lam     (deg 2)
              WS_C = 11,   // N nu lam^3       (deg 3)
              WS_D2 = 15,  // N nu^2 lam^2
              WS_D3 = 18,  // N nu^2 lam^3
              WS_D4 = 22,  // N nu^2 lam^4
              WS_NE = 27,  // dN/de_dev
              WS_LE = 28,  // dN/de_dev lam
              WS_BE = 30,  // dN/de_dev nu lam
              WS_AE = 32,  // dN/de_dev nu lam lam
              NWS = 35;
constexpr int WROW = 40;   // floats per (k, j): exponent coefficients of z1^2, z2^2, constant; 35 weights; pad
constexpr int WFR = 16;    // floats per k: T (row-major), K (3 x 3), g1, g2, pad
// K[e][p] = (T E_e T')_p for the pixel-frame shape directions E_e = (xx, xy + yx, yy)
// and the whitened pairs p = (11, 12, 22)
constexpr int WF_K = 4, WF_G = 13;
static_assert(3 + NWS <= WROW && WROW % 4 == 0 && WFR % 4 == 0 && WF_G + 2 <= WFR,
              "whitened rows are read as float4 from a 16-byte aligned array");

__host__ __device__ __forceinline__ int wpa(int p) { return p == 2 ? 1 : 0; }
__host__ __device__ __forceinline__ int wpb(int p) { return p == 0 ? 0 : 1; }
__host__ __device__ __forceinline__ float wmult(int p) { return p == 1 ? 2.f : 1.f; }
__host__ __device__ __forceinline__ float wdl(int a, int b) { return a == b ? 1.f : 0.f; }

// T_k from the Cholesky factor of the component's precision and one Jacobi rotation, in
// FP32 (a few threads per work item, before its pixels: FP64 square roots and divisions
// there would hold every warp of the item at the barrier; host-callable for tests)
__host__ __device__ void whiten_frame(const float* sT, int k, float* fr) {
    const float* S = sT + T_STAR + k * STAR_STRIDE;
    const float pxx = S[4], pxy = S[5], pyy = S[6];
    const float gxx = sT[T_G], gxy = sT[T_G + 1], gyy = sT[T_G + 2];
    // T0 = [[r11, r21], [0, r22]] with T0 Sigma T0' = I (r the lower factor of Sigma^-1)
    const float r11 = sqrtf(pxx), r21 = pxy / r11, r22 = sqrtf(fmaxf(pyy - r21 * r21, 0.f));
    const float u0 = r11 * gxx + r21 * gxy, u1 = r11 * gxy + r21 * gyy;
    const float b11 = u0 * r11 + u1 * r21, b12 = u1 * r22, b22 = r22 * gyy * r22;
    // Q = [[c, s], [-s, c]] with Q B Q' diagonal, B = T0 G T0' (the smaller rotation; an
    // infinite tau gives t = 0)
    float c = 1.f, s = 0.f;
    if (b12 != 0.f) {
        const float tau = (b22 - b11) / (2.f * b12);
        const float t = tau == 0.f ? 1.f : -copysignf(1.f, tau) / (fabsf(tau) + sqrtf(1.f + tau * tau));
        c = 1.f / sqrtf(1.f + t * t);
        s = t * c;
    }
    const float T[2][2] = {{c * r11, c * r21 + s * r22}, {-s * r11, -s * r21 + c * r22}};
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        fr[2 * a] = T[a][0];
        fr[2 * a + 1] = T[a][1];
        const float v0 = T[a][0] * gxx + T[a][1] * gxy, v1 = T[a][0] * gxy + T[a][1] * gyy;
        fr[WF_G + a] = fmaxf(v0 * T[a][0] + v1 * T[a][1], 0.f);
    }
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const int a = wpa(p), b = wpb(p);
        fr[WF_K + 0 * 3 + p] = T[a][0] * T[b][0];
        fr[WF_K + 1 * 3 + p] = T[a][0] * T[b][1] + T[a][1] * T[b][0];
        fr[WF_K + 2 * 3 + p] = T[a][1] * T[b][1];
    }
    fr[15] = 0.f;
}

// the row of galaxy component (k, j): exponent in z and the 35 monomial weights
__host__ __device__ void whiten_row(const float* G, const float* fr, float* row) {
    const float nu = G[9], w = G[7], dw = G[8];
    const float l1 = 1.f / (1.f + nu * fr[WF_G]), l2 = 1.f / (1.f + nu * fr[WF_G + 1]);
    float p1[5], p2[5];
    p1[0] = p2[0] = 1.f;
#pragma unroll
    for (int i = 1; i < 5; ++i) {
        p1[i] = p1[i - 1] * l1;
        p2[i] = p2[i - 1] * l2;
    }
    auto mono = [&](int deg, int i) { return p1[deg - i] * p2[i]; };
    const float wn = w * nu, wn2 = wn * nu, dwn = dw * nu;
    row[0] = -0.5f * (float)LOG2E_H * l1;
    row[1] = -0.5f * (float)LOG2E_H * l2;
    row[2] = G[3];
    float* c = row + 3;
    c[WS_N] = w;
    c[WS_NE] = dw;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        c[WS_L + i] = w * mono(1, i);
        c[WS_B + i] = wn * mono(1, i);
        c[WS_LE + i] = dw * mono(1, i);
        c[WS_BE + i] = dwn * mono(1, i);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        c[WS_LL + i] = w * mono(2, i);
        c[WS_A + i] = wn * mono(2, i);
        c[WS_D2 + i] = wn2 * mono(2, i);
        c[WS_AE + i] = dwn * mono(2, i);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        c[WS_C + i] = wn * mono(3, i);
        c[WS_D3 + i] = wn2 * mono(3, i);
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) c[WS_D4 + i] = wn2 * mono(4, i);
    row[3 + NWS] = 0.f;
    row[4 + NWS] = 0.f;
}

// adds PSF component k's galaxy terms at one pixel, from its 35 sums, to the pixel-frame
// value, gradient (mx, my, Gxx, Gxy, Gyy), e_dev derivatives and packed 5 x 5 Hessian
__host__ __device__ __forceinline__ void whitened_add(const float (&s)[NWS], float z1, float z2,
                                             const float* fr, float& g1, float (&d1)[5],
                                             float& de, float (&h1)[15], float (&he)[5]) {
    const float z[2] = {z1, z2};
    const float Z2[3] = {z1 * z1, z1 * z2, z2 * z2};
    const float Z3[4] = {z1 * Z2[0], z1 * Z2[1], z1 * Z2[2], z2 * Z2[2]};
    const float Z4[5] = {Z2[0] * Z2[0], Z2[0] * Z2[1], Z2[0] * Z2[2], Z2[1] * Z2[2], Z2[2] * Z2[2]};
    float T[2][2], K[3][3];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        T[a][0] = fr[2 * a];
        T[a][1] = fr[2 * a + 1];
    }
#pragma unroll
    for (int e = 0; e < 3; ++e)
#pragma unroll
        for (int p = 0; p < 3; ++p) K[e][p] = fr[WF_K + 3 * e + p];
    g1 += s[WS_N];
    de += s[WS_NE];
    // d/dmu = T' r-sums; d/dG[E] = K (W11, 2 W12, W22), W_ab = (z_a z_b A_ab - delta_ab B_a) / 2
    const float gm[2] = {z1 * s[WS_L], z2 * s[WS_L + 1]};
    const float ge[2] = {z1 * s[WS_LE], z2 * s[WS_LE + 1]};
    float Wv[3], Wev[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const int a = wpa(p), b = wpb(p);
        Wv[p] = 0.5f * wmult(p) * (Z2[a + b] * s[WS_A + a + b] - wdl(a, b) * s[WS_B + a]);
        Wev[p] = 0.5f * wmult(p) * (Z2[a + b] * s[WS_AE + a + b] - wdl(a, b) * s[WS_BE + a]);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        d1[i] += T[0][i] * gm[0] + T[1][i] * gm[1];
        he[i] += T[0][i] * ge[0] + T[1][i] * ge[1];
    }
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        d1[2 + e] += K[e][0] * Wv[0] + K[e][1] * Wv[1] + K[e][2] * Wv[2];
        he[2 + e] += K[e][0] * Wev[0] + K[e][1] * Wev[1] + K[e][2] * Wev[2];
    }
    // (mu, mu) = T' X T, X_ab = z_a z_b LL_ab - delta_ab L_a
    float XT[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            float v = 0.f;
#pragma unroll
            for (int b = 0; b < 2; ++b)
                v += (Z2[a + b] * s[WS_LL + a + b] - wdl(a, b) * s[WS_L + a]) * T[b][k];
            XT[a][k] = v;
        }
    h1[0] += T[0][0] * XT[0][0] + T[1][0] * XT[1][0];
    h1[1] += T[0][0] * XT[0][1] + T[1][0] * XT[1][1];
    h1[5] += T[0][1] * XT[0][1] + T[1][1] * XT[1][1];
    // (mu, G): T' (Yv K'), Y_{a,bc} = (z_a z_b z_c C_abc - delta_bc z_a A_ab - delta_ab z_c A_ac
    //                                  - delta_ac z_b A_ab) / 2
    float YK[2][3];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        float Yv[3];
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            const int b = wpa(p), c = wpb(p);
            Yv[p] = 0.5f * wmult(p) *
                    (Z3[a + b + c] * s[WS_C + a + b + c] - wdl(b, c) * z[a] * s[WS_A + a + b] -
                     wdl(a, b) * z[c] * s[WS_A + a + c] - wdl(a, c) * z[b] * s[WS_A + a + b]);
        }
#pragma unroll
        for (int e = 0; e < 3; ++e) YK[a][e] = K[e][0] * Yv[0] + K[e][1] * Yv[1] + K[e][2] * Yv[2];
    }
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        h1[2 + e] += T[0][0] * YK[0][e] + T[1][0] * YK[1][e];
        h1[6 + e] += T[0][1] * YK[0][e] + T[1][1] * YK[1][e];
    }
    // (G, G) = K Vm K', Vm_pq = m_p m_q V_{ab,cd} (pairs p = ab, q = cd)
    float KV[3][3];
    {
        float Vm[3][3];
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int a = wpa(p), b = wpb(p), c = wpa(q), d = wpb(q);
                const float* D2 = s + WS_D2;
                const float* D3 = s + WS_D3;
                const float v =
                    Z4[a + b + c + d] * s[WS_D4 + a + b + c + d] - wdl(c, d) * Z2[a + b] * D3[a + b + c] -
                    wdl(a, b) * Z2[c + d] * D3[a + c + d] + wdl(a, b) * wdl(c, d) * D2[a + c] -
                    wdl(b, c) * Z2[a + d] * D3[a + b + d] - wdl(a, c) * Z2[b + d] * D3[a + b + d] -
                    wdl(b, d) * Z2[a + c] * D3[a + b + c] - wdl(a, d) * Z2[b + c] * D3[a + b + c] +
                    (wdl(b, c) * wdl(a, d) + wdl(a, c) * wdl(b, d)) * D2[a + b];
                Vm[p][q] = 0.25f * wmult(p) * wmult(q) * v;
            }
#pragma unroll
        for (int e = 0; e < 3; ++e)
#pragma unroll
            for (int q = 0; q < 3; ++q) KV[e][q] = K[e][0] * Vm[0][q] + K[e][1] * Vm[1][q] + K[e][2] * Vm[2][q];
    }
    int c = 9;
#pragma unroll
    for (int e = 0; e < 3; ++e)
#pragma unroll
        for (int f = e; f < 3; ++f, ++c) h1[c] += KV[e][0] * K[f][0] + KV[e][1] * K[f][1] + KV[e][2] * K[f][2];
}

template <class R>
__global__ void __launch_bounds__(CHUNK) k_hess(const WorkItem* __restrict__ items,
                                                const PatchGeo* __restrict__ geo,
                                                const ImgMeta* __restrict__ img, int nprof,
                                                const float* __restrict__ pixels,
                                                const R* __restrict__ tbl,
                                                const R* __restrict__ emap,
                                                const R* __restrict__ vmap,
                                                double* __restrict__ part,
                                                const int32_t* __restrict__ src_active) {
    // FP32: the galaxy terms in the frame that whitens each PSF component
    constexpr bool WHITE = std::is_same<R, float>::value;
    __shared__ R sT[TBL_STRIDE];
    __shared__ double red[CHUNK / 32][HV];
    __shared__ __align__(16) float wsm[WHITE ? MAXPSF * WFR + MAXPSF * MAXPROF * WROW : 4];
    const WorkItem it = items[blockIdx.x];
    const PatchGeo g = geo[it.patch];
    if (src_active && !src_active[g.src]) return;
    const ImgMeta& im = img[g.img];
    const int npsf = im.npsf;
    {
        const R* gT = tbl + (size_t)it.patch * TBL_STRIDE;
        const int n = T_GAL + npsf * nprof * GAL_STRIDE;
        for (int i = threadIdx.x; i < n; i += blockDim.x) sT[i] = gT[i];
        __syncthreads();
    }
    if constexpr (WHITE) {
        if ((int)threadIdx.x < npsf) whiten_frame(sT, threadIdx.x, wsm + threadIdx.x * WFR);
        __syncthreads();
        for (int i = threadIdx.x; i < npsf * nprof; i += blockDim.x)
            whiten_row(sT + T_GAL + i * GAL_STRIDE, wsm + (i / nprof) * WFR, wsm + MAXPSF * WFR + i * WROW);
        __syncthreads();
    }
    R out[HV];
#pragma unroll
    for (int i = 0; i < HV; ++i) out[i] = 0;
    const int t = threadIdx.x;
    if (t < it.n) {
        const int q = it.q0 + t;
        const int yy = q / g.w, xx = q - yy * g.w;
        const int64_t m = im.px_off + (int64_t)(g.y0 + yy) * im.W + (g.x0 + xx);
        const R x = (R)pixels[m], E = emap[m], V = vmap[m];
        const R iE = (R)1 / E, iE2 = iE * iE;
        const R cE = x * (iE + V * iE2 * iE) - (R)1;
        const R cV = (R)-0.5 * x * iE2;
        const R hEE = -x * iE2 * ((R)1 + (R)3 * V * iE2);
        const R hEV = x * iE2 * iE;
        out[0] = x * (lgh(E) - (R)0.5 * V * iE2) - E;
        // star: value, gradient (mx, my), Hessian (xx, xy, yy)
        R g0 = 0, d0[2] = {0, 0}, h0[3] = {0, 0, 0};
        // galaxy: value; gradient over z5 = (mx, my, Gxx, Gxy, Gyy); e_dev derivative;
        // Hessian over z5 (packed 15); e_dev x z5
        R g1 = 0, d1[5] = {0, 0, 0, 0, 0}, de = 0, h1[15], he[5] = {0, 0, 0, 0, 0};
#pragma unroll
        for (int i = 0; i < 15; ++i) h1[i] = 0;
        for (int k = 0; k < npsf; ++k) {
            const R dx = (R)xx - sT[T_MEAN + 2 * k], dy = (R)yy - sT[T_MEAN + 2 * k + 1];
            const R dxx = dx * dx, dxy = dx * dy, dyy = dy * dy;
            {
                const R* S = sT + T_STAR + k * STAR_STRIDE;
                const R n = S[7] * ex2h(S[0] * dxx + S[1] * dxy + S[2] * dyy + S[3]);
                const R qx = S[4] * dx + S[5] * dy, qy = S[5] * dx + S[6] * dy;
                g0 += n;
                d0[0] += n * qx;
                d0[1] += n * qy;
                h0[0] += n * (qx * qx - S[4]);
                h0[1] += n * (qx * qy - S[5]);
                h0[2] += n * (qy * qy - S[6]);
            }
            if constexpr (WHITE) {
                const float* fr = wsm + k * WFR;
                const float z1 = fr[0] * dx + fr[1] * dy, z2 = fr[2] * dx + fr[3] * dy;
                const float z1s = z1 * z1, z2s = z2 * z2;
                float sw[NWS];
#pragma unroll
                for (int m = 0; m < NWS; ++m) sw[m] = 0.f;
                const float4* row = reinterpret_cast<const float4*>(wsm + MAXPSF * WFR + k * nprof * WROW);
                for (int j = 0; j < nprof; ++j, row += WROW / 4) {
                    float cw[WROW];
#pragma unroll
                    for (int u = 0; u < WROW / 4; ++u) {
                        const float4 v = row[u];
                        cw[4 * u] = v.x;
                        cw[4 * u + 1] = v.y;
                        cw[4 * u + 2] = v.z;
                        cw[4 * u + 3] = v.w;
                    }
                    const float e = ex2h(fmaf(cw[0], z1s, fmaf(cw[1], z2s, cw[2])));
#pragma unroll
                    for (int m = 0; m < NWS; ++m) sw[m] = fmaf(e, cw[3 + m], sw[m]);
                }
                whitened_add(sw, z1, z2, fr, g1, d1, de, h1, he);
                continue;
            }
            // FP64: the galaxy components one by one in the pixel frame
            const R* G = sT + T_GAL + k * nprof * GAL_STRIDE;
            for (int j = 0; j < nprof; ++j, G += GAL_STRIDE) {
                const R e = ex2h(G[0] * dxx + G[1] * dxy + G[2] * dyy + G[3]);
                const R n = G[7] * e, ne = G[8] * e;
                const R pxx = G[4], pxy = G[5], pyy = G[6], nu = G[9];
                const R qx = pxx * dx + pxy * dy, qy = pxy * dx + pyy * dy;
                R l[5];
                l[0] = qx;
                l[1] = qy;
                l[2] = (R)0.5 * nu * (qx * qx - pxx);
                l[3] = nu * (qx * qy - pxy);
                l[4] = (R)0.5 * nu * (qy * qy - pyy);
                const R nu2 = nu * nu;
                const R Pqy_x = pxx * qy + pxy * qx;   // (P (qy, qx))_x
                const R Pqy_y = pxy * qy + pyy * qx;   // (P (qy, qx))_y
                R L[15];
                L[0] = -pxx;                  // (mx, mx)
                L[1] = -pxy;                  // (mx, my)
                L[2] = -nu * pxx * qx;        // (mx, Gxx)
                L[3] = -nu * Pqy_x;           // (mx, Gxy)
                L[4] = -nu * pxy * qy;        // (mx, Gyy)
                L[5] = -pyy;                  // (my, my)
                L[6] = -nu * pxy * qx;        // (my, Gxx)
                L[7] = -nu * Pqy_y;           // (my, Gxy)
                L[8] = -nu * pyy * qy;        // (my, Gyy)
                L[9] = nu2 * ((R)0.5 * pxx * pxx - pxx * qx * qx);                           // (Gxx, Gxx)
                L[10] = nu2 * (pxx * pxy - qx * Pqy_x);                                      // (Gxx, Gxy)
                L[11] = nu2 * ((R)0.5 * pxy * pxy - pxy * qx * qy);                          // (Gxx, Gyy)
                L[12] = nu2 * (pxy * pxy + pxx * pyy - (qy * Pqy_x + qx * Pqy_y));            // (Gxy, Gxy)
                L[13] = nu2 * (pxy * pyy - qy * Pqy_y);                                      // (Gxy, Gyy)
                L[14] = nu2 * ((R)0.5 * pyy * pyy - pyy * qy * qy);                          // (Gyy, Gyy)
                g1 += n;
                de += ne;
                int c = 0;
#pragma unroll
                for (int a = 0; a < 5; ++a) {
                    d1[a] += n * l[a];
                    he[a] += ne * l[a];
#pragma unroll
                    for (int b = a; b < 5; ++b, ++c) h1[c] += n * (l[a] * l[b] + L[c]);
                }
            }
        }
        // ---- assemble the pixel's y-derivatives
        const R iota = sT[H_IOTA], a0 = sT[H_A0], a1 = sT[H_A1];
        const R el0 = sT[H_EL0], el20 = sT[H_EL20], el1 = sT[H_EL1], el21 = sT[H_EL21];
        const R i2 = iota * iota;
        const R f0 = iota * el0 * g0, f1 = iota * el1 * g1;
        const R Es = a0 * f0 + a1 * f1;
        const R w1 = cE - (R)2 * cV * Es, w2 = cV;
        // gradient of g_i over y (index 6..11), zero elsewhere
        R dg0[6] = {d0[0], d0[1], 0, 0, 0, 0};
        R dg1[6] = {d1[0], d1[1], de, d1[2], d1[3], d1[4]};
        // e = dE_s/dy, v2 = dE2_s/dy
        R e[NY], v2[NY];
        e[Y_A0] = f0;
        e[Y_A1] = f1;
        e[Y_EL0] = a0 * iota * g0;
        e[Y_EL20] = 0;
        e[Y_EL1] = a1 * iota * g1;
        e[Y_EL21] = 0;
        v2[Y_A0] = i2 * el20 * g0 * g0;
        v2[Y_A1] = i2 * el21 * g1 * g1;
        v2[Y_EL0] = 0;
        v2[Y_EL20] = a0 * i2 * g0 * g0;
        v2[Y_EL1] = 0;
        v2[Y_EL21] = a1 * i2 * g1 * g1;
        const R k0 = a0 * iota * el0, k1 = a1 * iota * el1;
        const R m0 = (R)2 * a0 * i2 * el20, m1 = (R)2 * a1 * i2 * el21;
#pragma unroll
        for (int z = 0; z < 6; ++z) {
            e[Y_MX + z] = k0 * dg0[z] + k1 * dg1[z];
            v2[Y_MX + z] = m0 * g0 * dg0[z] + m1 * g1 * dg1[z];
        }
        // gradient
#pragma unroll
        for (int y = 0; y < NY; ++y) out[1 + y] = w1 * e[y] + w2 * v2[y];
        // Hessian: outer-product part
        R v[NY];
#pragma unroll
        for (int y = 0; y < NY; ++y) v[y] = v2[y] - (R)2 * Es * e[y];
        const R c1 = hEE - (R)2 * cV;
        R* H = out + 1 + NY;
#pragma unroll
        for (int a = 0; a < NY; ++a)
#pragma unroll
            for (int b = a; b < NY; ++b)
                H[yh_index(a, b)] = c1 * e[a] * e[b] + hEV * (e[a] * v[b] + v[a] * e[b]);
        // second-derivative part  w1 DE + w2 DE2
        H[P2(Y_A0, Y_EL0)] += w1 * iota * g0;
        H[P2(Y_A1, Y_EL1)] += w1 * iota * g1;
        H[P2(Y_A0, Y_EL20)] += w2 * i2 * g0 * g0;
        H[P2(Y_A1, Y_EL21)] += w2 * i2 * g1 * g1;
        const R p0 = w1 * iota * el0 + (R)2 * w2 * i2 * el20 * g0;
        const R p1 = w1 * iota * el1 + (R)2 * w2 * i2 * el21 * g1;
        const R u0 = a0 * p0, u1 = a1 * p1;
        const R b0 = w2 * m0, b1 = w2 * m1;
#pragma unroll
        for (int z = 0; z < 6; ++z) {
            const int yz = Y_MX + z;
            H[P2(Y_A0, yz)] += p0 * dg0[z];
            H[P2(Y_A1, yz)] += p1 * dg1[z];
            H[P2(Y_EL0, yz)] += w1 * a0 * iota * dg0[z];
            H[P2(Y_EL1, yz)] += w1 * a1 * iota * dg1[z];
            H[P2(Y_EL20, yz)] += w2 * (R)2 * a0 * i2 * g0 * dg0[z];
            H[P2(Y_EL21, yz)] += w2 * (R)2 * a1 * i2 * g1 * dg1[z];
        }
        // z-z block: u0 d2g0 + b0 dg0 dg0' + u1 d2g1 + b1 dg1 dg1'
        // d2g1 over (mx, my, edev, Gxx, Gxy, Gyy) from h1 (z5 packed) and he (edev x z5)
        const int zmap[5] = {0, 1, 3, 4, 5};   // z5 position -> position among the six
        R d2g1[6][6];
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int b = 0; b < 6; ++b) d2g1[a][b] = 0;
        {
            int c = 0;
#pragma unroll
            for (int a = 0; a < 5; ++a) {
                d2g1[zmap[a]][2] = he[a];
                d2g1[2][zmap[a]] = he[a];
#pragma unroll
                for (int b = a; b < 5; ++b, ++c) {
                    d2g1[zmap[a]][zmap[b]] = h1[c];
                    d2g1[zmap[b]][zmap[a]] = h1[c];
                }
            }
        }
        const R d2g0[3] = {h0[0], h0[1], h0[2]};
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int b = a; b < 6; ++b) {
                R s = u1 * d2g1[a][b] + b1 * dg1[a] * dg1[b] + b0 * dg0[a] * dg0[b];
                if (a < 2 && b < 2) s += u0 * d2g0[a + b];
                H[yh_index(Y_MX + a, Y_MX + b)] += s;
            }
    }
    // ---- CTA reduction: in R within a warp (a reduce-scatter), FP64 across warps
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    R v[HVP];
#pragma unroll
    for (int i = 0; i < HVP; ++i) v[i] = i < HV ? out[i] : (R)0;
    warp_reduce_scatter(v, lane);
#pragma unroll
    for (int u = 0; u < HVP / 32; ++u)
        if (3 * lane + u < HV) red[warp][3 * lane + u] = (double)v[u];
    __syncthreads();
    for (int i = threadIdx.x; i < HV; i += blockDim.x) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][i];
        part[(size_t)blockIdx.x * NPART + i] = s;
    }
}

// ---------------------------------------------------------------------------------
// per-source chain rule and KL Hessian


// The pixel-frame ellipse is G = A W A' with W = ah I + bh (cos 2phi, sin 2phi; sin 2phi,
// -cos 2phi), ah = sigma^2 (1 + rho^2) / 2, bh = sigma^2 (1 - rho^2) / 2.  Its first and
// second derivatives over s = (e_axis, e_angle, e_scale) are A (dW) A' and A (d2W) A':
// dW and d2W depend on theta alone (computed once per source, by one thread), and each
// patch maps them through its own A (one output per thread).  Host-callable for tests.
__host__ __device__ void shape_w_derivs(const double* th, double dW[3][3], double d2W[3][3][3]) {
    const double rho = th[P_AXIS], phi = th[P_ANGLE], sg = th[P_SCALE];
    const double bh = 0.5 * sg * sg * (1.0 - rho * rho);
    double s2, c2;
    sincos(2.0 * phi, &s2, &c2);
    // first derivatives (index order rho = 0, phi = 1, sigma = 2; W as xx, xy, yy)
    {
        const double da = sg * sg * rho, db = -sg * sg * rho;
        dW[0][0] = da + db * c2; dW[0][1] = db * s2; dW[0][2] = da - db * c2;
    }
    dW[1][0] = -2.0 * bh * s2; dW[1][1] = 2.0 * bh * c2; dW[1][2] = 2.0 * bh * s2;
    {
        const double da = sg * (1.0 + rho * rho), db = sg * (1.0 - rho * rho);
        dW[2][0] = da + db * c2; dW[2][1] = db * s2; dW[2][2] = da - db * c2;
    }
    // second derivatives of ah, bh over (rho, sigma)
    const double bh_r = -sg * sg * rho, bh_s = sg * (1.0 - rho * rho);
    const double ah_rr = sg * sg, ah_ss = 1.0 + rho * rho, ah_rs = 2.0 * sg * rho;
    const double bh_rr = -sg * sg, bh_ss = 1.0 - rho * rho, bh_rs = -2.0 * sg * rho;
    auto set = [&](int a, int b, double xx, double xy, double yy) {
        d2W[a][b][0] = d2W[b][a][0] = xx;
        d2W[a][b][1] = d2W[b][a][1] = xy;
        d2W[a][b][2] = d2W[b][a][2] = yy;
    };
    set(0, 0, ah_rr + bh_rr * c2, bh_rr * s2, ah_rr - bh_rr * c2);
    set(2, 2, ah_ss + bh_ss * c2, bh_ss * s2, ah_ss - bh_ss * c2);
    set(0, 2, ah_rs + bh_rs * c2, bh_rs * s2, ah_rs - bh_rs * c2);
    set(0, 1, -2.0 * bh_r * s2, 2.0 * bh_r * c2, 2.0 * bh_r * s2);
    set(2, 1, -2.0 * bh_s * s2, 2.0 * bh_s * c2, 2.0 * bh_s * s2);
    set(1, 1, -4.0 * bh * c2, -4.0 * bh * s2, 4.0 * bh * c2);
}

// component c (xx, xy, yy) of A w A' for a symmetric w = (wxx, wxy, wyy)
__host__ __device__ __forceinline__ double a_transform(const double* A, const double* w, int c) {
    const double wxx = w[0], wxy = w[1], wyy = w[2];
    if (c == 0) return A[0] * A[0] * wxx + 2.0 * A[0] * A[1] * wxy + A[1] * A[1] * wyy;
    if (c == 1) return A[0] * A[2] * wxx + (A[0] * A[3] + A[1] * A[2]) * wxy + A[1] * A[3] * wyy;
    return A[2] * A[2] * wxx + 2.0 * A[2] * A[3] * wxy + A[3] * A[3] * wyy;
}

// Full KL Hessian (44 x 44, row-major) added into H (zeroed by the caller), by one warp
// (every lane calls it).  Lanes 8 i + d (i < 2, d < 8) hold the terms of type i's
// colour-prior component d, which touch disjoint entries (the k_d rows); the sums over
// components are shuffled within each group of eight, and lane 8 i then writes the
// type's a / r / c entries.  Every entry is written by exactly one lane.
__device__ void kl_hessian_warp(const ModelDev& md, const double* th, double* H) {
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    const int i = (lane >> 3) & 1, d = lane & 7;
    auto add = [&](int p, int q, double v) {
        H[p * NP + q] += v;
        if (p != q) H[q * NP + p] += v;
    };
    double c1[4], c2[4], ic2[4], slog = 0.0;
    for (int j = 0; j < 4; ++j) {
        c1[j] = th[P_C1 + 4 * i + j];
        c2[j] = th[P_C2 + 4 * i + j];
    }
    double sc1[4] = {0, 0, 0, 0}, sc2[4] = {0, 0, 0, 0}, Pk[16], ks = 0.0;
    for (int j = 0; j < 16; ++j) Pk[j] = 0.0;
    const double a = th[P_A + i];
    if (lane < 16) {
        for (int j = 0; j < 4; ++j) {
            slog += log(c2[j]);
            ic2[j] = 1.0 / c2[j];
        }
        const double k = th[P_K + NCOMP * i + d];
        const double* Pm = md.prior_P[i][d];
        const double* mu = md.prior_mu[i][d];
        double diff[4], Pd[4], quad = 0.0, tr = 0.0;
        for (int j = 0; j < 4; ++j) diff[j] = c1[j] - mu[j];
        for (int j = 0; j < 4; ++j) {
            double sj = 0.0;
            for (int l = 0; l < 4; ++l) sj += Pm[4 * j + l] * diff[l];
            Pd[j] = sj;
            quad += diff[j] * sj;
            tr += Pm[5 * j] * c2[j];
        }
        const double klc = 0.5 * (tr + quad - 4.0 + md.prior_logdet[i][d] - slog);
        const int ik = P_K + NCOMP * i + d;
        add(P_A + i, ik, log(k / md.prior_w[i][d]) + 1.0 + klc);
        add(ik, ik, a / k);
        for (int j = 0; j < 4; ++j) {
            add(ik, P_C1 + 4 * i + j, a * Pd[j]);
            add(ik, P_C2 + 4 * i + j, a * 0.5 * (Pm[5 * j] - ic2[j]));
            sc1[j] = k * Pd[j];
            sc2[j] = 0.5 * k * (Pm[5 * j] - ic2[j]);
        }
        for (int j = 0; j < 16; ++j) Pk[j] = k * Pm[j];
        ks = k;
    }
    for (int o = 1; o < 8; o <<= 1) {
        ks += __shfl_xor_sync(full, ks, o);
        for (int j = 0; j < 4; ++j) {
            sc1[j] += __shfl_xor_sync(full, sc1[j], o);
            sc2[j] += __shfl_xor_sync(full, sc2[j], o);
        }
        for (int j = 0; j < 16; ++j) Pk[j] += __shfl_xor_sync(full, Pk[j], o);
    }
    if (lane < 16 && d == 0) {
        const double r1 = th[P_R1 + i], r2 = th[P_R2 + i];
        const double pm = md.prior_r[i][0], pv = md.prior_r[i][1];
        const int ia = P_A + i, ir1 = P_R1 + i, ir2 = P_R2 + i;
        add(ia, ia, 1.0 / a);
        add(ia, ir1, (r1 - pm) / pv);
        add(ia, ir2, 0.5 * (1.0 / pv - 1.0 / r2));
        add(ir1, ir1, a / pv);
        add(ir2, ir2, a * 0.5 / (r2 * r2));
        for (int j = 0; j < 4; ++j) {
            add(ia, P_C1 + 4 * i + j, sc1[j]);
            add(ia, P_C2 + 4 * i + j, sc2[j]);
            add(P_C2 + 4 * i + j, P_C2 + 4 * i + j, a * 0.5 * ks * ic2[j] * ic2[j]);
            for (int l = j; l < 4; ++l) add(P_C1 + 4 * i + j, P_C1 + 4 * i + l, a * Pk[4 * j + l]);
        }
    }
    __syncwarp();
}

constexpr int FH_THREADS = 256;
// packed order of the 44 x 44 upper triangle (a << 8 | b, b <= a)
__device__ const PackedTriangle<NP> g_pkq = packed_triangle<NP>();

// d(m + v/2) / d theta_j (second = false) or d(2m + 2v) / d theta_j (second = true) of
// type ty in band `band`, where log l | ty ~ N(m, v), m = r1 + beta . c1, v = r2 + beta^2 . c2
__device__ __forceinline__ double bright_d(int band, int ty, int j, bool second) {
    if (j == P_R1 + ty) return second ? 2.0 : 1.0;
    if (j == P_R2 + ty) return second ? 2.0 : 0.5;
    if (j >= P_C1 + 4 * ty && j < P_C1 + 4 * ty + 4) {
        const double b = color_beta(band, j - P_C1 - 4 * ty);
        return second ? 2.0 * b : b;
    }
    if (j >= P_C2 + 4 * ty && j < P_C2 + 4 * ty + 4) {
        const double b = color_beta(band, j - P_C2 - 4 * ty);
        return second ? 2.0 * b * b : 0.5 * b * b;
    }
    return 0.0;
}

__global__ void __launch_bounds__(FH_THREADS)
k_finalize_hess(int n_src, const double* __restrict__ theta, const PatchGeo* __restrict__ geo,
                const int32_t* __restrict__ patch_off, const ImgMeta* __restrict__ img,
                const ModelDev* __restrict__ md, const double* __restrict__ part,
                double* __restrict__ kl_out, double* __restrict__ local_out,
                double* __restrict__ grad_out, double* __restrict__ hess_out,
                int32_t* __restrict__ status, const int32_t* __restrict__ src_active) {
    const int s = blockIdx.x;
    if (s >= n_src || (src_active && !src_active[s])) return;
    __shared__ double th[NP];
    __shared__ double Hy[NY][NY];
    __shared__ double Gy[NY + 1];
    __shared__ int nzn[NP];
    __shared__ int nzy[NP][3];
    __shared__ double nzv[NP][3];
    __shared__ double bmom[5][2][2];              // E[l_b | i], E[l_b^2 | i] per band and type
    __shared__ double dG[3][3], d2G[3][3][3];     // the patch map's shape derivatives
    __shared__ double dW[3][3], d2W[3][3][3];     // the same in the world frame (theta only)
    __shared__ double wd[2], we[2];
    __shared__ double S2[3][3];
    __shared__ double klH[NP * NP];
    __shared__ double Hacc[NP * NP];              // the pixel part of the 44 x 44 Hessian
    __shared__ double bd[2][2][NP];               // bright_d(band, type, j, second) of this patch
    __shared__ int act[NP], nact;                 // parameters this patch touches
    __shared__ double klg[NP];
    __shared__ double klv;
    // packed upper-triangle order of the active block: q = a (a + 1) / 2 + b, b <= a,
    // stored as a << 8 | b
    constexpr int NPK = NP * (NP + 1) / 2;
    __shared__ uint16_t pkq[NPK];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    for (int q = t; q < NPK; q += blockDim.x) pkq[q] = g_pkq.v[q];
    if (t < NP) {
        th[t] = theta[(size_t)NP * s + t];
        if (status) theta_domain_check(t, th[t], status);
    }
    for (int i = t; i < NP * NP; i += blockDim.x) {
        klH[i] = 0.0;
        Hacc[i] = 0.0;
    }
    __syncthreads();
    // the KL (warp 0: value and gradient; warp 1: Hessian) and the band moments of the
    // five bands (warp 2), each lane-parallel: the FP64 pipe costs a warp instruction
    // the same however few of its lanes are active
    if (warp == 0) {
        const double v = kl_warp<double>(*md, th, th, klg);
        if (lane == 0) klv = v;
    } else if (warp == 1) {
        kl_hessian_warp(*md, th, klH);
    } else if (warp == 2 && lane < 10) {
        const int b = lane >> 1, i = lane & 1;
        band_moments(th, b, i, bmom[b][i][0], bmom[b][i][1]);
    } else if (warp == 3 && lane == 0) {
        shape_w_derivs(th, dW, d2W);
    }
    double gacc = 0.0, lacc = 0.0;
    for (int p = patch_off[s]; p < patch_off[s + 1]; ++p) {
        __syncthreads();
        const PatchGeo g = geo[p];
        const ImgMeta& im = img[g.img];
        const double* A = im.A;
        if (t < 1 + NY + NYH) {
            // the patch's items in order, loaded eight at a time before any is added
            double v = 0.0;
            const int i1 = g.item0 + g.nitem;
            for (int i0 = g.item0; i0 < i1; i0 += 8) {
                double x[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) x[u] = i0 + u < i1 ? part[(size_t)(i0 + u) * NPART + t] : 0.0;
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (i0 + u < i1) v += x[u];
            }
            if (t == 0) lacc += v;
            else if (t < 1 + NY) Gy[t - 1] = v;
            else {
                // unpack the packed upper triangle
                int idx = t - 1 - NY, a = 0;
                while (idx >= NY - a) { idx -= NY - a; ++a; }
                const int b = a + idx;
                Hy[a][b] = v;
                Hy[b][a] = v;
            }
        } else if (t >= 128 && t < 128 + 9 + 27) {
            // the patch's shape derivatives through its map, one output per thread
            const int i = t - 128;
            if (i < 9) {
                dG[i / 3][i % 3] = a_transform(A, dW[i / 3], i % 3);
            } else {
                const int r = i - 9, a = r / 9, b = (r / 3) % 3, c = r % 3;
                d2G[a][b][c] = a_transform(A, d2W[a][b], c);
            }
        }
        __syncthreads();
        if (t < NP) {
            // column t of the sparse Jacobian dy / dtheta for this patch
            const int j = t;
            int n = 0;
            auto put = [&](int y, double val) {
                nzy[j][n] = y;
                nzv[j][n] = val;
                ++n;
            };
            if (j == 0) { put(Y_MX, A[0]); put(Y_MY, A[2]); }
            else if (j == 1) { put(Y_MX, A[1]); put(Y_MY, A[3]); }
            else if (j == P_EDEV) put(Y_EDEV, 1.0);
            else if (j >= P_AXIS && j <= P_SCALE) {
                const int q = j - P_AXIS;
                put(Y_GXX, dG[q][0]);
                put(Y_GXY, dG[q][1]);
                put(Y_GYY, dG[q][2]);
            } else if (j == P_A || j == P_A + 1) put(j == P_A ? Y_A0 : Y_A1, 1.0);
            else if (j < P_A) {
                const int i = (j < P_C1) ? ((j - P_R1) & 1) : (((j - (j >= P_C2 ? P_C2 : P_C1)) >> 2) & 1);
                const double dv = bright_d(im.band, i, j, false), ev = bright_d(im.band, i, j, true);
                if (dv != 0.0) put(i == 0 ? Y_EL0 : Y_EL1, bmom[im.band][i][0] * dv);
                if (ev != 0.0) put(i == 0 ? Y_EL20 : Y_EL21, bmom[im.band][i][1] * ev);
            }
            nzn[j] = n;
            for (int ty = 0; ty < 2; ++ty) {
                bd[ty][0][j] = bright_d(im.band, ty, j, false);
                bd[ty][1][j] = bright_d(im.band, ty, j, true);
            }
        } else if (t >= 64 && t < 73) {
            const int a = (t - 64) / 3, b = (t - 64) % 3;
            S2[a][b] = Gy[Y_GXX] * d2G[a][b][0] + Gy[Y_GXY] * d2G[a][b][1] + Gy[Y_GYY] * d2G[a][b][2];
        } else if (t >= 96 && t < 98) {
            const int i = t - 96;
            wd[i] = bmom[im.band][i][0] * Gy[i == 0 ? Y_EL0 : Y_EL1];
            we[i] = bmom[im.band][i][1] * Gy[i == 0 ? Y_EL20 : Y_EL21];
        }
        __syncthreads();
        if (t < NP)
            for (int n = 0; n < nzn[t]; ++n) gacc += nzv[t][n] * Gy[nzy[t][n]];
        if (warp == 0) {
            // the parameters with a nonzero Jacobian column, ascending: the only rows and
            // columns this patch adds to (every brightness and shape term lies among them)
            const unsigned b0 = __ballot_sync(0xffffffffu, nzn[lane] > 0);
            const unsigned b1 = __ballot_sync(0xffffffffu, lane + 32 < NP && nzn[lane + 32] > 0);
            const unsigned below = (1u << lane) - 1u;
            if (b0 >> lane & 1u) act[__popc(b0 & below)] = lane;
            if (b1 >> lane & 1u) act[__popc(b0) + __popc(b1 & below)] = lane + 32;
            if (lane == 0) nact = __popc(b0) + __popc(b1);
        }
        __syncthreads();
        // the upper triangle of the active block, each entry (and its mirror) by one thread
        const int na = nact, npair = na * (na + 1) / 2;
        for (int q = t; q < npair; q += blockDim.x) {
            const int a = pkq[q] >> 8, b = pkq[q] & 255;   // b <= a
            const int i = act[a], j = act[b];
            double h = 0.0;
            for (int u = 0; u < nzn[i]; ++u)
                for (int v = 0; v < nzn[j]; ++v)
                    h += nzv[i][u] * Hy[nzy[i][u]][nzy[j][v]] * nzv[j][v];
            // second derivatives of log E[l] and log E[l^2] (linear in the brightness
            // parameters, so only their products appear): w (dm)(dm)'
            for (int ty = 0; ty < 2; ++ty)
                h += wd[ty] * bd[ty][0][i] * bd[ty][0][j] + we[ty] * bd[ty][1][i] * bd[ty][1][j];
            if (i >= P_AXIS && i <= P_SCALE && j >= P_AXIS && j <= P_SCALE)
                h += S2[i - P_AXIS][j - P_AXIS];
            Hacc[i * NP + j] += h;
            if (i != j) Hacc[j * NP + i] += h;
        }
    }
    __syncthreads();
    double* Ho = hess_out + (size_t)NP * NP * s;
    for (int idx = t; idx < NP * NP; idx += blockDim.x) Ho[idx] = Hacc[idx] - klH[idx];
    if (t < NP && grad_out) grad_out[(size_t)NP * s + t] = gacc - klg[t];
    if (t == 0) {
        kl_out[s] = klv;
        if (local_out) local_out[s] = lacc - klv;
    }
}

cudaError_t launch_hess_pixels(const DevProblem& P, int precision, cudaStream_t st) {
    if (P.n_item == 0) return cudaSuccess;
    if (precision == CELESTE_FP64)
        k_hess<double><<<P.n_item, CHUNK, 0, st>>>(P.items, P.geo, P.img, P.nprof, P.pixels,
                                                   P.tbl64, (const double*)P.emap,
                                                   (const double*)P.vmap, P.item_part, P.src_active);
    else
        k_hess<float><<<P.n_item, CHUNK, 0, st>>>(P.items, P.geo, P.img, P.nprof, P.pixels,
                                                  P.tbl32, (const float*)P.emap,
                                                  (const float*)P.vmap, P.item_part, P.src_active);
    return cudaGetLastError();
}

cudaError_t launch_finalize_hess(const DevProblem& P, const double* d_theta, double* d_local,
                                 double* d_grad, double* d_hess, cudaStream_t st) {
    if (P.n_src == 0) return cudaSuccess;
    k_finalize_hess<<<P.n_src, FH_THREADS, 0, st>>>(P.n_src, d_theta, P.geo, P.patch_off, P.img,
                                                    P.model, P.item_part, P.kl, d_local, d_grad,
                                                    d_hess, P.status, P.src_active);
    return cudaGetLastError();
}

}  // namespace cel
