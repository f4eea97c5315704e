// FP32 value / gradient pass of the ELBO over the split work items, in the frame that
// whitens each PSF component (Section III model; Section VI-B: the cost is proportional
// to active pixel visits).
//
// Frame.  For PSF component k (covariance Sigma_k = L L^T) and the source's galaxy shape G
// in the patch's pixel frame, let L^-1 G L^-T = Q D Q^T (D = diag(D1, D2) >= 0) and
// T = Q^T L^-1.  Then T Sigma_k T^T = I and T G T^T = D, so every galaxy component j of
// PSF component k, covariance C_kj = Sigma_k + nu_j G, has precision T^T Lam_j T with
// Lam_j = diag(l1_j, l2_j), l_i = 1 / (1 + nu_j D_i), and det C_kj = det Sigma_k / (l1 l2).
// With z = T d (d = pixel - mean):
//   N_kj         = exp2(-log2(e)/2 (l1 z1^2 + l2 z2^2) + c_j)            (two FMAs)
//   dN/dmean     = N T^T (l1 z1, l2 z2)
//   dN/dG        = nu_j N T^T (Lam z z^T Lam - Lam) T / 2
// so per component only the sums over j of N times (1, l1, l2, nu (l1^2 z1^2 - l1),
// nu l1 l2, nu (l2^2 z2^2 - l2)) are accumulated (ten FMA-pipe operations), and T maps
// them back once per (pixel, k).  The star's component is the case nu = 0.  The same
// quantities as the packed kernels of pixel_kernels.cu, rearranged: fewer operations
// per component.
//
// Work.  k_ztab builds every patch's table (one warp per patch, in FP32 with the
// position in FP64) and the KL of every source (one warp per source).  k_items then takes
// one CTA per split item (<= 256 pixels of one patch): it copies its patch's table to
// shared memory, evaluates the mixture and its derivatives at its pixels, and for pixels
// that other patches also cover (multiply covered items) evaluates those patches' E_s,
// Var_s too, from their tables, summing E = sky + sum_s E_s and Var = sum_s Var_s in
// ascending source order (every covering item forms the same sum, bit for bit).  So the
// value / gradient pass has no map buffers between kernels; a per-source epilogue
// (k_finalize) and the total follow.  Packed FP32x2 arithmetic pairs two mixture
// components in one instruction (coefficients of adjacent components side by side in
// shared memory); FP64 only in the per-item sums.
#include <math.h>

#include "internal.cuh"
#include "source_math.cuh"
#include "epilogue.cuh"

namespace cel {

namespace {

constexpr float HL = -0.72134752044448170368f;   // -log2(e) / 2

// unroll factor of the component-pair loop of the gradient pass
#ifndef CEL_PAIR_UNROLL
#define CEL_PAIR_UNROLL 7
#endif
constexpr int PAIR_UNROLL = CEL_PAIR_UNROLL;

// table layout (floats).  Full record (the item's own patch):
//   header [0..31]: a0 a1 el0 el20 el1 el21 iota e_dev em0 em1 (1 - e_dev) band A[4]
//                   dG[3][3] at 16..24 (d(Gxx, Gxy, Gyy) / d(e_axis, e_angle, e_scale))
//   per PSF component k at ZH + k ZK:
//     [0..3] -mean_x -mean_y c_star sign   [4..7] T11 T12 T21 T22
//     [8..16] finishing coefficients of T^T W T (xx: T11^2, 2 T11 T21, T21^2; xy: T11 T12,
//             T11 T22 + T21 T12, T21 T22; yy: T12^2, 2 T12 T22, T22^2)
//     component pair q at 20 + 20 q, entries (component 2q, 2q+1) side by side:
//       [A A B B] [C C U1 U1] [U2 U2 Wa Wa] [Wb Wb W12 W12] [Va Va Vb Vb]
//       A, B = -log2(e)/2 (l1, l2); C = log2(|alpha_k| w_j) - log2(2 pi sqrt(det C_kj));
//       U1, U2 = s (l1, l2); Wa, Wb = s nu (l1^2, -l1); W12 = s nu l1 l2; Va, Vb = s nu (l2^2, -l2)
//       (s = sign(alpha_k) (1 - e_dev) for exp components, sign(alpha_k) e_dev for dev ones)
//     exp components fill pairs 0 .. npe-1, dev components pairs npe .. npe+npd-1, each
//     group padded to an even count with a component of weight zero (C = -1e30)
// Value record (shared-memory copy of another patch covering some of the pixels): the
// first 16 header floats, per k the first 8 floats, and per pair the first 8 floats
// [A A B B] [C C U1 U1].
constexpr int ZH = 32, ZKH = 20, ZPAIR = 20, ZMAXPAIR = (MAXPROF + 2) / 2;
constexpr int ZK = ZKH + ZMAXPAIR * ZPAIR;
constexpr int ZFULL = ZH + MAXPSF * ZK;
static_assert(ZFULL == ZFULL_FLOATS, "table size");
constexpr int VH = 16, VKH = 8, VPAIR = 8;
constexpr int VK = VKH + ZMAXPAIR * VPAIR;
constexpr int VFULL = VH + MAXPSF * VK;
constexpr int ZMAXC = 8;    // other patches' value records staged at once

__device__ __forceinline__ float ex2f(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float2 ex2x2(float2 a) { return make_float2(ex2f(a.x), ex2f(a.y)); }
__device__ __forceinline__ float2 dup(float a) { return make_float2(a, a); }
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// ---------------------------------------------------------------------------------
// table construction: one warp per patch, written to the table in global memory

// One patch's table, built by one warp.  Every lane first converts a share of theta to
// FP32 (FP64 -> FP32 conversions and FP64 arithmetic have ~70-cycle latencies on GB300's
// narrow FP64 pipe, so each is done once); lane 0 forms the position in FP64 (relative to
// the patch origin, so FP32 offsets stay exact).  Then, in parallel: lanes k < npsf build
// PSF component k's frame, lanes npsf, npsf + 1 the brightness moments of each type, lane
// npsf + 2 the weights, lane npsf + 3 the shape Jacobian; finally one lane per (PSF
// component, component slot) the slot's coefficients.  sm: 64 floats of this warp's
// shared memory.
__device__ __forceinline__ void build_patch_table(const double* __restrict__ theta, const PatchGeo* __restrict__ geo,
                                                  const ImgMeta* __restrict__ img, const ModelDev& md, int patch,
                                                  float* __restrict__ ztbl, float* sm) {
    const int lane = threadIdx.x & 31;
    const PatchGeo g = geo[patch];
    const ImgMeta& im = img[g.img];
    const double* th = theta + (size_t)NP * g.src;
    float* T = ztbl + (size_t)patch * ZFULL;
    float* thf = sm;        // [44] theta in FP32
    float* dscr = sm + 44;  // [8] D1, D2 per PSF component
    float* mu = sm + 52;    // [2] position relative to the patch origin
    // every global value this lane reads below, loaded together (one memory round trip)
    const int npsf = im.npsf, band = im.band;
    const float a0 = im.A_f[0], a1 = im.A_f[1], a2 = im.A_f[2], a3 = im.A_f[3];
    const int kk = lane < npsf ? lane : 0;
    const float li0 = im.psf_li[kk][0], li1 = im.psf_li[kk][1], li2 = im.psf_li[kk][2], dmk = im.psf_dm[kk];
    const float ps1 = im.psf_f[kk][1], ps2 = im.psf_f[kk][2], csk = im.psf_cs[kk], sgk = im.psf_sg[kk];
    const float iota = (float)im.iota;
    const int n_exp = md.n_exp, n_dev = md.n_dev;
    thf[lane] = (float)th[lane];
    if (lane + 32 < NP) thf[lane + 32] = (float)th[lane + 32];
    if (lane == 0) {
        const double u0 = th[0], u1 = th[1];
        mu[0] = (float)(im.A[0] * u0 + im.A[1] * u1 + im.t[0] - g.x0);
        mu[1] = (float)(im.A[2] * u0 + im.A[3] * u1 + im.t[1] - g.y0);
    }
    __syncwarp();
    const float rho = thf[P_AXIS], phi = thf[P_ANGLE], sg = thf[P_SCALE], ed = thf[P_EDEV];
    if (lane < npsf) {
        const int k = lane;
        // shape G = A W A^T in this patch's pixel frame, W = sigma^2 R(phi) diag(1, rho^2)
        // R(phi)^T = ah I + bh (cos 2phi, sin 2phi; sin 2phi, -cos 2phi)
        const float ah = 0.5f * sg * sg * (1.f + rho * rho), bh = 0.5f * sg * sg * (1.f - rho * rho);
        float s2, c2;
        sincosf(2.f * phi, &s2, &c2);
        const float wxx = ah + bh * c2, wxy = bh * s2, wyy = ah - bh * c2;
        const float gxx = a0 * a0 * wxx + 2.f * a0 * a1 * wxy + a1 * a1 * wyy;
        const float gxy = a0 * a2 * wxx + (a0 * a3 + a1 * a2) * wxy + a1 * a3 * wyy;
        const float gyy = a2 * a2 * wxx + 2.f * a2 * a3 * wxy + a3 * a3 * wyy;
        const float a = li0, b = li1, c = li2;
        // M = L^-1 G L^-T
        const float bxc = b * gxx + c * gxy, byc = b * gxy + c * gyy;
        const float m11 = a * a * gxx, m12 = a * bxc, m22 = bxc * b + byc * c;
        // Jacobi rotation diagonalising M (symmetric 2 x 2 Schur decomposition)
        float cs = 1.f, sn = 0.f, d1 = m11, d2 = m22;
        if (m12 != 0.f) {
            const float tau = __fdividef(m22 - m11, 2.f * m12);
            const float t = fabsf(tau) > 1e15f ? __fdividef(0.5f, tau)
                                               : copysignf(1.f, tau) * __frcp_rn(fabsf(tau) + sqrtf(1.f + tau * tau));
            cs = rsqrtf(1.f + t * t);
            sn = t * cs;
            d1 = m11 - t * m12;
            d2 = m22 + t * m12;
        }
        // the smaller eigenvalue from det M = psf_dm sigma^4 rho^2 (no cancellation)
        const float detm = dmk * (sg * sg * rho) * (sg * sg * rho);
        if (d1 >= d2 && d1 > 0.f) d2 = detm * __frcp_rn(d1);
        else if (d2 > d1 && d2 > 0.f) d1 = detm * __frcp_rn(d2);
        d1 = fmaxf(d1, 0.f);
        d2 = fmaxf(d2, 0.f);
        const float t11 = cs * a - sn * b, t12 = -sn * c, t21 = sn * a + cs * b, t22 = cs * c;
        float* K = T + ZH + k * ZK;
        K[0] = -(mu[0] + ps1);
        K[1] = -(mu[1] + ps2);
        K[2] = csk;
        K[3] = sgk;
        K[4] = t11; K[5] = t12; K[6] = t21; K[7] = t22;
        K[8] = t11 * t11; K[9] = 2.f * t11 * t21; K[10] = t21 * t21;
        K[11] = t11 * t12; K[12] = t11 * t22 + t21 * t12; K[13] = t21 * t22;
        K[14] = t12 * t12; K[15] = 2.f * t12 * t22; K[16] = t22 * t22;
        K[17] = K[18] = K[19] = 0.f;
        dscr[2 * k] = d1;
        dscr[2 * k + 1] = d2;
    } else if (lane < npsf + 2) {
        // brightness of type i in this band: log l ~ N(m, v); E[l] = e^{m+v/2},
        // E[l^2] = e^{2m+2v}, E[l^2] / E[l]^2 - 1 = e^v - 1
        const int i = lane - npsf;
        float m = thf[P_R1 + i], v = thf[P_R2 + i];
        for (int j = 0; j < 4; ++j) {
            const float bb = band_beta<float>(band, j);
            m += bb * thf[P_C1 + 4 * i + j];
            v += bb * bb * thf[P_C2 + 4 * i + j];
        }
        T[2 + 2 * i] = expf(m + 0.5f * v);
        T[3 + 2 * i] = expf(2.f * m + 2.f * v);
        T[8 + i] = expm1f(v);
    } else if (lane == npsf + 2) {
        T[0] = thf[P_A];
        T[1] = thf[P_A + 1];
        T[6] = iota;
        T[7] = ed;
        T[10] = 1.f - ed;
        T[11] = (float)band;   // the chain rule's band and image-frame map, for the epilogue
        T[12] = a0; T[13] = a1; T[14] = a2; T[15] = a3;
    } else if (lane == npsf + 3) {
        // dG = A dW A^T, dW = d(Wxx, Wxy, Wyy) / d(e_axis, e_angle, e_scale)
        const float bh = 0.5f * sg * sg * (1.f - rho * rho);
        float s2, c2;
        sincosf(2.f * phi, &s2, &c2);
        float dW[3][3];
        float da = sg * sg * rho, db = -sg * sg * rho;
        dW[0][0] = da + db * c2; dW[0][1] = db * s2; dW[0][2] = da - db * c2;
        dW[1][0] = -2.f * bh * s2; dW[1][1] = 2.f * bh * c2; dW[1][2] = 2.f * bh * s2;
        da = sg * (1.f + rho * rho); db = sg * (1.f - rho * rho);
        dW[2][0] = da + db * c2; dW[2][1] = db * s2; dW[2][2] = da - db * c2;
        for (int q = 0; q < 3; ++q) {
            const float ux = dW[q][0], uxy = dW[q][1], uy = dW[q][2];
            T[16 + 3 * q + 0] = a0 * a0 * ux + 2.f * a0 * a1 * uxy + a1 * a1 * uy;
            T[16 + 3 * q + 1] = a0 * a2 * ux + (a0 * a3 + a1 * a2) * uxy + a1 * a3 * uy;
            T[16 + 3 * q + 2] = a2 * a2 * ux + 2.f * a2 * a3 * uxy + a3 * a3 * uy;
        }
        for (int q = 25; q < 32; ++q) T[q] = 0.f;
    }
    // the coefficients of each (PSF component k, component slot): lane r takes slots r,
    // r + 32, ..., whose constants are read before the wait for phase one
    const int npe = (n_exp + 1) >> 1, nslot = 2 * (npe + ((n_dev + 1) >> 1));
    constexpr int NR = (MAXPSF * 2 * ZMAXPAIR + 31) / 32;   // rounds of 32 slots
    int sj[NR], sk[NR];
    float snu[NR], slw[NR], ssg[NR], scs[NR];
#pragma unroll
    for (int u = 0; u < NR; ++u) {
        const int r = lane + 32 * u;
        const int k = r / nslot, slot = r - k * nslot, q = slot >> 1;
        int j = -1;   // slot -> profile component j (or a padding slot)
        if (r < npsf * nslot) {
            if (q < npe) {
                if (slot < n_exp) j = slot;
            } else if (slot - 2 * npe < n_dev) {
                j = n_exp + slot - 2 * npe;
            }
        }
        sj[u] = j;
        sk[u] = k;
        snu[u] = j >= 0 ? md.prof_nu_f[j] : 0.f;
        slw[u] = j >= 0 ? md.prof_lw_f[j] : 0.f;
        ssg[u] = r < npsf * nslot ? im.psf_sg[k] : 0.f;
        scs[u] = r < npsf * nslot ? im.psf_cs[k] : 0.f;
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < NR; ++u) {
        const int r = lane + 32 * u;
        if (r >= npsf * nslot) break;
        const int k = sk[u], slot = r - k * nslot, q = slot >> 1, h = slot & 1, j = sj[u];
        const bool dev = j >= n_exp;
        float A = 0.f, B = 0.f, C = -1e30f, U1 = 0.f, U2 = 0.f, Wa = 0.f, Wb = 0.f, W12 = 0.f, Va = 0.f, Vb = 0.f;
        if (j >= 0) {
            const float nu = snu[u];
            const float l1 = __frcp_rn(1.f + nu * dscr[2 * k]), l2 = __frcp_rn(1.f + nu * dscr[2 * k + 1]);
            const float sgn = ssg[u] * (dev ? ed : 1.f - ed);
            A = HL * l1;
            B = HL * l2;
            C = scs[u] + slw[u] + 0.5f * (__log2f(l1) + __log2f(l2));
            U1 = sgn * l1;
            U2 = sgn * l2;
            const float snu = sgn * nu;
            Wa = snu * l1 * l1;
            Wb = -snu * l1;
            W12 = snu * l1 * l2;
            Va = snu * l2 * l2;
            Vb = -snu * l2;
        }
        float* pp = T + ZH + k * ZK + ZKH + q * ZPAIR + h;
        pp[0] = A; pp[2] = B; pp[4] = C; pp[6] = U1; pp[8] = U2; pp[10] = Wa; pp[12] = Wb; pp[14] = W12;
        pp[16] = Va; pp[18] = Vb;
    }
}

// Ready flags of the tables (one int per patch, 0 before the launch): the building warp
// publishes its table with a release (fence, then the flag); a reader acquires it, waiting
// at most ~1 s of SM clock, after which it records CELESTE_ERR_TIMEOUT and goes on.
__device__ __forceinline__ void publish_ready(int32_t* flag) {
    __threadfence();
    atomicExch(flag, 1);
}

__device__ __forceinline__ int load_acquire(const int32_t* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void wait_ready(const int32_t* flag, int32_t* status) {
    if (load_acquire(flag)) return;
    const long long t0 = clock64();
    for (int i = 0; i < (1 << 24); ++i) {
        __nanosleep(64);
        if (load_acquire(flag)) return;
        if (clock64() - t0 > 2000000000LL) break;
    }
    atomicExch(status, (int32_t)CELESTE_ERR_TIMEOUT);
}

// ---------------------------------------------------------------------------------
// per-pixel evaluation

// E_s and Var_s of a source at a pixel from its profile sums (every rounding written out,
// the same in every kernel of this file):
//   f_i = iota E[l_i] g_i,  E_s = a0 f0 + a1 f1,
//   Var_s = a0 f0^2 em0 + a1 f1^2 em1 + a0 (1 - a0) f0^2 + a1 (1 - a1) f1^2 - 2 a0 a1 f0 f1
__device__ __forceinline__ void source_ev(const float* H, float G0, float G1, float& f0, float& f1,
                                          float& es, float& vs) {
    const float a0 = H[0], a1 = H[1], iota = H[6];
    f0 = __fmul_rn(__fmul_rn(iota, H[2]), G0);
    f1 = __fmul_rn(__fmul_rn(iota, H[4]), G1);
    es = __fadd_rn(__fmul_rn(a0, f0), __fmul_rn(a1, f1));
    const float f00 = __fmul_rn(f0, f0), f11 = __fmul_rn(f1, f1);
    float v = __fmul_rn(__fmul_rn(a0, f00), H[8]);
    v = __fadd_rn(v, __fmul_rn(__fmul_rn(a1, f11), H[9]));
    v = __fadd_rn(v, __fmul_rn(__fmul_rn(a0, __fsub_rn(1.f, a0)), f00));
    v = __fadd_rn(v, __fmul_rn(__fmul_rn(a1, __fsub_rn(1.f, a1)), f11));
    vs = __fsub_rn(v, __fmul_rn(__fmul_rn(2.f, __fmul_rn(a0, a1)), __fmul_rn(f0, f1)));
}

// the profile sums g0 (star), g1 (galaxy) of one patch at PX pixels, value only
template <int PX, int NPE, int NPD>
__device__ __forceinline__ void profile_value(const float* H, const float* Kbase, int kstride, int pstride,
                                              int npsf, int npe_rt, int npd_rt, const float (&X)[PX],
                                              const float (&Y)[PX], float (&G0)[PX], float (&G1)[PX]) {
    const int npe = NPE >= 0 ? NPE : npe_rt, npd = NPD >= 0 ? NPD : npd_rt;
    float ge[PX], gd[PX];
#pragma unroll
    for (int p = 0; p < PX; ++p) G0[p] = ge[p] = gd[p] = 0.f;
    for (int k = 0; k < npsf; ++k) {
        const float* K = Kbase + k * kstride;
        const float4 h0 = ld4(K), h1 = ld4(K + 4);
        float2 Z1[PX], Z2[PX], xe[PX], xd[PX];
#pragma unroll
        for (int p = 0; p < PX; ++p) {
            const float dx = __fadd_rn(X[p], h0.x), dy = __fadd_rn(Y[p], h0.y);
            const float z1 = __fmaf_rn(h1.x, dx, __fmul_rn(h1.y, dy));
            const float z2 = __fmaf_rn(h1.z, dx, __fmul_rn(h1.w, dy));
            const float q1 = __fmul_rn(z1, z1), q2 = __fmul_rn(z2, z2);
            const float es = ex2f(__fmaf_rn(HL, __fadd_rn(q1, q2), h0.z));
            G0[p] = __fmaf_rn(h0.w, es, G0[p]);
            Z1[p] = dup(q1);
            Z2[p] = dup(q2);
            xe[p] = xd[p] = dup(0.f);
        }
        const float* Q = K + (kstride == ZK ? ZKH : VKH);
#pragma unroll
        for (int q = 0; q < (NPE >= 0 ? NPE + NPD : 1); ++q) {
            if (NPE < 0) break;
            const float4 ab = ld4(Q + q * pstride), cc = ld4(Q + q * pstride + 4);
            const float2 A = make_float2(ab.x, ab.y), B = make_float2(ab.z, ab.w), C = make_float2(cc.x, cc.y);
#pragma unroll
            for (int p = 0; p < PX; ++p) {
                const float2 e = ex2x2(__ffma2_rn(A, Z1[p], __ffma2_rn(B, Z2[p], C)));
                if (q < NPE) xe[p] = __fadd2_rn(xe[p], e);
                else xd[p] = __fadd2_rn(xd[p], e);
            }
        }
        if (NPE < 0) {
            for (int q = 0; q < npe + npd; ++q) {
                const float4 ab = ld4(Q + q * pstride), cc = ld4(Q + q * pstride + 4);
                const float2 A = make_float2(ab.x, ab.y), B = make_float2(ab.z, ab.w), C = make_float2(cc.x, cc.y);
#pragma unroll
                for (int p = 0; p < PX; ++p) {
                    const float2 e = ex2x2(__ffma2_rn(A, Z1[p], __ffma2_rn(B, Z2[p], C)));
                    if (q < npe) xe[p] = __fadd2_rn(xe[p], e);
                    else xd[p] = __fadd2_rn(xd[p], e);
                }
            }
        }
#pragma unroll
        for (int p = 0; p < PX; ++p) {
            ge[p] = __fmaf_rn(h0.w, __fadd_rn(xe[p].x, xe[p].y), ge[p]);
            gd[p] = __fmaf_rn(h0.w, __fadd_rn(xd[p].x, xd[p].y), gd[p]);
        }
    }
#pragma unroll
    for (int p = 0; p < PX; ++p) G1[p] = __fmaf_rn(H[10], ge[p], __fmul_rn(H[7], gd[p]));
}

struct ProfileGrad {
    float g0, gx0, gy0, g1, gx1, gy1, de, sxx, sxy, syy;
};

// the profile sums and their derivatives of the item's own patch at PX pixels; g0 and g1
// are formed with exactly the operations of profile_value
template <int PX, int NPE, int NPD>
__device__ __forceinline__ void profile_grad(const float* H, int npsf, int npe_rt, int npd_rt,
                                             const float (&X)[PX], const float (&Y)[PX],
                                             ProfileGrad (&o)[PX]) {
    const int npe = NPE >= 0 ? NPE : npe_rt, npd = NPD >= 0 ? NPD : npd_rt;
    float ge[PX], gd[PX];
#pragma unroll
    for (int p = 0; p < PX; ++p) {
        o[p].g0 = o[p].gx0 = o[p].gy0 = o[p].gx1 = o[p].gy1 = o[p].sxx = o[p].sxy = o[p].syy = 0.f;
        ge[p] = gd[p] = 0.f;
    }
    for (int k = 0; k < npsf; ++k) {
        const float* K = H + ZH + k * ZK;
        const float4 h0 = ld4(K), h1 = ld4(K + 4);
        float z1[PX], z2[PX];
        float2 Z1[PX], Z2[PX], xe[PX], xd[PX], u1[PX], u2[PX], w11[PX], w12[PX], w22[PX];
#pragma unroll
        for (int p = 0; p < PX; ++p) {
            const float dx = __fadd_rn(X[p], h0.x), dy = __fadd_rn(Y[p], h0.y);
            z1[p] = __fmaf_rn(h1.x, dx, __fmul_rn(h1.y, dy));
            z2[p] = __fmaf_rn(h1.z, dx, __fmul_rn(h1.w, dy));
            const float q1 = __fmul_rn(z1[p], z1[p]), q2 = __fmul_rn(z2[p], z2[p]);
            const float es = ex2f(__fmaf_rn(HL, __fadd_rn(q1, q2), h0.z));
            o[p].g0 = __fmaf_rn(h0.w, es, o[p].g0);
            // star: d/dmean = sign alpha N T^T z
            const float ge_ = __fmul_rn(h0.w, es);
            const float su = __fmul_rn(ge_, z1[p]), sv = __fmul_rn(ge_, z2[p]);
            o[p].gx0 = __fmaf_rn(h1.x, su, __fmaf_rn(h1.z, sv, o[p].gx0));
            o[p].gy0 = __fmaf_rn(h1.y, su, __fmaf_rn(h1.w, sv, o[p].gy0));
            Z1[p] = dup(q1);
            Z2[p] = dup(q2);
            xe[p] = xd[p] = u1[p] = u2[p] = w11[p] = w12[p] = w22[p] = dup(0.f);
        }
        const float* Q = K + ZKH;
        auto pair = [&](int q, bool is_exp) {
            const float* c = Q + q * ZPAIR;
            const float4 c0 = ld4(c), c1 = ld4(c + 4), c2 = ld4(c + 8), c3 = ld4(c + 12), c4 = ld4(c + 16);
            const float2 A = make_float2(c0.x, c0.y), B = make_float2(c0.z, c0.w);
            const float2 C = make_float2(c1.x, c1.y), U1 = make_float2(c1.z, c1.w);
            const float2 U2 = make_float2(c2.x, c2.y), Wa = make_float2(c2.z, c2.w);
            const float2 Wb = make_float2(c3.x, c3.y), W12 = make_float2(c3.z, c3.w);
            const float2 Va = make_float2(c4.x, c4.y), Vb = make_float2(c4.z, c4.w);
#pragma unroll
            for (int p = 0; p < PX; ++p) {
                const float2 e = ex2x2(__ffma2_rn(A, Z1[p], __ffma2_rn(B, Z2[p], C)));
                if (is_exp) xe[p] = __fadd2_rn(xe[p], e);
                else xd[p] = __fadd2_rn(xd[p], e);
                u1[p] = __ffma2_rn(U1, e, u1[p]);
                u2[p] = __ffma2_rn(U2, e, u2[p]);
                w11[p] = __ffma2_rn(__ffma2_rn(Wa, Z1[p], Wb), e, w11[p]);
                w12[p] = __ffma2_rn(W12, e, w12[p]);
                w22[p] = __ffma2_rn(__ffma2_rn(Va, Z2[p], Vb), e, w22[p]);
            }
        };
        if (NPE >= 0) {
#pragma unroll (PAIR_UNROLL)
            for (int q = 0; q < (NPE >= 0 ? NPE + NPD : 0); ++q) pair(q, q < NPE);
        } else {
            for (int q = 0; q < npe + npd; ++q) pair(q, q < npe);
        }
        // finish component k: map the whitened sums back with T
        const float4 f0 = ld4(K + 8), f1 = ld4(K + 12);
        const float f8 = K[16];
#pragma unroll
        for (int p = 0; p < PX; ++p) {
            ge[p] = __fmaf_rn(h0.w, __fadd_rn(xe[p].x, xe[p].y), ge[p]);
            gd[p] = __fmaf_rn(h0.w, __fadd_rn(xd[p].x, xd[p].y), gd[p]);
            const float a = __fmul_rn(z1[p], __fadd_rn(u1[p].x, u1[p].y));
            const float b = __fmul_rn(z2[p], __fadd_rn(u2[p].x, u2[p].y));
            o[p].gx1 = __fmaf_rn(h1.x, a, __fmaf_rn(h1.z, b, o[p].gx1));
            o[p].gy1 = __fmaf_rn(h1.y, a, __fmaf_rn(h1.w, b, o[p].gy1));
            const float W11 = __fadd_rn(w11[p].x, w11[p].y);
            const float W12 = __fmul_rn(__fmul_rn(z1[p], z2[p]), __fadd_rn(w12[p].x, w12[p].y));
            const float W22 = __fadd_rn(w22[p].x, w22[p].y);
            o[p].sxx = __fmaf_rn(f0.x, W11, __fmaf_rn(f0.y, W12, __fmaf_rn(f0.z, W22, o[p].sxx)));
            o[p].sxy = __fmaf_rn(f0.w, W11, __fmaf_rn(f1.x, W12, __fmaf_rn(f1.y, W22, o[p].sxy)));
            o[p].syy = __fmaf_rn(f1.z, W11, __fmaf_rn(f1.w, W12, __fmaf_rn(f8, W22, o[p].syy)));
        }
    }
#pragma unroll
    for (int p = 0; p < PX; ++p) {
        o[p].g1 = __fmaf_rn(H[10], ge[p], __fmul_rn(H[7], gd[p]));
        o[p].de = __fsub_rn(gd[p], ge[p]);
    }
}

// ll = x (log E - Var / (2 E^2)) - E and its weights c_E = x (1/E + Var/E^3) - 1,
// c_V = -x / (2 E^2)
__device__ __forceinline__ float pix_ll(float x, float E, float V) {
    const float iE = __fdiv_rn(1.f, E), iE2 = __fmul_rn(iE, iE);
    return __fsub_rn(__fmul_rn(x, __fsub_rn(logf(E), __fmul_rn(__fmul_rn(0.5f, V), iE2))), E);
}
__device__ __forceinline__ void pix_weights(float x, float E, float V, float& cE, float& cV) {
    const float iE = __fdiv_rn(1.f, E), iE2 = __fmul_rn(iE, iE);
    cE = __fsub_rn(__fmul_rn(x, __fadd_rn(iE, __fmul_rn(V, __fmul_rn(iE2, iE)))), 1.f);
    cV = __fmul_rn(__fmul_rn(-0.5f, x), iE2);
}

// Sum NV per-thread values over the CTA: FP32 within a warp, FP64 across warps in warp
// order.  Thread i < NV receives the CTA total of value i in out[i] (shared).
template <int NV, int NTH>
__device__ __forceinline__ void block_sum(const float (&v)[NV], double* out) {
    constexpr int NW = NTH / 32;
    __shared__ float red[NW][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        float s = v[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[warp][i] = s;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < NW; ++w) s += (double)red[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

struct ItemArgs {
    const ZItem* items;        // launch order: the most expensive items first
    const ZCand* cands;
    const int32_t* xy;         // gathered pixels: (row << 16) | column in the patch
    const float2* xs;          // gathered pixels: (counts, sky)
    const ModelDev* md;
    const double* theta;
    float* ztbl;               // [patch][ZFULL] tables (built by the table CTAs)
    int32_t* ready;            // [patch] table ready flags, 0 before the launch
    const PatchGeo* geo_tab;   // patch geometry and image records for the table CTAs
    const ImgMeta* img_tab;
    double* part;              // [item][NZPART]
    double* item_ll;           // ll of a singly covered item's pixels
    double* item_own;          // ll of the multiply covered pixels the item owns
    int n_order, n_multi;
    int npe, npd;              // exp / dev component pairs
    int n_patch, tab_blocks;   // table CTAs: the first tab_blocks of the launch
    int kl_blocks, n_src;      // KL CTAs: the next kl_blocks
    double* kl;
    double* kl_grad;
    int32_t* status;
    // the per-source epilogue, run by the last of a source's items and KL warp to finish
    int mode;
    const int32_t* patch_off;
    const int32_t* spatch_off;
    const int32_t* sitem_off;
    int32_t* src_done;         // [n_src] arrivals per source, 0 between launches
    int32_t* grp_done;         // [groups + 1] finished sources per group, finished groups
    double* src_total;
    double* grp_total;
    double* local_out;
    double* grad_out;
    double* total_out;
};

constexpr int IT_THREADS = 128;              // threads per CTA
static_assert(CHUNK == 2 * IT_THREADS, "item sizes");
// shared memory of a CTA (floats): four warp items' tables and sums, or a multiply covered
// item's table, the other patches' value records and the stashed profile derivatives
constexpr int PG_F = 10;   // floats of a ProfileGrad
constexpr int VSUM_F = 16;   // floats per thread of the running per-thread sums (ll, d ll / d y, owned ll)
constexpr int ZF_DBL_OUT = 1024;   // doubles of one epilogue warp's shared memory (at most)
template <int PX>
struct ItemSmem {
    static constexpr int tables = ZFULL + ZMAXC * VFULL + IT_THREADS * PX * PG_F;
    static constexpr int items = tables + IT_THREADS * VSUM_F;
    // the KL CTAs: four warps' KL arrays and epilogue space
    static constexpr int kl = 5 * (IT_THREADS / 32) * NP + 2 * (IT_THREADS / 32) * ZF_DBL_OUT;
    static constexpr int floats = items > kl ? items : kl;
};
static_assert(sizeof(ProfileGrad) == PG_F * sizeof(float), "ProfileGrad layout");

// ---------------------------------------------------------------------------------
// Per-source epilogue, run by one warp: the last of the source's items and its KL warp to
// finish (an arrival counter per source, released and acquired at gpu scope).  Per patch,
// the [ll, d ll / d y] sums of its items (FP64 in item order: a batch of up to ZF_BATCH
// patches has contiguous items, staged in chunks with coalesced L2 loads, lane c adding
// column c, so one FP64 instruction serves every column -- GB300's FP64 pipe costs a whole
// warp instruction however few lanes are active); then the chain rule dy/dtheta of each
// patch from its table header (band, map, brightness moments, shape Jacobian), accumulated
// per column over the source's patches in order; minus the KL.  The source's share of the
// total (the ll of its singly covered items and of the multiply covered pixels its items
// own, minus its KL) goes to src_total; the last source of each group of ZF_GROUP adds the
// group's shares in order, the last group adds the group sums in order (fixed order at
// every level), and the counters are reset for the next launch.

constexpr int ZF_COLS = NZPART + 1;   // ll, d ll / d y, the item's share of the total
constexpr int ZF_BATCH = 4;           // patches per batch
constexpr int ZF_CHUNK = 24;          // item partials staged at once
// shared memory of one epilogue warp (doubles): the batch's sums, a chunk of partials and
// their total shares, the batch's headers and item ranges, chain coefficients and indices
constexpr int ZF_YS = 0, ZF_SP = ZF_YS + ZF_BATCH * 32, ZF_SL = ZF_SP + ZF_CHUNK * NZPART,
              ZF_HD = ZF_SL + ZF_CHUNK, ZF_CF = ZF_HD + ZF_BATCH * 10 + 8, ZF_CY = ZF_CF + ZF_BATCH * NP * 2,
              ZF_DBL = ZF_CY + ZF_BATCH * NP / 2 + 2;

__device__ __forceinline__ double warp_dsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// one arrival of source s (the calling warp's writes -- and, after a block barrier, its
// CTA's -- are done); true on the warp that arrived last
__device__ __forceinline__ bool source_arrive(const ItemArgs& a, int s) {
    const int lane = threadIdx.x & 31;
    int last = 0;
    if (lane == 0) {
        const int target = a.sitem_off[s + 1] - a.sitem_off[s] + 1;   // items + the KL warp
        __threadfence();
        last = atomicAdd(a.src_done + s, 1) == target - 1;
        if (last) __threadfence();
    }
    return __shfl_sync(0xffffffffu, last, 0) != 0;
}

__device__ void source_epilogue(const ItemArgs& a, int s, double* sm /* ZF_DBL doubles */) {
    const int lane = threadIdx.x & 31, c = lane;
    double* ys = sm + ZF_YS;
    double* sp = sm + ZF_SP;
    double* sl = sm + ZF_SL;
    float* hd = reinterpret_cast<float*>(sm + ZF_HD);   // [ZF_BATCH][18]: 13 + band + A[4]
    int* ir = reinterpret_cast<int*>(sm + ZF_HD + ZF_BATCH * 9);   // [ZF_BATCH + 1]
    float* cf = reinterpret_cast<float*>(sm + ZF_CF);   // [ZF_BATCH * NP][4] chain coefficients
    int* cy = reinterpret_cast<int*>(sm + ZF_CY);       // [ZF_BATCH * NP] their y indices
    const int p0 = __ldcg(a.patch_off + s), p1 = __ldcg(a.patch_off + s + 1);
    const bool grad = a.mode >= MODE_GRAD;
    const double klv = __ldcg(a.kl + s);
    const double klg0 = grad ? __ldcg(a.kl_grad + (size_t)NP * s + lane) : 0.0;
    const double klg1 = grad && lane + 32 < NP ? __ldcg(a.kl_grad + (size_t)NP * s + 32 + lane) : 0.0;
    double g0 = 0.0, g1 = 0.0, lls = 0.0, tot = 0.0;
    for (int pb = p0; pb < p1; pb += ZF_BATCH) {
        const int np = min(ZF_BATCH, p1 - pb);
        if (lane <= np) ir[lane] = __ldcg(a.spatch_off + pb + lane);
        if (grad && lane < np) {
            const float* H = a.ztbl + (size_t)(pb + lane) * ZFULL;
            float* h = hd + 18 * lane;
            h[0] = __ldcg(H + 2); h[1] = __ldcg(H + 3); h[2] = __ldcg(H + 4); h[3] = __ldcg(H + 5);
            for (int e = 0; e < 9; ++e) h[4 + e] = __ldcg(H + 16 + e);
            for (int e = 0; e < 5; ++e) h[13 + e] = __ldcg(H + 11 + e);   // band, A[4]
        }
        __syncwarp();
        // per-patch column sums in item order (the batch's items are contiguous)
        // lane c (< 14) adds column c of the even items, lane 16 + c of the odd ones
        const int ib = ir[0], ie = ir[np];
        const int cc = c & 15, par = c >> 4;
        int j = 0, jend = ir[1];
        double acc = 0.0;
        for (int cs = ib; cs < ie; cs += ZF_CHUNK) {
            const int n = min(ZF_CHUNK, ie - cs);
            for (int e = lane; e < n * NZPART; e += 32) sp[e] = __ldcg(a.part + (size_t)cs * NZPART + e);
            for (int e = lane; e < n; e += 32) sl[e] = __ldcg(a.item_ll + cs + e) + __ldcg(a.item_own + cs + e);
            __syncwarp();
            if (cc < ZF_COLS && (grad || cc == 0 || cc == NZPART))
                for (int k = 0; k < n; ++k) {
                    while (cs + k >= jend) {   // the item starts a later patch of the batch
                        ys[16 * (2 * j + par) + cc] = acc;
                        acc = 0.0;
                        ++j;
                        jend = ir[j + 1];
                    }
                    if (((cs + k - ir[j]) & 1) == par) acc += cc < NZPART ? sp[k * NZPART + cc] : sl[k];
                }
            __syncwarp();
        }
        if (cc < ZF_COLS) {
            for (; j < np; ++j) {   // the last patch with items
                ys[16 * (2 * j + par) + cc] = acc;
                acc = 0.0;
            }
        }
        __syncwarp();
        // even + odd halves, in that order
        for (int r = lane; r < np * 16; r += 32) {
            const int q = r >> 4, col = r & 15;
            const double v = (col < ZF_COLS && (grad || col == 0 || col == NZPART))
                                 ? ys[16 * (2 * q) + col] + ys[16 * (2 * q + 1) + col] : 0.0;
            ys[16 * (2 * q) + col] = v;   // this lane's slot alone
        }
        __syncwarp();
        for (int q = 0; q < np; ++q) {
            lls += ys[32 * q];
            tot += ys[32 * q + NZPART];
        }
        if (grad) {
            // every (patch, column) pair's chain coefficients first (FP32, independent of the
            // sums, so the conversions below overlap), then per column three dependent FP64
            // FMAs per patch
            for (int r = lane; r < np * NP; r += 32) {
                const int q = r / NP, col = r - q * NP;
                const float* h = hd + 18 * q;
                const float el[2] = {h[0], h[2]}, el2[2] = {h[1], h[3]};
                float dG[3][3];
                for (int e = 0; e < 9; ++e) dG[e / 3][e % 3] = h[4 + e];
                int y0, y1, y2;
                float k0, k1, k2;
                chain_column<float>(col, (int)h[13], h + 14, el, el2, dG, &y0, &k0, &y1, &k1, &y2, &k2);
                cf[4 * r] = k0; cf[4 * r + 1] = k1; cf[4 * r + 2] = k2;
                cy[r] = y0 | (y1 << 4) | (y2 << 8);
            }
            __syncwarp();
            for (int q = 0; q < np; ++q) {
                const double* Y = ys + 32 * q;
                for (int half = 0; half < 2; ++half) {
                    const int col = lane + 32 * half;
                    if (col >= NP) break;
                    const int r = q * NP + col, yy = cy[r];
                    const double k0 = cf[4 * r], k1 = cf[4 * r + 1], k2 = cf[4 * r + 2];
                    double& gg = half == 0 ? g0 : g1;
                    gg = fma(k0, Y[1 + (yy & 15)], gg);
                    gg = fma(k1, Y[1 + ((yy >> 4) & 15)], gg);
                    gg = fma(k2, Y[1 + (yy >> 8)], gg);
                }
            }
        }
        __syncwarp();
    }
    if (lane == 0 && a.local_out) a.local_out[s] = lls - klv;
    if (grad && a.grad_out) {
        a.grad_out[(size_t)NP * s + lane] = g0 - klg0;
        if (lane + 32 < NP) a.grad_out[(size_t)NP * s + 32 + lane] = g1 - klg1;
    }
    if (lane == 0) a.src_done[s] = 0;
    if (!a.total_out) return;
    const int grp = s / ZF_GROUP, n_grp = (a.n_src + ZF_GROUP - 1) / ZF_GROUP;
    const int gb = grp * ZF_GROUP, gn = min(ZF_GROUP, a.n_src - gb);
    int last = 0;
    if (lane == 0) {
        a.src_total[s] = tot - klv;
        __threadfence();
        last = atomicAdd(a.grp_done + grp, 1) == gn - 1;
        if (last) __threadfence();
    }
    if (!__shfl_sync(0xffffffffu, last, 0)) return;
    // the group's shares in order: lane l adds shares l, l + 32, ..., then a shuffle tree
    double v = 0.0;
    for (int i = lane; i < gn; i += 32) v += __ldcg(a.src_total + gb + i);
    v = warp_dsum(v);
    last = 0;
    if (lane == 0) {
        a.grp_total[grp] = v;
        a.grp_done[grp] = 0;
        __threadfence();
        last = atomicAdd(a.grp_done + n_grp, 1) == n_grp - 1;
        if (last) __threadfence();
    }
    if (!__shfl_sync(0xffffffffu, last, 0)) return;
    v = 0.0;
    for (int i = lane; i < n_grp; i += 32) v += __ldcg(a.grp_total + i);
    v = warp_dsum(v);
    if (lane == 0) {
        *a.total_out = v;
        a.grp_done[n_grp] = 0;
    }
}

// this thread's pixels of an item (consecutive in the item's list, base = first index)
template <int PX>
__device__ __forceinline__ void item_pixels(const ItemArgs& a, const ZItem& it, int base, float (&X)[PX],
                                            float (&Y)[PX], float (&xv)[PX], float (&sky)[PX], bool (&ok)[PX]) {
#pragma unroll
    for (int p = 0; p < PX; ++p) {
        const int l = base + p;
        ok[p] = l < it.n;
        const int64_t j = it.pix + (ok[p] ? l : 0);
        const int q = a.xy[j];   // (row << 16) | column in the patch
        const float2 v = a.xs[j];
        X[p] = (float)(q & 0xffff);
        Y[p] = (float)(q >> 16);
        xv[p] = v.x;
        sky[p] = v.y;
    }
}

// copy a patch's table (header and the used part of each PSF component) to shared memory,
// threads `lane` of `nth`
__device__ __forceinline__ void stage_table(const float* __restrict__ src_tbl, float* dst_tbl, int npsf,
                                            int npair, int lane, int nth) {
    const float4* src = reinterpret_cast<const float4*>(src_tbl);
    float4* dst = reinterpret_cast<float4*>(dst_tbl);
    const int per_k = (ZKH + npair * ZPAIR) / 4;
    for (int i = lane; i < ZH / 4; i += nth) dst[i] = __ldcg(src + i);
    for (int k = 0; k < npsf; ++k)
        for (int i = lane; i < per_k; i += nth) dst[(ZH + k * ZK) / 4 + i] = __ldcg(src + (ZH + k * ZK) / 4 + i);
}

// the item's own source at this thread's pixels: E_s, Var_s, f_i and (gradient) the
// profile sums with their derivatives
template <int MODE, int PX, int NPE, int NPD>
__device__ __forceinline__ void own_source(const float* H, int npsf, int npe, int npd, const float (&X)[PX],
                                           const float (&Y)[PX], float (&Es)[PX], float (&Vs)[PX],
                                           float (&f0)[PX], float (&f1)[PX], ProfileGrad (&pg)[PX]) {
    if constexpr (MODE == MODE_LL) {
        float G0[PX], G1[PX];
        profile_value<PX, NPE, NPD>(H, H + ZH, ZK, ZPAIR, npsf, npe, npd, X, Y, G0, G1);
#pragma unroll
        for (int p = 0; p < PX; ++p) source_ev(H, G0[p], G1[p], f0[p], f1[p], Es[p], Vs[p]);
    } else {
        profile_grad<PX, NPE, NPD>(H, npsf, npe, npd, X, Y, pg);
#pragma unroll
        for (int p = 0; p < PX; ++p) source_ev(H, pg[p].g0, pg[p].g1, f0[p], f1[p], Es[p], Vs[p]);
    }
}

// the pixel's expected log-likelihood into v[0] and (gradient) its adjoint wrt the twelve
// y of the item's patch into v[1 ..]
template <int MODE, int NV>
__device__ __forceinline__ void pixel_terms(const float* H, float x, float E, float V, float Es, float f0,
                                            float f1, const ProfileGrad& q, float (&v)[NV], float& ll) {
    ll = pix_ll(x, E, V);
    v[0] += ll;
    if constexpr (MODE >= MODE_GRAD) {
        const float a0 = H[0], a1 = H[1], iota = H[6];
        const float el0 = H[2], el20 = H[3], el1 = H[4], el21 = H[5];
        const float i2 = iota * iota;
        float cE, cV;
        pix_weights(x, E, V, cE, cV);
        const float w1 = cE - 2.f * cV * Es, w2 = cV;
        const float s0 = i2 * q.g0 * q.g0, s1 = i2 * q.g1 * q.g1;
        v[1 + Y_A0] += w1 * f0 + w2 * el20 * s0;
        v[1 + Y_A1] += w1 * f1 + w2 * el21 * s1;
        v[1 + Y_EL0] += w1 * a0 * iota * q.g0;
        v[1 + Y_EL20] += w2 * a0 * s0;
        v[1 + Y_EL1] += w1 * a1 * iota * q.g1;
        v[1 + Y_EL21] += w2 * a1 * s1;
        const float u0 = a0 * iota * (w1 * el0 + 2.f * w2 * iota * el20 * q.g0);
        const float u1 = a1 * iota * (w1 * el1 + 2.f * w2 * iota * el21 * q.g1);
        v[1 + Y_MX] += u0 * q.gx0 + u1 * q.gx1;
        v[1 + Y_MY] += u0 * q.gy0 + u1 * q.gy1;
        v[1 + Y_EDEV] += u1 * q.de;
        v[1 + Y_GXX] += 0.5f * u1 * q.sxx;
        v[1 + Y_GXY] += u1 * q.sxy;
        v[1 + Y_GYY] += 0.5f * u1 * q.syy;
    }
}

// One singly covered item (<= FUSED_CHUNK pixels) on one CTA: no other source covers its
// pixels, so E = sky + E_s and Var = Var_s come from the item's own mixture sums.  Warp w
// takes the rounds of 32 PX pixels w, w + 4, ... (PX pixels per thread per round); the
// thread's running sums wait in shared memory while the mixture is evaluated; FP32 sums
// within a warp, FP64 across the warps in warp order.
template <int MODE, int PX, int NPE, int NPD>
__device__ __forceinline__ void single_item(const ItemArgs& a, const ZItem& it, float* sT, float* vs) {
    constexpr int NV = (MODE == MODE_LL) ? 1 : 1 + NY;
    constexpr int NW = IT_THREADS / 32;
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const int npsf = it.nc_npsf >> 24, n = it.n;
    float X[PX], Y[PX], xv[PX], sky[PX];
    bool ok[PX];
    item_pixels<PX>(a, it, w * 32 * PX + lane * PX, X, Y, xv, sky, ok);
    if (t == 0) wait_ready(a.ready + it.patch, a.status);
    __syncthreads();
    stage_table(a.ztbl + (size_t)it.patch * ZFULL, sT, npsf, a.npe + a.npd, t, IT_THREADS);
#pragma unroll
    for (int i = 0; i < NV; ++i) vs[i] = 0.f;
    __syncthreads();
    for (int r0 = w * 32 * PX; r0 < n; r0 += NW * 32 * PX) {
        if (r0 != w * 32 * PX) item_pixels<PX>(a, it, r0 + lane * PX, X, Y, xv, sky, ok);
        float Es[PX], Vs[PX], f0[PX], f1[PX];
        ProfileGrad pg[PX];
        own_source<MODE, PX, NPE, NPD>(sT, npsf, a.npe, a.npd, X, Y, Es, Vs, f0, f1, pg);
        float v[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i] = vs[i];
#pragma unroll
        for (int p = 0; p < PX; ++p) {
            if (!ok[p]) continue;
            float ll;
            pixel_terms<MODE, NV>(sT, xv[p], __fadd_rn(sky[p], Es[p]), Vs[p], Es[p], f0[p], f1[p], pg[p], v, ll);
        }
#pragma unroll
        for (int i = 0; i < NV; ++i) vs[i] = v[i];
    }
    float v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = vs[i];
    __shared__ double tot[NV];
    block_sum<NV, IT_THREADS>(v, tot);
    double* out = a.part + (size_t)it.out * NZPART;
    if (t < NV) out[t] = tot[t];
    if (t == 0) {
        a.item_ll[it.out] = tot[0];
        a.item_own[it.out] = 0.0;
    }
    __syncthreads();
    if (t >= 32) return;   // warp 0 arrives for the CTA (no block barrier after this)
    if (source_arrive(a, it.src)) source_epilogue(a, it.src, reinterpret_cast<double*>(sT));
}

// One multiply covered item (<= 256 pixels) on the whole CTA, PX pixels per thread per
// round: E and Var sum the item's source and every other covering source in ascending
// source order.
template <int MODE, int PX, int NPE, int NPD>
__device__ __forceinline__ void cta_item(const ItemArgs& a, const ZItem& it, float* sT, float* sVbase,
                                         float* vs) {
    constexpr int NTH = IT_THREADS;
    constexpr int NV = (MODE == MODE_LL) ? 1 : 1 + NY;
    __shared__ ZCand s_c[ZMAXC];
    const int npsf = it.nc_npsf >> 24, nc = it.nc_npsf & 0xffffff;
    const int npair = a.npe + a.npd;
    const int t = threadIdx.x;
    float X[PX], Y[PX], xv[PX], sky[PX];
    bool ok[PX];
    item_pixels<PX>(a, it, t * PX, X, Y, xv, sky, ok);
    if (t == 0) wait_ready(a.ready + it.patch, a.status);
    for (int ci = t; ci < nc; ci += NTH) wait_ready(a.ready + a.cands[it.c0 + ci].patch, a.status);
    __syncthreads();
    auto stage_others = [&](int cb, int cn) {
        if (t < cn) s_c[t] = a.cands[it.c0 + cb + t];
        // per record: 4 float4 of header, per k 2 float4 of header and 2 per pair
        const int per_k = 2 + 2 * npair, per_rec = 4 + MAXPSF * per_k;
        for (int i = t; i < cn * per_rec; i += NTH) {
            const int ci = i / per_rec, r = i - ci * per_rec;
            const float4* src = reinterpret_cast<const float4*>(a.ztbl + (size_t)a.cands[it.c0 + cb + ci].patch * ZFULL);
            float4* dst = reinterpret_cast<float4*>(sVbase + ci * VFULL);
            if (r < 4) {
                dst[r] = __ldcg(src + r);
            } else {
                const int k = (r - 4) / per_k, e = (r - 4) - k * per_k;
                const int so = (ZH + k * ZK) / 4 + (e < 2 ? e : ZKH / 4 + ((e - 2) >> 1) * (ZPAIR / 4) + ((e - 2) & 1));
                const int d = (VH + k * VK) / 4 + (e < 2 ? e : VKH / 4 + ((e - 2) >> 1) * (VPAIR / 4) + ((e - 2) & 1));
                dst[d] = __ldcg(src + so);
            }
        }
    };
    stage_table(a.ztbl + (size_t)it.patch * ZFULL, sT, npsf, npair, t, NTH);
    const int nc0 = nc < ZMAXC ? nc : ZMAXC;
    if (nc0 > 0) stage_others(0, nc0);
    __syncthreads();
    // the profile derivatives wait in shared memory while the other sources are evaluated,
    // and so do the thread's running sums
    ProfileGrad* spg = reinterpret_cast<ProfileGrad*>(sVbase + ZMAXC * VFULL) + t * PX;
#pragma unroll
    for (int i = 0; i <= NV; ++i) vs[i] = 0.f;
    for (int r0 = 0; r0 < it.n; r0 += NTH * PX) {
        if (r0 > 0) item_pixels<PX>(a, it, r0 + t * PX, X, Y, xv, sky, ok);
        const bool warp_on = r0 + (t >> 5) * 32 * PX < it.n;   // idle warps skip the work
        float Es[PX], Vs[PX], f0[PX], f1[PX];
        if (warp_on) {
            ProfileGrad pg[PX];
            own_source<MODE, PX, NPE, NPD>(sT, npsf, a.npe, a.npd, X, Y, Es, Vs, f0, f1, pg);
            if constexpr (MODE >= MODE_GRAD)
#pragma unroll
                for (int p = 0; p < PX; ++p) spg[p] = pg[p];
        }
        // E and Var over every covering source in ascending source order
        float E[PX], V[PX];
        bool owner[PX], added[PX];
#pragma unroll
        for (int p = 0; p < PX; ++p) {
            E[p] = sky[p];
            V[p] = 0.f;
            owner[p] = true;
            added[p] = false;
        }
        for (int cb = 0; cb < nc; cb += ZMAXC) {
            const int cn = min(ZMAXC, nc - cb);
            if (nc > ZMAXC && (cb > 0 || r0 > 0)) {
                __syncthreads();   // every thread is done with the previous round's records
                stage_others(cb, cn);
                __syncthreads();
            }
            if (!warp_on) continue;
            for (int ci = 0; ci < cn; ++ci) {
                const float* R = sVbase + ci * VFULL;
                const ZCand c = s_c[ci];
                float Xc[PX], Yc[PX];
                bool in[PX], any = false;
#pragma unroll
                for (int p = 0; p < PX; ++p) {
                    const int xx = (int)X[p] - c.dx, yy = (int)Y[p] - c.dy;
                    in[p] = ok[p] && xx >= 0 && xx < c.w && yy >= 0 && yy < c.h;
                    Xc[p] = (float)xx;
                    Yc[p] = (float)yy;
                    any = any || in[p];
                    // the item's own source enters the sum at its place in source order
                    if (!added[p] && c.src > it.src) {
                        E[p] = __fadd_rn(E[p], Es[p]);
                        V[p] = __fadd_rn(V[p], Vs[p]);
                        added[p] = true;
                    }
                    if (in[p] && c.src < it.src) owner[p] = false;
                }
                if (!__any_sync(0xffffffffu, any)) continue;
                float G0[PX], G1[PX];
                profile_value<PX, NPE, NPD>(R, R + VH, VK, VPAIR, c.npsf, a.npe, a.npd, Xc, Yc, G0, G1);
#pragma unroll
                for (int p = 0; p < PX; ++p) {
                    float q0, q1, ec, vc;
                    source_ev(R, G0[p], G1[p], q0, q1, ec, vc);
                    if (in[p]) {
                        E[p] = __fadd_rn(E[p], ec);
                        V[p] = __fadd_rn(V[p], vc);
                    }
                }
            }
        }
        if (warp_on) {
            float v[NV + 1];
#pragma unroll
            for (int i = 0; i <= NV; ++i) v[i] = vs[i];
#pragma unroll
            for (int p = 0; p < PX; ++p) {
                if (!ok[p]) continue;
                if (!added[p]) {
                    E[p] = __fadd_rn(E[p], Es[p]);
                    V[p] = __fadd_rn(V[p], Vs[p]);
                }
                float vv[NV], ll;
#pragma unroll
                for (int i = 0; i < NV; ++i) vv[i] = v[i];
                ProfileGrad q{};
                if constexpr (MODE >= MODE_GRAD) q = spg[p];
                pixel_terms<MODE, NV>(sT, xv[p], E[p], V[p], Es[p], f0[p], f1[p], q, vv, ll);
#pragma unroll
                for (int i = 0; i < NV; ++i) v[i] = vv[i];
                if (owner[p]) v[NV] += ll;
            }
#pragma unroll
            for (int i = 0; i <= NV; ++i) vs[i] = v[i];
        }
    }
    float v[NV + 1];
#pragma unroll
    for (int i = 0; i <= NV; ++i) v[i] = vs[i];
    __shared__ double tot[NV + 1];
    block_sum<NV + 1, NTH>(v, tot);
    double* out = a.part + (size_t)it.out * NZPART;
    if (t < NV) out[t] = tot[t];
    if (t == 0) {
        a.item_ll[it.out] = 0.0;
        a.item_own[it.out] = tot[NV];
    }
    __syncthreads();
    if (t >= 32) return;   // warp 0 arrives for the CTA (no block barrier after this)
    if (source_arrive(a, it.src)) source_epilogue(a, it.src, reinterpret_cast<double*>(sT));
}

// The whole FP32 value / gradient evaluation in one launch: CTAs [0, tab_blocks) build the
// patches' tables (one warp per patch) and publish them; the next kl_blocks CTAs compute
// the KL (one warp per source, with the domain check of theta); then one CTA per item, the
// most expensive first, each waiting for the tables it reads.  The last of each
// source's items and KL warp to finish runs the source's epilogue.  Waits are only on CTAs
// of lower index, which are dispatched first and wait on nothing.
template <int MODE, int PX, int NPE, int NPD, int MINB>
__global__ void __launch_bounds__(IT_THREADS, MINB) k_items(ItemArgs a) {
    __shared__ __align__(16) float smem[ItemSmem<PX>::floats];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int W = IT_THREADS / 32;
    if ((int)blockIdx.x < a.tab_blocks) {
        const int patch = (int)blockIdx.x * W + w;
        if (patch >= a.n_patch) return;   // whole warps leave; no block barrier in this branch
        build_patch_table(a.theta, a.geo_tab, a.img_tab, *a.md, patch, a.ztbl, smem + 64 * w);
        __syncwarp();
        if (lane == 0) publish_ready(a.ready + patch);
        return;
    }
    const int kb = (int)blockIdx.x - a.tab_blocks;
    if (kb < a.kl_blocks) {
        double (*kth)[NP] = reinterpret_cast<double (*)[NP]>(smem);
        double (*kg)[NP] = reinterpret_cast<double (*)[NP]>(smem + 2 * W * NP);
        float (*kthr)[NP] = reinterpret_cast<float (*)[NP]>(smem + 4 * W * NP);
        const int s = kb * W + w;
        if (s >= a.n_src) return;   // whole warps leave; no block barrier in this branch
        for (int i = lane; i < NP; i += 32) {
            const double v = a.theta[(size_t)NP * s + i];
            kth[w][i] = v;
            kthr[w][i] = (float)v;
            theta_domain_check(i, v, a.status);
        }
        __syncwarp();
        const double v = kl_warp<float>(*a.md, kth[w], kthr[w], kg[w]);
        __syncwarp();
        if (lane == 0) a.kl[s] = v;
        for (int i = lane; i < NP; i += 32) a.kl_grad[(size_t)NP * s + i] = kg[w][i];
        __syncwarp();
        // the epilogue's shared memory lies beyond every warp's KL arrays
        static_assert(ZF_DBL <= ZF_DBL_OUT, "epilogue shared memory");
        if (source_arrive(a, s)) source_epilogue(a, s, reinterpret_cast<double*>(smem + 5 * W * NP) + w * ZF_DBL);
        return;
    }
    const ZItem it = a.items[kb - a.kl_blocks];
    if ((it.nc_npsf & 0xffffff) > 0) {
        cta_item<MODE, PX, NPE, NPD>(a, it, smem, smem + ZFULL, smem + ItemSmem<PX>::tables + threadIdx.x * VSUM_F);
        return;
    }
    single_item<MODE, PX, NPE, NPD>(a, it, smem, smem + ItemSmem<PX>::tables + threadIdx.x * VSUM_F);
}

template <int MODE, int PX, int NPE, int NPD, int MINB>
cudaError_t items_launch_k(const ItemArgs& a, cudaStream_t st) {
    const int grid = a.tab_blocks + a.kl_blocks + a.n_order;
    if (grid == 0) return cudaSuccess;
    k_items<MODE, PX, NPE, NPD, MINB><<<grid, IT_THREADS, 0, st>>>(a);
    return cudaGetLastError();
}

// variant codes: 1, 2 two pixels per thread (at most 128 / 96 registers); 3, 4, 5 one pixel
// per thread (at most 64 / 72 / 80 registers)
template <int MODE, int PX, int MINB>
cudaError_t items_launch_v(const ItemArgs& a, cudaStream_t st) {
    if (a.npe == 3 && a.npd == 4) return items_launch_k<MODE, PX, 3, 4, MINB>(a, st);
    return items_launch_k<MODE, PX, -1, -1, MINB>(a, st);
}

template <int MODE>
cudaError_t items_launch(const ItemArgs& a, int code, cudaStream_t st) {
    switch (code) {
        case 1: return items_launch_v<MODE, 2, 4>(a, st);
        case 2: return items_launch_v<MODE, 2, 5>(a, st);
        case 4: return items_launch_v<MODE, 1, 7>(a, st);
        case 5: return items_launch_v<MODE, 1, 6>(a, st);
        default: return items_launch_v<MODE, 1, 8>(a, st);
    }
}

}  // namespace

cudaError_t launch_items(const DevProblem& P, int mode, cudaStream_t st, const double* d_theta, double* d_local,
                         double* d_grad, double* d_total) {
    if (P.n_src == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(P.zready, 0, sizeof(int32_t) * (size_t)(P.n_patch > 0 ? P.n_patch : 1), st);
    if (e != cudaSuccess) return e;
    ItemArgs a{};
    a.items = P.zitems;
    a.cands = P.zcands;
    a.xy = P.zxy;
    a.xs = P.zxs;
    a.md = P.model;
    a.theta = d_theta;
    a.ztbl = P.ztbl;
    a.ready = P.zready;
    a.geo_tab = P.geo;
    a.img_tab = P.img;
    a.part = P.spart;
    a.item_ll = P.sitem_ll;
    a.item_own = P.sitem_own;
    a.n_order = P.n_sitem;
    a.n_multi = P.n_smulti;
    a.npe = P.model_npe;
    a.npd = P.model_npd;
    a.n_patch = P.n_patch;
    a.tab_blocks = (P.n_patch + IT_THREADS / 32 - 1) / (IT_THREADS / 32);
    a.n_src = P.n_src;
    a.kl_blocks = (P.n_src + IT_THREADS / 32 - 1) / (IT_THREADS / 32);
    a.kl = P.kl;
    a.kl_grad = P.kl_grad;
    a.status = P.status;
    a.mode = mode;
    a.patch_off = P.patch_off;
    a.spatch_off = P.spatch_off;
    a.sitem_off = P.sitem_off;
    a.src_done = P.zsrc_done;
    a.grp_done = P.zf_done;
    a.src_total = P.src_total;
    a.grp_total = P.zf_grp_total;
    a.local_out = d_local;
    a.grad_out = mode >= MODE_GRAD ? d_grad : nullptr;
    a.total_out = d_total;
    if (mode == MODE_LL) return items_launch<MODE_LL>(a, P.tune_items, st);
    return items_launch<MODE_GRAD>(a, P.tune_items, st);
}

}  // namespace cel
