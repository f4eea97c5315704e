// FP32 value / gradient pass of the ELBO over every source's active pixels, in the frame
// that whitens each PSF component (Section III model; Section VI-B: the cost is
// proportional to active pixel visits).
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
// them back once per (pixel, k).  The star's component is the case nu = 0.  Packed FP32x2
// arithmetic pairs two mixture components per instruction (coefficients of adjacent
// components side by side in the table).
//
// Work.  Three launches.  k_tables builds every patch's table and chain-rule record (one
// warp per patch, FP32 with the position in FP64), publishing each with a ready flag, and
// every source's KL terms (one warp per source).  k_items, its programmatic dependent,
// runs on persistent CTAs of four compute warps and a producer warp that take items from
// a queue (a global counter over the items in decreasing cost): up to ZIMAX pixels of one
// patch, the multiply covered ones first.  The producer waits for the tables an item
// reads and copies its patch's table and chain-rule record, its pixel records and the
// value records of up to ZSTAGE other patches covering its pixels into a shared-memory
// stage with bulk asynchronous copies (two stages, completing on mbarriers), while the
// compute warps run the item in the other stage.  They evaluate the mixture and its
// derivatives at the item's pixels; where other patches cover a pixel, E = sky + sum_s
// E_s and Var = sum_s Var_s are summed over every covering source in ascending source
// order (every covering item forms the same sum, bit for bit).  Per warp FP32 sums; the
// producer adds the warps in FP64, applies the patch's chain rule dy/dtheta and writes the
// item's record.  k_finish, k_items' programmatic dependent, runs every
// source's epilogue once the items are done (one CTA per source: FP64 sums of its item
// records in a fixed order, minus the KL); the last CTA to finish adds the sources' shares
// of the total in source order.
// Every wait is bounded (~1 s), after which the kernel records CELESTE_ERR_TIMEOUT and
// ends.
#include <math.h>

#include "internal.cuh"
#include "source_math.cuh"
#include "epilogue.cuh"
#include "async_copy.cuh"

namespace cel {

namespace {

constexpr float HL = -0.72134752044448170368f;   // -log2(e) / 2


// Table layout (floats).  Value part (the prefix that another patch's items copy):
//   header [0..15]: a0 a1 el0 el20 el1 el21 iota e_dev em0 em1 (1 - e_dev) band A[4]
//   per PSF component k at VH + k VK:
//     [0..3] -mean_x -mean_y c_star sign   [4..7] T11 T12 T21 T22
//     profile component pair q at VKH + q VPAIR, the entries of components 2q and 2q + 1
//     side by side (so that one 8-byte half of a 16-byte load is a packed FP32x2 operand):
//       [A A B B] [C C U1 U1]
// Gradient part, per PSF component k at VFULL + k GK:
//     [0..8] finishing coefficients of T^T W T (xx: T11^2, 2 T11 T21, T21^2; xy: T11 T12,
//            T11 T22 + T21 T12, T21 T22; yy: T12^2, 2 T12 T22, T22^2), [9..11] unused
//     component pair q at GKH + q GPAIR: [U2 U2 Wa Wa] [Wb Wb W12 W12] [Va Va Vb Vb]
//   A, B = -log2(e)/2 (l1, l2); C = log2(|alpha_k| w_j) - log2(2 pi sqrt(det C_kj));
//   U1, U2 = s (l1, l2); Wa, Wb = s nu (l1^2, -l1); W12 = s nu l1 l2; Va, Vb = s nu (l2^2, -l2)
//   (s = sign(alpha_k) (1 - e_dev) for exp components, sign(alpha_k) e_dev for dev ones);
//   exp components fill pairs 0 .. npe-1, dev components pairs npe .. npe+npd-1, each
//   group padded to an even count with a component of weight zero (C = -1e30).
// Chain-rule record of a patch: per theta column j, (k0, k1, k2, y0 | y1 << 4 | y2 << 8):
// d y_{y_e} / d theta_j = k_e (unused pairs y = 0, k = 0).
constexpr int ZMAXPAIR = (MAXPROF + 2) / 2;
constexpr int VH = 16, VKH = 8, VPAIR = 8, VK = VKH + ZMAXPAIR * VPAIR, VFULL = VH + MAXPSF * VK;
constexpr int GKH = 12, GPAIR = 12, GK = GKH + ZMAXPAIR * GPAIR, GFULL = MAXPSF * GK;
constexpr int ZFULL = VFULL + GFULL;
static_assert(ZFULL == ZFULL_FLOATS, "table size");
static_assert(VFULL % 4 == 0 && ZFULL % 4 == 0, "tables are copied in 16-byte units");

// CTA shape: four compute warps and the producer warp
constexpr int NWC = 4;
constexpr int NTC = 32 * NWC;
constexpr int IT_THREADS = NTC + 32;

// One shared-memory stage (bytes): the item's table, its patch's chain-rule record, its
// pixel records, and its first ZSTAGE candidates' records and value tables.
constexpr int ST_TBL = 0;
constexpr int ST_CHAIN = ST_TBL + ZFULL * 4;
constexpr int ST_PX = ST_CHAIN + NP * 16;
constexpr int ST_ZC = ST_PX + ZIMAX * 16;
constexpr int ST_VREC = ST_ZC + ZSTAGE * (int)sizeof(ZCand);
constexpr int ST_BYTES = ST_VREC + ZSTAGE * VFULL * 4;
static_assert(ST_CHAIN % 16 == 0 && ST_PX % 16 == 0 && ST_ZC % 16 == 0 && ST_VREC % 16 == 0 && ST_BYTES % 16 == 0,
              "bulk copies land on 16-byte boundaries");
static_assert(sizeof(ZCand) == 32 && sizeof(ZTask) == 64, "record sizes");

constexpr int PG_F = 10;                 // floats of a ProfileGrad
constexpr int NSUM = 2 + NY;             // per-thread sums: ll, d ll / d y, owned ll
constexpr int SCR_W = 880;               // bytes per warp of the table kernel: KL arrays (2 x 44
                                         // doubles, 44 floats) or the table builder's 96 floats
constexpr int RED_W = 16;                // floats per warp of an item's warp sums

// the rest of the item kernel's shared memory (bytes), after the two stages
template <int PX>
struct Lay {
    static constexpr int vs = 2 * ST_BYTES;                        // running sums [NSUM][NTC]
    static constexpr int pg = vs + NSUM * NTC * 4;                 // stashed derivatives [PX PG_F][NTC]
    static constexpr int red = pg + PX * PG_F * NTC * 4;           // [2][NWC][RED_W] warp sums
    static constexpr int bar = red + 2 * NWC * RED_W * 4;          // full[2], reduced[2]
    static constexpr int task = bar + 4 * 8;                       // [2] ZTask
    static constexpr int bytes = task + 2 * (int)sizeof(ZTask);
    static_assert(task % 16 == 0 && bar % 8 == 0, "alignment");
};

// Registers per thread with MINB CTAs of IT_THREADS threads per SM: the SM's 64K
// registers, and each of its four sub-partitions' 16K over the warps it holds (warps are
// spread evenly), in multiples of 8.
constexpr int regs_for(int minb) {
    const int warps = minb * (IT_THREADS / 32), per_part = (warps + 3) / 4;
    const int a = 65536 / (minb * IT_THREADS), b = 16384 / (per_part * 32);
    return (a < b ? a : b) & ~7;
}

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

// One patch's table and chain-rule record, built by one warp.  Every lane first converts
// a share of theta to FP32 (FP64 -> FP32 conversions and FP64 arithmetic have ~70-cycle
// latencies on GB300's narrow FP64 pipe, so each is done once); lane 0 forms the position
// in FP64 (relative to the patch origin, so FP32 offsets stay exact).  Then every lane
// computes, and one lane each stores: PSF component k's frame (lanes k < npsf), the
// brightness moments of each type (lanes npsf, npsf + 1), the weights (lane npsf + 2)
// and the shape Jacobian (lane npsf + 3);
// finally one lane per (PSF component, component slot) the slot's coefficients and one
// lane per theta column its chain-rule pairs.  sm: 96 floats of this warp's shared memory.

__device__ __forceinline__ void build_patch_table(const double* __restrict__ theta, const ZBuild& g,
                                                  const ImgMeta* __restrict__ img, const ModelDev& md,
                                                  float* __restrict__ ztbl, float4* __restrict__ zchain,
                                                  float* sm) {
    const int lane = threadIdx.x & 31;
    const int patch = g.patch;
    const ImgMeta& im = img[g.img];
    const double* th = theta + (size_t)NP * g.src;
    float* T = ztbl + (size_t)patch * ZFULL;
    float* thf = sm;        // [44] theta in FP32
    float* dscr = sm + 44;  // [8] D1, D2 per PSF component
    float* mu = sm + 52;    // [2] position relative to the patch origin
    float* elv = sm + 56;   // [4] el0, el20, el1, el21
    float* dgs = sm + 60;   // [9] dG
    // every global value this lane reads below, loaded together (one memory round trip)
    const int npsf = im.npsf, band = im.band;
    const float a0 = im.A_f[0], a1 = im.A_f[1], a2 = im.A_f[2], a3 = im.A_f[3];
    const int kk = lane < npsf ? lane : 0;
    const float li0 = im.psf_li[kk][0], li1 = im.psf_li[kk][1], li2 = im.psf_li[kk][2], dmk = im.psf_dm[kk];
    const float ps1 = im.psf_f[kk][1], ps2 = im.psf_f[kk][2], csk = im.psf_cs[kk], sgk = im.psf_sg[kk];
    const float iota = im.iota_f;
    const int n_exp = md.n_exp, n_dev = md.n_dev;
    thf[lane] = (float)th[lane];
    if (lane + 32 < NP) thf[lane + 32] = (float)th[lane + 32];
    if (lane == 0) {
        const double u0 = th[0], u1 = th[1];
        mu[0] = (float)fma(im.A[0], u0, fma(im.A[1], u1, g.ox));
        mu[1] = (float)fma(im.A[2], u0, fma(im.A[3], u1, g.oy));
    }
    __syncwarp();
    const float rho = thf[P_AXIS], phi = thf[P_ANGLE], sg = thf[P_SCALE], ed = thf[P_EDEV];
    // Phase one, straight-line on every lane (the four parts are independent, so their
    // latencies overlap instead of adding up); each lane stores only its own part.
    float s2, c2;
    sincosf(2.f * phi, &s2, &c2);
    {
        // PSF component kk's frame: shape G = A W A^T in this patch's pixel frame,
        // W = sigma^2 R(phi) diag(1, rho^2), R(phi)^T = ah I + bh (cos 2phi, sin 2phi;
        // sin 2phi, -cos 2phi)
        const float ah = 0.5f * sg * sg * (1.f + rho * rho), bh = 0.5f * sg * sg * (1.f - rho * rho);
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
        if (lane < npsf) {
            const int k = lane;
            float4* K = reinterpret_cast<float4*>(T + VH + k * VK);
            K[0] = make_float4(-(mu[0] + ps1), -(mu[1] + ps2), csk, sgk);
            K[1] = make_float4(t11, t12, t21, t22);
            float4* KG = reinterpret_cast<float4*>(T + VFULL + k * GK);
            KG[0] = make_float4(t11 * t11, 2.f * t11 * t21, t21 * t21, t11 * t12);
            KG[1] = make_float4(t11 * t22 + t21 * t12, t21 * t22, t12 * t12, 2.f * t12 * t22);
            KG[2] = make_float4(t22 * t22, 0.f, 0.f, 0.f);
            dscr[2 * k] = d1;
            dscr[2 * k + 1] = d2;
        }
    }
    {
        // brightness of type i in this band: log l ~ N(m, v); E[l] = e^{m+v/2},
        // E[l^2] = e^{2m+2v}, E[l^2] / E[l]^2 - 1 = e^v - 1
        const int i = lane == npsf + 1 ? 1 : 0;
        float m = thf[P_R1 + i], v = thf[P_R2 + i];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float bb = band_beta<float>(band, j);
            m += bb * thf[P_C1 + 4 * i + j];
            v += bb * bb * thf[P_C2 + 4 * i + j];
        }
        const float el = expf(m + 0.5f * v), el2 = expf(2.f * m + 2.f * v), em = expm1f(v);
        if (lane == npsf || lane == npsf + 1) {
            T[2 + 2 * i] = el;
            T[3 + 2 * i] = el2;
            T[8 + i] = em;
            elv[2 * i] = el;
            elv[2 * i + 1] = el2;
        }
    }
    if (lane == npsf + 2) {
        T[0] = thf[P_A];
        T[1] = thf[P_A + 1];
        T[6] = iota;
        T[7] = ed;
        T[10] = 1.f - ed;
        T[11] = (float)band;
        T[12] = a0; T[13] = a1; T[14] = a2; T[15] = a3;
    }
    {
        // dG = A dW A^T, dW = d(Wxx, Wxy, Wyy) / d(e_axis, e_angle, e_scale)
        const float bh = 0.5f * sg * sg * (1.f - rho * rho);
        float dW[3][3];
        float da = sg * sg * rho, db = -sg * sg * rho;
        dW[0][0] = da + db * c2; dW[0][1] = db * s2; dW[0][2] = da - db * c2;
        dW[1][0] = -2.f * bh * s2; dW[1][1] = 2.f * bh * c2; dW[1][2] = 2.f * bh * s2;
        da = sg * (1.f + rho * rho); db = sg * (1.f - rho * rho);
        dW[2][0] = da + db * c2; dW[2][1] = db * s2; dW[2][2] = da - db * c2;
        if (lane == npsf + 3) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float ux = dW[q][0], uxy = dW[q][1], uy = dW[q][2];
                dgs[3 * q + 0] = a0 * a0 * ux + 2.f * a0 * a1 * uxy + a1 * a1 * uy;
                dgs[3 * q + 1] = a0 * a2 * ux + (a0 * a3 + a1 * a2) * uxy + a1 * a3 * uy;
                dgs[3 * q + 2] = a2 * a2 * ux + 2.f * a2 * a3 * uxy + a3 * a3 * uy;
            }
        }
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
            const float snu_ = sgn * nu;
            Wa = snu_ * l1 * l1;
            Wb = -snu_ * l1;
            W12 = snu_ * l1 * l2;
            Va = snu_ * l2 * l2;
            Vb = -snu_ * l2;
        }
        float* pv = T + VH + k * VK + VKH + q * VPAIR + h;
        pv[0] = A; pv[2] = B; pv[4] = C; pv[6] = U1;
        float* pq = T + VFULL + k * GK + GKH + q * GPAIR + h;
        pq[0] = U2; pq[2] = Wa; pq[4] = Wb; pq[6] = W12; pq[8] = Va; pq[10] = Vb;
    }
    // the chain-rule record: column j of dy/dtheta for this patch
    const float Af[4] = {a0, a1, a2, a3};
    const float el[2] = {elv[0], elv[2]}, el2[2] = {elv[1], elv[3]};
    float dG[3][3];
#pragma unroll
    for (int e = 0; e < 9; ++e) dG[e / 3][e % 3] = dgs[e];
    for (int j = lane; j < NP; j += 32) {
        int y0, y1, y2;
        float k0, k1, k2;
        chain_column<float>(j, band, Af, el, el2, dG, &y0, &k0, &y1, &k1, &y2, &k2);
        zchain[(size_t)patch * NP + j] = make_float4(k0, k1, k2, __int_as_float(y0 | (y1 << 4) | (y2 << 8)));
    }
}

// Ready flags of the tables (one int per patch, 0 before the launch): the building warp
// publishes its table and chain record with a release (fence, then the flag) and counts
// it in `built`; a reader acquires the flag, waiting at most ~1 s of SM clock (or less
// once another wait has given up), after which it records CELESTE_ERR_TIMEOUT and goes on.
__device__ __forceinline__ void publish_ready(int32_t* flag, int32_t* built) {
    asm volatile("st.release.gpu.global.s32 [%0], 1;" ::"l"(flag) : "memory");
    asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(built) : "memory");
}

__device__ __forceinline__ int load_acquire(const int32_t* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// another wait of the launch gave up, or a bounds check failed: waits end at once
__device__ __forceinline__ bool timed_out(const int32_t* status) {
    const int32_t v = *reinterpret_cast<const volatile int32_t*>(status);
    return v == (int32_t)CELESTE_ERR_TIMEOUT || v == (int32_t)CELESTE_ERR_BOUNDS;
}

// a wait that gave up records CELESTE_ERR_TIMEOUT unless an error is recorded already
__device__ __forceinline__ void record_timeout(int32_t* status) {
    atomicCAS(status, 0, (int32_t)CELESTE_ERR_TIMEOUT);
}

__device__ __forceinline__ void wait_ready(const int32_t* flag, int32_t* status) {
    if (load_acquire(flag)) return;
    const long long t0 = clock64();
    for (int i = 0; i < (1 << 24); ++i) {
        __nanosleep(64);
        if (load_acquire(flag)) return;
        if (timed_out(status) || clock64() - t0 > MBAR_MAX_CYCLES) break;
    }
    record_timeout(status);
}

// an mbarrier wait that also gives up once another wait of the launch has
__device__ __forceinline__ bool mbar_wait_launch(uint64_t* bar, unsigned parity, int32_t* status) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (int i = 0; i < MBAR_MAX_POLLS; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63) == 63 && timed_out(status)) break;
        if (clock64() - t0 > MBAR_MAX_CYCLES) break;
    }
    record_timeout(status);
    return false;
}

__device__ __forceinline__ void mbar_arrive_plain(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_arrive(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// one bulk copy completing on bar (whose expected bytes were announced already)
__device__ __forceinline__ void bulk_g2s_tx(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// order this thread's earlier (acquired) view of global memory before its async-proxy reads
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// ---------------------------------------------------------------------------------
// per-pixel evaluation: PX pixels per thread; a packed FP32x2 operation covers two
// profile components of one pixel

// E_s and Var_s of a source at a pixel from its profile sums (every rounding written out,
// the same wherever a source's E_s is formed):
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

// the profile sums g0 (star), g1 (galaxy) of one patch at PX pixels from its value part
// (an item's own table or another patch's value record: the same layout)
template <int PX, int NPE, int NPD>
__device__ __forceinline__ void profile_value(const float* H, int npsf, int npe_rt, int npd_rt,
                                              const float (&X)[PX], const float (&Y)[PX], float (&G0)[PX],
                                              float (&G1)[PX]) {
    const int npe = NPE >= 0 ? NPE : npe_rt, npd = NPD >= 0 ? NPD : npd_rt;
    float ge[PX], gd[PX];
#pragma unroll
    for (int p = 0; p < PX; ++p) G0[p] = ge[p] = gd[p] = 0.f;
    for (int k = 0; k < npsf; ++k) {
        const float* K = H + VH + k * VK;
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
        const float* Q = K + VKH;
        auto pair = [&](int q, bool is_exp) {
            const float4 ab = ld4(Q + q * VPAIR), cc = ld4(Q + q * VPAIR + 4);
            const float2 A = make_float2(ab.x, ab.y), B = make_float2(ab.z, ab.w), C = make_float2(cc.x, cc.y);
#pragma unroll
            for (int p = 0; p < PX; ++p) {
                const float2 e = ex2x2(__ffma2_rn(A, Z1[p], __ffma2_rn(B, Z2[p], C)));
                if (is_exp) xe[p] = __fadd2_rn(xe[p], e);
                else xd[p] = __fadd2_rn(xd[p], e);
            }
        };
        if (NPE >= 0) {
#pragma unroll
            for (int q = 0; q < (NPE >= 0 ? NPE + NPD : 0); ++q) pair(q, q < NPE);
        } else {
            for (int q = 0; q < npe + npd; ++q) pair(q, q < npe);
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
static_assert(sizeof(ProfileGrad) == PG_F * sizeof(float), "ProfileGrad layout");

// the profile sums and their derivatives of the item's own patch at PX pixels; g0 and g1
// are formed with exactly the operations of profile_value (UNR: unroll factor of the
// loop over component pairs)
template <int PX, int NPE, int NPD, int UNR>
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
        const float* K = H + VH + k * VK;
        const float* KG = H + VFULL + k * GK;
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
        const float* Q = K + VKH;
        const float* QG = KG + GKH;
        auto pair = [&](int q, bool is_exp) {
            const float4 c0 = ld4(Q + q * VPAIR), c1 = ld4(Q + q * VPAIR + 4);
            const float* cg = QG + q * GPAIR;
            const float4 c2 = ld4(cg), c3 = ld4(cg + 4), c4 = ld4(cg + 8);
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
#pragma unroll (UNR)
            for (int q = 0; q < (NPE >= 0 ? NPE + NPD : 0); ++q) pair(q, q < NPE);
        } else {
            for (int q = 0; q < npe + npd; ++q) pair(q, q < npe);
        }
        // finish component k: map the whitened sums back with T
        const float4 f0 = ld4(KG), f1 = ld4(KG + 4);
        const float f8 = KG[8];
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
    const float iE = __frcp_rn(E), iE2 = __fmul_rn(iE, iE);
    return __fsub_rn(__fmul_rn(x, __fsub_rn(logf(E), __fmul_rn(__fmul_rn(0.5f, V), iE2))), E);
}
__device__ __forceinline__ void pix_weights(float x, float E, float V, float& cE, float& cV) {
    const float iE = __frcp_rn(E), iE2 = __fmul_rn(iE, iE);
    cE = __fsub_rn(__fmul_rn(x, __fadd_rn(iE, __fmul_rn(V, __fmul_rn(iE2, iE)))), 1.f);
    cV = __fmul_rn(__fmul_rn(-0.5f, x), iE2);
}

// the item's own source at this thread's pixels: E_s, Var_s, f_i and (gradient) the
// profile sums with their derivatives
template <int MODE, int PX, int NPE, int NPD, int UNR>
__device__ __forceinline__ void own_source(const float* H, int npsf, int npe, int npd, const float (&X)[PX],
                                           const float (&Y)[PX], float (&Es)[PX], float (&Vs)[PX],
                                           float (&f0)[PX], float (&f1)[PX], ProfileGrad (&pg)[PX]) {
    if constexpr (MODE == MODE_LL) {
        float G0[PX], G1[PX];
        profile_value<PX, NPE, NPD>(H, npsf, npe, npd, X, Y, G0, G1);
#pragma unroll
        for (int p = 0; p < PX; ++p) source_ev(H, G0[p], G1[p], f0[p], f1[p], Es[p], Vs[p]);
    } else {
        profile_grad<PX, NPE, NPD, UNR>(H, npsf, npe, npd, X, Y, pg);
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

// ---------------------------------------------------------------------------------
// launch arguments

struct ItemArgs {
    const ZTask* tasks;
    int n_task;
    const ZBuild* torder;      // the patches' build records, in the order the items first read them
    const ZCand* cands;
    const float4* px;          // pixel records (column, row in the patch, counts, sky)
    const ModelDev* md;
    const double* theta;
    float* ztbl;               // [patch][ZFULL] tables
    float4* zchain;            // [patch][NP] chain-rule records
    int32_t* ready;            // [patch] table ready flags, then the queue counter and the
                               // count of built tables; all 0 before the launch
    const PatchGeo* geo_tab;
    const ImgMeta* img_tab;
    double* part;              // [item][ZPCOLS]
    int ne, nd;                // exp / dev profile components
    int n_patch, n_src;
    int64_t n_sp;              // pixel records (bounds checks)
    int n_zcand, n_sitem, n_img_rec;
    double* kl;
    double* kl_grad;
    int32_t* status;
    int mode;
    const int32_t* sitem_off;
    int32_t* grp_done;         // [0]: finished sources of the epilogue kernel, 0 between launches
    double* src_total;         // [n_src] each source's share of the total (epilogue kernel)
    double* local_out;
    double* grad_out;
    double* total_out;
};

// ---------------------------------------------------------------------------------
// per-source epilogue and the total

__device__ __forceinline__ double warp_dsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// an arrival counter increment with release (this thread's, and what it has seen of its
// CTA's, writes become visible first) and acquire (the other arrivals' writes become
// visible to the caller) at gpu scope; returns the count before it
__device__ __forceinline__ int arrive_acq_rel(int32_t* ctr) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], 1;" : "=r"(old) : "l"(ctr) : "memory");
    return old;
}


// ---------------------------------------------------------------------------------
// tasks of the compute warps

// One item on the four compute warps: warp w takes the chunks of 32 PX pixels w, w + 4,
// ... (PX consecutive pixels per thread); the thread's running sums wait in shared memory
// between chunks; a chunk that holds multiply covered pixels (warp-uniform) stashes its
// derivatives in shared memory while the other covering patches are evaluated.  Each
// warp leaves its FP32 sums (ll, d ll / d y, owned ll) in red (lane 0).
template <int MODE, int PX, int NPE, int NPD, int UNR>
__device__ __forceinline__ void item_compute(const ItemArgs& a, const ZItem& it, const uint8_t* stage,
                                             float* vs, float* spg, float* red) {
    constexpr int NV = (MODE == MODE_LL) ? 1 : 1 + NY;   // ll (+ d ll / d y)
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const int n = it.n_nm & 0xffff, nm = it.n_nm >> 16;
    const int npsf = it.nc_npsf >> 24, nc = it.nc_npsf & 0xffffff;
    const int npe = (a.ne + 1) >> 1, npd = (a.nd + 1) >> 1;
    const float* T = reinterpret_cast<const float*>(stage + ST_TBL);
    const float4* pxr = reinterpret_cast<const float4*>(stage + ST_PX);
    const ZCand* zc = reinterpret_cast<const ZCand*>(stage + ST_ZC);
    const float* vrec = reinterpret_cast<const float*>(stage + ST_VREC);
#pragma unroll
    for (int i = 0; i <= NV; ++i) vs[i * NTC] = 0.f;
    for (int c0 = w * 32 * PX; c0 < n; c0 += NWC * 32 * PX) {
        float X[PX], Y[PX], xv[PX], sky[PX];
        bool ok[PX];
#pragma unroll
        for (int p = 0; p < PX; ++p) {
            const int l = c0 + lane * PX + p;
            ok[p] = l < n;
            const float4 r = pxr[ok[p] ? l : n - 1];
            X[p] = r.x;
            Y[p] = r.y;
            xv[p] = r.z;
            sky[p] = r.w;
        }
        float Es[PX], Vs[PX], f0[PX], f1[PX];
        ProfileGrad pg[PX];
        own_source<MODE, PX, NPE, NPD, UNR>(T, npsf, npe, npd, X, Y, Es, Vs, f0, f1, pg);
        float E[PX], V[PX];
        bool owner[PX];
        if (c0 < nm) {
            // E and Var over every covering source in ascending source order; the item's
            // own source enters at its place
            if constexpr (MODE >= MODE_GRAD) {
#pragma unroll
                for (int p = 0; p < PX; ++p) {
                    const float* q = reinterpret_cast<const float*>(&pg[p]);
#pragma unroll
                    for (int f = 0; f < PG_F; ++f) spg[(p * PG_F + f) * NTC] = q[f];
                }
            }
            bool added = false;
#pragma unroll
            for (int p = 0; p < PX; ++p) {
                E[p] = sky[p];
                V[p] = 0.f;
                owner[p] = true;
            }
            for (int ci = 0; ci < nc; ++ci) {
                const ZCand c = ci < ZSTAGE ? zc[ci] : a.cands[it.c0 + ci];
                const float* R = ci < ZSTAGE ? vrec + ci * VFULL : a.ztbl + (size_t)c.patch * ZFULL;
                if (!added && c.src > it.src) {
#pragma unroll
                    for (int p = 0; p < PX; ++p) {
                        E[p] = __fadd_rn(E[p], Es[p]);
                        V[p] = __fadd_rn(V[p], Vs[p]);
                    }
                    added = true;
                }
                float Xc[PX], Yc[PX];
                bool in[PX], any = false;
#pragma unroll
                for (int p = 0; p < PX; ++p) {
                    const int xx = (int)X[p] - c.dx, yy = (int)Y[p] - c.dy;
                    in[p] = ok[p] && xx >= 0 && xx < c.w && yy >= 0 && yy < c.h;
                    Xc[p] = (float)xx;
                    Yc[p] = (float)yy;
                    any = any || in[p];
                    if (in[p] && c.src < it.src) owner[p] = false;
                }
                if (!__any_sync(0xffffffffu, any)) continue;
                float G0[PX], G1[PX];
                profile_value<PX, NPE, NPD>(R, c.npsf, npe, npd, Xc, Yc, G0, G1);
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
            if (!added)
#pragma unroll
                for (int p = 0; p < PX; ++p) {
                    E[p] = __fadd_rn(E[p], Es[p]);
                    V[p] = __fadd_rn(V[p], Vs[p]);
                }
            if constexpr (MODE >= MODE_GRAD) {
#pragma unroll
                for (int p = 0; p < PX; ++p) {
                    float* q = reinterpret_cast<float*>(&pg[p]);
#pragma unroll
                    for (int f = 0; f < PG_F; ++f) q[f] = spg[(p * PG_F + f) * NTC];
                }
            }
        } else {
#pragma unroll
            for (int p = 0; p < PX; ++p) {
                E[p] = __fadd_rn(sky[p], Es[p]);
                V[p] = Vs[p];
                owner[p] = true;
            }
        }
        float v[NV + 1];
#pragma unroll
        for (int i = 0; i <= NV; ++i) v[i] = vs[i * NTC];
#pragma unroll
        for (int p = 0; p < PX; ++p) {
            if (!ok[p]) continue;
            float vv[NV], ll;
#pragma unroll
            for (int i = 0; i < NV; ++i) vv[i] = v[i];
            pixel_terms<MODE, NV>(T, xv[p], E[p], V[p], Es[p], f0[p], f1[p], pg[p], vv, ll);
#pragma unroll
            for (int i = 0; i < NV; ++i) v[i] = vv[i];
            if (owner[p]) v[NV] += ll;
        }
#pragma unroll
        for (int i = 0; i <= NV; ++i) vs[i * NTC] = v[i];
    }
    // the warp's sums (FP32 shuffle tree) to red
#pragma unroll
    for (int i = 0; i <= NV; ++i) {
        float s = vs[i * NTC];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) red[i] = s;
    }
}

// the KL value and gradient of source s on one warp (with the domain check of its theta)
__device__ __forceinline__ void kl_task(const ItemArgs& a, int s, float* scr) {
    const int lane = threadIdx.x & 31;
    double* kth = reinterpret_cast<double*>(scr);
    double* kg = kth + NP;
    float* kthr = reinterpret_cast<float*>(kg + NP);
    for (int i = lane; i < NP; i += 32) {
        const double v = a.theta[(size_t)NP * s + i];
        kth[i] = v;
        kthr[i] = (float)v;
        theta_domain_check(i, v, a.status);
    }
    __syncwarp();
    const double v = kl_warp<float>(*a.md, kth, kthr, kg);
    __syncwarp();
    if (lane == 0) a.kl[s] = v;
    for (int i = lane; i < NP; i += 32) a.kl_grad[(size_t)NP * s + i] = kg[i];
}

// After an item, on the producer warp: the compute warps' sums added in warp order
// (FP64), the patch's chain rule applied (column j of d ll / d theta =
// sum_e k_e d ll / d y_{y_e}, FP64) and the item's record written.  In two parts: what
// the record needs from the item's stage and warp sums, read into registers (so that the
// stage can take its next item at once), then the FP64 arithmetic and the stores.
struct ItemSums {
    float r[NWC];       // lane < NS: the warps' sums of column lane
    float4 ch[2];       // the chain-rule columns lane, lane + 32
};

template <int MODE>
__device__ __forceinline__ ItemSums finish_load(const uint8_t* stage, const float* red) {
    const int lane = threadIdx.x & 31;
    constexpr int NS = (MODE == MODE_LL) ? 2 : 2 + NY;   // ll, (d ll / d y), owned ll
    ItemSums q;
#pragma unroll
    for (int w = 0; w < NWC; ++w) q.r[w] = lane < NS ? red[w * RED_W + lane] : 0.f;
    if constexpr (MODE >= MODE_GRAD) {
        const float4* ch = reinterpret_cast<const float4*>(stage + ST_CHAIN);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = lane + 32 * h;
            q.ch[h] = ch[c < NP ? c : 0];
        }
    }
    return q;
}

template <int MODE>
__device__ __forceinline__ void finish_store(const ItemArgs& a, int out, const ItemSums& q) {
    const int lane = threadIdx.x & 31;
    constexpr int NS = (MODE == MODE_LL) ? 2 : 2 + NY;
    double y = 0.0;
    if (lane < NS)
#pragma unroll
        for (int w = 0; w < NWC; ++w) y += (double)q.r[w];
    double* rec = a.part + (size_t)out * ZPCOLS;
    if (lane == 0) rec[0] = y;
    if (lane == NS - 1) rec[1] = y;
    if constexpr (MODE >= MODE_GRAD) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = lane + 32 * h;
            const float4 r = q.ch[h];
            const int yy = __float_as_int(r.w);
            const double y0 = __shfl_sync(0xffffffffu, y, 1 + (yy & 15));
            const double y1 = __shfl_sync(0xffffffffu, y, 1 + ((yy >> 4) & 15));
            const double y2 = __shfl_sync(0xffffffffu, y, 1 + ((yy >> 8) & 15));
            double g = (double)r.x * y0;
            g = fma((double)r.y, y1, g);
            g = fma((double)r.z, y2, g);
            if (c < NP) rec[2 + c] = g;
        }
    }
}

// ---------------------------------------------------------------------------------
// the producer warp

// the 64-byte record of queue slot q, a quarter per lane 0 .. 3 (past the end: an end
// marker)
__device__ __forceinline__ int4 load_task(const ItemArgs& a, int q) {
    const int lane = threadIdx.x & 31;
    if (q >= a.n_task) return make_int4(ZT_END, 0, 0, 0);
    return lane < 4 ? __ldcg(reinterpret_cast<const int4*>(a.tasks + q) + lane) : make_int4(0, 0, 0, 0);
}

// Put a task record (lanes 0 .. 3) in a stage and, for an item, wait for the tables it
// reads and start the bulk copies of its data into the stage; the stage's full barrier
// completes when they land (at once for the end marker).  Whole warp, every lane one of
// the item's patches (lane 0 its own, lane 1 + e candidate e), so that the patch ids,
// the ready flags and the copies of the candidates' value records take one memory round
// trip each instead of one per candidate.  all_built (every lane): every table was seen
// built, so no flag need be read.
template <int MODE>
__device__ void prepare(const ItemArgs& a, int4 rec, uint8_t* stage, ZTask* tk, uint64_t* full, bool& all_built) {
    const int lane = threadIdx.x & 31;
    const unsigned fullmask = 0xffffffffu;
    if (lane < 4) reinterpret_cast<int4*>(tk)[lane] = rec;
    __syncwarp();
    if (tk->kind != ZT_ITEM) {
        if (lane == 0) mbar_arrive_plain(full);
        return;
    }
    const ZItem it = tk->item;
    const int n = it.n_nm & 0xffff, nc = it.nc_npsf & 0xffffff, nc0 = nc < ZSTAGE ? nc : ZSTAGE;
    // candidate e's patch: named in the record for e < ZMAXC, else in the candidate list
    auto cand_patch = [&](int e) { return e < ZMAXC ? tk->cand[e] : a.cands[it.c0 + e].patch; };
#ifdef CELESTE_CHECK_BOUNDS
    {
        // the record's offsets into the pixel records, candidates, tables and item records;
        // a bad record ends this CTA's work (the status tells the caller)
        const int nm = it.n_nm >> 16, npsf = it.nc_npsf >> 24;
        bool ok = it.patch >= 0 && it.patch < a.n_patch && n >= 1 && n <= ZIMAX && nm <= n && it.pix >= 0 &&
                  it.pix + n <= a.n_sp && it.c0 >= 0 && (int64_t)it.c0 + nc <= a.n_zcand && it.out >= 0 &&
                  it.out < a.n_sitem && it.src >= 0 && it.src < a.n_src && npsf >= 1 && npsf <= MAXPSF;
        for (int j = lane; ok && j <= nc; j += 32) {
            const int pe = j == 0 ? it.patch : cand_patch(j - 1);
            ok = pe >= 0 && pe < a.n_patch;
        }
        ok = __all_sync(fullmask, ok);
        if (!ok) {
            if (lane == 0) {
                CEL_IN_BOUNDS(false, a.status);
                tk->kind = ZT_END;
                mbar_arrive_plain(full);
            }
            return;
        }
    }
#endif
    // this lane's patch: 0 the item's own, 1 + e candidate e (staged ones: e < nc0 <= 31)
    const int pl = lane == 0 ? it.patch : (lane - 1 < nc ? cand_patch(lane - 1) : -1);
    if (!all_built) {
        // lane 0 reads the built counter while the lanes read the flags of their patches
        bool built = false;
        if (lane == 0) built = load_acquire(a.ready + a.n_patch + 1) >= a.n_patch;
        else if (pl >= 0) wait_ready(a.ready + pl, a.status);
        for (int j = lane + 32; j <= nc; j += 32) wait_ready(a.ready + cand_patch(j - 1), a.status);
        if (lane == 0 && !built) wait_ready(a.ready + it.patch, a.status);
        all_built = __shfl_sync(fullmask, built, 0);
    }
    __syncwarp();
    // lane 0 announces the bytes before any copy is issued
    const unsigned tbl_bytes = MODE == MODE_LL ? VFULL * 4 : ZFULL * 4;
    const unsigned chain_bytes = MODE == MODE_LL ? 0u : NP * 16;
    if (lane == 0) {
        const unsigned bytes =
            tbl_bytes + chain_bytes + (unsigned)n * 16u + (unsigned)nc0 * (unsigned)(sizeof(ZCand) + VFULL * 4);
        mbar_expect_arrive(full, bytes);
    }
    __syncwarp();
    fence_proxy_async_global();
    fence_proxy_async_smem();   // the stage was last read through the generic proxy
    if (lane == 0) {
        bulk_g2s_tx(stage + ST_TBL, a.ztbl + (size_t)it.patch * ZFULL, tbl_bytes, full);
        if (chain_bytes) bulk_g2s_tx(stage + ST_CHAIN, a.zchain + (size_t)it.patch * NP, chain_bytes, full);
        bulk_g2s_tx(stage + ST_PX, a.px + it.pix, (unsigned)n * 16u, full);
        if (nc0 > 0) bulk_g2s_tx(stage + ST_ZC, a.cands + it.c0, (unsigned)nc0 * (unsigned)sizeof(ZCand), full);
    } else if (lane - 1 < nc0) {
        bulk_g2s_tx(stage + ST_VREC + (lane - 1) * VFULL * 4, a.ztbl + (size_t)pl * ZFULL, VFULL * 4, full);
    }
}

// ---------------------------------------------------------------------------------
// the kernels

// Tables and KL terms: warp u < n_patch builds the table and chain-rule record of the
// patch of torder[u] (the patches in the order the items first read them) and publishes
// it; warp n_patch + s computes the KL terms of source s (with the domain check of its
// theta).  The item kernel is launched as this kernel's programmatic dependent and waits
// for each table's flag, not for this kernel.
__global__ void __launch_bounds__(128) k_tables(ItemArgs a) {
    __shared__ __align__(16) float scr[4][SCR_W / 4];
    pdl_trigger();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int u = (int)blockIdx.x * 4 + w;
    if (u < a.n_patch) {
        const ZBuild g = a.torder[u];
        if (!CEL_IN_BOUNDS(g.patch >= 0 && g.patch < a.n_patch && g.img >= 0 && g.img < a.n_img_rec && g.src >= 0 &&
                               g.src < a.n_src,
                           a.status))
            return;
        build_patch_table(a.theta, g, a.img_tab, *a.md, a.ztbl, a.zchain, scr[w]);
        __syncwarp();
        if (lane == 0) publish_ready(a.ready + g.patch, a.ready + a.n_patch + 1);
    } else if (u < a.n_patch + a.n_src) {
        kl_task(a, u - a.n_patch, scr[w]);
    }
}

// The per-source epilogues and the total, after every item: the item kernel's
// programmatic dependent, waiting for it to finish.  One CTA of FIN_W warps per source:
// warp w adds the columns of the source's items w, w + FIN_W, ... in item order (FP64;
// lane c columns c and c + 32, loaded FIN_WIN items at a time before any is added), the
// CTA then adds the warps' sums in warp order and subtracts the KL: the local objective
// and gradient, and the source's share of the total (the ll of the pixels its items own,
// minus its KL).  The last CTA to finish adds the shares in source order (its warps over
// contiguous ranges, lanes strided, then warp order) and resets the counter.
constexpr int FIN_W = 4, FIN_WIN = 16;
__global__ void __launch_bounds__(32 * FIN_W) k_finish(ItemArgs a) {
    __shared__ double sh[FIN_W][64];
    __shared__ int s_last;
    pdl_wait();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, s = (int)blockIdx.x;
    const bool grad = a.mode >= MODE_GRAD;
    const int ncol = grad ? ZPCOLS : 2;
    int i0 = __ldcg(a.sitem_off + s), i1 = __ldcg(a.sitem_off + s + 1);
    if (!CEL_IN_BOUNDS(i0 >= 0 && i0 <= i1 && i1 <= a.n_sitem, a.status)) i0 = i1 = 0;
    const int cA = lane, cB = lane + 32;
    double sA = 0.0, sB = 0.0;
    for (int k0 = i0 + w; k0 < i1; k0 += FIN_W * FIN_WIN) {
        double vA[FIN_WIN], vB[FIN_WIN];
#pragma unroll
        for (int u = 0; u < FIN_WIN; ++u) {
            const int k = k0 + FIN_W * u;
            const double* r = a.part + (size_t)k * ZPCOLS;
            vA[u] = (k < i1 && cA < ncol) ? __ldcg(r + cA) : 0.0;
            vB[u] = (k < i1 && cB < ncol) ? __ldcg(r + cB) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < FIN_WIN; ++u) {
            if (k0 + FIN_W * u >= i1) break;
            sA += vA[u];
            sB += vB[u];
        }
    }
    sh[w][cA] = sA;
    sh[w][cB] = sB;
    s_last = 0;
    __syncthreads();
    if (w == 0) {
        double tA = 0.0, tB = 0.0;
#pragma unroll
        for (int v = 0; v < FIN_W; ++v) {
            tA += sh[v][cA];
            tB += sh[v][cB];
        }
        const double klv = __ldcg(a.kl + s);
        if (lane == 0 && a.local_out) a.local_out[s] = tA - klv;   // column 0: ll
        if (grad && a.grad_out) {
            if (cA >= 2) a.grad_out[(size_t)NP * s + cA - 2] = tA - __ldcg(a.kl_grad + (size_t)NP * s + cA - 2);
            if (cB < ncol) a.grad_out[(size_t)NP * s + cB - 2] = tB - __ldcg(a.kl_grad + (size_t)NP * s + cB - 2);
        }
        if (lane == 1 && a.total_out) {
            a.src_total[s] = tA - klv;   // column 1: owned ll
            s_last = arrive_acq_rel(a.grp_done) == (int)gridDim.x - 1;
        }
    }
    if (!a.total_out) return;
    __syncthreads();
    if (!s_last) return;
    const int n = a.n_src, per = (n + FIN_W - 1) / FIN_W;
    const int b0 = w * per, b1 = min(n, b0 + per);
    double acc = 0.0;
    for (int c0 = b0; c0 < b1; c0 += 32 * 16) {
        double x[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int i = c0 + lane + 32 * u;
            x[u] = i < b1 ? __ldcg(a.src_total + i) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) acc += x[u];
    }
    acc = warp_dsum(acc);
    __syncthreads();   // every warp is past its reads of sh
    if (lane == 0) sh[w][0] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int v = 0; v < FIN_W; ++v) t += sh[v][0];
        *a.total_out = t;
        a.grp_done[0] = 0;
    }
}

// The items, on persistent CTAs of four compute warps and a producer warp.  The producer
// keeps the next two items in the two stages: once the compute warps are done with item
// i it writes item i's record (the warps' sums in FP64, the chain rule) and puts item
// i + 2 in that stage; it holds one task record ahead in registers and one queue slot
// claimed beyond that.  CTA c's first two items are slots c and c + G (G CTAs); later
// slots come from the queue counter.
template <int MODE, int PX, int NPE, int NPD, int MINB, int UNR>
__global__ void __launch_bounds__(IT_THREADS) __maxnreg__(regs_for(MINB)) k_items(ItemArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    using L = Lay<PX>;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::bar);
    uint64_t* reduced = full + 2;
    ZTask* tasks = reinterpret_cast<ZTask*>(smem + L::task);
    float* red = reinterpret_cast<float*>(smem + L::red);
    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    pdl_trigger();   // the epilogue kernel may start (it waits for this grid to finish)
    if (t == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&reduced[0], NTC);
        mbar_init(&reduced[1], NTC);
        mbar_init_fence();
    }
    __syncthreads();
    int32_t* queue = a.ready + a.n_patch;
    if (w == NWC) {
        bool all_built = false;
        // slots 0 .. 2 G - 1 (G CTAs) are dealt out, one per stage of every CTA, so that
        // a queue of few items spreads over all CTAs; the rest are claimed one at a time
        const int G = (int)gridDim.x, base = 2 * G;
        int qa = 0;
        if (lane == 0) qa = base + atomicAdd(queue, 1);
        qa = __shfl_sync(0xffffffffu, qa, 0);
        const int4 r0 = load_task(a, (int)blockIdx.x), r1 = load_task(a, (int)blockIdx.x + G);
        int4 ra = load_task(a, qa);   // the record of the next item to prepare
        prepare<MODE>(a, r0, smem, &tasks[0], &full[0], all_built);
        prepare<MODE>(a, r1, smem + ST_BYTES, &tasks[1], &full[1], all_built);
        int qb = 0;   // lane 0: the slot after that
        if (lane == 0) qb = base + atomicAdd(queue, 1);
        for (int i = 0;; ++i) {
            const int b = i & 1;
            __syncwarp();
            if (tasks[b].kind == ZT_END) break;
            if (!mbar_wait_launch(&reduced[b], (i >> 1) & 1, a.status)) break;
            // item i is done: what its record needs, read from the stage; item i + 2's
            // copies into the stage; item i's record (FP64, off the compute warps)
            const int out = tasks[b].item.out;
            const ItemSums q = finish_load<MODE>(smem + b * ST_BYTES, red + b * NWC * RED_W);
            __syncwarp();
            prepare<MODE>(a, ra, smem + b * ST_BYTES, &tasks[b], &full[b], all_built);
            finish_store<MODE>(a, out, q);
            ra = load_task(a, __shfl_sync(0xffffffffu, qb, 0));
            if (lane == 0) qb = base + atomicAdd(queue, 1);
        }
        // this grid completes only after the table kernel (and its KL terms) has, so the
        // epilogue kernel that waits for this grid sees both, and the next evaluation's
        // flag reset follows both
        pdl_wait();
        return;
    }
    // compute warps
    float* vs = reinterpret_cast<float*>(smem + L::vs) + t;
    float* spg = reinterpret_cast<float*>(smem + L::pg) + t;
    for (int i = 0;; ++i) {
        const int b = i & 1;
        if (!mbar_wait_launch(&full[b], (i >> 1) & 1, a.status)) break;
        if (tasks[b].kind == ZT_END) break;
        const ZItem it = tasks[b].item;
        const uint8_t* stage = smem + b * ST_BYTES;
        float* rb = red + b * NWC * RED_W;
        item_compute<MODE, PX, NPE, NPD, UNR>(a, it, stage, vs, spg, rb + w * RED_W);
        // the producer adds the warps' sums and writes the item's record
        __syncwarp();
        mbar_arrive_plain(&reduced[b]);
    }
}

// ---------------------------------------------------------------------------------
// launch

template <int MODE, int PX, int NPE, int NPD, int MINB, int UNR>
struct ItemsKernel {
    static int per_sm;   // resident CTAs per SM (0: not yet set up)
    static cudaError_t setup() {
        if (per_sm > 0) return cudaSuccess;
        auto* fn = k_items<MODE, PX, NPE, NPD, MINB, UNR>;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, Lay<PX>::bytes);
        if (e != cudaSuccess) return e;
        int per = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, IT_THREADS, Lay<PX>::bytes);
        if (e != cudaSuccess) return e;
        per_sm = per > 0 ? per : 1;
        return cudaSuccess;
    }
    // a programmatic dependent launch of the table kernel before it on st
    static cudaError_t launch(const ItemArgs& a, int n_sm, cudaStream_t st) {
        cudaError_t e = setup();
        if (e != cudaSuccess) return e;
        int grid = per_sm * n_sm;
        if (grid > a.n_task) grid = a.n_task;
        if (grid < 1) return cudaSuccess;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3(IT_THREADS);
        cfg.dynamicSmemBytes = Lay<PX>::bytes;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k_items<MODE, PX, NPE, NPD, MINB, UNR>, a);
    }
};
template <int MODE, int PX, int NPE, int NPD, int MINB, int UNR>
int ItemsKernel<MODE, PX, NPE, NPD, MINB, UNR>::per_sm = 0;

// the model of the synthetic workloads and of the paper (6 exp + 8 dev profile
// components: 3 + 4 pairs) gets its loops unrolled for those counts
template <int MODE, int PX, int MINB, int UNR>
cudaError_t items_launch_v(const ItemArgs& a, int n_sm, cudaStream_t st) {
    if ((a.ne + 1) / 2 == 3 && (a.nd + 1) / 2 == 4) return ItemsKernel<MODE, PX, 3, 4, MINB, UNR>::launch(a, n_sm, st);
    return ItemsKernel<MODE, PX, -1, -1, MINB, 1>::launch(a, n_sm, st);
}

#define CEL_ITEM_VARIANTS(X)   \
    X(1, 2, 2, 7)              \
    X(2, 3, 2, 3)              \
    X(3, 2, 3, 2)              \
    X(4, 3, 2, 7)              \
    X(5, 3, 2, 2)
// variant codes (code, pixels per thread, CTAs per SM, unroll of the component-pair loop):
// 1 (2, 2, 7), 2 (3, 2, 3), 3 (2, 3, 2), 4 (3, 2, 7), 5 (3, 2, 2); two CTAs per SM leave
// 168 registers per thread, three 128
template <int MODE>
cudaError_t items_launch(const ItemArgs& a, int code, int n_sm, cudaStream_t st) {
    switch (code) {
#define CEL_CASE(c, px, minb, unr) \
    case c: return items_launch_v<MODE, px, minb, unr>(a, n_sm, st);
        CEL_ITEM_VARIANTS(CEL_CASE)
#undef CEL_CASE
        default: return items_launch_v<MODE, 2, 2, 7>(a, n_sm, st);
    }
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            n = v;
        else
            n = 1;
    }
    return n;
}

template <int MODE>
cudaError_t items_setup_mode() {
    cudaError_t e = cudaSuccess;
#define CEL_SETUP(c, px, minb, unr)                                                    \
    if (e == cudaSuccess) e = ItemsKernel<MODE, px, 3, 4, minb, unr>::setup();           \
    if (e == cudaSuccess) e = ItemsKernel<MODE, px, -1, -1, minb, 1>::setup();
    CEL_ITEM_VARIANTS(CEL_SETUP)
#undef CEL_SETUP
    return e;
}

}  // namespace

// shared-memory limits and resident CTAs of every item-kernel variant, set once outside
// any stream capture
cudaError_t prime_items_kernels() {
    cudaError_t e = items_setup_mode<MODE_LL>();
    if (e == cudaSuccess) e = items_setup_mode<MODE_GRAD>();
    return e;
}

cudaError_t launch_items_stage(const DevProblem& P, int stage, int mode, cudaStream_t st, const double* d_theta,
                               double* d_local, double* d_grad, double* d_total) {
    if (P.n_src == 0 || !P.ztasks) return cudaSuccess;
    ItemArgs a{};
    a.tasks = P.ztasks;
    a.n_task = P.n_task;
    a.torder = P.ztorder;
    a.cands = P.zcands;
    a.px = P.zpx;
    a.md = P.model;
    a.theta = d_theta;
    a.ztbl = P.ztbl;
    a.zchain = P.zchain;
    a.ready = P.zready;
    a.geo_tab = P.geo;
    a.img_tab = P.img;
    a.part = P.spart;
    a.ne = P.model_ne;
    a.nd = P.model_nd;
    a.n_patch = P.n_patch;
    a.n_src = P.n_src;
    a.n_sp = P.n_sp;
    a.n_zcand = P.n_zcand;
    a.n_sitem = P.n_sitem;
    a.n_img_rec = P.n_img_rec;
    a.kl = P.kl;
    a.kl_grad = P.kl_grad;
    a.status = P.status;
    a.mode = mode;
    a.sitem_off = P.sitem_off;
    a.grp_done = P.zf_done;
    a.src_total = P.src_total;
    a.local_out = d_local;
    a.grad_out = mode >= MODE_GRAD ? d_grad : nullptr;
    a.total_out = d_total;
    if (stage == 0) {
        // ready flags, the queue counter and the built-table count start at 0
        cudaError_t e = cudaMemsetAsync(P.zready, 0, sizeof(int32_t) * ((size_t)P.n_patch + 2), st);
        if (e != cudaSuccess) return e;
        k_tables<<<(P.n_patch + P.n_src + 3) / 4, 128, 0, st>>>(a);
        return cudaGetLastError();
    }
    if (stage == 1) {
        const int n_sm = sm_count();
        return mode == MODE_LL ? items_launch<MODE_LL>(a, P.tune_items, n_sm, st)
                               : items_launch<MODE_GRAD>(a, P.tune_items, n_sm, st);
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)P.n_src);
    cfg.blockDim = dim3(32 * FIN_W);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_finish, a);
}

cudaError_t launch_items(const DevProblem& P, int mode, cudaStream_t st, const double* d_theta, double* d_local,
                         double* d_grad, double* d_total) {
    for (int stage = 0; stage < 3; ++stage) {
        const cudaError_t e = launch_items_stage(P, stage, mode, st, d_theta, d_local, d_grad, d_total);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace cel
