// Internal layout shared by the CUDA translation units of libceleste (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "celeste.h"

namespace cel {

// Device-side bounds checks, compiled in with -DCELESTE_CHECK_BOUNDS: an index outside its
// buffer (a pixel outside its patch, a tile-list or candidate entry out of range, a table
// or record offset past its array) records CELESTE_ERR_BOUNDS in the status word and the
// access is skipped; nothing traps.  Without the flag every check is the constant true.
#ifdef CELESTE_CHECK_BOUNDS
__device__ __forceinline__ bool bound_ok(bool c, int32_t* status) {
    if (!c) atomicExch(status, (int32_t)CELESTE_ERR_BOUNDS);
    return c;
}
#define CEL_IN_BOUNDS(cond, status) ::cel::bound_ok((cond), (status))
#else
#define CEL_IN_BOUNDS(cond, status) true
#endif

constexpr int NP = CELESTE_NPARAM;      // 44 constrained parameters per source
constexpr int NT = CELESTE_NFREE;       // 41 free parameters (trust-region coordinates)
constexpr int MAXPSF = CELESTE_MAX_PSF;
constexpr int MAXPROF = CELESTE_MAX_PROFILE;
constexpr int NCOMP = CELESTE_NPRIOR_COMP;

// constrained parameter indices (see celeste.h)
enum : int { P_U = 0, P_EDEV = 2, P_AXIS = 3, P_ANGLE = 4, P_SCALE = 5, P_R1 = 6, P_R2 = 8,
             P_C1 = 10, P_C2 = 18, P_A = 26, P_K = 28 };

// Per (source, image) the pixel terms depend on theta only through twelve
// intermediate variables y; the kernels differentiate wrt y and a per-source
// epilogue applies the chain rule dy/dtheta.
enum : int { Y_A0 = 0, Y_A1, Y_EL0, Y_EL20, Y_EL1, Y_EL21, Y_MX, Y_MY, Y_EDEV, Y_GXX, Y_GXY,
             Y_GYY, NY };
constexpr int NYH = NY * (NY + 1) / 2;   // packed upper triangle of the y-Hessian

// Work-item partial record (doubles): [0] sum of ll over the item's pixels; gradient
// mode: [1..44] gradient wrt theta (the chain rule applied per item); Hessian mode:
// [1..NY] gradient wrt y, [1+NY ..) packed y-Hessian.
constexpr int PART_LL = 0, PART_G = 1, PART_H = 1 + NY, PART_TH = 1;
constexpr int NPART = 1 + NY + NYH;
// Per-item partial record of the FP32 value / gradient kernel (doubles): [0] ll of the
// item's pixels, [1] ll of the pixels the item owns (its share of the total), [2 .. 2 + NP)
// d ll / d theta of its source (the patch's chain rule applied per item).
constexpr int ZPCOLS = 2 + NP;

// Mixture table of one (source, patch), in units of the pixel precision R:
//   header [0..7]: a0 a1 E[l|star] E[l^2|star] E[l|gal] E[l^2|gal] iota 0
//   means  [8..15]: pixel-frame mean of PSF component k (x, y)
//   star   [16 + 8k]: qa qb qc qd pxx pxy pyy c
//   dG     [48 + 3q + c]: d(Gxx, Gxy, Gyy)[c] / d(e_axis, e_angle, e_scale)[q] (chain rule)
//   G      [57..59]: the galaxy covariance Gxx Gxy Gyy in the pixel frame
//   galaxy [64 + 12 (k nprof + j)]: qa qb qc qd pxx pxy pyy c dc nu 0 0
// Component density: c * exp2(qa dx^2 + qb dx dy + qc dy^2 + qd) with
// (qa, qb, qc) = -log2(e) (Pxx/2, Pxy, Pyy/2) and qd = -log2(2 pi sqrt(det C)).
constexpr int T_HDR = 0, T_MEAN = 8, T_STAR = 16, STAR_STRIDE = 8, T_DG = 48, T_G = 57, T_GAL = 64,
              GAL_STRIDE = 12;
constexpr int TBL_STRIDE = T_GAL + MAXPSF * MAXPROF * GAL_STRIDE;   // 832
static_assert(T_MEAN + 2 * MAXPSF <= T_STAR && T_STAR + MAXPSF * STAR_STRIDE <= T_DG &&
                  T_DG + 9 <= T_G && T_G + 3 <= T_GAL,
              "mixture-table fields overlap");
constexpr int H_A0 = 0, H_A1 = 1, H_EL0 = 2, H_EL20 = 3, H_EL1 = 4, H_EL21 = 5, H_IOTA = 6;

// floats of one patch's whitened-frame table (item_kernels.cu): a value part (header 16,
// per PSF component 8 + 8 per pair of profile components) and a gradient part (per PSF
// component 12 + 12 per pair); each profile group padded to an even count
constexpr int ZFULL_FLOATS = 16 + MAXPSF * (8 + ((MAXPROF + 2) / 2) * 8) + MAXPSF * (12 + ((MAXPROF + 2) / 2) * 12);
constexpr int CHUNK = 256;   // pixels per work item (one CTA)
constexpr int ZIMAX = 512;   // most pixels per item of the FP32 value / gradient kernel
constexpr int ZMAXC = 4;     // other covering patches named inline in such an item's queue record
constexpr int ZSTAGE = 12;   // other covering patches whose value records an item stages (more are
                             // read in place)
constexpr int TILE = 16;     // gather tiles are TILE x TILE pixels

struct ImgMeta {
    int64_t px_off;          // offset of the image in the concatenated pixel / map buffers
    int64_t tg_off;          // offset of the image's tile grid (tile id per cell, -1 = none)
    int32_t H, W, band, npsf;
    int32_t has_sky_map, tgw; // tgw: tile-grid cells per row
    double sky, iota;
    double A[4], t[2];
    double psf[MAXPSF][6];
    float psf_f[MAXPSF][6];  // the same in FP32 (conversions run on the narrow FP64 pipe)
    float A_f[4];
    // whitened-frame constants of PSF component k (item_kernels.cu), from FP64 on the host:
    //   psf_li:  L^-1 = [[li0, 0], [li1, li2]] with Sigma_k = L L^T (Cholesky)
    //   psf_cs:  log2|alpha_k| - log2(2 pi) - log2(det Sigma_k) / 2 (-inf for alpha_k = 0)
    //   psf_sg:  sign of alpha_k (+1 for alpha_k = 0)
    //   psf_dm:  (det A / sqrt(det Sigma_k))^2, so det(L^-1 G L^-T) = psf_dm sigma^4 rho^2
    float psf_li[MAXPSF][3];
    float psf_cs[MAXPSF];
    float psf_sg[MAXPSF];
    float psf_dm[MAXPSF];
    float sky_f;
    float iota_f;
};

struct PatchGeo {
    int32_t img, x0, y0, w, h, src;
    int64_t sp_off;          // offset in the per-(source, pixel) buffers
    int32_t item0, nitem;    // work items covering this patch
};

struct WorkItem {
    int32_t patch, q0, n, src;
};

// One item of the FP32 value / gradient kernel: n <= ZIMAX consecutive pixel records of
// one patch (from pix; the patch's multiply covered pixels come first, nm of them), its
// partial record (out), source, the other patches covering any of its multiply covered
// pixels (zcands[c0 .. c0 + nc), ascending patch id) and npsf of its image.
struct ZItem {
    int32_t patch, n_nm, out, src;   // n_nm = n | nm << 16
    int64_t pix;
    int32_t c0, nc_npsf;             // nc | npsf << 24
};

// One entry of the FP32 value / gradient kernel's queue: an item (kind ZT_ITEM) with the
// patches of its first ZMAXC candidates, so that one 64-byte load gives everything the
// item's copies need; ZT_END marks the end of the queue.
enum : int32_t { ZT_ITEM = 0, ZT_END = 3 };
struct ZTask {
    int32_t kind, index, pad0, pad1;
    ZItem item;
    int32_t cand[ZMAXC];
};

// Another patch covering pixels of a multiply covered item: its table index, its origin
// relative to the item's patch origin, size, source and PSF component count.
struct ZCand {
    int32_t patch, dx, dy, w, h, src, npsf, pad;
};

// What the table kernel needs of a patch to build its table: the patch, its image and
// source, and its origin in the image.
struct ZBuild {
    int32_t patch, img, src, pad;
    double ox, oy;   // the image map's translation minus the patch origin (FP64, from the host)
};

struct Tile {
    int32_t img, x0, y0, list_off, list_n, pad[3];
};

struct ModelDev {
    int32_t n_exp, n_dev;
    double prof_w[MAXPROF], prof_nu[MAXPROF];
    double prior_star;
    double prior_r[2][2];
    double prior_w[2][NCOMP];
    double prior_mu[2][NCOMP][4];
    double prior_P[2][NCOMP][16];     // inverse covariances
    double prior_logdet[2][NCOMP];
    double prior_logw[2][NCOMP];      // log w_id, log Phi_i, log pv_i
    double prior_logphi[2];
    double prior_logpv[2];
    double prior_inv_pv[2];
    // FP32 copies for the FP32 path
    float prof_w_f[MAXPROF], prof_nu_f[MAXPROF];
    float prior_star_f;
    float prior_r_f[2][2];
    float prior_w_f[2][NCOMP];
    float prior_mu_f[2][NCOMP][4];
    float prior_P_f[2][NCOMP][16];
    float prior_logdet_f[2][NCOMP];
    float prof_lw_f[MAXPROF];         // log2 of the profile weights (-inf for a zero weight)
};

// FP32 copies of the model / image constants, filled once on the host
inline void fill_float_copies(ModelDev& m) {
    for (int i = 0; i < 2; ++i) {
        for (int d = 0; d < NCOMP; ++d) m.prior_logw[i][d] = std::log(m.prior_w[i][d]);
        m.prior_logphi[i] = std::log(i == 0 ? m.prior_star : 1.0 - m.prior_star);
        m.prior_logpv[i] = std::log(m.prior_r[i][1]);
        m.prior_inv_pv[i] = 1.0 / m.prior_r[i][1];
    }
    for (int j = 0; j < MAXPROF; ++j) {
        m.prof_w_f[j] = (float)m.prof_w[j];
        m.prof_nu_f[j] = (float)m.prof_nu[j];
        m.prof_lw_f[j] = (float)std::log2(m.prof_w[j]);
    }
    m.prior_star_f = (float)m.prior_star;
    for (int i = 0; i < 2; ++i) {
        for (int c = 0; c < 2; ++c) m.prior_r_f[i][c] = (float)m.prior_r[i][c];
        for (int d = 0; d < NCOMP; ++d) {
            m.prior_w_f[i][d] = (float)m.prior_w[i][d];
            m.prior_logdet_f[i][d] = (float)m.prior_logdet[i][d];
            for (int j = 0; j < 4; ++j) m.prior_mu_f[i][d][j] = (float)m.prior_mu[i][d][j];
            for (int j = 0; j < 16; ++j) m.prior_P_f[i][d][j] = (float)m.prior_P[i][d][j];
        }
    }
}
inline void fill_float_copies(ImgMeta& im) {
    for (int k = 0; k < MAXPSF; ++k)
        for (int c = 0; c < 6; ++c) im.psf_f[k][c] = (float)im.psf[k][c];
    for (int k = 0; k < 4; ++k) im.A_f[k] = (float)im.A[k];
    im.sky_f = (float)im.sky;
    im.iota_f = (float)im.iota;
    const double detA = im.A[0] * im.A[3] - im.A[1] * im.A[2];
    for (int k = 0; k < MAXPSF; ++k) {
        im.psf_li[k][0] = im.psf_li[k][1] = im.psf_li[k][2] = 0.f;
        im.psf_cs[k] = -INFINITY;
        im.psf_sg[k] = 1.f;
        im.psf_dm[k] = 0.f;
        if (k >= im.npsf) continue;
        const double* ps = im.psf[k];
        const double l11 = std::sqrt(ps[3]), l21 = ps[4] / l11, l22 = std::sqrt(ps[5] - l21 * l21);
        const double det = ps[3] * ps[5] - ps[4] * ps[4];
        im.psf_li[k][0] = (float)(1.0 / l11);
        im.psf_li[k][1] = (float)(-l21 / (l11 * l22));
        im.psf_li[k][2] = (float)(1.0 / l22);
        im.psf_cs[k] = (float)(std::log2(std::fabs(ps[0])) - 2.6514961294723187 /* log2(2 pi) */ - 0.5 * std::log2(det));
        im.psf_sg[k] = ps[0] < 0 ? -1.f : 1.f;
        im.psf_dm[k] = (float)(detA * detA / det);
    }
}

// precision-selected views of those constants
__device__ inline const double* psf_row(const ImgMeta& im, int k, double) { return im.psf[k]; }
__device__ inline const float* psf_row(const ImgMeta& im, int k, float) { return im.psf_f[k]; }
__device__ inline double wcs_of(const ImgMeta& im, int k, double) { return im.A[k]; }
__device__ inline float wcs_of(const ImgMeta& im, int k, float) { return im.A_f[k]; }
__device__ inline double prof_w_of(const ModelDev& m, int j, double) { return m.prof_w[j]; }
__device__ inline float prof_w_of(const ModelDev& m, int j, float) { return m.prof_w_f[j]; }
__device__ inline double prof_nu_of(const ModelDev& m, int j, double) { return m.prof_nu[j]; }
__device__ inline float prof_nu_of(const ModelDev& m, int j, float) { return m.prof_nu_f[j]; }

// colour coefficient beta_bj: log l_b = log r + sum_j beta_bj c_j, colours c_j the
// log ratio of band j+1 to band j and r the reference (r, index 2) band brightness.
__host__ __device__ inline double color_beta(int band, int j) {
    const int ref = 2;
    if (band < ref) return (j >= band && j < ref) ? -1.0 : 0.0;
    if (band > ref) return (j >= ref && j < band) ? 1.0 : 0.0;
    return 0.0;
}

__host__ __device__ inline int yh_index(int a, int b) {   // packed upper triangle, a <= b
    return a * NY - (a * (a - 1)) / 2 + (b - a);
}

// ---------------------------------------------------------------------------------
// launchers (pixel_kernels.cu, source_kernels.cu)

enum Mode : int { MODE_LL = 0, MODE_GRAD = 1, MODE_HESS = 2 };

struct DevProblem {
    int32_t n_img, n_src, n_patch, n_item, n_tile, npsf_max, nprof;
    int32_t tune_contrib, tune_adjoint;   // FP32 map-pass / adjoint kernel codes of the Hessian, fit
                                          // and allocation-free paths (0 = default)
    int64_t n_px, n_sp;
    int32_t max_src_patches;              // most patches of one source (k_prep's grid)
    const ImgMeta* img;
    const float* pixels;
    const float* sky_map;
    const PatchGeo* geo;
    const WorkItem* items;
    const Tile* tiles;
    const int32_t* tile_list;
    const int32_t* tile_grid;
    const int32_t* patch_off;
    const ModelDev* model;
    double* tbl64;
    float* tbl32;
    void* spE;
    void* spE2;
    void* emap;
    void* vmap;
    const uint8_t* single;   // per (source, pixel): 1 when no other patch covers the pixel (nullable)
    double* item_ll;         // per work item: ll summed over its singly covered pixels
    double* item_part;
    double* tile_ll;
    double* kl;
    double* kl_grad;         // [n_src][44] KL gradient, written by k_prep (nullable: no KL in prep)
    double* src_total;       // [n_src] each source's share of the total ELBO (k_finalize)
    int32_t* done;           // k_finalize completion counter, 0 between launches
    double* tot_part;        // [64] k_total slice sums
    int32_t* tot_done;       // k_total completion counter, 0 between launches
    // The FP32 value / gradient kernel's work (item_kernels.cu): a source's items are
    // contiguous in partial order (sitem_off); ztasks null when there is none.
    const int32_t* sitem_off;    // [n_src + 1]
    int n_sitem, n_smulti;       // items; those holding multiply covered pixels
    double* spart;               // [n_sitem][ZPCOLS] per-item partials
    int32_t* zf_done;            // finished sources of the FP32 epilogue kernel, 0 between launches
    const int32_t* src_active;   // per source: 0 = skip its work (the fit's converged batch
                                 // sources); nullable = every source works
    // the FP32 value / gradient item kernel (item_kernels.cu)
    const ZTask* ztasks;         // [n_task] the work queue
    int32_t n_task;
    const ZBuild* ztorder;       // [n_patch] the patches' build records, in the order the items first read them
    const ZCand* zcands;
    const float4* zpx;           // per item pixel: (column, row in the patch, counts, sky)
    float* ztbl;                 // [n_patch][ZFULL_FLOATS] whitened-frame tables (FP32)
    float4* zchain;              // [n_patch][NP] chain-rule records of the patches
    int32_t* zready;             // [n_patch] table ready flags, then the queue counter and the
                                 // count of built tables (reset before each launch)
    int32_t tune_items;          // item kernel variant, 1 .. 5 (pixels per thread, CTAs per SM,
                                 // unroll; item_kernels.cu); 0 = the default, 1
    int32_t model_ne, model_nd;     // exp / dev profile components of the model
    int32_t* queue;          // [2] work queue of the FP64 / Hessian map pass's persistent variants
                             // (next item, finished CTAs), 0 between launches (nullable: those
                             // variants fall back to one CTA per item)
    int32_t* status;
    // sizes the bounds checks compare against (CELESTE_CHECK_BOUNDS)
    int32_t n_img_rec;           // image records (the images, then per-patch map copies)
    int32_t n_zcand;             // candidate records of the FP32 items
    int64_t n_tile_list;         // entries of tile_list
    int64_t n_tile_grid;         // entries of tile_grid
};

// Packed lower-triangle order of a side-N triangle, built at compile time: entry
// idx = a (a + 1) / 2 + b (0 <= b <= a < N) holds a << 8 | b.  A triangle of side m < N
// is the first m (m + 1) / 2 entries.
template <int N>
struct PackedTriangle {
    uint16_t v[N * (N + 1) / 2];
};
template <int N>
constexpr PackedTriangle<N> packed_triangle() {
    PackedTriangle<N> t{};
    int idx = 0;
    for (int a = 0; a < N; ++a)
        for (int b = 0; b <= a; ++b) t.v[idx++] = (uint16_t)(a << 8 | b);
    return t;
}

// What the tile-list (CSR) bounds checks of k_gather and k_other compare against
struct CsrBounds {
    int32_t n_patch, n_tile;
    int64_t n_tile_list, n_tile_grid;
    int32_t* status;
};
inline CsrBounds csr_bounds(const DevProblem& P) {
    return CsrBounds{P.n_patch, P.n_tile, P.n_tile_list, P.n_tile_grid, P.status};
}

void set_last_error(const char* msg);

// 4 x 4 symmetric positive-definite inverse and log-determinant by Cholesky (false when
// not positive definite)
bool chol_inverse4(const double* S, double* inv, double* logdet);
// The model's device record, with every check of the model description (profile
// weights finite and >= 0, variances > 0, prior_star in (0, 1), brightness-prior
// variances > 0, colour-prior weights > 0 and covariances positive definite); on a
// failure the status and *why (a static message).  Shared by every entry point.
celeste_status build_model_dev(const celeste_model* model, ModelDev& md, const char** why);

// task_of (host, one entry per source, nullable): a region-task stage, every task fitted
// against the stage-start parameters of the sources outside it
celeste_status fit_sources_impl(celeste_problem* pr, double* theta_inout, const int32_t* which,
                                int32_t n_which, const celeste_fit_options* opts,
                                int32_t* iters_out, int32_t* status_out, double* elbo_out,
                                celeste_status (*elbo_fn)(celeste_problem*, const double*, int32_t,
                                                          double*, double*),
                                const int32_t* task_of = nullptr);
// celeste_fit_sources with its argument checks, and the region-task stage mode above
celeste_status fit_sources_checked(celeste_problem* pr, double* theta_inout, const int32_t* which,
                                   int32_t n_which, const celeste_fit_options* opts, int32_t* iters_out,
                                   int32_t* status_out, double* elbo_out, const int32_t* task_of);

void prime_persistent_grids();
cudaError_t prime_items_kernels();
// total = tile ll sums + item ll sums - KL (after the gather and every item ll)
cudaError_t launch_total(const DevProblem& P, double* d_total, cudaStream_t st);
// tables (and, with_kl, the KL value / gradient and the domain check) of every source
cudaError_t launch_prep(const DevProblem& P, const double* d_theta, int precision,
                        cudaStream_t st, bool with_kl = true);
// contrib / adjoint over the items idx[0 .. n) (idx null: items 0 .. n; n < 0: all items)
cudaError_t launch_contrib(const DevProblem& P, int precision, cudaStream_t st,
                           const int32_t* idx = nullptr, int n = -1);
// The FP32 value (MODE_LL) or value + gradient (MODE_GRAD) evaluation (item_kernels.cu):
// the patches' whitened-frame tables, the KL value / gradient and the domain check of
// theta, every item, the per-source epilogue (local objective, gradient; each nullable)
// and the total (nullable); launch_items_stage below launches them one stage at a time
cudaError_t launch_items(const DevProblem& P, int mode, cudaStream_t st, const double* d_theta, double* d_local,
                         double* d_grad, double* d_total);
// its three launches one at a time: stage 0 the tables and KL terms (after resetting the
// ready flags), 1 the items, 2 the per-source epilogues and the total
cudaError_t launch_items_stage(const DevProblem& P, int stage, int mode, cudaStream_t st, const double* d_theta,
                               double* d_local, double* d_grad, double* d_total);
cudaError_t launch_gather(const DevProblem& P, int precision, cudaStream_t st);
cudaError_t launch_adjoint(const DevProblem& P, int precision, int mode, cudaStream_t st,
                           const int32_t* idx = nullptr, int n = -1);
cudaError_t launch_hess_pixels(const DevProblem& P, int precision, cudaStream_t st);
cudaError_t launch_finalize(const DevProblem& P, const double* d_theta, int precision, int mode,
                            double* d_total, double* d_local, double* d_grad, double* d_hess,
                            cudaStream_t st);

// catalog rows (one thread per source) and the Table II error summary (one CTA)
cudaError_t launch_catalog(int n, const double* d_theta, double* d_cat, int32_t* d_status, cudaStream_t st);
cudaError_t launch_score(int n, const double* d_est, const double* d_true, double* d_score, cudaStream_t st);
// E = sky and Var = 0 over every pixel of every image (FP64, concatenated image layout)
cudaError_t launch_fill_sky(const DevProblem& P, double* d_e, double* d_v, cudaStream_t st);

// Programmatic dependent launch (sm_90 and later): a kernel launched with the
// programmatic-serialization attribute may start while its predecessor in the stream is
// still running; pdl_wait() blocks until that predecessor has completed and its writes are
// visible (a no-op for an ordinary launch), pdl_trigger() lets the dependent start early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

}  // namespace cel
