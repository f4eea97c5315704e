/*
 * celeste.h -- C ABI of the GB300 Celeste hot path: the variational objective (ELBO)
 * of the Celeste astronomical-catalog model over every active pixel of every
 * source's patch, its gradient and per-source Hessian, and the per-source
 * trust-region Newton fit that consumes them.
 *
 * Paper: Regier et al., "Cataloging the Visible Universe through Bayesian Inference
 * at Petascale" (arXiv 1801.10277).
 *   - Section III: pixels x_nm ~ Poisson(F_nm); per source a star/galaxy indicator,
 *     log-normal reference-band brightness, Gaussian colours (log ratios of adjacent
 *     bands), position and galaxy shape; image metadata Lambda_n (PSF, sky,
 *     calibration, WCS); ELBO  L(theta) = E_q[log p(x, z) - log q(z)]  (Eq. 1).
 *   - Section IV: 44 parameters per source.
 *   - Section IV-D: block coordinate ascent, one source's 44 parameters per block;
 *     Newton steps with exact Hessians inside a trust region.
 *   - Section VI-B: cost counted per active pixel visit.
 * The paper defers the exact variational family and the expected log-likelihood to
 * Regier et al. (ICML 2015).  This library implements the reading:
 *     E[F]   = sky + iota * sum_s sum_i a_i E[l_si] g_si(pixel)
 *     Var[F] = sum_s ( sum_i a_i iota^2 E[l_si^2] g_si^2 - (sum_i a_i iota E[l_si] g_si)^2 )
 *     E_q[log F] ~= log E[F] - Var[F] / (2 E[F]^2)          (second-order delta method)
 *     ELBO = sum over the union of patches of  x (log E - Var / (2 E^2)) - E
 *            - sum_s KL(q_s || prior)                      (log x! dropped)
 * with g the PSF mixture (star) or the PSF convolved with exp/dev Gaussian-mixture
 * profiles (galaxy), evaluated at integer pixel centres and truncated to the
 * source's patch.
 *
 * PARAMETER LAYOUT (44 doubles per source, row-major [n_src][44], constrained):
 *   0,1 u (world position)   2 e_dev   3 e_axis (minor/major)   4 e_angle (radians,
 *   counter-clockwise from +x)   5 e_scale (half-light radius, px)
 *   6,7 r1[type]  8,9 r2[type] (mean, variance of log r-band brightness, nmgy)
 *   10..17 c1[type][4]  18..25 c2[type][4] (colour means, variances; colours are
 *   u-g, g-r, r-i, i-z log ratios)   26,27 a[type] (P(star), P(galaxy))
 *   28..43 k[type][8] (colour-prior component responsibilities).  type 0 = star.
 * Bands: 0..4 = u g r i z; the reference band is r (2).
 *
 * CONVENTIONS
 *   - Ownership: every pointer argument is owned by the caller.  celeste_problem_create
 *     copies what it needs to the current CUDA device; the caller may free its
 *     arrays afterwards.  The problem owns its device memory until destroy.
 *   - Host vs device: functions without the _device suffix take HOST pointers and
 *     synchronise before returning.  _device variants take DEVICE pointers and a
 *     cudaStream_t (passed as void*), enqueue work on that stream and return
 *     without synchronising.
 *   - Errors: every call returns a celeste_status; nothing aborts and no kernel
 *     traps.  celeste_last_error() returns a thread-local message for the last
 *     failure of the calling thread.
 *   - Threading: calls on one problem handle are not thread-safe; different handles
 *     are independent.
 *   - Precision: CELESTE_FP64 evaluates every pixel in double; CELESTE_FP32_ACC64
 *     evaluates per-pixel mixture and likelihood arithmetic in float and keeps
 *     per-source accumulation (across warps, work items and patches), the chain rule,
 *     the KL terms and the trust-region solve in double.
 */
#ifndef CELESTE_H
#define CELESTE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t celeste_status;

enum {
    CELESTE_OK = 0,
    CELESTE_ERR_ARG = -1,        /* invalid argument, size or parameter value */
    CELESTE_ERR_NOT_PD = -2,     /* a PSF or prior covariance is not positive definite */
    CELESTE_ERR_NONFINITE = -3,  /* NaN/Inf in inputs, or produced for some source */
    CELESTE_ERR_CUDA = -4,       /* a CUDA runtime call failed */
    CELESTE_ERR_TIMEOUT = -5,    /* a bounded device-side wait gave up */
    CELESTE_ERR_NOMEM = -6,      /* device allocation failed */
    CELESTE_ERR_BOUNDS = -7      /* a device-side bounds check failed (libraries built with
                                    CELESTE_CHECK_BOUNDS only; the access was skipped) */
};

enum { CELESTE_FP64 = 0, CELESTE_FP32_ACC64 = 1 };

enum { CELESTE_NPARAM = 44, CELESTE_NFREE = 41, CELESTE_MAX_PSF = 4, CELESTE_MAX_PROFILE = 16,
       CELESTE_NPRIOR_COMP = 8 };

/* One image (Section III, metadata Lambda_n). */
typedef struct {
    int32_t band;              /* 0..4 = u g r i z */
    int32_t height, width;     /* pixels */
    const float* pixels;       /* [height][width] photon counts, row-major */
    double sky;                /* sky background, counts per pixel (used when sky_map is NULL) */
    const float* sky_map;      /* optional [height][width] sky counts, or NULL */
    double nmgy_per_count;     /* calibration; iota = 1 / nmgy_per_count counts per nanomaggy */
    double wcs[6];             /* affine world->pixel: pixel = A u + t, A = {wcs[0] wcs[1]; wcs[2] wcs[3]}, t = {wcs[4], wcs[5]} */
    int32_t n_psf;             /* 1..CELESTE_MAX_PSF */
    const double* psf;         /* [n_psf][6]: weight, offset x, offset y, Sxx, Sxy, Syy (pixels) */
} celeste_image;

/* Galaxy profiles and priors (Section III: Phi, Upsilon, Xi). */
typedef struct {
    int32_t n_exp, n_dev;      /* n_exp + n_dev <= CELESTE_MAX_PROFILE */
    const double* exp_mix;     /* [n_exp][2]: weight, variance of a circular Gaussian, unit half-light radius */
    const double* dev_mix;     /* [n_dev][2] */
    double prior_star;         /* Phi: prior P(star), in (0, 1) */
    const double* prior_r;     /* [2][2]: mean, variance of log r-band brightness per type */
    int32_t n_color_comp;      /* must be CELESTE_NPRIOR_COMP (8) */
    const double* prior_c;     /* [2][n_color_comp][21]: weight, mean[4], covariance[4][4] */
} celeste_model;

/* One source's active region in one image: a rectangle of pixel centres, inside the image. */
typedef struct {
    int32_t image;
    int32_t x0, y0, w, h;
} celeste_patch;

typedef struct celeste_problem celeste_problem;   /* opaque; owns device copies */

/*
 * Copy a problem to the current device and build its work lists.
 *   imgs[n_img]; model; n_src sources; patch_offsets[n_src + 1] (CSR into patches[]);
 *   nbr_offsets[n_src + 1] / nbrs: neighbour lists (sources whose patches intersect
 *   in some image; Section IV-D's conflict graph); every list must be symmetric.
 * Errors: CELESTE_ERR_ARG (sizes, a patch outside its image, bad band, weights),
 * CELESTE_ERR_NOT_PD (PSF / prior covariance), CELESTE_ERR_NOMEM, CELESTE_ERR_CUDA.
 */
celeste_status celeste_problem_create(const celeste_image* imgs, int32_t n_img,
                                      const celeste_model* model, int32_t n_src,
                                      const int32_t* patch_offsets, const celeste_patch* patches,
                                      const int32_t* nbr_offsets, const int32_t* nbrs,
                                      celeste_problem** out);
/*
 * The same with a world -> pixel map per patch (multi-epoch data whose images carry a
 * non-linear WCS: the caller linearises each image's map at the patch's source,
 * pixel = A_p u + t_p near the source, Section III's image metadata Lambda_n evaluated
 * per source).  patch_wcs[n_patches][6] in celeste_image.wcs layout, or NULL (every
 * patch uses its image's wcs).  Position and galaxy shape of the source in that patch
 * use its map; everything else is as in celeste_problem_create.  Errors as there, plus
 * CELESTE_ERR_ARG for a non-finite or singular patch map.
 */
celeste_status celeste_problem_create_ex(const celeste_image* imgs, int32_t n_img,
                                         const celeste_model* model, int32_t n_src,
                                         const int32_t* patch_offsets, const celeste_patch* patches,
                                         const double* patch_wcs, const int32_t* nbr_offsets,
                                         const int32_t* nbrs, celeste_problem** out);
void celeste_problem_destroy(celeste_problem* prob);

/* Number of (source, active pixel) pairs: the unit of the cost accounting (Section VI-B). */
int64_t celeste_source_pixels(const celeste_problem* prob);

/*
 * Work decomposition of a problem (host read, no GPU work), for cost accounting:
 * out[0] sources, [1] patches, [2] work items of the FP64 and Hessian paths (<= 256
 * pixels of one patch each), [3] items of the FP32 value / gradient path (<= 512 pixels
 * of one patch each, fewer on a problem too small to give every resident CTA two),
 * [4] singly covered source-pixels, [5] 16 x 16 tiles covered by two or more patches,
 * [6] source-pixels in all, [7] (source-pixel, other covering patch) pairs: the other
 * sources' E and Var the FP32 value / gradient path evaluates at multiply covered pixels.
 * Writes min(n, 8) entries; returns the number written, or CELESTE_ERR_ARG for a null
 * problem / out.
 */
int32_t celeste_problem_stats(const celeste_problem* prob, int64_t* out, int32_t n);

/*
 * ELBO (Eq. 1, the reading above) at theta[n_src][44] (host).
 *   elbo_total: sum over the union of patches of the expected log-likelihood minus the
 *     sum of KL terms.
 *   elbo_per_source (nullable, [n_src]): local objective of each source, the sum over
 *     its own patch pixels (neighbours' light included in E and Var) minus its KL.
 * Errors: CELESTE_ERR_ARG for parameters outside their domain (r2, c2, e_scale <= 0,
 * a or k outside (0,1), e_axis outside (0,1], e_dev outside [0,1]); CELESTE_ERR_NONFINITE.
 * The domain is checked on the device during the evaluation and read back with the
 * results (with several violations either code may be reported); on an error the
 * outputs hold the evaluation at the invalid parameters and must not be used.
 */
celeste_status celeste_elbo(celeste_problem* prob, const double* theta, int32_t precision,
                            double* elbo_total, double* elbo_per_source);

/*
 * ELBO and its gradient wrt every source's 44 constrained parameters (Section IV-D:
 * one block per source; d ELBO_total / d theta_s = d ELBO_s / d theta_s because each
 * source's light is truncated to its patch).  grad[n_src][44] (host).
 */
celeste_status celeste_elbo_grad(celeste_problem* prob, const double* theta, int32_t precision,
                                 double* elbo_total, double* elbo_per_source, double* grad);

/*
 * Per-source exact Hessians (Section IV-D: 44 x 44, dense symmetric) of ELBO_s wrt
 * theta_s, with the gradient.  hess[n_src][44][44] full symmetric (host); grad and
 * elbo_per_source nullable.
 */
celeste_status celeste_hess(celeste_problem* prob, const double* theta, int32_t precision,
                            double* elbo_per_source, double* grad, double* hess);

/* Trust-region Newton options (Section IV-D; Nocedal & Wright, Algorithm 4.1). */
typedef struct {
    int32_t max_iter;          /* Newton iterations per source per sweep (default 50) */
    double grad_tol;           /* stop when max |dELBO_s/dt| <= grad_tol (free coords) */
    double pred_tol_rel;       /* stop when the model's predicted gain <= pred_tol_rel (1 + |ELBO_s|) */
    double delta0, delta_max;  /* initial and largest trust radius (free coords) */
    double eta;                /* accept a step when actual/predicted gain > eta */
    double f_noise_rel;        /* predicted gains below f_noise_rel (1+|ELBO_s|) skip the ratio test */
    int32_t precision;         /* CELESTE_FP64 or CELESTE_FP32_ACC64 */
    int32_t max_sweeps;        /* block-coordinate sweeps over all colour classes */
    double sweep_tol;          /* stop sweeping when |dELBO_total| / max(1,|ELBO_total|) < sweep_tol */
    int32_t refine_fp64;       /* with CELESTE_FP32_ACC64: after the FP32 sweeps converge, polish with
                                  FP64 sweeps (Newton needs one or two steps from there), so poorly
                                  constrained parameters are not left at FP32 rounding noise */
    int32_t schedule;          /* CELESTE_SCHED_COLOUR (default) or CELESTE_SCHED_CYCLADES */
    int32_t sample_size;       /* Cyclades: sources per random sample, >= 1 (default 64) */
    uint64_t seed;             /* Cyclades with order == NULL: sweep g visits the moving sources
                                  (ascending ids) shuffled by Fisher-Yates with SplitMix64
                                  draws keyed by (seed, g) */
    const int32_t* order;      /* Cyclades, nullable: [max_sweeps][n_moving] host array; sweep g
                                  (counted over both precision phases) uses row g mod max_sweeps,
                                  each row a permutation of the moving sources */
} celeste_fit_options;

/* Conflict-free update schedules of the block-coordinate fit (Section IV-D). */
enum { CELESTE_SCHED_COLOUR = 0, CELESTE_SCHED_CYCLADES = 1 };

/* Fill opts with the defaults documented above. */
void celeste_fit_options_default(celeste_fit_options* opts);

/*
 * Block-coordinate trust-region Newton fit (Section IV-D).  Each sweep runs a sequence
 * of batches; the sources of one batch never overlap and take their Newton iterations
 * together with every other source fixed; E and Var are updated after each batch.
 * Schedules:
 *   CELESTE_SCHED_COLOUR: sources greedily coloured in ascending id over the
 *     neighbour graph; one batch per colour, colours in order, the same every sweep.
 *   CELESTE_SCHED_CYCLADES: the conflict-free sampling of Section IV-D (Pan et al.,
 *     Cyclades): the sweep's order is cut into consecutive samples of sample_size
 *     sources; each sample is split into the connected components of the neighbour
 *     graph restricted to it; the sources of one component are updated one after
 *     another in sample order, different components concurrently: batch r of a sample
 *     holds the r-th source of every component that has one (celeste_cyclades_batches).
 * theta_inout[n_src][44] (host) is read and overwritten.  which[n_which] restricts the
 * moving sources (NULL: all).  iters_out / status_out ([n_src], nullable) receive
 * Newton iterations and 0 converged / 1 iteration limit / 2 non-finite.  The fit
 * restarts from theta_inout, so it can be resumed (also from its own result, whose
 * bounded parameters may sit on their bounds).  The fit works inside a box: e_dev and
 * e_axis in [0.01, 0.99], a_star in [0.005, 0.995]; a start outside it, a Cyclades order
 * row that is not a permutation of the moving sources, or sample_size < 1, is
 * CELESTE_ERR_ARG.
 */
celeste_status celeste_fit_sources(celeste_problem* prob, double* theta_inout,
                                   const int32_t* which, int32_t n_which,
                                   const celeste_fit_options* opts, int32_t* iters_out,
                                   int32_t* status_out, double* elbo_out);

/*
 * Region tasks (Section IV-A; host logic, no device work).  The sources' positions
 * pos[n][2] (world coordinates) and expected work work[n] >= 0 (e.g. each source's
 * active pixel count, or its bright pixels from an existing catalog) cut the bounding
 * box of the positions recursively into regions of work <= max_work (or a single
 * source): each cut runs across the longer side of a region's box, at the weighted
 * median (sources sorted by that coordinate, ties by index; the first prefix whose work
 * reaches half the region's goes to the lower side; the cut lies halfway between the
 * two sources it separates); the leaves, depth first, lower side first, are tasks
 * 0 .. n_tasks - 1.  task_of[s] = the task whose region holds pos[s] - shift (shift
 * NULL = (0, 0)): the first stage with no shift, the second with the same regions
 * shifted by a fixed amount.  Errors: CELESTE_ERR_ARG (null pointers, n < 0,
 * max_work <= 0, non-finite positions, shift or work, negative work).
 */
celeste_status celeste_make_tasks(const double* pos, const double* work, int32_t n, double max_work,
                                  const double* shift, int32_t* task_of, int32_t* n_tasks);

/*
 * One stage of region tasks (Section IV-A): every task (the sources s with
 * task_of[s] == k, k >= 0; -1 = the source stays fixed) is fitted as
 * celeste_fit_sources would with `which` = its sources, starting from theta_inout with
 * every other source held at its starting value, as tasks running side by side on
 * separate nodes see each other; the tasks' results are merged into theta_inout.  The
 * tasks run side by side on the device: one sweep schedule over all their sources, a
 * source of another task contributing its stage-start E_s / Var_s, so each task's
 * iterates equal those of its own fit.  Sweeps end for all tasks together: after
 * max_sweeps, or once the merged parameters' total ELBO changes by less than
 * sweep_tol (relative) in a sweep.  iters_out / status_out ([n_src], nullable) as
 * celeste_fit_sources (0 for fixed sources); elbo_out (nullable) = the total ELBO of
 * the merged parameters (FP64 when FP32 sweeps are polished, else in the fit's
 * precision).  Errors as celeste_fit_sources; task ids below -1 are CELESTE_ERR_ARG.
 */
celeste_status celeste_fit_tasks(celeste_problem* prob, double* theta_inout, const int32_t* task_of,
                                 const celeste_fit_options* opts, int32_t* iters_out,
                                 int32_t* status_out, double* elbo_out);

/*
 * The Cyclades batches of one sweep (host logic, no device work, no CUDA context
 * needed) over the neighbour graph nbr_offsets[n_src + 1] / nbrs (the CSR lists given
 * to celeste_problem_create, symmetric): order[n_order] lists distinct source ids in
 * [0, n_src); positions [k sample_size, (k+1) sample_size) form sample k.  On
 * return batch_of[i] is the batch of order[i]: samples take consecutive batch ranges
 * in order, and within a sample the r-th member (in order) of a connected component of
 * the neighbour graph restricted to the sample goes to the sample's batch r.
 * *n_batches = the number of batches.  comp_of (nullable, [n_order]) receives the
 * position in order of the first member of order[i]'s component.  Errors:
 * CELESTE_ERR_ARG (null pointers, n_src < 0, sample_size < 1, an id out of range or
 * repeated, a neighbour id out of range).
 */
celeste_status celeste_cyclades_batches(const int32_t* nbr_offsets, const int32_t* nbrs, int32_t n_src,
                                        const int32_t* order, int32_t n_order, int32_t sample_size,
                                        int32_t* batch_of, int32_t* comp_of, int32_t* n_batches);

/* Device-pointer variants: same semantics, pointers on the problem's device, work
 * enqueued on `stream` (a cudaStream_t; NULL = legacy default stream), no synchronisation.
 * Parameter-domain checks read theta on the device and report through
 * celeste_device_status() after the stream completes. */
celeste_status celeste_elbo_device(celeste_problem* prob, const double* d_theta, int32_t precision,
                                   double* d_elbo_total, double* d_elbo_per_source, void* stream);
celeste_status celeste_elbo_grad_device(celeste_problem* prob, const double* d_theta,
                                        int32_t precision, double* d_elbo_total,
                                        double* d_elbo_per_source, double* d_grad, void* stream);
celeste_status celeste_hess_device(celeste_problem* prob, const double* d_theta, int32_t precision,
                                   double* d_elbo_per_source, double* d_grad, double* d_hess,
                                   void* stream);
/*
 * Backward half of an ELBO evaluation (the adjoint, Section IV-D's gradient): the
 * gradient wrt every source's 44 parameters, reusing the mixture tables and the
 * E / Var maps that the immediately preceding celeste_elbo_device call on this problem
 * left behind, which must have used the same d_theta contents and precision.  The
 * per-pixel mixture terms are recomputed, never stored.  elbo_per_source nullable.
 */
celeste_status celeste_grad_device(celeste_problem* prob, const double* d_theta, int32_t precision,
                                   double* d_elbo_per_source, double* d_grad, void* stream);

/*
 * Autotuner, at theta (host), with CUDA events on the problem's stream.
 *   contrib_code: the FP32 map-pass kernel of the Hessian and fit paths, timed over reps
 *     launches: 1, 2, 4 pixels per thread (CTAs of 256, 128, 64 threads over the same
 *     256-pixel work items), 3, 5 two or four pixels per thread in packed FP32x2
 *     instructions, 6, 7 the same as persistent CTAs taking items from a work queue.
 *   items_code: the variant of the persistent FP32 value / gradient item kernel (CTAs
 *     of four compute warps and one producer warp), as (pixels per thread, CTAs per SM,
 *     unroll of the loop over profile-component pairs): 1 (2, 2, 7), 2 (3, 2, 3),
 *     3 (2, 3, 2), 4 (3, 2, 7), 5 (3, 2, 2); timed on whole FP32 value + gradient
 *     evaluations as the calls run them (the captured CUDA graph).
 * The choices are kept for later FP32 calls and returned (nullable outputs);
 * celeste_set_tuning restores them (contrib 0 .. 7, items 0 .. 5; 0 = the built-in
 * defaults 2 and 1; anything else is CELESTE_ERR_ARG).
 */
celeste_status celeste_autotune(celeste_problem* prob, const double* theta, int32_t reps,
                                int32_t* contrib_code, int32_t* items_code);
celeste_status celeste_set_tuning(celeste_problem* prob, int32_t contrib_code, int32_t items_code);

/* Status word written by the device-side checks of the last _device call (host read;
 * synchronises the problem's last stream).  CELESTE_OK or a negative status. */
celeste_status celeste_device_status(celeste_problem* prob);

/*
 * Per-kernel timing (tracing aid).  With profiling on, every stage launch of the
 * calls above (prep, contrib, gather, adjoint / ll_sum / hess_adjoint, finalize) is
 * bracketed by CUDA events on its launch stream.  on = 1: the stages run as in a
 * normal call (the FP32 value / gradient path's fused pass and total on a second
 * stream, concurrently with the others), so a stage's time includes waiting for SM
 * slots that the concurrent stages hold; on = 2: every stage runs on the calling
 * stream, one after another, so the times add up to a serialised evaluation (results
 * identical to the concurrent order's); on = 0: off; anything else is CELESTE_ERR_ARG.
 * celeste_profile_read waits for the
 * recorded events, writes up to max_kernels entries (names[k*32 .. k*32+31]
 * NUL-terminated, total milliseconds, kernel launches), resets the accumulators and
 * returns the number of distinct stages (negative status on error).
 */
celeste_status celeste_profile_enable(celeste_problem* prob, int32_t on);
int32_t celeste_profile_read(celeste_problem* prob, int32_t max_kernels, char* names,
                             double* ms_total, int32_t* launches);

/*
 * Allocation-free variant (no counterpart in the paper): the ELBO, local objective
 * and gradient of ONE source whose light falls in ONE patch, for callers that cannot
 * call cudaMalloc -- a program whose device memory is owned by another allocator, or
 * code that must not allocate on a latency-critical path.  celeste_problem_create
 * allocates the problem's device copies; this call allocates nothing.  It takes:
 *   im, model, patch: host structs as for celeste_problem_create (im->pixels and
 *     im->sky_map are ignored; the patch rectangle is in im's pixel frame);
 *   d_pixels: DEVICE [patch->h][patch->w] counts of the patch's pixels (row-major);
 *   d_sky_map: DEVICE [patch->h][patch->w] sky counts, or NULL for the scalar im->sky;
 *   d_theta: DEVICE [44] parameters of the source (domain as in celeste_elbo; not
 *     checked here);
 *   outputs (DEVICE): d_elbo_total (nullable, [1]: the patch's expected
 *     log-likelihood minus the KL), d_elbo_local (nullable, [1]: the same here, since
 *     the patch is the source's only one), d_grad ([44]);
 *   stream: cudaStream_t for the launches (NULL = legacy default stream); the call
 *     returns without synchronising.
 * Every intermediate buffer lives in one file-scope device array of
 * CELESTE_NOALLOC_SCRATCH_BYTES, which each GPU that loads the library holds until the
 * process exits; the largest patch it serves is 101 x 101 pixels (larger sides return
 * CELESTE_ERR_ARG with a message).  A call made outside a stream capture looks up that
 * array's device address (cudaGetSymbolAddress) with the device current, every time; a
 * call inside a capture uses the address of the last uncaptured call on that device, so
 * make the first call on a device before any stream capture (a first call inside one
 * returns CELESTE_ERR_ARG).  The model is checked as by celeste_problem_create.  All
 * calls on a device share the array and it keeps
 * the last call's contents (every value a call reads is written by the same call
 * first): calls whose work overlaps on the GPU race on it, so order them on one
 * stream or synchronise between them.  Errors: CELESTE_ERR_ARG, CELESTE_ERR_NOT_PD,
 * CELESTE_ERR_CUDA; message via celeste_last_error().
 */
enum { CELESTE_NOALLOC_SCRATCH_BYTES = 393216 };
celeste_status celeste_patch_elbo_grad_noalloc(const celeste_image* im, const celeste_model* model,
                                               const celeste_patch* patch, const float* d_pixels,
                                               const float* d_sky_map, const double* d_theta,
                                               int32_t precision, double* d_elbo_total,
                                               double* d_elbo_local, double* d_grad, void* stream);

/*
 * Catalog with posterior uncertainty (Section VIII: besides point estimates the
 * variational posterior gives the probability of each type and the uncertainty of
 * brightness and colours).  One row of CELESTE_CAT_NFIELD doubles per source, from
 * theta alone:
 *   CAT_U0, CAT_U1        position u (world coordinates)
 *   CAT_PSTAR             q(star) = a_star;  CAT_IS_STAR = 1 if a_star >= 0.5 else 0
 *   per type t (CAT_STAR + k, CAT_GAL + k): under q, log l_b | t is Gaussian with mean
 *   r1_t + beta_b . c1_t and variance r2_t + sum_j beta_bj^2 c2_tj (log-normal
 *   brightness, colours as adjacent-band log ratios), so the magnitude
 *   m_b = 22.5 - 2.5 log10(l_b [nmgy]) is Gaussian:
 *     k = CAT_RMAG, CAT_RMAG_SD     r-band magnitude mean and standard deviation
 *     k = CAT_RFLUX, CAT_RFLUX_SD   r-band flux E[l_r | t] and its standard deviation (nmgy)
 *     k = CAT_COLOR + j, CAT_COLOR_SD + j   magnitude colours m_j - m_{j+1}
 *                                   (u-g, g-r, r-i, i-z): 2.5 / ln 10 * c1_tj, sd from c2_tj
 *     k = CAT_MAG + b, CAT_MAG_SD + b       magnitude in band b (u g r i z)
 *   CAT_RFLUX_MIX, CAT_RFLUX_MIX_SD   r-band flux mean and sd with the type marginalised
 *                                     (weights a_star, a_gal, which sum to 1 in the model)
 *   CAT_EDEV, CAT_AXIS, CAT_ANGLE_DEG (in [0, 180)), CAT_SCALE (world units)
 */
enum {
    CELESTE_CAT_U0 = 0, CELESTE_CAT_U1 = 1, CELESTE_CAT_PSTAR = 2, CELESTE_CAT_IS_STAR = 3,
    CELESTE_CAT_STAR = 4, CELESTE_CAT_GAL = 26, CELESTE_CAT_TYPE_NFIELD = 22,
    /* offsets within a type block */
    CELESTE_CAT_RMAG = 0, CELESTE_CAT_RMAG_SD = 1, CELESTE_CAT_RFLUX = 2, CELESTE_CAT_RFLUX_SD = 3,
    CELESTE_CAT_COLOR = 4, CELESTE_CAT_COLOR_SD = 8, CELESTE_CAT_MAG = 12, CELESTE_CAT_MAG_SD = 17,
    /* after both type blocks */
    CELESTE_CAT_RFLUX_MIX = 48, CELESTE_CAT_RFLUX_MIX_SD = 49, CELESTE_CAT_EDEV = 50,
    CELESTE_CAT_AXIS = 51, CELESTE_CAT_ANGLE_DEG = 52, CELESTE_CAT_SCALE = 53,
    CELESTE_CAT_NFIELD = 54
};

/* catalog[n_src][CELESTE_CAT_NFIELD] (host) from theta[n_src][44] (host); one kernel
 * thread per source.  Errors: CELESTE_ERR_ARG (null pointers, theta outside the
 * parameter domain: r2, c2 <= 0 or non-finite entries), CELESTE_ERR_CUDA. */
celeste_status celeste_catalog(celeste_problem* prob, const double* theta, double* catalog);
/* Same with device pointers, enqueued on `stream`, no synchronisation; domain errors
 * are reported through celeste_device_status(). */
celeste_status celeste_catalog_device(celeste_problem* prob, const double* d_theta,
                                      double* d_catalog, void* stream);

/*
 * Fit quality against a known truth, the error summary of Table II: from an estimated
 * and a true catalog ([n][CELESTE_CAT_NFIELD] each, host) of the same sources, the
 * types taken from each catalog's CAT_IS_STAR and brightness / colours from each
 * catalog's own classified type:
 *   SCORE_POSITION      mean distance between positions (world units)
 *   SCORE_MISSED_GAL    fraction of true galaxies classified as stars
 *   SCORE_MISSED_STAR   fraction of true stars classified as galaxies
 *   SCORE_BRIGHTNESS    mean |r-band magnitude error|
 *   SCORE_COLOR + j     mean |colour error| for u-g, g-r, r-i, i-z (magnitudes)
 *   SCORE_PROFILE, SCORE_AXIS, SCORE_SCALE, SCORE_ANGLE_DEG   mean |e_dev|, |axis
 *                       ratio|, |scale| and angle (degrees, modulo 180) errors over
 *                       the true galaxies
 *   SCORE_N_GAL, SCORE_N_STAR   counts of true galaxies and stars
 * Means over an empty set are 0.  One CTA with a fixed-order FP64 reduction, so the
 * result does not depend on timing.  Errors: CELESTE_ERR_ARG, CELESTE_ERR_CUDA.
 */
enum {
    CELESTE_SCORE_POSITION = 0, CELESTE_SCORE_MISSED_GAL = 1, CELESTE_SCORE_MISSED_STAR = 2,
    CELESTE_SCORE_BRIGHTNESS = 3, CELESTE_SCORE_COLOR = 4, CELESTE_SCORE_PROFILE = 8,
    CELESTE_SCORE_AXIS = 9, CELESTE_SCORE_SCALE = 10, CELESTE_SCORE_ANGLE_DEG = 11,
    CELESTE_SCORE_N_GAL = 12, CELESTE_SCORE_N_STAR = 13, CELESTE_SCORE_NFIELD = 14
};
celeste_status celeste_catalog_score(celeste_problem* prob, const double* cat_est,
                                     const double* cat_true, int32_t n, double* score);

/*
 * The model's expected image and its variance under q (Section III: E[F] and Var[F]
 * per pixel, sources independent): e[m] = sky_m + sum over the patches covering pixel m
 * of the source's E[F_s], v[m] = sum of Var[F_s] (0 outside every patch), FP64, for
 * every pixel of every image, images concatenated in creation order, each row-major
 * ([sum_n height_n * width_n]).  Used to draw data from the model itself (e.g. Poisson
 * counts around e).  The evaluation overwrites the problem's per-source scratch, so it
 * must not fall between celeste_elbo_device and celeste_grad_device.  Host pointers;
 * v nullable.  Errors as celeste_elbo.
 */
celeste_status celeste_render(celeste_problem* prob, const double* theta, double* e, double* v);
/* Same with device pointers on `stream` (e and v: [sum_n height_n * width_n] doubles, v
 * nullable), no synchronisation; domain errors via celeste_device_status(). */
celeste_status celeste_render_device(celeste_problem* prob, const double* d_theta, double* d_e,
                                     double* d_v, void* stream);

/*
 * Self-test of failure detection without a fault: one kernel waits, through the same
 * bounded wait the persistent work-queue kernels use (a poll and ~1 s clock limit), on a
 * shared-memory mbarrier that nothing arrives on.  Returns CELESTE_ERR_TIMEOUT when the
 * wait gave up and reported it through a status word (the expected outcome, after about
 * a second; the context stays usable), CELESTE_OK if the barrier completed (a defect),
 * CELESTE_ERR_CUDA on a launch error.  Runs on the current device.
 */
celeste_status celeste_selftest_bounded_wait(void);

/* Thread-local message describing the calling thread's last error. */
const char* celeste_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CELESTE_H */
