// C ABI of libceleste: problem creation (validation, device copies, work lists) and
// the ELBO / gradient / Hessian / fit entry points declared in celeste.h.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace cel;

namespace {

thread_local std::string g_err;

celeste_status fail(celeste_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

celeste_status cuda_fail(cudaError_t e, const char* where) {
    if (e == cudaErrorMemoryAllocation)
        return fail(CELESTE_ERR_NOMEM, "%s: %s", where, cudaGetErrorString(e));
    return fail(CELESTE_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CEL_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)


template <class T>
celeste_status upload(T** dst, const T* src, size_t n) {
    *dst = nullptr;
    if (n == 0) return CELESTE_OK;
    CEL_CUDA(cudaMalloc((void**)dst, n * sizeof(T)));
    CEL_CUDA(cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
    return CELESTE_OK;
}

}  // namespace

namespace cel {
// 2x2 / 4x4 symmetric positive-definiteness and inverse by Cholesky
bool chol_inverse4(const double* S, double* inv, double* logdet) {
    double L[4][4] = {{0}};
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = S[4 * i + j];
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            if (i == j) {
                if (!(s > 0)) return false;
                L[i][i] = sqrt(s);
            } else {
                L[i][j] = s / L[j][j];
            }
        }
    double ld = 0;
    for (int i = 0; i < 4; ++i) ld += 2.0 * log(L[i][i]);
    *logdet = ld;
    // inverse of L, then L^-T L^-1
    double Li[4][4] = {{0}};
    for (int i = 0; i < 4; ++i) {
        Li[i][i] = 1.0 / L[i][i];
        for (int j = 0; j < i; ++j) {
            double s = 0;
            for (int k = j; k < i; ++k) s -= L[i][k] * Li[k][j];
            Li[i][j] = s / L[i][i];
        }
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double s = 0;
            for (int k = std::max(i, j); k < 4; ++k) s += Li[k][i] * Li[k][j];
            inv[4 * i + j] = s;
        }
    return true;
}

celeste_status build_model_dev(const celeste_model* model, ModelDev& md, const char** why) {
    auto bad = [&](celeste_status st, const char* msg) {
        *why = msg;
        return st;
    };
    if (model->n_exp < 1 || model->n_dev < 1 || model->n_exp + model->n_dev > MAXPROF ||
        !model->exp_mix || !model->dev_mix)
        return bad(CELESTE_ERR_ARG, "profile mixtures: need 1 <= n_exp, n_dev and n_exp + n_dev <= CELESTE_MAX_PROFILE");
    if (model->n_color_comp != NCOMP || !model->prior_c || !model->prior_r)
        return bad(CELESTE_ERR_ARG, "colour prior must have 8 components per type");
    if (!(model->prior_star > 0 && model->prior_star < 1)) return bad(CELESTE_ERR_ARG, "prior_star outside (0,1)");
    md = ModelDev{};
    md.n_exp = model->n_exp;
    md.n_dev = model->n_dev;
    for (int j = 0; j < model->n_exp + model->n_dev; ++j) {
        const double* m = j < model->n_exp ? model->exp_mix + 2 * j : model->dev_mix + 2 * (j - model->n_exp);
        if (!(m[0] >= 0 && isfinite(m[0]) && m[1] > 0 && isfinite(m[1])))
            return bad(CELESTE_ERR_ARG, "profile components need weight >= 0 and variance > 0");
        md.prof_w[j] = m[0];
        md.prof_nu[j] = m[1];
    }
    md.prior_star = model->prior_star;
    for (int i = 0; i < 2; ++i) {
        md.prior_r[i][0] = model->prior_r[2 * i];
        md.prior_r[i][1] = model->prior_r[2 * i + 1];
        if (!(md.prior_r[i][1] > 0) || !isfinite(md.prior_r[i][0]) || !isfinite(md.prior_r[i][1]))
            return bad(CELESTE_ERR_ARG, "prior_r variance must be > 0");
        for (int d = 0; d < NCOMP; ++d) {
            const double* pc = model->prior_c + (size_t)(i * NCOMP + d) * 21;
            if (!(pc[0] > 0) || !isfinite(pc[0])) return bad(CELESTE_ERR_ARG, "colour prior weight must be > 0");
            md.prior_w[i][d] = pc[0];
            for (int j = 0; j < 4; ++j) {
                if (!isfinite(pc[1 + j])) return bad(CELESTE_ERR_ARG, "colour prior mean not finite");
                md.prior_mu[i][d][j] = pc[1 + j];
            }
            if (!chol_inverse4(pc + 5, md.prior_P[i][d], &md.prior_logdet[i][d]))
                return bad(CELESTE_ERR_NOT_PD, "colour prior covariance not positive definite");
        }
    }
    fill_float_copies(md);
    return CELESTE_OK;
}

// lets other translation units report through celeste_last_error()
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace cel

#include "problem.cuh"

namespace {

celeste_status dalloc(celeste_problem* pr, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    pr->owned.push_back(*p);
    return CELESTE_OK;
}

template <class T>
celeste_status dupload(celeste_problem* pr, T** dst, const T* src, size_t n) {
    void* p;
    celeste_status st = dalloc(pr, &p, n * sizeof(T));
    if (st) return st;
    *dst = (T*)p;
    if (n) CEL_CUDA(cudaMemcpy(p, src, n * sizeof(T), cudaMemcpyHostToDevice));
    return CELESTE_OK;
}

bool psd2(double xx, double xy, double yy) { return xx > 0 && yy > 0 && xx * yy - xy * xy > 0; }

cudaEvent_t take_event(celeste_problem* pr) {
    if (!pr->pool.empty()) {
        cudaEvent_t e = pr->pool.back();
        pr->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Run a launcher of n_kernels kernels; with profiling on, bracket it with events on the
// launch stream.
template <class F>
cudaError_t timed(celeste_problem* pr, const char* name, cudaStream_t st, F&& f, int n_kernels = 1) {
    if (!pr->profile) return f();
    cudaEvent_t a = take_event(pr), b = take_event(pr);
    cudaEventRecord(a, st);
    cudaError_t e = f();
    cudaEventRecord(b, st);
    pr->pending.push_back({name, a, b, n_kernels});
    return e;
}

celeste_status check_theta_host(const double* theta, int n_src) {
    for (int s = 0; s < n_src; ++s) {
        const double* th = theta + (size_t)NP * s;
        for (int i = 0; i < NP; ++i)
            if (!isfinite(th[i])) return fail(CELESTE_ERR_NONFINITE, "theta[%d][%d] is not finite", s, i);
        if (!(th[P_EDEV] >= 0 && th[P_EDEV] <= 1)) return fail(CELESTE_ERR_ARG, "theta[%d]: e_dev outside [0,1]", s);
        if (!(th[P_AXIS] > 0 && th[P_AXIS] <= 1)) return fail(CELESTE_ERR_ARG, "theta[%d]: e_axis outside (0,1]", s);
        if (!(th[P_SCALE] > 0)) return fail(CELESTE_ERR_ARG, "theta[%d]: e_scale <= 0", s);
        for (int i = 0; i < 2; ++i) {
            if (!(th[P_R2 + i] > 0)) return fail(CELESTE_ERR_ARG, "theta[%d]: r2 <= 0", s);
            if (!(th[P_A + i] > 0 && th[P_A + i] < 1)) return fail(CELESTE_ERR_ARG, "theta[%d]: a outside (0,1)", s);
            for (int j = 0; j < 4; ++j)
                if (!(th[P_C2 + 4 * i + j] > 0)) return fail(CELESTE_ERR_ARG, "theta[%d]: c2 <= 0", s);
            for (int d = 0; d < NCOMP; ++d)
                if (!(th[P_K + NCOMP * i + d] > 0)) return fail(CELESTE_ERR_ARG, "theta[%d]: k <= 0", s);
        }
    }
    return CELESTE_OK;
}

celeste_status ensure_out(celeste_problem* pr) {
    size_t need = 1 + (size_t)pr->P.n_src * (1 + NP + NP * NP);
    if (pr->out_cap >= need) return CELESTE_OK;
    void* p;
    celeste_status st = dalloc(pr, &p, need * sizeof(double));
    if (st) return st;
    pr->d_out = (double*)p;
    pr->out_cap = need;
    return CELESTE_OK;
}

celeste_status run(celeste_problem* pr, const double* d_theta, int precision, int mode,
                   double* d_total, double* d_local, double* d_grad, double* d_hess,
                   cudaStream_t st) {
    if (precision != CELESTE_FP64 && precision != CELESTE_FP32_ACC64)
        return fail(CELESTE_ERR_ARG, "precision must be CELESTE_FP64 or CELESTE_FP32_ACC64");
    CEL_CUDA(cudaSetDevice(pr->device));
    pr->last_stream = st;
    const DevProblem& P = pr->P;
    // FP32 value / gradient: the item kernels (item_kernels.cu) -- tables and KL terms,
    // the items (a programmatic dependent of the tables), the per-source epilogues and
    // the total (a programmatic dependent of the items); timed as three stages when
    // profiling.  FP64 and the Hessian: the map / gather / adjoint pipeline below.
    const bool fused = precision == CELESTE_FP32_ACC64 && mode != MODE_HESS && P.ztasks;
    if (fused) {
        static const char* const names[3] = {"tables", "items", "finish"};
        for (int stage = 0; stage < 3; ++stage)
            CEL_CUDA(timed(pr, names[stage], st, [&] {
                return launch_items_stage(P, stage, mode, st, d_theta, d_local, d_grad, d_total);
            }));
        return CELESTE_OK;
    }
    CEL_CUDA(timed(pr, "prep", st, [&] { return launch_prep(P, d_theta, precision, st); }));
    CEL_CUDA(timed(pr, "contrib", st, [&] { return launch_contrib(P, precision, st); }));
    CEL_CUDA(timed(pr, "gather", st, [&] { return launch_gather(P, precision, st); }));
    if (mode == MODE_HESS)
        CEL_CUDA(timed(pr, "hess_adjoint", st, [&] { return launch_hess_pixels(P, precision, st); }));
    else
        CEL_CUDA(timed(pr, mode == MODE_LL ? "ll_sum" : "adjoint", st,
                       [&] { return launch_adjoint(P, precision, mode, st); }));
    CEL_CUDA(timed(pr, "finalize", st, [&] {
        return launch_finalize(P, d_theta, precision, mode, d_total, d_local, d_grad, d_hess, st);
    }));
    return CELESTE_OK;
}

// run() through the graph cache: the first call with an argument set captures the
// evaluation (with the status reset when reset_status) on the private capture stream and
// instantiates it; every call launches the graph on st.  With profiling on, run() is
// called directly (its per-kernel events are recorded at launch time).
constexpr size_t MAX_GRAPHS = 8;

void drop_graphs(celeste_problem* pr) {
    for (auto& g : pr->graphs) cudaGraphExecDestroy(g.second);
    pr->graphs.clear();
}

celeste_status run_cached(celeste_problem* pr, const double* d_theta, int precision, int mode,
                          double* d_total, double* d_local, double* d_grad, double* d_hess,
                          cudaStream_t st, bool reset_status) {
    const DevProblem& P = pr->P;
    if (pr->profile || !pr->capture) {
        if (reset_status) CEL_CUDA(cudaMemsetAsync(P.status, 0, sizeof(int32_t), st));
        return run(pr, d_theta, precision, mode, d_total, d_local, d_grad, d_hess, st);
    }
    celeste_problem::GraphKey key{precision, mode, P.tune_contrib, P.tune_adjoint, P.tune_items,
                                  {d_theta, d_total, d_local, d_grad, d_hess}};
    if (!reset_status) key.mode |= 0x100;
    cudaGraphExec_t exec = nullptr;
    for (auto& g : pr->graphs)
        if (g.first == key) exec = g.second;
    if (!exec) {
        cudaStream_t cs = pr->capture;
        CEL_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        cudaError_t ce = reset_status ? cudaMemsetAsync(P.status, 0, sizeof(int32_t), cs) : cudaSuccess;
        celeste_status rs = ce == cudaSuccess
                                ? run(pr, d_theta, precision, mode, d_total, d_local, d_grad, d_hess, cs)
                                : CELESTE_ERR_CUDA;
        cudaGraph_t graph = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(cs, &graph);
        if (rs != CELESTE_OK || ce != cudaSuccess || ee != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            if (rs != CELESTE_OK) return rs;
            return cuda_fail(ce != cudaSuccess ? ce : ee, "evaluation capture");
        }
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return cuda_fail(ie, "cudaGraphInstantiate");
        if (pr->graphs.size() >= MAX_GRAPHS) {
            cudaGraphExecDestroy(pr->graphs.front().second);
            pr->graphs.erase(pr->graphs.begin());
        }
        pr->graphs.push_back({key, exec});
    }
    CEL_CUDA(cudaGraphLaunch(exec, st));
    pr->last_stream = st;
    return CELESTE_OK;
}

celeste_status run_host(celeste_problem* pr, const double* theta, int precision, int mode,
                        double* total, double* local, double* grad, double* hess) {
    if (!pr || !theta) return fail(CELESTE_ERR_ARG, "null problem or theta");
    // the parameter domain is checked on the device by the evaluation itself (every
    // entry of every source, the same rules as the host check), read back with the results
    celeste_status s = ensure_out(pr);
    if (s) return s;
    const int n = pr->P.n_src;
    double* o_total = pr->d_out;
    double* o_local = o_total + 1;
    double* o_grad = o_local + n;
    double* o_hess = o_grad + (size_t)n * NP;
    CEL_CUDA(cudaSetDevice(pr->device));
    CEL_CUDA(cudaMemcpyAsync(pr->d_theta, theta, sizeof(double) * NP * n, cudaMemcpyHostToDevice,
                             pr->stream));
    s = run_cached(pr, pr->d_theta, precision, mode, o_total, o_local,
                   mode >= MODE_GRAD ? o_grad : nullptr, mode >= MODE_HESS ? o_hess : nullptr,
                   pr->stream, true);
    if (s) return s;
    if (total) CEL_CUDA(cudaMemcpyAsync(total, o_total, sizeof(double), cudaMemcpyDeviceToHost, pr->stream));
    if (local) CEL_CUDA(cudaMemcpyAsync(local, o_local, sizeof(double) * n, cudaMemcpyDeviceToHost, pr->stream));
    if (grad && mode >= MODE_GRAD)
        CEL_CUDA(cudaMemcpyAsync(grad, o_grad, sizeof(double) * n * NP, cudaMemcpyDeviceToHost, pr->stream));
    if (hess && mode >= MODE_HESS)
        CEL_CUDA(cudaMemcpyAsync(hess, o_hess, sizeof(double) * n * NP * NP, cudaMemcpyDeviceToHost, pr->stream));
    CEL_CUDA(cudaMemcpyAsync(pr->h_status, pr->P.status, sizeof(int32_t), cudaMemcpyDeviceToHost, pr->stream));
    CEL_CUDA(cudaStreamSynchronize(pr->stream));
    if (*pr->h_status != 0)
        return fail(*pr->h_status, "theta outside the parameter domain (status %d from the device check)",
                    *pr->h_status);
    if (total && !isfinite(*total)) return fail(CELESTE_ERR_NONFINITE, "ELBO is not finite");
    return CELESTE_OK;
}

}  // namespace

extern "C" {

const char* celeste_last_error(void) { return g_err.c_str(); }

int64_t celeste_source_pixels(const celeste_problem* pr) { return pr ? pr->P.n_sp : 0; }

int32_t celeste_problem_stats(const celeste_problem* pr, int64_t* out, int32_t n) {
    if (!pr || !out) return fail(CELESTE_ERR_ARG, "null problem or output");
    const DevProblem& P = pr->P;
    const int64_t v[8] = {P.n_src, P.n_patch, P.n_item, (int64_t)P.n_sitem, pr->sp_single, P.n_tile, P.n_sp,
                          pr->other_evals};
    const int m = n < 8 ? (n > 0 ? n : 0) : 8;
    for (int i = 0; i < m; ++i) out[i] = v[i];
    return m;
}

void celeste_problem_destroy(celeste_problem* pr) {
    if (!pr) return;
    cudaSetDevice(pr->device);
    if (pr->stream) cudaStreamSynchronize(pr->stream);
    cudaDeviceSynchronize();
    for (auto& r : pr->pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : pr->pool) cudaEventDestroy(e);
    drop_graphs(pr);
    for (void* p : pr->owned) cudaFree(p);
    if (pr->side) cudaStreamDestroy(pr->side);
    if (pr->capture) cudaStreamDestroy(pr->capture);
    for (cudaEvent_t e : {pr->ev_prep, pr->ev_fused, pr->ev_gather, pr->ev_join})
        if (e) cudaEventDestroy(e);
    if (pr->stream) cudaStreamDestroy(pr->stream);
    if (pr->h_status) cudaFreeHost(pr->h_status);
    delete pr;
}

celeste_status celeste_problem_create(const celeste_image* imgs, int32_t n_img,
                                      const celeste_model* model, int32_t n_src,
                                      const int32_t* patch_offsets, const celeste_patch* patches,
                                      const int32_t* nbr_offsets, const int32_t* nbrs,
                                      celeste_problem** out) {
    return celeste_problem_create_ex(imgs, n_img, model, n_src, patch_offsets, patches, nullptr,
                                     nbr_offsets, nbrs, out);
}

celeste_status celeste_problem_create_ex(const celeste_image* imgs, int32_t n_img,
                                         const celeste_model* model, int32_t n_src,
                                         const int32_t* patch_offsets, const celeste_patch* patches,
                                         const double* patch_wcs, const int32_t* nbr_offsets,
                                         const int32_t* nbrs, celeste_problem** out) {
    if (!out) return fail(CELESTE_ERR_ARG, "out is null");
    *out = nullptr;
    if (n_img <= 0 || !imgs) return fail(CELESTE_ERR_ARG, "need at least one image");
    if (n_src < 0 || !model || !patch_offsets || !nbr_offsets)
        return fail(CELESTE_ERR_ARG, "null model / offsets or negative n_src");
    // ---- model
    ModelDev md{};
    {
        const char* why = nullptr;
        const celeste_status ms = build_model_dev(model, md, &why);
        if (ms != CELESTE_OK) return fail(ms, "%s", why);
    }
    fill_float_copies(md);
    // ---- images
    std::vector<ImgMeta> im(n_img);
    int64_t n_px = 0;
    bool any_sky_map = false;
    int npsf_max = 0;
    for (int n = 0; n < n_img; ++n) {
        const celeste_image& I = imgs[n];
        if (I.band < 0 || I.band > 4) return fail(CELESTE_ERR_ARG, "image %d: band must be 0..4", n);
        if (I.height <= 0 || I.width <= 0 || !I.pixels) return fail(CELESTE_ERR_ARG, "image %d: bad size or pixels", n);
        if (I.n_psf < 1 || I.n_psf > MAXPSF || !I.psf) return fail(CELESTE_ERR_ARG, "image %d: n_psf must be 1..%d", n, MAXPSF);
        if (!(I.nmgy_per_count > 0) || !isfinite(I.nmgy_per_count)) return fail(CELESTE_ERR_ARG, "image %d: calibration must be > 0", n);
        if (!I.sky_map && !(I.sky > 0 && isfinite(I.sky))) return fail(CELESTE_ERR_ARG, "image %d: sky must be > 0", n);
        const double detA = I.wcs[0] * I.wcs[3] - I.wcs[1] * I.wcs[2];
        for (int k = 0; k < 6; ++k)
            if (!isfinite(I.wcs[k])) return fail(CELESTE_ERR_ARG, "image %d: wcs not finite", n);
        if (detA == 0) return fail(CELESTE_ERR_ARG, "image %d: singular wcs", n);
        ImgMeta& M = im[n];
        memset(&M, 0, sizeof M);
        M.px_off = n_px;
        M.H = I.height;
        M.W = I.width;
        M.band = I.band;
        M.npsf = I.n_psf;
        M.has_sky_map = I.sky_map != nullptr;
        any_sky_map = any_sky_map || M.has_sky_map;
        M.sky = I.sky;
        M.iota = 1.0 / I.nmgy_per_count;
        for (int k = 0; k < 4; ++k) M.A[k] = I.wcs[k];
        M.t[0] = I.wcs[4];
        M.t[1] = I.wcs[5];
        for (int k = 0; k < I.n_psf; ++k) {
            const double* ps = I.psf + 6 * k;
            for (int c = 0; c < 6; ++c) {
                if (!isfinite(ps[c])) return fail(CELESTE_ERR_ARG, "image %d psf %d not finite", n, k);
                M.psf[k][c] = ps[c];
            }
            if (!psd2(ps[3], ps[4], ps[5])) return fail(CELESTE_ERR_NOT_PD, "image %d psf %d covariance not positive definite", n, k);
        }
        fill_float_copies(M);
        npsf_max = std::max(npsf_max, (int)I.n_psf);
        n_px += (int64_t)I.height * I.width;
    }
    // ---- patches, work items, tiles
    if (patch_offsets[0] != 0) return fail(CELESTE_ERR_ARG, "patch_offsets[0] must be 0");
    for (int s = 0; s < n_src; ++s)
        if (patch_offsets[s + 1] < patch_offsets[s]) return fail(CELESTE_ERR_ARG, "patch_offsets must be non-decreasing");
    const int n_patch = patch_offsets[n_src];
    if (n_patch > 0 && !patches) return fail(CELESTE_ERR_ARG, "patches is null");
    std::vector<PatchGeo> geo(n_patch);
    std::vector<WorkItem> items;
    int64_t n_sp = 0;
    for (int s = 0; s < n_src; ++s)
        for (int p = patch_offsets[s]; p < patch_offsets[s + 1]; ++p) {
            const celeste_patch& c = patches[p];
            if (c.image < 0 || c.image >= n_img) return fail(CELESTE_ERR_ARG, "patch %d: bad image", p);
            const ImgMeta& M = im[c.image];
            if (c.w <= 0 || c.h <= 0 || c.x0 < 0 || c.y0 < 0 || c.x0 + c.w > M.W || c.y0 + c.h > M.H)
                return fail(CELESTE_ERR_ARG, "patch %d lies outside image %d", p, c.image);
            if (c.w > 32767 || c.h > 32767)
                return fail(CELESTE_ERR_ARG, "patch %d: sides above 32767 pixels are not supported", p);
            PatchGeo& g = geo[p];
            g.img = c.image; g.x0 = c.x0; g.y0 = c.y0; g.w = c.w; g.h = c.h; g.src = s;
            g.sp_off = n_sp;
            g.item0 = (int)items.size();
            const int npx = c.w * c.h;
            for (int q0 = 0; q0 < npx; q0 += CHUNK) items.push_back({p, q0, std::min(CHUNK, npx - q0), s});
            g.nitem = (int)items.size() - g.item0;
            n_sp += npx;
        }
    // per-(source, pixel) flag: 1 when no other patch covers the pixel (those pixels are
    // finished by k_contrib; k_gather visits only cells that two or more patches touch)
    std::vector<uint8_t> single((size_t)n_sp, 0);
    {
        std::vector<std::vector<uint8_t>> cover(n_img);
        for (int p = 0; p < n_patch; ++p) {
            const PatchGeo& g = geo[p];
            auto& c = cover[g.img];
            if (c.empty()) c.assign((size_t)im[g.img].H * im[g.img].W, 0);
            for (int yy = 0; yy < g.h; ++yy)
                for (int xx = 0; xx < g.w; ++xx) {
                    uint8_t& v = c[(size_t)(g.y0 + yy) * im[g.img].W + g.x0 + xx];
                    if (v < 255) ++v;
                }
        }
        for (int p = 0; p < n_patch; ++p) {
            const PatchGeo& g = geo[p];
            const auto& c = cover[g.img];
            for (int yy = 0; yy < g.h; ++yy)
                for (int xx = 0; xx < g.w; ++xx)
                    single[(size_t)g.sp_off + (size_t)yy * g.w + xx] =
                        c[(size_t)(g.y0 + yy) * im[g.img].W + g.x0 + xx] == 1;
        }
    }
    // The FP32 value / gradient kernel's items: per source, per patch, the patch's pixels
    // with the multiply covered ones first (row-major), then the singly covered ones, cut
    // into ceil(n / cap) items of near-equal size.  cap = ZIMAX, or for a problem too small
    // to give two items to each of the kernel's resident CTAs (two per SM), the pixel count
    // that would, rounded up to 64 and at least 128.
    int item_cap = ZIMAX;
    {
        int dev = 0, n_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm <= 0)
            n_sm = 152;
        const int64_t per = (n_sp + 4LL * n_sm - 1) / (4LL * n_sm);
        item_cap = (int)std::min<int64_t>(ZIMAX, std::max<int64_t>(128, (per + 63) / 64 * 64));
    }
    struct SItem {
        int32_t patch, src, n, nm;
        int64_t q0;   // first pixel (spix)
    };
    std::vector<SItem> sitems;
    std::vector<int32_t> spix, sitem_off(1, 0);
    int n_smulti = 0;
    spix.reserve((size_t)n_sp);
    int64_t sp_single = 0;
    for (int s = 0; s < n_src; ++s) {
        for (int p = patch_offsets[s]; p < patch_offsets[s + 1]; ++p) {
            const PatchGeo& g = geo[p];
            const uint8_t* f = single.data() + g.sp_off;
            const int64_t first = (int64_t)spix.size();
            const int npx = g.w * g.h;
            for (int q = 0; q < npx; ++q)
                if (!f[q]) spix.push_back(((q / g.w) << 16) | (q % g.w));
            const int nm_all = (int)((int64_t)spix.size() - first);
            for (int q = 0; q < npx; ++q)
                if (f[q]) spix.push_back(((q / g.w) << 16) | (q % g.w));
            sp_single += npx - nm_all;
            const int k = (npx + item_cap - 1) / item_cap, base = npx / k, rem = npx % k;
            for (int j = 0, o = 0; j < k; ++j) {
                const int n = base + (j < rem ? 1 : 0);
                const int nm = std::max(0, std::min(n, nm_all - o));
                sitems.push_back({p, s, n, nm, first + o});
                if (nm > 0) ++n_smulti;
                o += n;
            }
        }
        sitem_off.push_back((int32_t)sitems.size());
    }
    // tiles: per image a dense grid of TILE x TILE cells, each with its covering patches
    std::vector<Tile> tiles;
    std::vector<int32_t> tile_list;
    std::vector<int32_t> tile_grid;
    {
        std::vector<std::vector<int32_t>> per_img(n_img);   // patch ids per image in order
        for (int p = 0; p < n_patch; ++p) per_img[geo[p].img].push_back(p);
        for (int n = 0; n < n_img; ++n) {
            if (per_img[n].empty()) continue;
            const int tw = (im[n].W + TILE - 1) / TILE, th = (im[n].H + TILE - 1) / TILE;
            im[n].tg_off = (int64_t)tile_grid.size();
            im[n].tgw = tw;
            tile_grid.resize(tile_grid.size() + (size_t)tw * th, -1);
            std::vector<std::vector<int32_t>> cell((size_t)tw * th);
            for (int p : per_img[n]) {
                const PatchGeo& g = geo[p];
                for (int ty = g.y0 / TILE; ty <= (g.y0 + g.h - 1) / TILE; ++ty)
                    for (int tx = g.x0 / TILE; tx <= (g.x0 + g.w - 1) / TILE; ++tx)
                        cell[(size_t)ty * tw + tx].push_back(p);
            }
            for (int ty = 0; ty < th; ++ty)
                for (int tx = 0; tx < tw; ++tx) {
                    auto& c = cell[(size_t)ty * tw + tx];
                    if (c.size() < 2) continue;   // a lone patch's pixels are done in k_contrib
                    Tile t{};
                    tile_grid[im[n].tg_off + (size_t)ty * tw + tx] = (int32_t)tiles.size();
                    t.img = n; t.x0 = tx * TILE; t.y0 = ty * TILE;
                    t.list_off = (int)tile_list.size(); t.list_n = (int)c.size();
                    tile_list.insert(tile_list.end(), c.begin(), c.end());
                    tiles.push_back(t);
                }
        }
    }
    // Per item, the other patches covering any of its multiply covered pixels (ascending
    // patch id = ascending source id within an image) and its cost: its pixels plus about
    // a third of a pixel per (64-pixel warp chunk, other patch touching the chunk).
    std::vector<int32_t> zc_off(1, 0), zc_list, zorder;
    int64_t other_evals = 0;   // (pixel, other covering patch) pairs the item kernel evaluates
    std::vector<double> zcost(sitems.size());
    {
        std::vector<int32_t> cand, chunk;
        for (size_t i = 0; i < sitems.size(); ++i) {
            const SItem& it = sitems[i];
            const PatchGeo& g = geo[it.patch];
            const ImgMeta& M = im[g.img];
            cand.clear();
            double extra = 0.0;
            for (int c0 = 0; c0 < it.nm; c0 += 64) {
                chunk.clear();
                for (int l = c0; l < std::min(it.nm, c0 + 64); ++l) {
                    const int xx = spix[it.q0 + l] & 0xffff, yy = spix[it.q0 + l] >> 16;
                    const int gx = g.x0 + xx, gy = g.y0 + yy;
                    const int tid = tile_grid[M.tg_off + (size_t)(gy / TILE) * M.tgw + gx / TILE];
                    if (tid < 0) continue;
                    const Tile& tl = tiles[tid];
                    for (int e = 0; e < tl.list_n; ++e) {
                        const int pe = tile_list[tl.list_off + e];
                        if (pe == it.patch) continue;
                        const PatchGeo& G = geo[pe];
                        if (gx >= G.x0 && gx < G.x0 + G.w && gy >= G.y0 && gy < G.y0 + G.h) {
                            chunk.push_back(pe);
                            ++other_evals;
                        }
                    }
                }
                std::sort(chunk.begin(), chunk.end());
                chunk.erase(std::unique(chunk.begin(), chunk.end()), chunk.end());
                extra += 64.0 * (double)chunk.size();
                cand.insert(cand.end(), chunk.begin(), chunk.end());
            }
            std::sort(cand.begin(), cand.end());
            cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
            zc_list.insert(zc_list.end(), cand.begin(), cand.end());
            zc_off.push_back((int32_t)zc_list.size());
            zcost[i] = (double)it.n + 0.3 * extra;
        }
        // the most expensive items first, so the last items taken are short ones
        for (size_t i = 0; i < sitems.size(); ++i) zorder.push_back((int32_t)i);
        std::stable_sort(zorder.begin(), zorder.end(), [&](int32_t a, int32_t b) { return zcost[a] > zcost[b]; });
    }
    // The work queue: the items in cost order, each with the patches of its first ZMAXC
    // candidates; and the order in which the table kernel builds the patches' tables (by
    // the first item that reads each).
    std::vector<ZTask> ztasks;
    std::vector<ZCand> zcands;
    std::vector<int32_t> ztorder;   // the table kernel's order of the patches
    std::vector<float4> zpx(spix.size());
    {
        const int n_it = (int)sitems.size();
        const int64_t never = INT64_MAX / 4;
        std::vector<int64_t> pneed((size_t)n_patch, never);
        for (int j = 0; j < n_it; ++j) {
            const int i = zorder[j];
            const SItem& it = sitems[i];
            pneed[it.patch] = std::min<int64_t>(pneed[it.patch], j);
            for (int e = zc_off[i]; e < zc_off[i + 1]; ++e)
                pneed[zc_list[e]] = std::min<int64_t>(pneed[zc_list[e]], j);
        }
        for (int p = 0; p < n_patch; ++p) ztorder.push_back(p);
        std::stable_sort(ztorder.begin(), ztorder.end(), [&](int32_t a, int32_t b) { return pneed[a] < pneed[b]; });
        for (int j = 0; j < n_it; ++j) {
            ZTask t{};
            t.kind = ZT_ITEM;
            t.index = j;
            for (int e = 0; e < ZMAXC; ++e) t.cand[e] = -1;
            const int i = zorder[j];
            const SItem& it = sitems[i];
            const PatchGeo& g = geo[it.patch];
            const int nc = zc_off[i + 1] - zc_off[i];
            t.item.patch = it.patch;
            t.item.n_nm = it.n | (it.nm << 16);
            t.item.out = i;
            t.item.src = it.src;
            t.item.pix = it.q0;
            t.item.c0 = (int32_t)zcands.size();
            t.item.nc_npsf = nc | (im[g.img].npsf << 24);
            for (int e = zc_off[i]; e < zc_off[i + 1]; ++e) {
                const PatchGeo& G = geo[zc_list[e]];
                if (e - zc_off[i] < ZMAXC) t.cand[e - zc_off[i]] = zc_list[e];
                zcands.push_back(ZCand{zc_list[e], G.x0 - g.x0, G.y0 - g.y0, G.w, G.h, G.src, im[G.img].npsf, 0});
            }
            ztasks.push_back(t);
        }
        // pixel records in item order: (column, row in the patch, counts, sky)
        for (const SItem& it : sitems) {
            const PatchGeo& g = geo[it.patch];
            const ImgMeta& M = im[g.img];
            const float* px = imgs[g.img].pixels;
            const float* sm = imgs[g.img].sky_map;
            for (int l = 0; l < it.n; ++l) {
                const int xx = spix[it.q0 + l] & 0xffff, yy = spix[it.q0 + l] >> 16;
                const size_t m = (size_t)(g.y0 + yy) * M.W + (g.x0 + xx);
                zpx[it.q0 + l] = make_float4((float)xx, (float)yy, px[m], sm ? sm[m] : (float)M.sky);
            }
        }
    }
    // neighbours
    if (nbr_offsets[0] != 0) return fail(CELESTE_ERR_ARG, "nbr_offsets[0] must be 0");
    const int n_edge = nbr_offsets[n_src];
    if (n_edge > 0 && !nbrs) return fail(CELESTE_ERR_ARG, "nbrs is null");
    for (int s = 0; s < n_src; ++s) {
        if (nbr_offsets[s + 1] < nbr_offsets[s]) return fail(CELESTE_ERR_ARG, "nbr_offsets must be non-decreasing");
        for (int e = nbr_offsets[s]; e < nbr_offsets[s + 1]; ++e)
            if (nbrs[e] < 0 || nbrs[e] >= n_src || nbrs[e] == s) return fail(CELESTE_ERR_ARG, "bad neighbour of source %d", s);
    }

    // Per-patch world -> pixel maps (each image's map linearised at the patch's source):
    // a patch whose map differs from its image's points at a copy of the image record
    // carrying that map (appended after the images, sharing their pixels, sky, PSF and
    // tile grid).  Every kernel reads a patch's map from img[geo.img], so nothing else
    // changes; the tiles and the coverage flags above keep the real image ids.
    if (patch_wcs) {
        for (int p = 0; p < n_patch; ++p) {
            const double* w = patch_wcs + 6 * (size_t)p;
            for (int k = 0; k < 6; ++k)
                if (!isfinite(w[k])) return fail(CELESTE_ERR_ARG, "patch %d: wcs not finite", p);
            if (w[0] * w[3] - w[1] * w[2] == 0) return fail(CELESTE_ERR_ARG, "patch %d: singular wcs", p);
            const ImgMeta& base = im[geo[p].img];
            if (w[0] == base.A[0] && w[1] == base.A[1] && w[2] == base.A[2] && w[3] == base.A[3] &&
                w[4] == base.t[0] && w[5] == base.t[1])
                continue;
            ImgMeta V = base;
            for (int k = 0; k < 4; ++k) V.A[k] = w[k];
            V.t[0] = w[4];
            V.t[1] = w[5];
            fill_float_copies(V);
            geo[p].img = (int)im.size();
            im.push_back(V);
        }
    }

    celeste_problem* pr = new (std::nothrow) celeste_problem();
    if (!pr) return fail(CELESTE_ERR_NOMEM, "host allocation failed");
    auto bail = [&](celeste_status st) { celeste_problem_destroy(pr); return st; };
    if (cudaGetDevice(&pr->device) != cudaSuccess) return bail(fail(CELESTE_ERR_CUDA, "no CUDA device"));
    if (cudaStreamCreateWithFlags(&pr->stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(fail(CELESTE_ERR_CUDA, "cudaStreamCreate failed"));
    {
        int least = 0, greatest = 0;   // numerically greatest = lowest priority
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        // graphs are captured with the critical chain on the highest-priority stream and the
        // fused pass on the lowest, and instantiated to keep those per-node priorities
        if (cudaStreamCreateWithPriority(&pr->side, cudaStreamNonBlocking, least) != cudaSuccess ||
            cudaStreamCreateWithPriority(&pr->capture, cudaStreamNonBlocking, greatest) != cudaSuccess)
            return bail(fail(CELESTE_ERR_CUDA, "cudaStreamCreate failed"));
        for (cudaEvent_t* e : {&pr->ev_prep, &pr->ev_fused, &pr->ev_gather, &pr->ev_join})
            if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess)
                return bail(fail(CELESTE_ERR_CUDA, "cudaEventCreate failed"));
    }
    pr->last_stream = pr->stream;
    if (cudaMallocHost((void**)&pr->h_status, sizeof(int32_t)) != cudaSuccess)
        return bail(fail(CELESTE_ERR_NOMEM, "pinned host allocation failed"));
    pr->patch_off.assign(patch_offsets, patch_offsets + n_src + 1);
    pr->nbr_off.assign(nbr_offsets, nbr_offsets + n_src + 1);
    pr->nbrs.assign(nbrs ? nbrs : nbr_offsets, nbrs ? nbrs + n_edge : nbr_offsets);
    if (!nbrs) pr->nbrs.clear();
    pr->geo = geo;
    pr->imgs = im;
    DevProblem& P = pr->P;
    P.n_img = n_img; P.n_src = n_src; P.n_patch = n_patch; P.n_item = (int)items.size();
    P.n_tile = (int)tiles.size(); P.npsf_max = npsf_max; P.nprof = model->n_exp + model->n_dev;
    P.model_ne = model->n_exp;
    P.model_nd = model->n_dev;
    P.n_px = n_px; P.n_sp = n_sp;
    P.max_src_patches = 0;
    for (int s = 0; s < n_src; ++s)
        P.max_src_patches = std::max(P.max_src_patches, patch_offsets[s + 1] - patch_offsets[s]);
    celeste_status st;
    // pixels (and optional sky maps) concatenated
    {
        void* p;
        if ((st = dalloc(pr, &p, sizeof(float) * n_px))) return bail(st);
        P.pixels = (float*)p;
        void* sm = nullptr;
        if (any_sky_map) {
            if ((st = dalloc(pr, &sm, sizeof(float) * n_px))) return bail(st);
            P.sky_map = (float*)sm;
        }
        for (int n = 0; n < n_img; ++n) {
            const size_t cnt = (size_t)im[n].H * im[n].W;
            if (cudaMemcpy((float*)p + im[n].px_off, imgs[n].pixels, cnt * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
                return bail(fail(CELESTE_ERR_CUDA, "pixel upload failed"));
            if (imgs[n].sky_map &&
                cudaMemcpy((float*)sm + im[n].px_off, imgs[n].sky_map, cnt * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
                return bail(fail(CELESTE_ERR_CUDA, "sky map upload failed"));
        }
    }
    ImgMeta* d_img; PatchGeo* d_geo; WorkItem* d_items; Tile* d_tiles; int32_t* d_tl; int32_t* d_po; ModelDev* d_md;
    int32_t* d_tg;
    if ((st = dupload(pr, &d_img, im.data(), im.size()))) return bail(st);
    if ((st = dupload(pr, &d_geo, geo.data(), geo.size()))) return bail(st);
    if ((st = dupload(pr, &d_items, items.data(), items.size()))) return bail(st);
    if ((st = dupload(pr, &d_tiles, tiles.data(), tiles.size()))) return bail(st);
    if ((st = dupload(pr, &d_tl, tile_list.data(), tile_list.size()))) return bail(st);
    if ((st = dupload(pr, &d_tg, tile_grid.data(), tile_grid.size()))) return bail(st);
    uint8_t* d_single;
    if ((st = dupload(pr, &d_single, single.data(), single.size()))) return bail(st);
    P.single = d_single;
    if (!sitems.empty()) {
        int32_t* d_soff = nullptr;
        ZBuild* d_tord = nullptr;
        ZTask* d_zt = nullptr;
        ZCand* d_zc = nullptr;
        float4* d_zpx = nullptr;
        if ((st = dupload(pr, &d_soff, sitem_off.data(), sitem_off.size()))) return bail(st);
        // build records from the final patch geometry (a patch with its own linearised map
        // refers to the image copy that carries it)
        std::vector<ZBuild> zb;
        for (const int32_t p : ztorder)
            zb.push_back(ZBuild{p, geo[p].img, geo[p].src, 0, im[geo[p].img].t[0] - (double)geo[p].x0,
                                im[geo[p].img].t[1] - (double)geo[p].y0});
        if ((st = dupload(pr, &d_tord, zb.data(), zb.size()))) return bail(st);
        if ((st = dupload(pr, &d_zt, ztasks.data(), ztasks.size()))) return bail(st);
        if (!zcands.empty() && (st = dupload(pr, &d_zc, zcands.data(), zcands.size()))) return bail(st);
        if ((st = dupload(pr, &d_zpx, zpx.data(), zpx.size()))) return bail(st);
        P.sitem_off = d_soff;
        P.ztorder = d_tord;
        P.ztasks = d_zt;
        P.n_task = (int32_t)ztasks.size();
        P.zcands = d_zc;
        P.zpx = d_zpx;
        P.n_sitem = (int)sitems.size();
        P.n_smulti = n_smulti;
        void* q;
        if ((st = dalloc(pr, &q, sizeof(double) * ZPCOLS * (size_t)P.n_sitem))) return bail(st);
        P.spart = (double*)q;
        if ((st = dalloc(pr, &q, sizeof(int32_t)))) return bail(st);
        P.zf_done = (int32_t*)q;
        if (cudaMemset(P.zf_done, 0, sizeof(int32_t)) != cudaSuccess)
            return bail(fail(CELESTE_ERR_CUDA, "memset"));
        if ((st = dalloc(pr, &q, sizeof(int32_t) * ((size_t)n_patch + 2)))) return bail(st);
        P.zready = (int32_t*)q;
        if ((st = dalloc(pr, &q, sizeof(float4) * NP * (size_t)n_patch))) return bail(st);
        P.zchain = (float4*)q;
    }
    pr->sp_single = sp_single;
    pr->other_evals = other_evals;
    if ((st = dupload(pr, &d_po, patch_offsets, (size_t)n_src + 1))) return bail(st);
    if ((st = dupload(pr, &d_md, &md, 1))) return bail(st);
    P.img = d_img; P.geo = d_geo; P.items = d_items; P.tiles = d_tiles; P.tile_list = d_tl;
    P.tile_grid = d_tg;
    P.patch_off = d_po; P.model = d_md;
    P.n_img_rec = (int32_t)im.size();
    P.n_zcand = (int32_t)zcands.size();
    P.n_tile_list = (int64_t)tile_list.size();
    P.n_tile_grid = (int64_t)tile_grid.size();
    void* p;
    if ((st = dalloc(pr, &p, sizeof(double) * TBL_STRIDE * (size_t)n_patch))) return bail(st);
    P.tbl64 = (double*)p;
    if ((st = dalloc(pr, &p, sizeof(float) * TBL_STRIDE * (size_t)n_patch))) return bail(st);
    P.tbl32 = (float*)p;
    if ((st = dalloc(pr, &p, sizeof(float) * ZFULL_FLOATS * (size_t)n_patch))) return bail(st);
    P.ztbl = (float*)p;
    if ((st = dalloc(pr, &P.spE, sizeof(double) * (size_t)n_sp))) return bail(st);
    if ((st = dalloc(pr, &P.spE2, sizeof(double) * (size_t)n_sp))) return bail(st);
    if ((st = dalloc(pr, &P.emap, sizeof(double) * (size_t)n_px))) return bail(st);
    if ((st = dalloc(pr, &P.vmap, sizeof(double) * (size_t)n_px))) return bail(st);
    if ((st = dalloc(pr, &p, sizeof(double) * NPART * (size_t)P.n_item))) return bail(st);
    P.item_part = (double*)p;
    if ((st = dalloc(pr, &p, sizeof(double) * (size_t)P.n_tile))) return bail(st);
    P.tile_ll = (double*)p;
    if ((st = dalloc(pr, &p, sizeof(double) * (size_t)P.n_item))) return bail(st);
    P.item_ll = (double*)p;

    if ((st = dalloc(pr, &p, sizeof(double) * (size_t)n_src))) return bail(st);
    P.kl = (double*)p;
    if ((st = dalloc(pr, &p, sizeof(double) * NP * (size_t)n_src))) return bail(st);
    P.kl_grad = (double*)p;
    if ((st = dalloc(pr, &p, sizeof(double) * (size_t)n_src))) return bail(st);
    P.src_total = (double*)p;
    if ((st = dalloc(pr, &p, sizeof(int32_t)))) return bail(st);
    P.done = (int32_t*)p;
    if (cudaMemset(P.done, 0, sizeof(int32_t)) != cudaSuccess) return bail(fail(CELESTE_ERR_CUDA, "memset"));
    if ((st = dalloc(pr, &p, sizeof(double) * 64))) return bail(st);
    P.tot_part = (double*)p;
    if ((st = dalloc(pr, &p, sizeof(int32_t)))) return bail(st);
    P.tot_done = (int32_t*)p;
    if (cudaMemset(P.tot_done, 0, sizeof(int32_t)) != cudaSuccess) return bail(fail(CELESTE_ERR_CUDA, "memset"));
    if ((st = dalloc(pr, &p, 2 * sizeof(int32_t)))) return bail(st);
    P.queue = (int32_t*)p;
    prime_persistent_grids();
    {
        const cudaError_t pe = prime_items_kernels();
        if (pe != cudaSuccess) return bail(fail(CELESTE_ERR_CUDA, "item kernel set-up: %s", cudaGetErrorString(pe)));
    }
    if (cudaMemset(P.queue, 0, 2 * sizeof(int32_t)) != cudaSuccess) return bail(fail(CELESTE_ERR_CUDA, "memset"));
    if ((st = dalloc(pr, &p, sizeof(int32_t)))) return bail(st);
    P.status = (int32_t*)p;
    if (cudaMemset(P.status, 0, sizeof(int32_t)) != cudaSuccess) return bail(fail(CELESTE_ERR_CUDA, "memset"));
    if ((st = dalloc(pr, &p, sizeof(double) * NP * (size_t)n_src))) return bail(st);
    pr->d_theta = (double*)p;
    if ((st = ensure_out(pr))) return bail(st);
    *out = pr;
    return CELESTE_OK;
}

celeste_status celeste_elbo(celeste_problem* pr, const double* theta, int32_t precision,
                            double* elbo_total, double* elbo_per_source) {
    return run_host(pr, theta, precision, MODE_LL, elbo_total, elbo_per_source, nullptr, nullptr);
}

celeste_status celeste_elbo_grad(celeste_problem* pr, const double* theta, int32_t precision,
                                 double* elbo_total, double* elbo_per_source, double* grad) {
    return run_host(pr, theta, precision, MODE_GRAD, elbo_total, elbo_per_source, grad, nullptr);
}

celeste_status celeste_hess(celeste_problem* pr, const double* theta, int32_t precision,
                            double* elbo_per_source, double* grad, double* hess) {
    return run_host(pr, theta, precision, MODE_HESS, nullptr, elbo_per_source, grad, hess);
}

static celeste_status run_device(celeste_problem* pr, const double* d_theta, int precision,
                                 int mode, double* d_total, double* d_local, double* d_grad,
                                 double* d_hess, void* stream) {
    if (!pr || !d_theta) return fail(CELESTE_ERR_ARG, "null problem or theta");
    cudaStream_t st = (cudaStream_t)stream;
    CEL_CUDA(cudaSetDevice(pr->device));
    // the status word (checked on the device) is reset first
    return run_cached(pr, d_theta, precision, mode, d_total, d_local, d_grad, d_hess, st, true);
}

celeste_status celeste_elbo_device(celeste_problem* pr, const double* d_theta, int32_t precision,
                                   double* d_total, double* d_local, void* stream) {
    return run_device(pr, d_theta, precision, MODE_LL, d_total, d_local, nullptr, nullptr, stream);
}

celeste_status celeste_elbo_grad_device(celeste_problem* pr, const double* d_theta,
                                        int32_t precision, double* d_total, double* d_local,
                                        double* d_grad, void* stream) {
    if (!d_grad) return fail(CELESTE_ERR_ARG, "d_grad is null");
    return run_device(pr, d_theta, precision, MODE_GRAD, d_total, d_local, d_grad, nullptr, stream);
}

celeste_status celeste_hess_device(celeste_problem* pr, const double* d_theta, int32_t precision,
                                   double* d_local, double* d_grad, double* d_hess, void* stream) {
    if (!d_hess) return fail(CELESTE_ERR_ARG, "d_hess is null");
    return run_device(pr, d_theta, precision, MODE_HESS, nullptr, d_local, d_grad, d_hess, stream);
}

celeste_status celeste_fit_sources(celeste_problem* pr, double* theta_inout, const int32_t* which,
                                   int32_t n_which, const celeste_fit_options* opts,
                                   int32_t* iters_out, int32_t* status_out, double* elbo_out) {
    return fit_sources_checked(pr, theta_inout, which, n_which, opts, iters_out, status_out, elbo_out, nullptr);
}

}  // extern "C"

celeste_status cel::fit_sources_checked(celeste_problem* pr, double* theta_inout, const int32_t* which,
                                        int32_t n_which, const celeste_fit_options* opts, int32_t* iters_out,
                                        int32_t* status_out, double* elbo_out, const int32_t* task_of) {
    if (!pr || !theta_inout) return fail(CELESTE_ERR_ARG, "null problem or theta");
    celeste_fit_options o;
    if (opts) o = *opts;
    else celeste_fit_options_default(&o);
    if (o.precision != CELESTE_FP64 && o.precision != CELESTE_FP32_ACC64)
        return fail(CELESTE_ERR_ARG, "precision must be CELESTE_FP64 or CELESTE_FP32_ACC64");
    if (o.max_iter < 1 || o.max_sweeps < 1 || !(o.delta0 > 0) || !(o.delta_max >= o.delta0))
        return fail(CELESTE_ERR_ARG, "bad fit options");
    if (which && n_which < 0) return fail(CELESTE_ERR_ARG, "n_which < 0");
    if (o.schedule != CELESTE_SCHED_COLOUR && o.schedule != CELESTE_SCHED_CYCLADES)
        return fail(CELESTE_ERR_ARG, "schedule must be CELESTE_SCHED_COLOUR or CELESTE_SCHED_CYCLADES");
    if (o.schedule == CELESTE_SCHED_CYCLADES && o.sample_size < 1)
        return fail(CELESTE_ERR_ARG, "Cyclades sample_size must be >= 1");
    celeste_status s = check_theta_host(theta_inout, pr->P.n_src);
    if (s) return s;
    for (int i = 0; i < pr->P.n_src; ++i) {
        const double* th = theta_inout + (size_t)NP * i;
        if (!(th[P_EDEV] >= 0.01 && th[P_EDEV] <= 0.99 && th[P_AXIS] >= 0.01 && th[P_AXIS] <= 0.99 &&
              th[P_A] >= 0.005 && th[P_A] <= 0.995))
            return fail(CELESTE_ERR_ARG,
                        "theta[%d]: the fit needs e_dev, e_axis in [0.01, 0.99] and a_star in [0.005, 0.995]", i);
    }
    CEL_CUDA(cudaSetDevice(pr->device));
    s = ensure_out(pr);
    if (s) return s;
    return fit_sources_impl(pr, theta_inout, which, n_which, &o, iters_out, status_out, elbo_out,
                            celeste_elbo, task_of);
}

extern "C" {

celeste_status celeste_profile_enable(celeste_problem* pr, int32_t on) {
    if (!pr) return fail(CELESTE_ERR_ARG, "null problem");
    if (on < 0 || on > 2) return fail(CELESTE_ERR_ARG, "profiling mode must be 0, 1 or 2");
    pr->profile = on != 0;
    pr->profile_serial = on == 2;
    return CELESTE_OK;
}

int32_t celeste_profile_read(celeste_problem* pr, int32_t max_kernels, char* names,
                             double* ms_total, int32_t* launches) {
    if (!pr) return fail(CELESTE_ERR_ARG, "null problem");
    cudaSetDevice(pr->device);
    for (auto& r : pr->pending) {
        if (cudaEventSynchronize(r.b) != cudaSuccess) return fail(CELESTE_ERR_CUDA, "event sync");
        float t = 0.f;
        cudaEventElapsedTime(&t, r.a, r.b);
        size_t k = 0;
        while (k < pr->names.size() && pr->names[k] != r.name) ++k;
        if (k == pr->names.size()) {
            pr->names.push_back(r.name);
            pr->ms.push_back(0.0);
            pr->launches.push_back(0);
        }
        pr->ms[k] += t;
        pr->launches[k] += r.n_kernels;
        pr->pool.push_back(r.a);
        pr->pool.push_back(r.b);
    }
    pr->pending.clear();
    const int n = (int)pr->names.size();
    for (int k = 0; k < n && k < max_kernels; ++k) {
        if (names) {
            strncpy(names + 32 * k, pr->names[k].c_str(), 31);
            names[32 * k + 31] = 0;
        }
        if (ms_total) ms_total[k] = pr->ms[k];
        if (launches) launches[k] = pr->launches[k];
    }
    pr->names.clear();
    pr->ms.clear();
    pr->launches.clear();
    return n;
}

celeste_status celeste_grad_device(celeste_problem* pr, const double* d_theta, int32_t precision,
                                  double* d_elbo_per_source, double* d_grad, void* stream) {
    if (!pr || !d_theta || !d_grad) return fail(CELESTE_ERR_ARG, "null problem, theta or grad");
    if (precision != CELESTE_FP64 && precision != CELESTE_FP32_ACC64)
        return fail(CELESTE_ERR_ARG, "precision must be CELESTE_FP64 or CELESTE_FP32_ACC64");
    cudaStream_t st = (cudaStream_t)stream;
    CEL_CUDA(cudaSetDevice(pr->device));
    pr->last_stream = st;
    const DevProblem& P = pr->P;
    CEL_CUDA(cudaMemsetAsync(P.status, 0, sizeof(int32_t), st));
    // FP64: the mixture tables and the E / Var maps of the preceding celeste_elbo_device
    // call are reused; the mixture terms themselves are recomputed by the adjoint.  FP32:
    // the item kernel of celeste_elbo_grad runs again (it recomputes its tables, E and Var
    // from theta; the KL of the preceding forward call is reused), so the gradient is
    // bit-identical to the one-call gradient.
    const bool fused = precision == CELESTE_FP32_ACC64 && P.ztasks;
    if (fused) {
        static const char* const names[3] = {"tables", "items", "finish"};
        for (int stage = 0; stage < 3; ++stage)
            CEL_CUDA(timed(pr, names[stage], st, [&] {
                return launch_items_stage(P, stage, MODE_GRAD, st, d_theta, d_elbo_per_source, d_grad, nullptr);
            }));
        return CELESTE_OK;
    }
    CEL_CUDA(timed(pr, "adjoint", st, [&] { return launch_adjoint(P, precision, MODE_GRAD, st); }));
    CEL_CUDA(timed(pr, "finalize", st, [&] {
        return launch_finalize(P, d_theta, precision, MODE_GRAD, nullptr, d_elbo_per_source, d_grad,
                               nullptr, st);
    }));
    return CELESTE_OK;
}

celeste_status celeste_autotune(celeste_problem* pr, const double* theta, int32_t reps,
                                int32_t* contrib_code, int32_t* items_code) {
    if (!pr || !theta) return fail(CELESTE_ERR_ARG, "null problem or theta");
    celeste_status s = check_theta_host(theta, pr->P.n_src);
    if (s) return s;
    if (reps < 1) reps = 5;
    CEL_CUDA(cudaSetDevice(pr->device));
    cudaStream_t st = pr->stream;
    DevProblem& P = pr->P;
    s = ensure_out(pr);
    if (s) return s;
    CEL_CUDA(cudaMemcpyAsync(pr->d_theta, theta, sizeof(double) * NP * P.n_src,
                             cudaMemcpyHostToDevice, st));
    CEL_CUDA(launch_prep(P, pr->d_theta, CELESTE_FP32_ACC64, st));
    cudaEvent_t a, b;
    CEL_CUDA(cudaEventCreate(&a));
    CEL_CUDA(cudaEventCreate(&b));
    cudaError_t e = cudaSuccess;
    // the FP32 map pass of the Hessian and fit paths: 1, 2, 4 pixels per thread; 3, 5: two
    // and four pixels per thread in packed FP32x2; 6, 7: the packed kernels as persistent
    // CTAs on a work queue
    const int cands[7] = {1, 2, 4, 3, 5, 6, 7};
    float best_c = 1e30f;
    int pick_c = 2;
    for (int ci = 0; ci < 7 && e == cudaSuccess; ++ci) {
        P.tune_contrib = cands[ci];
        float tc = 0.f;
        e = launch_contrib(P, CELESTE_FP32_ACC64, st);   // warm
        if (e == cudaSuccess) e = cudaEventRecord(a, st);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_contrib(P, CELESTE_FP32_ACC64, st);
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&tc, a, b);
        if (e == cudaSuccess && tc < best_c) { best_c = tc; pick_c = cands[ci]; }
    }
    P.tune_contrib = pick_c;
    // the item kernel's register budget (codes 1 .. 5), timed on whole value + gradient
    // evaluations as the calls run them (the captured graph)
    int pick_i = 1;
    if (P.ztasks) {
        float best = 1e30f;
        double* o = pr->d_out;
        for (int code = 1; code <= 5 && e == cudaSuccess; ++code) {
            P.tune_items = code;
            celeste_status rs = run_cached(pr, pr->d_theta, CELESTE_FP32_ACC64, MODE_GRAD, o, o + 1,
                                           o + 1 + P.n_src, nullptr, st, false);
            float t = 0.f;
            if (rs == CELESTE_OK) e = cudaEventRecord(a, st);
            for (int r = 0; r < 2 * reps && rs == CELESTE_OK && e == cudaSuccess; ++r)
                rs = run_cached(pr, pr->d_theta, CELESTE_FP32_ACC64, MODE_GRAD, o, o + 1, o + 1 + P.n_src,
                                nullptr, st, false);
            if (rs != CELESTE_OK) e = cudaErrorUnknown;
            if (e == cudaSuccess) e = cudaEventRecord(b, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(b);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
            if (e == cudaSuccess && t < best) {
                best = t;
                pick_i = code;
            }
        }
    }
    P.tune_items = pick_i;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    if (contrib_code) *contrib_code = pick_c;
    if (items_code) *items_code = pick_i;
    return CELESTE_OK;
}

celeste_status celeste_set_tuning(celeste_problem* pr, int32_t contrib_code, int32_t items_code) {
    if (!pr) return fail(CELESTE_ERR_ARG, "null problem");
    if (contrib_code < 0 || contrib_code > 7)
        return fail(CELESTE_ERR_ARG,
                    "contrib code: 0 default, 1 / 2 / 4 pixels per thread, 3 / 5 packed FP32x2 (2 / 4 "
                    "pixels), 6 / 7 the same as persistent CTAs on a work queue");
    if (items_code < 0 || items_code > 5)
        return fail(CELESTE_ERR_ARG,
                    "items code: 0 default, 1 .. 5 the item kernel's variant (pixels per thread, CTAs per SM, "
                    "unroll)");
    pr->P.tune_contrib = contrib_code;
    pr->P.tune_items = items_code;
    return CELESTE_OK;
}

celeste_status celeste_catalog_device(celeste_problem* pr, const double* d_theta, double* d_cat,
                                      void* stream) {
    if (!pr || (pr->P.n_src > 0 && (!d_theta || !d_cat))) return fail(CELESTE_ERR_ARG, "null problem or pointer");
    CEL_CUDA(cudaSetDevice(pr->device));
    cudaStream_t st = (cudaStream_t)stream;
    pr->last_stream = st;
    CEL_CUDA(cudaMemsetAsync(pr->P.status, 0, sizeof(int32_t), st));
    CEL_CUDA(launch_catalog(pr->P.n_src, d_theta, d_cat, pr->P.status, st));
    return CELESTE_OK;
}

celeste_status celeste_catalog(celeste_problem* pr, const double* theta, double* cat) {
    if (!pr || !theta || !cat) return fail(CELESTE_ERR_ARG, "null problem or pointer");
    const int n = pr->P.n_src;
    for (int s = 0; s < n; ++s) {
        const double* th = theta + (size_t)NP * s;
        for (int i = 0; i < NP; ++i)
            if (!isfinite(th[i])) return fail(CELESTE_ERR_ARG, "theta[%d][%d] is not finite", s, i);
        for (int t = 0; t < 2; ++t) {
            if (!(th[P_R2 + t] > 0)) return fail(CELESTE_ERR_ARG, "theta[%d]: r2 <= 0", s);
            for (int j = 0; j < 4; ++j)
                if (!(th[P_C2 + 4 * t + j] > 0)) return fail(CELESTE_ERR_ARG, "theta[%d]: c2 <= 0", s);
        }
    }
    celeste_status s = ensure_out(pr);   // n * (1 + 44 + 44^2) doubles: room for the rows
    if (s) return s;
    CEL_CUDA(cudaSetDevice(pr->device));
    CEL_CUDA(cudaMemcpyAsync(pr->d_theta, theta, sizeof(double) * NP * n, cudaMemcpyHostToDevice, pr->stream));
    s = celeste_catalog_device(pr, pr->d_theta, pr->d_out, pr->stream);
    if (s) return s;
    CEL_CUDA(cudaMemcpyAsync(cat, pr->d_out, sizeof(double) * CELESTE_CAT_NFIELD * n, cudaMemcpyDeviceToHost,
                             pr->stream));
    CEL_CUDA(cudaStreamSynchronize(pr->stream));
    return CELESTE_OK;
}

celeste_status celeste_catalog_score(celeste_problem* pr, const double* est, const double* tru, int32_t n,
                                     double* score) {
    if (!pr || !score || n < 0 || (n > 0 && (!est || !tru))) return fail(CELESTE_ERR_ARG, "null pointer or n < 0");
    CEL_CUDA(cudaSetDevice(pr->device));
    const size_t rows = (size_t)CELESTE_CAT_NFIELD * n;
    const size_t need = 2 * rows + CELESTE_SCORE_NFIELD;
    if (pr->scr_cap < need) {
        void* p;
        celeste_status s = dalloc(pr, &p, need * sizeof(double));
        if (s) return s;
        pr->d_scr = (double*)p;
        pr->scr_cap = need;
    }
    double* d_est = pr->d_scr;
    double* d_tru = d_est + rows;
    double* d_score = d_tru + rows;
    if (n > 0) {
        CEL_CUDA(cudaMemcpyAsync(d_est, est, sizeof(double) * rows, cudaMemcpyHostToDevice, pr->stream));
        CEL_CUDA(cudaMemcpyAsync(d_tru, tru, sizeof(double) * rows, cudaMemcpyHostToDevice, pr->stream));
    }
    CEL_CUDA(launch_score(n, d_est, d_tru, d_score, pr->stream));
    CEL_CUDA(cudaMemcpyAsync(score, d_score, sizeof(double) * CELESTE_SCORE_NFIELD, cudaMemcpyDeviceToHost,
                             pr->stream));
    CEL_CUDA(cudaStreamSynchronize(pr->stream));
    pr->last_stream = pr->stream;
    return CELESTE_OK;
}

celeste_status celeste_render_device(celeste_problem* pr, const double* d_theta, double* d_e, double* d_v,
                                     void* stream) {
    if (!pr || !d_theta || !d_e) return fail(CELESTE_ERR_ARG, "null problem, theta or E image");
    CEL_CUDA(cudaSetDevice(pr->device));
    cudaStream_t st = (cudaStream_t)stream;
    pr->last_stream = st;
    // the FP64 evaluation's map passes with the caller's images as the maps: k_contrib
    // writes the singly covered pixels, k_gather the multiply covered ones
    DevProblem R = pr->P;
    R.emap = d_e;
    R.vmap = d_v ? d_v : pr->P.vmap;
    CEL_CUDA(cudaMemsetAsync(R.status, 0, sizeof(int32_t), st));
    CEL_CUDA(launch_fill_sky(R, d_e, (double*)R.vmap, st));
    CEL_CUDA(launch_prep(R, d_theta, CELESTE_FP64, st));
    CEL_CUDA(launch_contrib(R, CELESTE_FP64, st));
    CEL_CUDA(launch_gather(R, CELESTE_FP64, st));
    return CELESTE_OK;
}

celeste_status celeste_render(celeste_problem* pr, const double* theta, double* e, double* v) {
    if (!pr || !theta || !e) return fail(CELESTE_ERR_ARG, "null problem, theta or E image");
    celeste_status s = check_theta_host(theta, pr->P.n_src);
    if (s) return s;
    CEL_CUDA(cudaSetDevice(pr->device));
    const size_t npx = (size_t)pr->P.n_px;
    const size_t need = 2 * npx;
    if (pr->scr_cap < need) {
        void* p;
        s = dalloc(pr, &p, need * sizeof(double));
        if (s) return s;
        pr->d_scr = (double*)p;
        pr->scr_cap = need;
    }
    CEL_CUDA(cudaMemcpyAsync(pr->d_theta, theta, sizeof(double) * NP * pr->P.n_src, cudaMemcpyHostToDevice,
                             pr->stream));
    s = celeste_render_device(pr, pr->d_theta, pr->d_scr, pr->d_scr + npx, pr->stream);
    if (s) return s;
    CEL_CUDA(cudaMemcpyAsync(e, pr->d_scr, sizeof(double) * npx, cudaMemcpyDeviceToHost, pr->stream));
    if (v) CEL_CUDA(cudaMemcpyAsync(v, pr->d_scr + npx, sizeof(double) * npx, cudaMemcpyDeviceToHost, pr->stream));
    CEL_CUDA(cudaStreamSynchronize(pr->stream));
    return celeste_device_status(pr);
}

celeste_status celeste_device_status(celeste_problem* pr) {
    if (!pr) return fail(CELESTE_ERR_ARG, "null problem");
    CEL_CUDA(cudaSetDevice(pr->device));
    CEL_CUDA(cudaStreamSynchronize(pr->last_stream));
    int32_t v = 0;
    CEL_CUDA(cudaMemcpy(&v, pr->P.status, sizeof v, cudaMemcpyDeviceToHost));
    if (v != 0) return fail(v, "device-side check failed with status %d", v);
    return CELESTE_OK;
}

}  // extern "C"
