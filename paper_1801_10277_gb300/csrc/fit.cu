// Block-coordinate trust-region Newton fit (Section IV-D): each source's 44 parameters
// form a block; sources whose patches never intersect (one colour of a greedy colouring
// of the neighbour graph) are optimised together, each with the others fixed; a
// source's step is a Newton step with its exact Hessian inside a trust region
// (Nocedal & Wright, Chapter 4).
//
// Per colour the batch runs in lock step; one iteration is
//   k_prep / k_contrib   E_s, Var_s of every batch source at theta
//   k_batch_maps         E = E_other + E_s and Var at the batch pixels (patches of one
//                        colour are disjoint, so every pixel has one writer)
//   k_hess / k_finalize_hess   ELBO_s, gradient and Hessian (44 x 44)
//   k_tr_step            one CTA per source: free coordinates (41), the trust-region
//                        subproblem (More-Sorensen with Cholesky factorisations), the
//                        candidate point
//   k_prep / k_contrib   E_s, Var_s at the candidate
//   k_batch_dll          per-pixel change of the log-likelihood (stable difference form)
//   k_tr_accept          actual / predicted gain, radius update, accept or reject
// The iteration is captured once per colour as a CUDA graph and replayed; the host
// reads one counter (sources still iterating) per replay.  A per-source mask
// (k_mark_active, after the step and after the acceptance) lets every pixel kernel skip
// the items of a source that has stopped iterating, so a replay costs in proportion to
// the sources still active.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <vector>

#include "internal.cuh"
#include "problem.cuh"
#include "source_math.cuh"

namespace cel {

cudaError_t launch_finalize_hess(const DevProblem& P, const double* d_theta, double* d_local,
                                 double* d_grad, double* d_hess, cudaStream_t st);

namespace {

// K_LO: added to every softmax weight, so that a weight whose softmax underflows keeps
// 1 / k and 1 / k^2 (the KL's derivatives in k) finite in FP64 (above ~1e-104 the sum is
// the softmax itself)
constexpr double BOX_LO = 0.01, BOX_HI = 0.99, A_LO = 0.005, A_HI = 0.995, K_LO = 1e-120;
enum : int { ST_ACTIVE = -1, ST_CONVERGED = 0, ST_MAXITER = 1, ST_NONFINITE = 2 };

__device__ __forceinline__ double sigm(double x) { return 1.0 / (1.0 + exp(-x)); }

// theta(t): identity for u, angle, r1, c1; exp for scale, r2, c2; box sigmoids for
// e_dev, e_axis and the star probability; softmax (last logit 0) plus K_LO for k.
// One warp (every lane calls it): lane j < 28 writes parameter j, lanes 8 i + d (< 16)
// the weight k_id.  Every exponential of the map is one lane's, so the warp runs two
// FP64 exp sequences instead of thirty on one lane (the FP64 pipe charges a warp
// instruction the same however few lanes are active); the softmax denominator is summed
// in component order on every lane of its group.
__device__ void free_to_theta_warp(const double* t, double* th) {
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    if (lane < 28) {
        const int j = lane;
        double v;
        if (j == P_EDEV || j == P_AXIS) v = BOX_LO + (BOX_HI - BOX_LO) * sigm(t[j]);
        else if (j == P_SCALE || j == P_R2 || j == P_R2 + 1 || (j >= P_C2 && j < P_C2 + 8)) v = exp(t[j]);
        else if (j == P_A) v = A_LO + (A_HI - A_LO) * sigm(t[26]);
        else if (j == P_A + 1) v = 1.0 - (A_LO + (A_HI - A_LO) * sigm(t[26]));
        else v = t[j];
        th[j] = v;
    }
    const int i = (lane >> 3) & 1, d = lane & 7;
    double ex = 0.0;
    if (lane < 16) {
        double m = 0.0;
        for (int e = 0; e < 7; ++e) m = fmax(m, t[27 + 7 * i + e]);
        ex = exp((d < 7 ? t[27 + 7 * i + d] : 0.0) - m);
    }
    double den = 0.0;
    for (int e = 0; e < 8; ++e) den += __shfl_sync(full, ex, 8 * i + e);
    if (lane < 16) th[P_K + 8 * i + d] = K_LO + ex / den;
}

__device__ void theta_to_free(const double* th, double* t) {
    // a fitted parameter can sit on its bound after rounding (the sigmoid of a large free
    // coordinate is 1 in FP64); the fraction is kept 1e-15 inside so the free coordinate
    // stays finite and a fit can resume from its own result
    auto logit = [](double p) {
        p = fmin(fmax(p, 1e-15), 1.0 - 1e-15);
        return log(p / (1.0 - p));
    };
    t[0] = th[0];
    t[1] = th[1];
    t[2] = logit((th[P_EDEV] - BOX_LO) / (BOX_HI - BOX_LO));
    t[3] = logit((th[P_AXIS] - BOX_LO) / (BOX_HI - BOX_LO));
    t[4] = th[P_ANGLE];
    t[5] = log(th[P_SCALE]);
    t[6] = th[P_R1];
    t[7] = th[P_R1 + 1];
    t[8] = log(th[P_R2]);
    t[9] = log(th[P_R2 + 1]);
    for (int j = 0; j < 8; ++j) {
        t[10 + j] = th[P_C1 + j];
        t[18 + j] = log(th[P_C2 + j]);
    }
    t[26] = logit((th[P_A] - A_LO) / (A_HI - A_LO));
    for (int i = 0; i < 2; ++i)
        for (int e = 0; e < 7; ++e) t[27 + 7 * i + e] = log(th[P_K + 8 * i + e] / th[P_K + 8 * i + 7]);
}

// ------------------------------------------------------------------------------------
// batch kernels

// E_other, Var_other at every batch pixel: sky plus every other source covering it
// (tile lists, ascending source order), from the current global E_s / Var_s buffers.
// Region-task stages (task non-null): a covering source of another task than the batch
// source's contributes its stage-start terms (spEs, spVs), as if it had not moved.
template <class R>
__global__ void k_other(const WorkItem* __restrict__ bitems, const PatchGeo* __restrict__ bgeo,
                        const PatchGeo* __restrict__ geo, const ImgMeta* __restrict__ img,
                        const Tile* __restrict__ tiles, const int32_t* __restrict__ tile_list,
                        const int32_t* __restrict__ tile_grid, const float* __restrict__ sky_map,
                        const R* __restrict__ spE, const R* __restrict__ spV, R* __restrict__ eo,
                        R* __restrict__ vo, CsrBounds cb, const int32_t* __restrict__ task,
                        const R* __restrict__ spEs, const R* __restrict__ spVs) {
    const WorkItem it = bitems[blockIdx.x];
    const int t = threadIdx.x;
    if (t >= it.n) return;
    const PatchGeo g = bgeo[it.patch];
    const ImgMeta& im = img[g.img];
    const int q = it.q0 + t;
    const int yy = q / g.w, xx = q - yy * g.w;
    const int gx = g.x0 + xx, gy = g.y0 + yy;
    if (!CEL_IN_BOUNDS(q < g.w * g.h && gx >= 0 && gx < im.W && gy >= 0 && gy < im.H, cb.status)) return;
    const int64_t m = im.px_off + (int64_t)gy * im.W + gx;
    R E = im.has_sky_map ? (R)sky_map[m] : (R)im.sky;
    R V = 0;
    const int64_t gi = im.tg_off + (int64_t)(gy / TILE) * im.tgw + gx / TILE;
    const int tid = CEL_IN_BOUNDS(gi >= 0 && gi < cb.n_tile_grid, cb.status) ? tile_grid[gi] : -1;
    if (tid >= 0 && CEL_IN_BOUNDS(tid < cb.n_tile, cb.status)) {
        Tile tl = tiles[tid];
        if (!CEL_IN_BOUNDS(tl.list_off >= 0 && tl.list_n >= 0 && (int64_t)tl.list_off + tl.list_n <= cb.n_tile_list,
                           cb.status))
            tl.list_n = 0;
        for (int e = 0; e < tl.list_n; ++e) {
            const int pe = tile_list[tl.list_off + e];
            if (!CEL_IN_BOUNDS(pe >= 0 && pe < cb.n_patch, cb.status)) continue;
            const PatchGeo o = geo[pe];
            if (o.src == it.src) continue;
            const int ox = gx - o.x0, oy = gy - o.y0;
            if (ox >= 0 && ox < o.w && oy >= 0 && oy < o.h) {
                const int64_t qq = o.sp_off + (int64_t)oy * o.w + ox;
                const bool start = task && task[o.src] != task[it.src];
                E += start ? spEs[qq] : spE[qq];
                V += start ? spVs[qq] : spV[qq];
            }
        }
    }
    eo[g.sp_off + q] = E;
    vo[g.sp_off + q] = V;
}

// E, Var maps at the batch pixels from E_other and the batch sources' own terms
template <class R>
__global__ void k_batch_maps(const WorkItem* __restrict__ bitems, const PatchGeo* __restrict__ bgeo,
                             const ImgMeta* __restrict__ img, const R* __restrict__ eo,
                             const R* __restrict__ vo, const R* __restrict__ se,
                             const R* __restrict__ sv, R* __restrict__ emap, R* __restrict__ vmap,
                             const int32_t* __restrict__ src_active) {
    const WorkItem it = bitems[blockIdx.x];
    const int t = threadIdx.x;
    if (t >= it.n) return;
    const PatchGeo g = bgeo[it.patch];
    if (!src_active[g.src]) return;   // a converged source's maps do not change
    const ImgMeta& im = img[g.img];
    const int q = it.q0 + t;
    const int yy = q / g.w, xx = q - yy * g.w;
    const int64_t m = im.px_off + (int64_t)(g.y0 + yy) * im.W + (g.x0 + xx);
    const int64_t b = g.sp_off + q;
    emap[m] = eo[b] + se[b];
    vmap[m] = vo[b] + sv[b];
}

// per-item sum of ll(E', V') - ll(E, V) at the candidate, in a difference form that
// does not cancel:  x (log1p(dE/E) - (dV E^2 - V dE (E + E')) / (2 E^2 E'^2)) - dE
template <class R>
__global__ void k_batch_dll(const WorkItem* __restrict__ bitems, const PatchGeo* __restrict__ bgeo,
                            const ImgMeta* __restrict__ img, const float* __restrict__ pixels,
                            const R* __restrict__ eo, const R* __restrict__ vo,
                            const R* __restrict__ se, const R* __restrict__ sv,
                            const R* __restrict__ ce, const R* __restrict__ cv,
                            double* __restrict__ dll, const int32_t* __restrict__ src_active) {
    __shared__ double red[CHUNK / 32];
    const WorkItem it = bitems[blockIdx.x];
    const int t = threadIdx.x;
    if (!src_active[bgeo[it.patch].src]) return;   // no candidate for a converged source
    R v = 0;
    if (t < it.n) {
        const PatchGeo g = bgeo[it.patch];
        const ImgMeta& im = img[g.img];
        const int q = it.q0 + t;
        const int yy = q / g.w, xx = q - yy * g.w;
        const int64_t m = im.px_off + (int64_t)(g.y0 + yy) * im.W + (g.x0 + xx);
        const int64_t b = g.sp_off + q;
        const R x = (R)pixels[m];
        const R E = eo[b] + se[b], V = vo[b] + sv[b];
        const R dE = ce[b] - se[b], dV = cv[b] - sv[b];
        const R E1 = E + dE;
        const R num = dV * E * E - V * dE * (E + E1);
        v = x * (log1p(dE / E) - num / ((R)2 * E * E * E1 * E1)) - dE;
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((t & 31) == 0) red[t >> 5] = (double)v;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        dll[blockIdx.x] = s;
    }
}

__global__ void k_to_free(int nb, const double* __restrict__ th, double* __restrict__ t) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) theta_to_free(th + (size_t)NP * b, t + (size_t)NT * b);
}

// ------------------------------------------------------------------------------------
// trust-region step: one CTA per batch source

constexpr int TR_THREADS = 128;
constexpr int TRN = NT;   // 41
// k_tr_step's dynamic shared memory: the source's 44 x 44 Hessian and H T (44 x 41)
constexpr size_t TR_DYN_BYTES = sizeof(double) * (NP * NP + NP * TRN);

struct TrState {
    double delta;   // trust radius (free coordinates)
    double pred;    // predicted gain of the candidate
    double pnorm;   // |p|
    double f;       // ELBO_s at theta
    double kl;      // KL at theta
    int32_t status; // ST_*
    int32_t iters;
    int32_t cand;   // a candidate was produced this iteration
    int32_t pad;
    double lam;     // multiplier of the last boundary step (warm start of the next), 0 inside
};

// Packed lower-triangle order of side 40 (every trailing triangle of n = 41), copied
// into shared memory by each CTA
constexpr int PK_N = (TRN - 1) * TRN / 2;
__device__ const PackedTriangle<TRN - 1> g_pk = packed_triangle<TRN - 1>();

__device__ void packed_table(uint16_t* pk) {
    for (int idx = threadIdx.x; idx < PK_N; idx += blockDim.x) pk[idx] = g_pk.v[idx];
}

// Cholesky of (B + lam I) into L (lower, row-major n x n, n <= TRN); returns success to
// all threads.  Right-looking, two barriers per column: step k scales column k by the
// pivot's 1 / sqrt(d_k) (its diagonal becomes sqrt(d_k)), then updates the trailing
// triangle with one FMA per entry, L_ij -= L_ik L_jk (entries dealt out in packed order,
// pk).  The thread that updates (k + 1, k + 1), the next pivot, takes its FP64 rsqrt at
// once, so the pivot is ready at the barrier.  On GB300's narrow FP64 pipe the
// factorisation is bound by its FP64 instruction count (a warp instruction costs the
// same however few lanes are active), so each pivot's square root and reciprocal come
// from one thread and the update is a single FMA.
// T = double, or float for the multiplier search (the same steps, FP32's reciprocal
// square root).
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }

template <class T>
__device__ bool block_chol(const T* B, T lam, T* L, int n, int* flag, T* rcp, const uint16_t* pk) {
    const int tid = threadIdx.x, nt = blockDim.x;
    auto pivot = [&](int k, T d) {
        if (!(d > (T)0) || !isfinite(d)) {
            *flag = 0;
        } else {
            const T r = rsqrt_t(d);
            rcp[k] = r;           // 1 / sqrt(d)
            rcp[n + k] = r * r;   // 1 / d
        }
    };
    for (int i = tid; i < n * n; i += nt) {
        const int r = i / n, c = i - r * n;
        L[i] = (c <= r) ? B[i] + (r == c ? lam : (T)0) : (T)0;
    }
    if (tid == 0) {
        *flag = 1;
        pivot(0, L[0]);   // this thread wrote L[0]
    }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (!*flag) return false;
        const T r = rcp[k];
        for (int i = k + tid; i < n; i += nt) L[i * n + k] *= r;
        __syncthreads();
        const int m = n - k - 1;
        const int cnt = m * (m + 1) / 2;
        for (int idx = tid; idx < cnt; idx += nt) {
            const int ab = pk[idx];
            const int i = k + 1 + (ab >> 8), j = k + 1 + (ab & 255);
            const T v = fma(-L[i * n + k], L[j * n + k], L[i * n + j]);
            L[i * n + j] = v;
            if (idx == 0) pivot(k + 1, v);
        }
        __syncthreads();
    }
    return true;
}

// Warp-level triangular solves (every lane of the calling warp calls them): lane l holds
// rows l and l + 32 of the right-hand side; one column of L per step (column-oriented
// substitution), the solved entry broadcast by shuffle.  invd[k] = 1 / L[k][k].  The
// arrays must not overlap.
template <class T>
__device__ void warp_fwd(const T* __restrict__ L, const T* __restrict__ invd, const T* __restrict__ b,
                         T* __restrict__ y, int n) {
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    T r0 = lane < n ? b[lane] : (T)0, r1 = lane + 32 < n ? b[lane + 32] : (T)0;
    for (int k = 0; k < n; ++k) {
        const T rk = __shfl_sync(full, k < 32 ? r0 : r1, k & 31);
        const T yk = rk * invd[k];
        if (lane == (k & 31)) y[k] = yk;
        if (lane > k && lane < n) r0 -= L[lane * n + k] * yk;
        if (lane + 32 > k && lane + 32 < n) r1 -= L[(lane + 32) * n + k] * yk;
    }
    __syncwarp();
}

template <class T>
__device__ void warp_bwd(const T* __restrict__ L, const T* __restrict__ invd, const T* __restrict__ y,
                         T* __restrict__ x, int n) {
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    T r0 = lane < n ? y[lane] : (T)0, r1 = lane + 32 < n ? y[lane + 32] : (T)0;
    for (int k = n - 1; k >= 0; --k) {
        const T rk = __shfl_sync(full, k < 32 ? r0 : r1, k & 31);
        const T xk = rk * invd[k];
        if (lane == (k & 31)) x[k] = xk;
        if (lane < k) r0 -= L[k * n + lane] * xk;
        if (lane + 32 < k) r1 -= L[k * n + lane + 32] * xk;
    }
    __syncwarp();
}

// Sum over the 32 lanes of a warp (every lane gets it).  The FP64 pipe charges a warp
// instruction whatever the active lanes, so a vector of 41 is summed lane-parallel (two
// entries a lane) and reduced in five steps rather than looped on one lane.
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(TR_THREADS)
k_tr_step(int nb, const double* __restrict__ theta, const double* __restrict__ tfree,
          const double* __restrict__ f_in, const double* __restrict__ g_in,
          const double* __restrict__ h_in, const double* __restrict__ kl_in,
          double* __restrict__ theta_c, double* __restrict__ tfree_c, TrState* __restrict__ st,
          celeste_fit_options o, int32_t* __restrict__ active) {
    const int b = blockIdx.x;
    if (b >= nb) return;
    __shared__ TrState S;
    __shared__ double gt[TRN], Ht[TRN * TRN], L[TRN * TRN], cvec[TRN], p[TRN], w[TRN];
    __shared__ double th[NP], tt[TRN], g44[NP];
    __shared__ int tn[TRN], tj[TRN][8];
    __shared__ double tv[TRN][8];
    __shared__ int flag, done;
    __shared__ double lam_s, pn_s;
    __shared__ uint16_t pk[PK_N];
    extern __shared__ double tr_dyn[];
    double* Hs = tr_dyn;             // [NP][NP] the source's Hessian
    double* X = tr_dyn + NP * NP;    // [NP][TRN] H T
    const int tid = threadIdx.x;
    if (tid == 0) S = st[b];
    __syncthreads();
    if (S.status != ST_ACTIVE) {
        if (tid == 0) st[b].cand = 0;
        return;
    }
    for (int i = tid; i < NP; i += blockDim.x) {
        th[i] = theta[(size_t)NP * b + i];
        g44[i] = g_in[(size_t)NP * b + i];
    }
    for (int i = tid; i < TRN; i += blockDim.x) tt[i] = tfree[(size_t)NT * b + i];
    {
        const double* H44 = h_in + (size_t)NP * NP * b;
        for (int i = tid; i < NP * NP; i += blockDim.x) Hs[i] = H44[i];
    }
    packed_table(pk);
    __syncthreads();
    // columns of T = d theta / d t
    if (tid < TRN) {
        const int a = tid;
        int n = 0;
        auto put = [&](int j, double v) {
            tj[a][n] = j;
            tv[a][n] = v;
            ++n;
        };
        if (a == 2 || a == 3) {
            const double s = sigm(tt[a]);
            put(a, (BOX_HI - BOX_LO) * s * (1.0 - s));
        } else if (a == 5 || a == 8 || a == 9 || (a >= 18 && a < 26)) {
            put(a, th[a]);
        } else if (a == 26) {
            const double s = sigm(tt[26]);
            const double d = (A_HI - A_LO) * s * (1.0 - s);
            put(P_A, d);
            put(P_A + 1, -d);
        } else if (a >= 27) {
            const int i = (a - 27) / 7, e = (a - 27) % 7;
            const double pe = th[P_K + 8 * i + e];
            for (int d = 0; d < 8; ++d) {
                const double pd = th[P_K + 8 * i + d];
                put(P_K + 8 * i + d, pd * ((d == e ? 1.0 : 0.0) - pe));
            }
        } else {
            put(a, 1.0);
        }
        tn[a] = n;
        double s = 0.0;
        for (int u = 0; u < n; ++u) s += tv[a][u] * g44[tj[a][u]];
        gt[a] = s;
    }
    __syncthreads();
    // Ht = T' H T + sum_j g_j d2 theta_j / dt dt, T' H T as two sparse products from
    // shared memory: X = H T, then T' X
    for (int idx = tid; idx < NP * TRN; idx += blockDim.x) {
        const int r = idx / TRN, c = idx - r * TRN;
        double x = 0.0;
        for (int v = 0; v < tn[c]; ++v) x += Hs[r * NP + tj[c][v]] * tv[c][v];
        X[idx] = x;
    }
    __syncthreads();
    for (int idx = tid; idx < TRN * TRN; idx += blockDim.x) {
        const int a = idx / TRN, c = idx % TRN;
        double s = 0.0;
        for (int u = 0; u < tn[a]; ++u) s += tv[a][u] * X[tj[a][u] * TRN + c];
        if (a == c) {
            if (a == 2 || a == 3) {
                const double sg = sigm(tt[a]);
                s += g44[a] * (BOX_HI - BOX_LO) * sg * (1.0 - sg) * (1.0 - 2.0 * sg);
            } else if (a == 5 || a == 8 || a == 9 || (a >= 18 && a < 26)) {
                s += g44[a] * th[a];
            } else if (a == 26) {
                const double sg = sigm(tt[26]);
                s += (g44[P_A] - g44[P_A + 1]) * (A_HI - A_LO) * sg * (1.0 - sg) * (1.0 - 2.0 * sg);
            }
        }
        if (a >= 27 && c >= 27 && (a - 27) / 7 == (c - 27) / 7) {
            const int i = (a - 27) / 7, e = (a - 27) % 7, f = (c - 27) % 7;
            const double pe = th[P_K + 8 * i + e], pf = th[P_K + 8 * i + f];
            for (int d = 0; d < 8; ++d) {
                const double pd = th[P_K + 8 * i + d];
                const double de = (d == e) ? 1.0 : 0.0, df = (d == f) ? 1.0 : 0.0;
                const double ef = (e == f) ? 1.0 : 0.0;
                s += g44[P_K + 8 * i + d] * pd * ((de - pe) * (df - pf) - pe * (ef - pf));
            }
        }
        Ht[idx] = s;
    }
    __syncthreads();
    // convergence checks (every thread a share of the entries)
    {
        bool bad = false;
        for (int i = tid; i < TRN * TRN; i += blockDim.x) bad = bad || !isfinite(Ht[i]);
        bool gbig = false;
        if (tid < TRN) {
            bad = bad || !isfinite(gt[tid]);
            gbig = !(fabs(gt[tid]) <= o.grad_tol);
        }
        const int any_bad = __syncthreads_or(bad || (tid == 0 && !isfinite(f_in[b])));
        const int any_big = __syncthreads_or(gbig);
        if (tid == 0) {
            done = 0;
            if (any_bad) {
                S.status = ST_NONFINITE;
                done = 1;
            } else if (!any_big) {
                S.status = ST_CONVERGED;
                done = 1;
            }
            S.f = f_in[b];
            S.kl = kl_in[b];
        }
    }
    __syncthreads();
    if (done) {
        if (tid == 0) {
            S.cand = 0;
            st[b] = S;
        }
        return;
    }
    // minimise m(p) = c.p + p.B p / 2, |p| <= Delta with c = -gt, B = -Ht
    for (int i = tid; i < TRN * TRN; i += blockDim.x) Ht[i] = -Ht[i];   // Ht now holds B
    for (int i = tid; i < TRN; i += blockDim.x) cvec[i] = -gt[i];
    __syncthreads();
    const double Delta = S.delta;
    // |c|, the largest absolute row sum of B and its smallest diagonal entry: one row per
    // thread, then combined in row order
    __shared__ double rs[TRN], invd[TRN];
    if (tid < TRN) {
        double r = 0.0;
        for (int j = 0; j < TRN; ++j) r += fabs(Ht[tid * TRN + j]);
        rs[tid] = r;
    }
    __syncthreads();
    __shared__ double bnd[3];
    if (tid < 32) {
        double c2 = 0.0, bn = 0.0, bd = 1e300;
        for (int i = tid; i < TRN; i += 32) {
            c2 += cvec[i] * cvec[i];
            bn = fmax(bn, rs[i]);
            bd = fmin(bd, Ht[i * TRN + i]);
        }
        c2 = warp_sum_d(c2);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            bn = fmax(bn, __shfl_xor_sync(0xffffffffu, bn, o));
            bd = fmin(bd, __shfl_xor_sync(0xffffffffu, bd, o));
        }
        if (tid == 0) {
            bnd[0] = c2;
            bnd[1] = bn;
            bnd[2] = bd;
        }
    }
    __syncthreads();
    const double cn = sqrt(bnd[0]), bnorm = bnd[1], bdmin = bnd[2];
    double lamL = fmax(0.0, fmax(-bdmin, cn / Delta - bnorm));
    double lamU = cn / Delta + bnorm;
    double lam = 0.0;
    for (int i = tid; i < TRN; i += blockDim.x) p[i] = 0.0;   // a zero step if nothing factors
    if (tid == 0) pn_s = 0.0;
    __syncthreads();
    __shared__ double rcp[2 * TRN];
    bool ok = block_chol(Ht, 0.0, L, TRN, &flag, rcp, pk);
    bool solved = false;
    if (ok) {
        if (tid < TRN) invd[tid] = rcp[tid];
        __syncthreads();
        if (tid < 32) {
            warp_fwd(L, invd, cvec, w, TRN);
            warp_bwd(L, invd, w, p, TRN);
            double s = 0.0;
            for (int i = tid; i < TRN; i += 32) {
                p[i] = -p[i];
                s += p[i] * p[i];
            }
            s = warp_sum_d(s);
            if (tid == 0) pn_s = sqrt(s);
        }
        __syncthreads();
        if (pn_s <= Delta) solved = true;
        else lam = fmax(lamL, 0.0);
    }
    if (!solved) {
        lam = fmax(lamL, fmax(1e-3 * lamU, sqrt(fmax(lamL, 1e-300) * lamU)));
        // the previous iteration's multiplier, when still inside the bracket, is usually
        // close: the Hessian and the radius change little between Newton iterations
        if (S.lam > lamL && S.lam < lamU) lam = S.lam;
        if (ok) lamL = fmax(lamL, 0.0);
        // The multiplier search in FP32 (a pipe 64 times the FP64 pipe's width): the same
        // safeguarded Newton iteration on 1 / |p(lam)| - 1 / Delta, to |p| within 1e-4 of
        // Delta (at most 16 factorisations); its multiplier starts the FP64 loop below,
        // which then needs one or two.  The FP32 bracket is not kept: FP32 rounding can
        // misjudge definiteness near the smallest eigenvalue.
        {
            float* B32 = reinterpret_cast<float*>(tr_dyn);   // H and H T are dead by now
            float* L32 = B32 + TRN * TRN;
            float* c32 = L32 + TRN * TRN;
            float *y32 = c32 + TRN, *p32 = y32 + TRN, *w32 = p32 + TRN, *r32 = w32 + TRN;   // r32: 2 TRN
            for (int i = tid; i < TRN * TRN; i += blockDim.x) B32[i] = (float)Ht[i];
            for (int i = tid; i < TRN; i += blockDim.x) c32[i] = (float)cvec[i];
            __syncthreads();
            double l = lam, lo = lamL, hi = lamU;
            for (int it = 0; it < 16; ++it) {
                const bool pd = block_chol<float>(B32, (float)l, L32, TRN, &flag, r32, pk);
                if (tid < 32) {
                    double nl = l;
                    int dn = 0;
                    if (!pd) {
                        lo = fmax(lo, l);
                        nl = fmax(sqrt(fmax(lo, 1e-300) * hi), lo + 0.01 * (hi - lo));
                    } else {
                        warp_fwd<float>(L32, r32, c32, y32, TRN);
                        warp_bwd<float>(L32, r32, y32, p32, TRN);
                        float sp = 0.f;
                        for (int i = tid; i < TRN; i += 32) sp += p32[i] * p32[i];
                        const double pn = sqrt((double)warp_sum_f(sp));
                        if (fabs(pn - Delta) <= 1e-4 * Delta) {
                            dn = 1;
                        } else {
                            if (pn < Delta) hi = l;
                            else lo = l;
                            warp_fwd<float>(L32, r32, p32, w32, TRN);
                            float sw = 0.f;
                            for (int i = tid; i < TRN; i += 32) sw += w32[i] * w32[i];
                            const double wn = (double)warp_sum_f(sw);
                            nl = l + (pn * pn / wn) * (pn - Delta) / Delta;
                            if (!(nl > lo && nl < hi)) nl = fmax(sqrt(fmax(lo, 1e-300) * hi), lo + 0.01 * (hi - lo));
                            if (hi - lo <= 1e-6 * fmax(1.0, hi)) dn = 1;
                        }
                    }
                    if (tid == 0) {
                        done = dn;
                        lam_s = nl;
                    }
                }
                __syncthreads();
                l = lam_s;
                const int stop = done;
                __syncthreads();   // every thread has read done and lam_s
                if (stop) break;
            }
            if (l > lamL && l < lamU) lam = l;
        }
        for (int it = 0; it < 200; ++it) {
            const bool pd = block_chol(Ht, lam, L, TRN, &flag, rcp, pk);
            if (pd && tid < TRN) invd[tid] = rcp[tid];
            __syncthreads();
            if (tid < 32) {
                double nl = 0.0;
                if (!pd) {
                    lamL = fmax(lamL, lam);
                    nl = fmax(sqrt(fmax(lamL, 1e-300) * lamU), lamL + 0.01 * (lamU - lamL));
                    if (tid == 0) done = 0;
                } else {
                    // p = -(B + lam I)^-1 c, then w = L^-1 p for Newton's step on 1/|p|
                    warp_fwd(L, invd, cvec, w, TRN);
                    warp_bwd(L, invd, w, p, TRN);
                    double s = 0.0;
                    for (int i = tid; i < TRN; i += 32) {
                        p[i] = -p[i];
                        s += p[i] * p[i];
                    }
                    const double pn = sqrt(warp_sum_d(s));
                    if (tid == 0) pn_s = pn;
                    __syncwarp();
                    int dn;
                    // |p| within 1e-6 of the radius: the step's model value is then
                    // within ~1e-6 of the subproblem's optimum, far below what the
                    // ratio test resolves; the bracket stops at 1e-10 relative
                    if (fabs(pn - Delta) <= 1e-6 * Delta) {
                        dn = 1;
                    } else {
                        if (pn < Delta) lamU = lam;
                        else lamL = lam;
                        warp_fwd(L, invd, p, w, TRN);
                        double wn = 0.0;
                        for (int i = tid; i < TRN; i += 32) wn += w[i] * w[i];
                        wn = warp_sum_d(wn);
                        nl = lam + (pn * pn / wn) * (pn - Delta) / Delta;
                        if (!(nl > lamL && nl < lamU))
                            nl = fmax(sqrt(fmax(lamL, 1e-300) * lamU), lamL + 0.01 * (lamU - lamL));
                        dn = (lamU - lamL <= 1e-10 * fmax(1.0, lamU)) ? 2 : 0;
                    }
                    if (tid == 0) done = dn;
                }
                if (tid == 0 && !done) lam_s = nl;
            }
            __syncthreads();
            if (done) break;
            lam = lam_s;
            // every thread follows warp 0's bracket (warp 0 updated its own copies)
            if (tid == 0) { rs[0] = lamL; rs[1] = lamU; }
            __syncthreads();
            lamL = rs[0];
            lamU = rs[1];
            __syncthreads();
        }
        // hard case: |p| < Delta with lambda pinned at -lambda_min: add tau z, z from
        // inverse iteration with the last factorisation
        if (done == 2 && pn_s < Delta) {
            __shared__ double zs[TRN], ys[TRN];
            if (tid < 32) {
                for (int i = tid; i < TRN; i += 32) zs[i] = 1.0 + 0.01 * i;
                __syncwarp();
                for (int r = 0; r < 6; ++r) {
                    warp_fwd(L, invd, zs, ys, TRN);
                    warp_bwd(L, invd, ys, w, TRN);
                    double zn = 0.0;
                    for (int i = 0; i < TRN; ++i) zn += w[i] * w[i];
                    zn = sqrt(zn);
                    __syncwarp();
                    for (int i = tid; i < TRN; i += 32) zs[i] = w[i] / zn;
                    __syncwarp();
                }
            }
            __syncthreads();
            if (tid == 0) {
                double z[TRN];
                for (int i = 0; i < TRN; ++i) z[i] = zs[i];
                double pz = 0.0, pp = 0.0;
                for (int i = 0; i < TRN; ++i) {
                    pz += p[i] * z[i];
                    pp += p[i] * p[i];
                }
                const double disc = sqrt(fmax(0.0, pz * pz + Delta * Delta - pp));
                const double t1 = -pz + disc, t2 = -pz - disc;
                // pick the root with the lower model value: m(p + t z) - m(p) = -lam t p.z + t^2 z'Bz/2
                double zbz = 0.0;
                for (int i = 0; i < TRN; ++i) {
                    double s = 0.0;
                    for (int j = 0; j < TRN; ++j) s += Ht[i * TRN + j] * z[j];
                    zbz += z[i] * s;
                }
                const double m1 = -lam * t1 * pz + 0.5 * t1 * t1 * zbz;
                const double m2 = -lam * t2 * pz + 0.5 * t2 * t2 * zbz;
                const double tau = (m1 <= m2) ? t1 : t2;
                for (int i = 0; i < TRN; ++i) p[i] += tau * z[i];
                pn_s = Delta;
            }
            __syncthreads();
        }
    }
    // predicted gain of the maximisation: g.p + p.H p / 2 = -(c.p + p.B p / 2); the rows
    // of B p one per thread, the sum in row order
    if (tid < TRN) {
        double s = 0.0;
        for (int j = 0; j < TRN; ++j) s += Ht[tid * TRN + j] * p[j];
        rs[tid] = s;
    }
    __syncthreads();
    double pred = 0.0;
    if (tid < 32) {
        for (int i = tid; i < TRN; i += 32) pred -= cvec[i] * p[i] + 0.5 * p[i] * rs[i];
        pred = warp_sum_d(pred);
    }
    if (tid == 0) {
        S.pred = pred;
        S.pnorm = pn_s;
        S.lam = solved ? 0.0 : lam;
        if (pred <= o.pred_tol_rel * (1.0 + fabs(S.f))) {
            S.status = ST_CONVERGED;
            S.cand = 0;
            done = 1;
        } else {
            S.cand = 1;
            done = 0;
        }
        st[b] = S;
    }
    __syncthreads();
    if (done) return;
    if (tid < TRN) tfree_c[(size_t)NT * b + tid] = tt[tid] + p[tid];
    __syncthreads();
    if (tid < TRN) tt[tid] += p[tid];
    __syncthreads();
    if (tid < 32) free_to_theta_warp(tt, theta_c + (size_t)NP * b);
    if (tid == 0) atomicAdd(active, 1);
}

// ratio of actual to predicted gain, radius update, acceptance: one warp per source (the
// candidate's KL lane-parallel in FP64, the log-likelihood change summed over the
// source's items by the lanes), so the FP64 work spreads over every SM
__global__ void __launch_bounds__(32)
k_tr_accept(int nb, const int32_t* __restrict__ bpatch_off, const PatchGeo* __restrict__ bgeo,
            const double* __restrict__ dll, const ModelDev* __restrict__ md, double* __restrict__ theta,
            double* __restrict__ tfree, const double* __restrict__ theta_c,
            const double* __restrict__ tfree_c, TrState* __restrict__ st, celeste_fit_options o) {
    const int b = blockIdx.x;
    if (b >= nb) return;
    const int lane = threadIdx.x;
    __shared__ TrState S;
    __shared__ double thc[NP], kg[NP];
    __shared__ int accept;
    if (lane == 0) S = st[b];
    __syncwarp();
    if (S.status != ST_ACTIVE || !S.cand) return;
    for (int i = lane; i < NP; i += 32) thc[i] = theta_c[(size_t)NP * b + i];
    __syncwarp();
    double d = 0.0;
    for (int p = bpatch_off[b]; p < bpatch_off[b + 1]; ++p) {
        const PatchGeo g = bgeo[p];
        for (int it = g.item0 + lane; it < g.item0 + g.nitem; it += 32) d += dll[it];
    }
    d = warp_sum_d(d);
    const double klc = kl_warp<double>(*md, thc, thc, kg);
    if (lane == 0) {
        const double df = d - (klc - S.kl);
        const double scale = 1.0 + fabs(S.f);
        double rho = (S.pred <= o.f_noise_rel * scale) ? 1.0 : df / S.pred;
        if (!isfinite(df)) rho = -1.0;
        if (rho < 0.25) S.delta = 0.25 * S.delta;
        else if (rho > 0.75 && S.pnorm >= (1.0 - 1e-9) * S.delta) S.delta = fmin(2.0 * S.delta, o.delta_max);
        accept = rho > o.eta;
        S.iters += 1;
        if (S.iters >= o.max_iter) S.status = ST_MAXITER;
        S.cand = 0;
        st[b] = S;
    }
    __syncwarp();
    if (accept) {
        for (int i = lane; i < NP; i += 32) theta[(size_t)NP * b + i] = thc[i];
        for (int i = lane; i < NT; i += 32) tfree[(size_t)NT * b + i] = tfree_c[(size_t)NT * b + i];
    }
}

__global__ void k_gather_theta(int nb, const int32_t* __restrict__ bsrc,
                               const double* __restrict__ theta, double* __restrict__ bth) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nb * NP) bth[i] = theta[(size_t)NP * bsrc[i / NP] + i % NP];
}

__global__ void k_scatter_theta(int nb, const int32_t* __restrict__ bsrc,
                                const double* __restrict__ bth, double* __restrict__ theta) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nb * NP) theta[(size_t)NP * bsrc[i / NP] + i % NP] = bth[i];
}

// per batch source: 1 while its Newton iterations continue (its pixel work is skipped after)
__global__ void k_mark_active(int nb, const TrState* __restrict__ st, int32_t* __restrict__ act) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) act[b] = st[b].status == ST_ACTIVE ? 1 : 0;
}

__global__ void k_init_state(int nb, TrState* st, double delta0) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    TrState S{};
    S.delta = delta0;
    S.status = ST_ACTIVE;
    st[b] = S;
}

// ------------------------------------------------------------------------------------
// host side

struct DevBuf {
    std::vector<void*> ptrs;
    ~DevBuf() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <class T>
    cudaError_t alloc(T** p, size_t n) {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
        if (e == cudaSuccess) ptrs.push_back(q);
        *p = (T*)q;
        return e;
    }
};

struct Batch {
    std::vector<int32_t> src;        // global ids
    std::vector<int32_t> patch_off;  // batch CSR
    std::vector<PatchGeo> geo;       // batch patches (src = batch index, sp_off batch-local)
    std::vector<WorkItem> items;     // patch = batch patch, src = GLOBAL id
    int64_t n_sp = 0;
};

Batch make_batch(const celeste_problem* pr, const std::vector<int32_t>& members) {
    Batch B;
    B.src = members;
    B.patch_off.push_back(0);
    for (int bi = 0; bi < (int)members.size(); ++bi) {
        const int s = members[bi];
        for (int p = pr->patch_off[s]; p < pr->patch_off[s + 1]; ++p) {
            PatchGeo g = pr->geo[p];
            g.src = bi;
            g.sp_off = B.n_sp;
            g.item0 = (int)B.items.size();
            const int npx = g.w * g.h;
            for (int q0 = 0; q0 < npx; q0 += CHUNK)
                B.items.push_back({(int)B.geo.size(), q0, std::min(CHUNK, npx - q0), s});
            g.nitem = (int)B.items.size() - g.item0;
            B.n_sp += npx;
            B.geo.push_back(g);
        }
        B.patch_off.push_back((int)B.geo.size());
    }
    return B;
}

// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the output for counter c is the
// finaliser applied to seed + (c + 1) * golden gamma.
uint64_t splitmix64(uint64_t seed, uint64_t c) {
    uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Sweep g's visiting order when the caller gives none: Fisher-Yates over the moving
// sources in ascending id, draw i of sweep g keyed by counter (g << 32) + i.
void shuffled_order(const std::vector<int32_t>& moving, uint64_t seed, int g, std::vector<int32_t>& out) {
    out = moving;
    for (int i = (int)out.size() - 1; i > 0; --i) {
        const uint64_t r = splitmix64(seed, ((uint64_t)(uint32_t)g << 32) + (uint64_t)i);
        std::swap(out[i], out[(size_t)(r % (uint64_t)(i + 1))]);
    }
}

int uf_find(std::vector<int>& up, int i) {
    while (up[i] != i) {
        up[i] = up[up[i]];
        i = up[i];
    }
    return i;
}

// Cyclades batches of one order (documented with celeste_cyclades_batches).  pos[s] is
// scratch of size n_src, -1 on entry and on return.  Union-find over the sample's
// internal edges; a component's root is its earliest member, so ranks follow order.
int cyclades_batches(const int32_t* nbr_off, const int32_t* nbrs, const int32_t* order, int m, int B,
                     std::vector<int>& pos, int32_t* batch_of, int32_t* comp_of) {
    std::vector<int> up, cnt;
    int base = 0;
    for (int k0 = 0; k0 < m; k0 += B) {
        const int k1 = std::min(m, k0 + B);
        const int L = k1 - k0;
        for (int i = 0; i < L; ++i) pos[order[k0 + i]] = i;
        up.resize(L);
        for (int i = 0; i < L; ++i) up[i] = i;
        for (int i = 0; i < L; ++i) {
            const int s = order[k0 + i];
            for (int e = nbr_off[s]; e < nbr_off[s + 1]; ++e) {
                const int j = pos[nbrs[e]];
                if (j < 0) continue;
                const int a = uf_find(up, i), b = uf_find(up, j);
                if (a != b) up[std::max(a, b)] = std::min(a, b);   // keep the earliest member
            }
        }
        cnt.assign(L, 0);
        int rounds = 0;
        for (int i = 0; i < L; ++i) {
            const int root = uf_find(up, i);
            batch_of[k0 + i] = base + cnt[root];
            if (comp_of) comp_of[k0 + i] = k0 + root;
            rounds = std::max(rounds, ++cnt[root]);
        }
        for (int i = 0; i < L; ++i) pos[order[k0 + i]] = -1;
        base += rounds;
    }
    return base;
}

}  // namespace

}  // namespace cel

using namespace cel;

celeste_status cel::fit_sources_impl(celeste_problem* pr, double* theta, const int32_t* which,
                                     int32_t n_which, const celeste_fit_options* opts,
                                     int32_t* iters_out, int32_t* status_out, double* elbo_out,
                                     celeste_status (*elbo_fn)(celeste_problem*, const double*, int32_t, double*, double*),
                                     const int32_t* task_of) {
    const DevProblem& P = pr->P;
    const int n = P.n_src;
    int prec = opts->precision;
    cudaStream_t st = pr->stream;
    auto cuda_err = [&](cudaError_t e, const char* w) -> celeste_status {
        char buf[256];
        snprintf(buf, sizeof buf, "%s: %s", w, cudaGetErrorString(e));
        set_last_error(buf);
        return e == cudaErrorMemoryAllocation ? CELESTE_ERR_NOMEM : CELESTE_ERR_CUDA;
    };
#define FIT_CUDA(x)                                          \
    do {                                                     \
        cudaError_t e_ = (x);                                \
        if (e_ != cudaSuccess) return cuda_err(e_, #x);      \
    } while (0)
    std::vector<char> moves(n, which ? 0 : 1);
    if (which)
        for (int k = 0; k < n_which; ++k) {
            if (which[k] < 0 || which[k] >= n) {
                set_last_error("which[] holds an invalid source index");
                return CELESTE_ERR_ARG;
            }
            moves[which[k]] = 1;
        }
    std::vector<int32_t> moving;
    for (int s = 0; s < n; ++s)
        if (moves[s]) moving.push_back(s);
    const int m = (int)moving.size();
    const bool cyclades = opts->schedule == CELESTE_SCHED_CYCLADES;
    // colour schedule: greedy colouring in ascending id over the neighbour graph, one
    // batch per colour, built once
    std::vector<Batch> colour_batches;
    if (!cyclades) {
        std::vector<int32_t> colour(n, 0);
        int ncol = 0;
        for (int s = 0; s < n; ++s) {
            std::vector<char> used(ncol + 2, 0);
            for (int e = pr->nbr_off[s]; e < pr->nbr_off[s + 1]; ++e) {
                const int o = pr->nbrs[e];
                if (o < s && colour[o] <= ncol) used[colour[o]] = 1;
            }
            int c = 0;
            while (used[c]) ++c;
            colour[s] = c;
            ncol = std::max(ncol, c + 1);
        }
        std::vector<std::vector<int32_t>> members(ncol);
        for (int s : moving) members[colour[s]].push_back(s);
        for (int c = 0; c < ncol; ++c) colour_batches.push_back(make_batch(pr, members[c]));
    } else if (opts->order) {
        // every row must be a permutation of the moving sources
        std::vector<int> seen(n, -1);
        for (int r = 0; r < opts->max_sweeps; ++r)
            for (int i = 0; i < m; ++i) {
                const int s = opts->order[(size_t)r * m + i];
                if (s < 0 || s >= n || !moves[s] || seen[s] == r) {
                    char buf[96];
                    snprintf(buf, sizeof buf, "order row %d is not a permutation of the moving sources", r);
                    set_last_error(buf);
                    return CELESTE_ERR_ARG;
                }
                seen[s] = r;
            }
    }
    // device buffers for the largest batch: a colour, or (Cyclades: at most one source
    // per component of a sample) the sample_size moving sources with the most work
    size_t maxB = 1, maxP = 1, maxI = 1;
    int64_t maxSp = 1;
    if (!cyclades) {
        for (const Batch& B : colour_batches) {
            maxB = std::max(maxB, B.src.size());
            maxP = std::max(maxP, B.geo.size());
            maxI = std::max(maxI, B.items.size());
            maxSp = std::max(maxSp, B.n_sp);
        }
    } else {
        std::vector<int64_t> np_, ni_, nsp_;
        for (int s : moving) {
            int64_t a = 0, b = 0, c = 0;
            for (int p = pr->patch_off[s]; p < pr->patch_off[s + 1]; ++p) {
                const int64_t npx = (int64_t)pr->geo[p].w * pr->geo[p].h;
                ++a;
                b += (npx + CHUNK - 1) / CHUNK;
                c += npx;
            }
            np_.push_back(a);
            ni_.push_back(b);
            nsp_.push_back(c);
        }
        const size_t top = std::min<size_t>((size_t)opts->sample_size, moving.size());
        auto top_sum = [&](std::vector<int64_t>& v) {
            std::sort(v.begin(), v.end(), std::greater<int64_t>());
            int64_t t = 0;
            for (size_t i = 0; i < top; ++i) t += v[i];
            return t;
        };
        maxB = std::max<size_t>(1, top);
        maxP = std::max<size_t>(1, (size_t)top_sum(np_));
        maxI = std::max<size_t>(1, (size_t)top_sum(ni_));
        maxSp = std::max<int64_t>(1, top_sum(nsp_));
    }
    // the batches of sweep g (counted over both precision phases)
    std::vector<int> pos(n, -1);
    std::vector<int32_t> ord, bof;
    auto sweep_batches = [&](int g, std::vector<Batch>& out) {
        if (!cyclades) {
            out = colour_batches;
            return;
        }
        if (opts->order) ord.assign(opts->order + (size_t)(g % opts->max_sweeps) * m,
                                    opts->order + (size_t)(g % opts->max_sweeps + 1) * m);
        else shuffled_order(moving, opts->seed, g, ord);
        bof.resize(m);
        const int nbt = cyclades_batches(pr->nbr_off.data(), pr->nbrs.data(), ord.data(), m,
                                         opts->sample_size, pos, bof.data(), nullptr);
        std::vector<std::vector<int32_t>> members(nbt);
        for (int i = 0; i < m; ++i) members[bof[i]].push_back(ord[i]);
        out.clear();
        for (int b = 0; b < nbt; ++b) out.push_back(make_batch(pr, members[b]));
    };
    // device buffers for the largest batch
    DevBuf mem;
    const size_t rs = sizeof(double);   // per-pixel batch buffers serve both precisions
    int32_t *d_bsrc, *d_bpo, *d_active, *d_srcact;
    PatchGeo* d_bgeo;
    WorkItem* d_bitems;
    double *d_bth, *d_bthc, *d_bt, *d_btc, *d_f, *d_g, *d_h, *d_kl, *d_part, *d_dll, *d_tbl64;
    float* d_tbl32;
    TrState* d_st;
    unsigned char *d_eo, *d_vo, *d_se, *d_sv, *d_ce, *d_cv;
    FIT_CUDA(mem.alloc(&d_bsrc, maxB));
    FIT_CUDA(mem.alloc(&d_bpo, maxB + 1));
    FIT_CUDA(mem.alloc(&d_active, 1));
    FIT_CUDA(mem.alloc(&d_srcact, maxB));
    FIT_CUDA(mem.alloc(&d_bgeo, maxP));
    FIT_CUDA(mem.alloc(&d_bitems, maxI));
    FIT_CUDA(mem.alloc(&d_bth, maxB * NP));
    FIT_CUDA(mem.alloc(&d_bthc, maxB * NP));
    FIT_CUDA(mem.alloc(&d_bt, maxB * NT));
    FIT_CUDA(mem.alloc(&d_btc, maxB * NT));
    FIT_CUDA(mem.alloc(&d_f, maxB));
    FIT_CUDA(mem.alloc(&d_g, maxB * NP));
    FIT_CUDA(mem.alloc(&d_h, maxB * NP * NP));
    FIT_CUDA(mem.alloc(&d_kl, maxB));
    FIT_CUDA(mem.alloc(&d_part, maxI * NPART));
    FIT_CUDA(mem.alloc(&d_dll, maxI));
    FIT_CUDA(mem.alloc(&d_tbl64, maxP * TBL_STRIDE));
    FIT_CUDA(mem.alloc(&d_tbl32, maxP * TBL_STRIDE));
    FIT_CUDA(mem.alloc(&d_st, maxB));
    FIT_CUDA(mem.alloc(&d_eo, maxSp * rs));
    FIT_CUDA(mem.alloc(&d_vo, maxSp * rs));
    FIT_CUDA(mem.alloc(&d_se, maxSp * rs));
    FIT_CUDA(mem.alloc(&d_sv, maxSp * rs));
    FIT_CUDA(mem.alloc(&d_ce, maxSp * rs));
    FIT_CUDA(mem.alloc(&d_cv, maxSp * rs));
    int32_t* h_active = nullptr;
    FIT_CUDA(cudaMallocHost((void**)&h_active, sizeof(int32_t)));
    struct HostFree {
        int32_t* p;
        ~HostFree() { cudaFreeHost(p); }
    } hf{h_active};

    // region-task stage: every source's task id, the stage-start parameters and, per
    // precision phase, every source's E_s / Var_s at them
    int32_t* d_task = nullptr;
    double* d_th0 = nullptr;
    unsigned char *d_se0 = nullptr, *d_sv0 = nullptr;
    if (task_of) {
        FIT_CUDA(mem.alloc(&d_task, n));
        FIT_CUDA(mem.alloc(&d_th0, (size_t)n * NP));
        FIT_CUDA(mem.alloc(&d_se0, (size_t)P.n_sp * rs));
        FIT_CUDA(mem.alloc(&d_sv0, (size_t)P.n_sp * rs));
        FIT_CUDA(cudaMemcpyAsync(d_task, task_of, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
        FIT_CUDA(cudaMemcpyAsync(d_th0, theta, sizeof(double) * NP * n, cudaMemcpyHostToDevice, st));
    }
    FIT_CUDA(cudaFuncSetAttribute(k_tr_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TR_DYN_BYTES));
    FIT_CUDA(cudaMemcpyAsync(pr->d_theta, theta, sizeof(double) * NP * n, cudaMemcpyHostToDevice, st));
    std::vector<int32_t> iters(n, 0), status(n, ST_CONVERGED);
    double prev = 0.0;
    {
        celeste_status s0 = elbo_fn(pr, theta, prec, &prev, nullptr);
        if (s0) return s0;
    }
    std::vector<TrState> hst(maxB);
    // phase 0 in the requested precision; with FP32 and refine_fp64, phase 1 polishes in FP64
    const int nphase = (opts->precision == CELESTE_FP32_ACC64 && opts->refine_fp64) ? 2 : 1;
    std::vector<Batch> batches;
    int g_sweep = 0;
    for (int phase = 0; phase < nphase; ++phase) {
    prec = (phase == 0) ? opts->precision : CELESTE_FP64;
    if (phase == 1) {
        celeste_status s2 = elbo_fn(pr, theta, prec, &prev, nullptr);
        if (s2) return s2;
    }
    if (task_of) {
        // the stage-start E_s / Var_s in this phase's precision
        const size_t bytes = (size_t)P.n_sp * (prec == CELESTE_FP64 ? sizeof(double) : sizeof(float));
        FIT_CUDA(launch_prep(P, d_th0, prec, st));
        FIT_CUDA(launch_contrib(P, prec, st));
        FIT_CUDA(cudaMemcpyAsync(d_se0, P.spE, bytes, cudaMemcpyDeviceToDevice, st));
        FIT_CUDA(cudaMemcpyAsync(d_sv0, P.spE2, bytes, cudaMemcpyDeviceToDevice, st));
    }
    int sw = 0;
    for (; sw < opts->max_sweeps; ++sw, ++g_sweep) {
        sweep_batches(g_sweep, batches);
        for (size_t c = 0; c < batches.size(); ++c) {
            const Batch& B = batches[c];
            const int nb = (int)B.src.size();
            if (nb == 0) continue;
            // current E_s / Var_s of every source (global buffers)
            FIT_CUDA(launch_prep(P, pr->d_theta, prec, st));
            FIT_CUDA(launch_contrib(P, prec, st));
            FIT_CUDA(cudaMemcpyAsync(d_bsrc, B.src.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, st));
            FIT_CUDA(cudaMemcpyAsync(d_bpo, B.patch_off.data(), sizeof(int32_t) * (nb + 1), cudaMemcpyHostToDevice, st));
            FIT_CUDA(cudaMemcpyAsync(d_bgeo, B.geo.data(), sizeof(PatchGeo) * B.geo.size(), cudaMemcpyHostToDevice, st));
            FIT_CUDA(cudaMemcpyAsync(d_bitems, B.items.data(), sizeof(WorkItem) * B.items.size(), cudaMemcpyHostToDevice, st));
            const int nI = (int)B.items.size();
            if (nI > 0) {
                if (prec == CELESTE_FP64)
                    k_other<double><<<nI, CHUNK, 0, st>>>(d_bitems, d_bgeo, P.geo, P.img, P.tiles, P.tile_list,
                                                         P.tile_grid, P.sky_map, (const double*)P.spE,
                                                         (const double*)P.spE2, (double*)d_eo, (double*)d_vo,
                                                         csr_bounds(P), d_task, (const double*)d_se0,
                                                         (const double*)d_sv0);
                else
                    k_other<float><<<nI, CHUNK, 0, st>>>(d_bitems, d_bgeo, P.geo, P.img, P.tiles, P.tile_list,
                                                        P.tile_grid, P.sky_map, (const float*)P.spE,
                                                        (const float*)P.spE2, (float*)d_eo, (float*)d_vo,
                                                        csr_bounds(P), d_task, (const float*)d_se0,
                                                        (const float*)d_sv0);
            }
            k_gather_theta<<<(nb * NP + 255) / 256, 256, 0, st>>>(nb, d_bsrc, pr->d_theta, d_bth);
            k_to_free<<<(nb + 127) / 128, 128, 0, st>>>(nb, d_bth, d_bt);
            k_init_state<<<(nb + 127) / 128, 128, 0, st>>>(nb, d_st, opts->delta0);
            k_mark_active<<<(nb + 127) / 128, 128, 0, st>>>(nb, d_st, d_srcact);
            FIT_CUDA(cudaGetLastError());
            // batch views of the problem
            DevProblem Pb = P;
            Pb.n_src = nb;
            Pb.n_patch = (int)B.geo.size();
            Pb.n_item = nI;
            Pb.n_sp = B.n_sp;
            Pb.geo = d_bgeo;
            Pb.items = d_bitems;
            Pb.patch_off = d_bpo;
            Pb.tbl64 = d_tbl64;
            Pb.tbl32 = d_tbl32;
            Pb.spE = d_se;
            Pb.spE2 = d_sv;
            Pb.item_part = d_part;
            Pb.kl = d_kl;
            Pb.kl_grad = nullptr;   // k_finalize_hess and k_tr_accept take the KL themselves
            Pb.single = nullptr;    // batch buffers keep every E_s / Var_s
            Pb.item_ll = nullptr;
            Pb.status = nullptr;
            // a source that stopped iterating keeps its theta: its pixel work is skipped
            Pb.src_active = d_srcact;
            DevProblem Pc = Pb;
            Pc.spE = d_ce;
            Pc.spE2 = d_cv;
            // one Newton iteration, captured as a graph
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            FIT_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            cudaError_t ce = cudaSuccess;
            auto chk = [&](cudaError_t e) {
                if (ce == cudaSuccess && e != cudaSuccess) ce = e;
            };
            chk(cudaMemsetAsync(d_active, 0, sizeof(int32_t), st));
            chk(launch_prep(Pb, d_bth, prec, st));
            chk(launch_contrib(Pb, prec, st));
            if (nI > 0) {
                if (prec == CELESTE_FP64)
                    k_batch_maps<double><<<nI, CHUNK, 0, st>>>(d_bitems, d_bgeo, P.img, (const double*)d_eo,
                                                               (const double*)d_vo, (const double*)d_se,
                                                               (const double*)d_sv, (double*)P.emap, (double*)P.vmap,
                                                               d_srcact);
                else
                    k_batch_maps<float><<<nI, CHUNK, 0, st>>>(d_bitems, d_bgeo, P.img, (const float*)d_eo,
                                                              (const float*)d_vo, (const float*)d_se,
                                                              (const float*)d_sv, (float*)P.emap, (float*)P.vmap,
                                                              d_srcact);
            }
            chk(launch_hess_pixels(Pb, prec, st));
            chk(launch_finalize_hess(Pb, d_bth, d_f, d_g, d_h, st));
            k_tr_step<<<nb, TR_THREADS, TR_DYN_BYTES, st>>>(nb, d_bth, d_bt, d_f, d_g, d_h, d_kl, d_bthc, d_btc,
                                                 d_st, *opts, d_active);
            // only sources with a candidate evaluate it
            k_mark_active<<<(nb + 127) / 128, 128, 0, st>>>(nb, d_st, d_srcact);
            chk(launch_prep(Pc, d_bthc, prec, st));
            chk(launch_contrib(Pc, prec, st));
            if (nI > 0) {
                if (prec == CELESTE_FP64)
                    k_batch_dll<double><<<nI, CHUNK, 0, st>>>(d_bitems, d_bgeo, P.img, P.pixels,
                                                              (const double*)d_eo, (const double*)d_vo,
                                                              (const double*)d_se, (const double*)d_sv,
                                                              (const double*)d_ce, (const double*)d_cv, d_dll,
                                                              d_srcact);
                else
                    k_batch_dll<float><<<nI, CHUNK, 0, st>>>(d_bitems, d_bgeo, P.img, P.pixels,
                                                             (const float*)d_eo, (const float*)d_vo,
                                                             (const float*)d_se, (const float*)d_sv,
                                                             (const float*)d_ce, (const float*)d_cv, d_dll,
                                                             d_srcact);
            }
            k_tr_accept<<<nb, 32, 0, st>>>(nb, d_bpo, d_bgeo, d_dll, P.model, d_bth, d_bt, d_bthc, d_btc,
                                           d_st, *opts);
            k_mark_active<<<(nb + 127) / 128, 128, 0, st>>>(nb, d_st, d_srcact);
            chk(cudaGetLastError());
            chk(cudaMemcpyAsync(h_active, d_active, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            cudaError_t ee = cudaStreamEndCapture(st, &graph);
            if (ce != cudaSuccess || ee != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return cuda_err(ce != cudaSuccess ? ce : ee, "fit iteration capture");
            }
            ee = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ee != cudaSuccess) return cuda_err(ee, "cudaGraphInstantiate");
            int it = 0;
            for (; it < opts->max_iter + 1; ++it) {
                ee = cudaGraphLaunch(exec, st);
                if (ee == cudaSuccess) ee = cudaStreamSynchronize(st);
                if (ee != cudaSuccess) {
                    cudaGraphExecDestroy(exec);
                    return cuda_err(ee, "fit iteration");
                }
                if (*h_active == 0) break;
            }
            cudaGraphExecDestroy(exec);
            // results of this colour
            k_scatter_theta<<<(nb * NP + 255) / 256, 256, 0, st>>>(nb, d_bsrc, d_bth, pr->d_theta);
            FIT_CUDA(cudaGetLastError());
            FIT_CUDA(cudaMemcpyAsync(hst.data(), d_st, sizeof(TrState) * nb, cudaMemcpyDeviceToHost, st));
            FIT_CUDA(cudaStreamSynchronize(st));
            for (int bi = 0; bi < nb; ++bi) {
                iters[B.src[bi]] += hst[bi].iters;
                status[B.src[bi]] = hst[bi].status == ST_ACTIVE ? ST_MAXITER : hst[bi].status;
            }
        }
        FIT_CUDA(cudaMemcpyAsync(theta, pr->d_theta, sizeof(double) * NP * n, cudaMemcpyDeviceToHost, st));
        FIT_CUDA(cudaStreamSynchronize(st));
        double cur = 0.0;
        celeste_status s1 = elbo_fn(pr, theta, prec, &cur, nullptr);
        if (s1) return s1;
        const double rel = fabs(cur - prev) / fmax(1.0, fabs(cur));
        prev = cur;
        if (rel < opts->sweep_tol) {
            ++sw;
            ++g_sweep;
            break;
        }
    }
    }
    if (iters_out) memcpy(iters_out, iters.data(), sizeof(int32_t) * n);
    if (status_out) memcpy(status_out, status.data(), sizeof(int32_t) * n);
    if (elbo_out) *elbo_out = prev;
    return CELESTE_OK;
#undef FIT_CUDA
}

extern "C" {

void celeste_fit_options_default(celeste_fit_options* o) {
    o->max_iter = 50;
    o->grad_tol = 1e-8;
    o->pred_tol_rel = 1e-12;
    o->delta0 = 1.0;
    o->delta_max = 1e3;
    o->eta = 1e-4;
    o->f_noise_rel = 1e-13;
    o->precision = CELESTE_FP64;
    o->max_sweeps = 20;
    o->sweep_tol = 1e-8;
    o->refine_fp64 = 1;
    o->schedule = CELESTE_SCHED_COLOUR;
    o->sample_size = 64;
    o->seed = 0;
    o->order = nullptr;
}

celeste_status celeste_cyclades_batches(const int32_t* nbr_off, const int32_t* nbrs, int32_t n,
                                        const int32_t* order, int32_t n_order, int32_t sample_size,
                                        int32_t* batch_of, int32_t* comp_of, int32_t* n_batches) {
    if (!nbr_off || !n_batches || n < 0 || n_order < 0 || (n_order > 0 && (!order || !batch_of)) ||
        sample_size < 1) {
        set_last_error("celeste_cyclades_batches: null pointer, n_src or n_order < 0, or sample_size < 1");
        return CELESTE_ERR_ARG;
    }
    if (nbr_off[0] != 0 || (nbr_off[n] > 0 && !nbrs)) {
        set_last_error("celeste_cyclades_batches: bad neighbour offsets");
        return CELESTE_ERR_ARG;
    }
    for (int s = 0; s < n; ++s) {
        if (nbr_off[s + 1] < nbr_off[s]) {
            set_last_error("celeste_cyclades_batches: neighbour offsets decrease");
            return CELESTE_ERR_ARG;
        }
    }
    for (int e = 0; e < nbr_off[n]; ++e)
        if (nbrs[e] < 0 || nbrs[e] >= n) {
            set_last_error("celeste_cyclades_batches: neighbour id out of range");
            return CELESTE_ERR_ARG;
        }
    std::vector<int> pos(n, -1);
    for (int i = 0; i < n_order; ++i) {
        const int s = order[i];
        if (s < 0 || s >= n || pos[s] >= 0) {
            char buf[96];
            snprintf(buf, sizeof buf, "celeste_cyclades_batches: order[%d] = %d is out of range or repeated", i, s);
            set_last_error(buf);
            return CELESTE_ERR_ARG;
        }
        pos[s] = i;
    }
    for (int i = 0; i < n_order; ++i) pos[order[i]] = -1;
    *n_batches = cyclades_batches(nbr_off, nbrs, order, n_order, sample_size, pos, batch_of, comp_of);
    return CELESTE_OK;
}

}  // extern "C"
