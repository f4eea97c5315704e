// celeste_patch_elbo_grad_noalloc: the ELBO + gradient path for one source whose
// light falls in one patch, with every intermediate buffer taken from a fixed
// device array compiled into the library instead of from cudaMalloc.
//
// Who needs it: a host program whose device memory is owned by another allocator
// (a framework's caching pool that hands out every byte), or code that must not
// call cudaMalloc / cudaFree on a latency-critical path, cannot use
// celeste_problem_create, which allocates the problem's device copies.  This entry
// point allocates nothing: the caller passes its inputs and outputs as device
// pointers, and the scratch lives in g_noalloc_scratch below.
//
// The scratch array is a file-scope __device__ array, so every GPU that loads the
// library holds it (CELESTE_NOALLOC_SCRATCH_BYTES) until the process exits.  In host
// code its name is only a host-side stand-in for the symbol; the device address is
// obtained with cudaGetSymbolAddress on every call made outside a stream capture (with
// the device current), so a device reset or a recreated context is picked up; a call
// inside a capture uses the address of the last uncaptured call on that device (the
// first call on a device must therefore be uncaptured).  The model is checked and
// converted by build_model_dev, as in celeste_problem_create.
#include <math.h>
#include <string.h>

#include <mutex>

#include "internal.cuh"

using namespace cel;

namespace {

// ---- scratch layout (bytes, 256-aligned pieces) ------------------------------------
constexpr int NA_MAX_SIDE = 101;                                  // largest patch side
constexpr int NA_MAX_PX = NA_MAX_SIDE * NA_MAX_SIDE;              // 10201 pixels
constexpr int NA_MAX_ITEMS = (NA_MAX_PX + CHUNK - 1) / CHUNK;     // 40 work items
constexpr int NA_TILES_SIDE = (NA_MAX_SIDE + TILE - 1) / TILE;    // 7
constexpr int NA_MAX_TILES = NA_TILES_SIDE * NA_TILES_SIDE;       // 49 tiles

constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t OFF_IMG = 0;
constexpr size_t OFF_GEO = OFF_IMG + al(sizeof(ImgMeta));
constexpr size_t OFF_ITEMS = OFF_GEO + al(sizeof(PatchGeo));
constexpr size_t OFF_TILES = OFF_ITEMS + al(sizeof(WorkItem) * NA_MAX_ITEMS);
constexpr size_t OFF_TLIST = OFF_TILES + al(sizeof(Tile) * NA_MAX_TILES);
constexpr size_t OFF_POFF = OFF_TLIST + al(sizeof(int32_t) * NA_MAX_TILES);
constexpr size_t OFF_MODEL = OFF_POFF + al(sizeof(int32_t) * 2);
constexpr size_t OFF_TBL64 = OFF_MODEL + al(sizeof(ModelDev));
constexpr size_t OFF_TBL32 = OFF_TBL64 + al(sizeof(double) * TBL_STRIDE);
constexpr size_t OFF_SPE = OFF_TBL32 + al(sizeof(float) * TBL_STRIDE);
constexpr size_t OFF_SPV = OFF_SPE + al(sizeof(double) * NA_MAX_PX);
constexpr size_t OFF_EMAP = OFF_SPV + al(sizeof(double) * NA_MAX_PX);
constexpr size_t OFF_VMAP = OFF_EMAP + al(sizeof(double) * NA_MAX_PX);
constexpr size_t OFF_PART = OFF_VMAP + al(sizeof(double) * NA_MAX_PX);
constexpr size_t OFF_TILELL = OFF_PART + al(sizeof(double) * NPART * NA_MAX_ITEMS);
constexpr size_t OFF_KL = OFF_TILELL + al(sizeof(double) * NA_MAX_TILES);
constexpr size_t OFF_KLG = OFF_KL + al(sizeof(double));
constexpr size_t OFF_SRCTOT = OFF_KLG + al(sizeof(double) * NP);
constexpr size_t OFF_DONE = OFF_SRCTOT + al(sizeof(double));
constexpr size_t OFF_STATUS = OFF_DONE + al(sizeof(int32_t));
constexpr size_t NA_BYTES = OFF_STATUS + al(sizeof(int32_t));

}  // namespace

// The shared scratch of every call on a device (see the header for the limits).
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

namespace {

static_assert(NA_BYTES <= (size_t)CELESTE_NOALLOC_SCRATCH_BYTES, "scratch larger than documented");

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
unsigned char* g_na_ptr[NA_MAX_DEVICES] = {nullptr};

celeste_status na_fail(celeste_status st, const char* msg) {
    set_last_error(msg);   // read back with celeste_last_error()
    return st;
}

// Writes the problem description (kernel parameters) into the scratch array and
// builds the work items and tiles of the single patch.
__global__ void k_noalloc_setup(unsigned char* base, ImgMeta im, ModelDev md, int w, int h) {
    ImgMeta* d_img = (ImgMeta*)(base + OFF_IMG);
    PatchGeo* d_geo = (PatchGeo*)(base + OFF_GEO);
    WorkItem* d_items = (WorkItem*)(base + OFF_ITEMS);
    Tile* d_tiles = (Tile*)(base + OFF_TILES);
    int32_t* d_tlist = (int32_t*)(base + OFF_TLIST);
    int32_t* d_poff = (int32_t*)(base + OFF_POFF);
    ModelDev* d_md = (ModelDev*)(base + OFF_MODEL);
    const int npx = w * h, nitem = (npx + CHUNK - 1) / CHUNK;
    const int tw = (w + TILE - 1) / TILE, th = (h + TILE - 1) / TILE;
    if (threadIdx.x == 0) {
        *d_img = im;
        *d_md = md;
        PatchGeo g{};
        g.img = 0; g.x0 = 0; g.y0 = 0; g.w = w; g.h = h; g.src = 0;
        g.sp_off = 0; g.item0 = 0; g.nitem = nitem;
        *d_geo = g;
        d_poff[0] = 0;
        d_poff[1] = 1;
        *(int32_t*)(base + OFF_STATUS) = 0;
        *(int32_t*)(base + OFF_DONE) = 0;
    }
    for (int i = threadIdx.x; i < nitem; i += blockDim.x)
        d_items[i] = WorkItem{0, i * CHUNK, min(CHUNK, npx - i * CHUNK), 0};
    for (int i = threadIdx.x; i < tw * th; i += blockDim.x) {
        Tile t{};
        t.img = 0; t.x0 = (i % tw) * TILE; t.y0 = (i / tw) * TILE; t.list_off = i; t.list_n = 1;
        d_tiles[i] = t;
        d_tlist[i] = 0;
    }
}


}  // namespace

extern "C" celeste_status celeste_patch_elbo_grad_noalloc(
    const celeste_image* im, const celeste_model* model, const celeste_patch* patch,
    const float* d_pixels, const float* d_sky_map, const double* d_theta, int32_t precision,
    double* d_elbo_total, double* d_elbo_local, double* d_grad, void* stream) {
    if (!im || !model || !patch || !d_pixels || !d_theta || !d_grad)
        return na_fail(CELESTE_ERR_ARG, "null argument");
    if (precision != CELESTE_FP64 && precision != CELESTE_FP32_ACC64)
        return na_fail(CELESTE_ERR_ARG, "precision must be CELESTE_FP64 or CELESTE_FP32_ACC64");
    const int w = patch->w, h = patch->h;
    if (w < 1 || h < 1 || w > NA_MAX_SIDE || h > NA_MAX_SIDE)
        return na_fail(CELESTE_ERR_ARG,
                       "patch side outside 1..101: the allocation-free entry point's scratch holds "
                       "at most a 101 x 101 patch");
    if (im->band < 0 || im->band > 4 || im->n_psf < 1 || im->n_psf > MAXPSF || !im->psf ||
        !(im->nmgy_per_count > 0) || (!d_sky_map && !(im->sky > 0)))
        return na_fail(CELESTE_ERR_ARG, "bad image description");
    // the patch is the whole image of this call: shift the WCS so pixel (x0, y0) is the origin
    ImgMeta M;
    memset(&M, 0, sizeof M);
    M.px_off = 0;
    M.H = h;
    M.W = w;
    M.band = im->band;
    M.npsf = im->n_psf;
    M.has_sky_map = d_sky_map != nullptr;
    M.sky = im->sky;
    M.iota = 1.0 / im->nmgy_per_count;
    for (int k = 0; k < 4; ++k) M.A[k] = im->wcs[k];
    M.t[0] = im->wcs[4] - patch->x0;
    M.t[1] = im->wcs[5] - patch->y0;
    for (int k = 0; k < im->n_psf; ++k) {
        const double* ps = im->psf + 6 * k;
        if (!(ps[3] > 0 && ps[5] > 0 && ps[3] * ps[5] - ps[4] * ps[4] > 0))
            return na_fail(CELESTE_ERR_NOT_PD, "PSF covariance not positive definite");
        for (int c = 0; c < 6; ++c) M.psf[k][c] = ps[c];
    }
    fill_float_copies(M);
    ModelDev md;
    {
        const char* why = nullptr;
        const celeste_status ms = build_model_dev(model, md, &why);
        if (ms != CELESTE_OK) return na_fail(ms, why);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES)
        return na_fail(CELESTE_ERR_CUDA, "no current CUDA device");
    cudaStream_t st = (cudaStream_t)stream;
    // The scratch array's address: looked up on every call made outside stream capture
    // (so a device reset or a recreated context is picked up); inside a capture the
    // address of the last uncaptured call on this device is used.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess)
        return na_fail(CELESTE_ERR_CUDA, "cudaStreamIsCapturing failed");
    unsigned char* base;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (cap == cudaStreamCaptureStatusNone) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return na_fail(CELESTE_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
            g_na_ptr[dev] = (unsigned char*)p;
        } else if (!g_na_ptr[dev]) {
            return na_fail(CELESTE_ERR_ARG,
                           "the first call on a device must be made outside a stream capture");
        }
        base = g_na_ptr[dev];
    }
    k_noalloc_setup<<<1, 64, 0, st>>>(base, M, md, w, h);
    DevProblem P{};
    P.n_img = 1; P.n_src = 1; P.n_patch = 1;
    P.n_item = (w * h + CHUNK - 1) / CHUNK;
    P.n_tile = ((w + TILE - 1) / TILE) * ((h + TILE - 1) / TILE);
    P.n_tile_list = P.n_tile;   // tile i lists the patch at entry i
    P.n_img_rec = 1;
    P.npsf_max = im->n_psf;
    P.nprof = model->n_exp + model->n_dev;
    P.n_px = (int64_t)w * h;
    P.n_sp = (int64_t)w * h;
    P.img = (const ImgMeta*)(base + OFF_IMG);
    P.pixels = d_pixels;
    P.sky_map = d_sky_map;
    P.geo = (const PatchGeo*)(base + OFF_GEO);
    P.items = (const WorkItem*)(base + OFF_ITEMS);
    P.tiles = (const Tile*)(base + OFF_TILES);
    P.tile_list = (const int32_t*)(base + OFF_TLIST);
    P.patch_off = (const int32_t*)(base + OFF_POFF);
    P.model = (const ModelDev*)(base + OFF_MODEL);
    P.tbl64 = (double*)(base + OFF_TBL64);
    P.tbl32 = (float*)(base + OFF_TBL32);
    P.spE = base + OFF_SPE;
    P.spE2 = base + OFF_SPV;
    P.emap = base + OFF_EMAP;
    P.vmap = base + OFF_VMAP;
    P.item_part = (double*)(base + OFF_PART);
    P.tile_ll = (double*)(base + OFF_TILELL);
    P.kl = (double*)(base + OFF_KL);
    P.kl_grad = (double*)(base + OFF_KLG);
    P.src_total = (double*)(base + OFF_SRCTOT);
    P.done = (int32_t*)(base + OFF_DONE);
    P.status = (int32_t*)(base + OFF_STATUS);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_prep(P, d_theta, precision, st);
    if (e == cudaSuccess) e = launch_contrib(P, precision, st);
    if (e == cudaSuccess) e = launch_gather(P, precision, st);
    if (e == cudaSuccess) e = launch_adjoint(P, precision, MODE_GRAD, st);
    if (e == cudaSuccess)
        e = launch_finalize(P, d_theta, precision, MODE_GRAD, d_elbo_total, d_elbo_local, d_grad, nullptr, st);
    if (e != cudaSuccess) return na_fail(CELESTE_ERR_CUDA, cudaGetErrorString(e));
    return CELESTE_OK;
}
