// Host-side problem object shared by the C-ABI translation units (not installed).
#pragma once

#include <string>
#include <vector>

#include "internal.cuh"

struct celeste_problem {
    using PatchGeo = cel::PatchGeo;
    using ImgMeta = cel::ImgMeta;
    using DevProblem = cel::DevProblem;
    int device = 0;
    DevProblem P{};
    cudaStream_t stream = nullptr;       // stream of the host-pointer entry points
    cudaStream_t last_stream = nullptr;  // stream of the last enqueued call
    // the fused FP32 pass and the total run on a low-priority side stream, forked from and
    // joined back into the caller's stream by these events
    cudaStream_t side = nullptr;
    cudaEvent_t ev_prep = nullptr, ev_fused = nullptr, ev_gather = nullptr, ev_join = nullptr;
    // one evaluation (status reset + every launch of both streams) captured as a CUDA graph
    // per argument set, replayed by later calls with the same arguments
    struct GraphKey {
        int precision, mode, tune_c, tune_a, cap;
        const void* ptr[5];   // theta, total, local, grad, hess
        bool operator==(const GraphKey& o) const {
            if (precision != o.precision || mode != o.mode || tune_c != o.tune_c || tune_a != o.tune_a ||
                cap != o.cap)
                return false;
            for (int i = 0; i < 5; ++i)
                if (ptr[i] != o.ptr[i]) return false;
            return true;
        }
    };
    std::vector<std::pair<GraphKey, cudaGraphExec_t>> graphs;
    cudaStream_t capture = nullptr;       // private stream the graphs are captured on
    // host copies used by the fit's host loop and validation
    std::vector<int32_t> patch_off, nbr_off, nbrs;
    std::vector<PatchGeo> geo;
    std::vector<ImgMeta> imgs;
    int64_t sp_single = 0;               // singly covered source-pixels
    int64_t other_evals = 0;             // (pixel, other covering patch) pairs of the item kernel
    // device buffers owned by the problem
    std::vector<void*> owned;
    double* d_theta = nullptr;
    double* d_out = nullptr;     // total(1) | local(n_src) | grad(n_src*44) | hess(n_src*44*44)
    size_t out_cap = 0;
    int32_t* h_status = nullptr; // pinned copy of the device status word (host-pointer calls)
    double* d_scr = nullptr;     // catalog / score scratch, grown on demand
    size_t scr_cap = 0;
    // per-kernel CUDA-event timing (celeste_profile_*)
    bool profile = false;
    bool profile_serial = false;   // every stage on the calling stream, one after another
    struct Rec { std::string name; cudaEvent_t a, b; int n_kernels; };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    std::vector<std::string> names;
    std::vector<double> ms;
    std::vector<int32_t> launches;
};
