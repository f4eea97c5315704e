// Region tasks (Section IV-A): the sky is cut recursively into regions of roughly equal
// expected work, each region's sources form one task optimised with every other source
// held fixed, and a second stage repeats this on the same regions shifted by a fixed
// amount, so that sources near a first-stage border lie inside a second-stage region.
//
// On one GPU a stage's tasks run one after another from the same starting parameters
// (each task sees its neighbours' stage-start values, as tasks on different nodes do)
// and their results are merged; within a task the fit batches its sources as usual.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "internal.cuh"
#include "problem.cuh"

namespace cel {

namespace {

// One node of the recursive partition: a leaf is a task; an inner node cuts its box at
// `cut` along `axis` (points with coordinate < cut go left).
struct TaskNode {
    int axis = -1;       // -1 = leaf
    double cut = 0.0;
    int left = -1, right = -1;
    int task = -1;
};

// Split the sources idx (all inside the box of node `me`) until a region's work is at
// most max_work or it holds one source.  The cut runs across the box's longer side, at
// the weighted median: sources sorted by that coordinate (ties by id), the first prefix
// whose work reaches half the region's goes left, and the cut lies halfway between the
// last source on the left and the first on the right.
int build(std::vector<TaskNode>& nodes, const double* pos, const double* work, std::vector<int> idx,
          double x0, double x1, double y0, double y1, double max_work, int* n_tasks) {
    const int me = (int)nodes.size();
    nodes.emplace_back();
    double total = 0.0;
    for (int s : idx) total += work[s];
    if (idx.size() <= 1 || total <= max_work) {
        nodes[me].task = (*n_tasks)++;
        return me;
    }
    const int axis = (x1 - x0 >= y1 - y0) ? 0 : 1;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) {
        const double pa = pos[2 * a + axis], pb = pos[2 * b + axis];
        return pa < pb || (pa == pb && a < b);
    });
    const int m = (int)idx.size();
    double acc = 0.0;
    int k = 0;
    for (; k < m - 1; ++k) {
        acc += work[idx[k]];
        if (acc >= 0.5 * total) break;
    }
    k = std::min(k, m - 2);   // both sides keep a source
    const double cut = 0.5 * (pos[2 * idx[k] + axis] + pos[2 * idx[k + 1] + axis]);
    std::vector<int> lo(idx.begin(), idx.begin() + k + 1), hi(idx.begin() + k + 1, idx.end());
    // equal coordinates on both sides of the cut cannot be told apart by a point
    // location: keep the region whole
    if (!(pos[2 * idx[k] + axis] < cut) || !(pos[2 * idx[k + 1] + axis] >= cut)) {
        nodes[me].task = (*n_tasks)++;
        return me;
    }
    nodes[me].axis = axis;
    nodes[me].cut = cut;
    int l, r;
    if (axis == 0) {
        l = build(nodes, pos, work, std::move(lo), x0, cut, y0, y1, max_work, n_tasks);
        r = build(nodes, pos, work, std::move(hi), cut, x1, y0, y1, max_work, n_tasks);
    } else {
        l = build(nodes, pos, work, std::move(lo), x0, x1, y0, cut, max_work, n_tasks);
        r = build(nodes, pos, work, std::move(hi), x0, x1, cut, y1, max_work, n_tasks);
    }
    nodes[me].left = l;
    nodes[me].right = r;
    return me;
}

int locate(const std::vector<TaskNode>& nodes, double x, double y) {
    int n = 0;
    while (nodes[n].axis >= 0) n = ((nodes[n].axis == 0 ? x : y) < nodes[n].cut) ? nodes[n].left : nodes[n].right;
    return nodes[n].task;
}

}  // namespace

}  // namespace cel

using namespace cel;

extern "C" {

celeste_status celeste_make_tasks(const double* pos, const double* work, int32_t n, double max_work,
                                  const double* shift, int32_t* task_of, int32_t* n_tasks) {
    if (n < 0 || !n_tasks || (n > 0 && (!pos || !work || !task_of)) || !(max_work > 0)) {
        set_last_error("celeste_make_tasks: null pointer, n < 0 or max_work <= 0");
        return CELESTE_ERR_ARG;
    }
    for (int s = 0; s < n; ++s)
        if (!isfinite(pos[2 * s]) || !isfinite(pos[2 * s + 1]) || !(work[s] >= 0) || !isfinite(work[s])) {
            char buf[96];
            snprintf(buf, sizeof buf, "celeste_make_tasks: source %d has a non-finite position or bad work", s);
            set_last_error(buf);
            return CELESTE_ERR_ARG;
        }
    if (shift && (!isfinite(shift[0]) || !isfinite(shift[1]))) {
        set_last_error("celeste_make_tasks: shift not finite");
        return CELESTE_ERR_ARG;
    }
    *n_tasks = 0;
    if (n == 0) return CELESTE_OK;
    double x0 = pos[0], x1 = pos[0], y0 = pos[1], y1 = pos[1];
    for (int s = 1; s < n; ++s) {
        x0 = fmin(x0, pos[2 * s]);
        x1 = fmax(x1, pos[2 * s]);
        y0 = fmin(y0, pos[2 * s + 1]);
        y1 = fmax(y1, pos[2 * s + 1]);
    }
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::vector<TaskNode> nodes;
    build(nodes, pos, work, std::move(idx), x0, x1, y0, y1, max_work, n_tasks);
    const double dx = shift ? shift[0] : 0.0, dy = shift ? shift[1] : 0.0;
    for (int s = 0; s < n; ++s)
        task_of[s] = locate(nodes, pos[2 * s] - dx, pos[2 * s + 1] - dy);
    return CELESTE_OK;
}

celeste_status celeste_fit_tasks(celeste_problem* pr, double* theta, const int32_t* task_of,
                                 const celeste_fit_options* opts, int32_t* iters_out, int32_t* status_out,
                                 double* elbo_out) {
    if (!pr || !theta || !task_of) {
        set_last_error("celeste_fit_tasks: null problem, theta or task_of");
        return CELESTE_ERR_ARG;
    }
    const int n = pr->P.n_src;
    std::vector<int32_t> members;
    for (int s = 0; s < n; ++s) {
        if (task_of[s] < -1) {
            set_last_error("celeste_fit_tasks: task ids must be >= -1");
            return CELESTE_ERR_ARG;
        }
        if (task_of[s] >= 0) members.push_back(s);
    }
    if (iters_out) memset(iters_out, 0, sizeof(int32_t) * n);
    if (status_out) memset(status_out, 0, sizeof(int32_t) * n);
    // Every task side by side in one fit over the union of the tasks' sources: the
    // colour batches are those of the whole neighbour graph, so a batch mixes tasks
    // without two of its sources overlapping, and each source sees the sources of other
    // tasks at their stage-start terms.  A source's iterates are then those of its
    // task's own fit from the stage start.
    if (members.empty()) {
        if (!elbo_out) return CELESTE_OK;
        celeste_fit_options o;
        if (opts) o = *opts;
        else celeste_fit_options_default(&o);
        const int prec = (o.precision == CELESTE_FP32_ACC64 && o.refine_fp64) ? CELESTE_FP64 : o.precision;
        return celeste_elbo(pr, theta, prec, elbo_out, nullptr);
    }
    std::vector<int32_t> it(n), st(n);
    const celeste_status e = cel::fit_sources_checked(pr, theta, members.data(), (int32_t)members.size(), opts,
                                                      it.data(), st.data(), elbo_out, task_of);
    if (e) return e;
    for (int s : members) {
        if (iters_out) iters_out[s] = it[s];
        if (status_out) status_out[s] = st[s];
    }
    return CELESTE_OK;
}

}  // extern "C"
