"""Region tasks (Section IV-A) written out plainly: the recursive weighted-median cut of
the sky into tasks, the shifted second stage, and a stage of task fits.

TEST INFRASTRUCTURE ONLY: the tests compare the library's task generation and task
fits with these functions.

Definitions (the paper describes the idea; the details are this reading):
* a region is cut while its sources' work exceeds max_work and it holds more than one
  source;
* the cut runs across the longer side of the region's box (x when the box is at least
  as wide as it is tall), at the weighted median: the sources sorted by that coordinate
  (ties by index); the shortest prefix whose work reaches half of the region's goes to
  the lower side (at least one source stays on the upper side); the cut value is the
  midpoint of the two neighbouring coordinates; equal coordinates there leave the
  region whole;
* tasks are the leaves numbered depth first, lower side first; the root box is the
  bounding box of all positions;
* stage two uses the same regions shifted by a fixed vector: a source belongs to the
  task whose region contains its position minus the shift.
"""
from __future__ import annotations

import numpy as np


def partition(pos, work, max_work):
    """The task tree as nested tuples: ("leaf", task) or ("cut", axis, value, lo, hi)."""
    pos = np.asarray(pos, np.float64).reshape(-1, 2)
    work = np.asarray(work, np.float64)
    counter = [0]

    def leaf():
        counter[0] += 1
        return ("leaf", counter[0] - 1)

    def split(members, box):
        total = 0.0
        for s in members:
            total += work[s]
        if len(members) <= 1 or total <= max_work:
            return leaf()
        (x0, x1), (y0, y1) = box
        axis = 0 if (x1 - x0) >= (y1 - y0) else 1
        order = sorted(members, key=lambda s: (pos[s, axis], s))
        acc = 0.0
        k = 0
        while k < len(order) - 1:
            acc += work[order[k]]
            if acc >= 0.5 * total:
                break
            k += 1
        k = min(k, len(order) - 2)
        a, b = pos[order[k], axis], pos[order[k + 1], axis]
        cut = 0.5 * (a + b)
        if not (a < cut <= b):
            return leaf()
        lo_box = [list(box[0]), list(box[1])]
        hi_box = [list(box[0]), list(box[1])]
        lo_box[axis][1] = cut
        hi_box[axis][0] = cut
        lo = split(order[:k + 1], lo_box)
        hi = split(order[k + 1:], hi_box)
        return ("cut", axis, cut, lo, hi)

    if len(pos) == 0:
        return None, 0
    box = [[pos[:, 0].min(), pos[:, 0].max()], [pos[:, 1].min(), pos[:, 1].max()]]
    tree = split(list(range(len(pos))), box)
    return tree, counter[0]


def task_of_point(tree, x, y):
    node = tree
    while node[0] == "cut":
        _, axis, cut, lo, hi = node
        node = lo if (x if axis == 0 else y) < cut else hi
    return node[1]


def make_tasks(pos, work, max_work, shift=(0.0, 0.0)):
    """(task of every source, number of tasks) for one stage."""
    pos = np.asarray(pos, np.float64).reshape(-1, 2)
    tree, n = partition(pos, work, max_work)
    out = np.array([task_of_point(tree, p[0] - shift[0], p[1] - shift[1]) for p in pos], np.int32)
    return out, n


def fit_stage(orc, theta, task_of, **fit_kw):
    """Every task fitted from the same starting parameters with all other sources held
    there, the results merged (tasks side by side on separate nodes)."""
    theta = np.asarray(theta, np.float64)
    out = theta.copy()
    iters = np.zeros(theta.shape[0], np.int32)
    status = np.zeros(theta.shape[0], np.int32)
    for k in range(int(np.max(task_of)) + 1 if len(task_of) else 0):
        members = np.flatnonzero(np.asarray(task_of) == k).astype(np.int32)
        if len(members) == 0:
            continue
        th, it, st, _, _ = orc.fit(theta, which=members, **fit_kw)
        out[members] = th[members]
        iters[members] = it[members]
        status[members] = st[members]
    return out, iters, status
