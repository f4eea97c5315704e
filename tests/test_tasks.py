"""Region tasks (Section IV-A): the oracle's partition pinned by hand-worked cases and
its defining properties, the library's host partition bit for bit against it, and the
oracle's stage of task fits (tasks from one snapshot, results merged) against its own
per-task fits."""
import numpy as np
import pytest

from oracle import tasks as OT
from paper_1801_10277_gb300 import synth


_PROBS = {}


def _prob(cfg):
    if cfg not in _PROBS:   # the multi-epoch layout with fewer sources keeps this quick
        _PROBS[cfg] = synth.config(cfg, n_src=3000) if cfg == 3 else synth.config(cfg)
    return _PROBS[cfg]


def _work(prob):
    w = (prob.patches[:, 3].astype(np.int64) * prob.patches[:, 4]).astype(np.float64)
    out = np.zeros(prob.n_src)
    np.add.at(out, np.repeat(np.arange(prob.n_src), np.diff(prob.patch_offsets)), w)
    return out


def test_hand_worked_partition():
    # four unit-work sources at the corners of a 10 x 8 box: the first cut is along x
    # (the wider side) between x = 0 and x = 10, then each 5 x 8 half along y
    pos = np.array([[0, 0], [10, 0], [0, 8], [10, 8]], np.float64)
    t, n = OT.make_tasks(pos, np.ones(4), max_work=1.0)
    assert n == 4 and list(t) == [0, 2, 1, 3]
    tree, _ = OT.partition(pos, np.ones(4), 1.0)
    assert tree[0] == "cut" and tree[1] == 0 and tree[2] == 5.0
    # everything fits one task
    t, n = OT.make_tasks(pos, np.ones(4), max_work=4.0)
    assert n == 1 and set(t) == {0}
    # a heavy source takes a side of its own
    t, n = OT.make_tasks(np.array([[0, 0], [1, 0], [2, 0], [3, 0]], float), [10, 1, 1, 1], max_work=5.0)
    assert n == 2 and list(t) == [0, 1, 1, 1]
    # identical positions cannot be separated
    t, n = OT.make_tasks(np.zeros((3, 2)), np.ones(3), max_work=1.0)
    assert n == 1


def test_shifted_stage():
    pos = np.array([[0, 0], [10, 0], [0, 8], [10, 8]], np.float64)
    t0, _ = OT.make_tasks(pos, np.ones(4), 1.0)
    t1, _ = OT.make_tasks(pos, np.ones(4), 1.0, shift=(0.0, 0.0))
    assert list(t0) == list(t1)
    # shifted by (6, 0): the right column's points land left of the x cut at 5
    t2, _ = OT.make_tasks(pos, np.ones(4), 1.0, shift=(6.0, 0.0))
    assert list(t2) == [0, 0, 1, 1]


@pytest.mark.parametrize("cfg,parts", [(1, 4), (1, 16), (2, 4), (3, 64)])
def test_partition_properties(cfg, parts):
    prob = _prob(cfg)
    pos, work = prob.theta[:, 0:2], _work(prob)
    mw = work.sum() / parts
    t, n = OT.make_tasks(pos, work, mw)
    assert t.min() == 0 and t.max() == n - 1 and len(np.unique(t)) == n
    per = np.bincount(t, weights=work, minlength=n)
    cnt = np.bincount(t, minlength=n)
    assert np.all((per <= mw) | (cnt == 1))
    # a weighted-median cut splits work into near halves: no task below a tenth of the cap
    assert per.min() >= 0.1 * mw
    # every source lies in its task's region: points located through the tree agree
    tree, _ = OT.partition(pos, work, mw)
    for s in range(0, prob.n_src, max(1, prob.n_src // 200)):
        assert OT.task_of_point(tree, *pos[s]) == t[s]


@pytest.mark.parametrize("cfg,parts,shift", [(1, 4, None), (1, 16, (150.0, 90.0)), (2, 8, (20.0, -7.5)),
                                             (3, 64, (200.0, 0.0))])
def test_library_partition_matches_oracle(cfg, parts, shift):
    from paper_1801_10277_gb300 import celeste
    prob = _prob(cfg)
    pos, work = prob.theta[:, 0:2], _work(prob)
    lt, ln = celeste.make_tasks(pos, work, work.sum() / parts, shift)
    ot, on = OT.make_tasks(pos, work, work.sum() / parts, (0.0, 0.0) if shift is None else shift)
    assert ln == on
    np.testing.assert_array_equal(lt, ot)


def test_library_partition_rejects_bad_input():
    from paper_1801_10277_gb300 import celeste
    with pytest.raises(celeste.CelesteError):
        celeste.make_tasks(np.zeros((2, 2)), [1.0, -1.0], 1.0)
    with pytest.raises(celeste.CelesteError):
        celeste.make_tasks(np.array([[0, np.nan], [1, 1]]), [1.0, 1.0], 1.0)
    with pytest.raises(celeste.CelesteError):
        celeste.make_tasks(np.zeros((2, 2)), [1.0, 1.0], 0.0)
    t, n = celeste.make_tasks(np.zeros((0, 2)), np.zeros(0), 1.0)
    assert n == 0 and len(t) == 0
