"""The Cyclades schedule of the block-coordinate fit (Section IV-D): the oracle's
batches pinned against connected components from networkx, hand-worked cases and the
schedule's defining properties; the library's host scheduler (no GPU needed) against
the oracle, bit for bit."""
import networkx as nx
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1801_10277_gb300 import synth


@pytest.fixture(scope="module")
def crowded():
    return synth.config(2)


def _graph(prob):
    g = nx.Graph()
    g.add_nodes_from(range(prob.n_src))
    for s in range(prob.n_src):
        for o in prob.nbrs[prob.nbr_offsets[s]:prob.nbr_offsets[s + 1]]:
            g.add_edge(s, int(o))
    return g


def _csr(n, edges):
    adj = [[] for _ in range(n)]
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    off = np.zeros(n + 1, np.int32)
    off[1:] = np.cumsum([len(a) for a in adj])
    return off, np.array([o for a in adj for o in sorted(a)], np.int32)


class _Graph:
    """Just the neighbour CSR of a problem, for the oracle's scheduler."""

    def __init__(self, n, edges):
        base = synth.config(0)
        self.n_src = n
        self.nbr_offsets, self.nbrs = _csr(n, edges)
        self.theta = np.repeat(base.theta[:1], n, axis=0)
        self.patches = np.zeros((0, 5), np.int32)
        self.patch_offsets = np.zeros(n + 1, np.int32)
        for k in ("images", "exp_mix", "dev_mix", "prior_star", "prior_r", "prior_c"):
            setattr(self, k, getattr(base, k))


def test_symmetric_neighbour_lists(crowded):
    g = _graph(crowded)
    for s in range(crowded.n_src):
        for o in crowded.nbrs[crowded.nbr_offsets[s]:crowded.nbr_offsets[s + 1]]:
            assert s in crowded.nbrs[crowded.nbr_offsets[o]:crowded.nbr_offsets[o + 1]]
    assert g.number_of_edges() > crowded.n_src   # a crowded case: many conflicts


def test_hand_worked_cases():
    # path 0-1-2, isolated 3, edge 4-5
    G = _Graph(6, [(0, 1), (1, 2), (4, 5)])
    orc = Oracle(G)
    order = [2, 0, 3, 1, 5, 4]
    b, c, nb = orc.cyclades_batches(order, 6)
    # one sample: {2, 0, 1} connected through 1; 3 alone; {5, 4}
    assert list(c) == [0, 0, 2, 0, 4, 4]
    assert list(b) == [0, 1, 0, 2, 0, 1] and nb == 3
    b, c, nb = orc.cyclades_batches(order, 3)
    # samples [2, 0, 3] (2 and 0 do not touch without 1) and [1, 5, 4]
    assert list(c) == [0, 1, 2, 3, 4, 4]
    assert list(b) == [0, 0, 0, 1, 1, 2] and nb == 3
    b, c, nb = orc.cyclades_batches(order, 1)   # one source at a time: sequential sweep
    assert list(b) == list(range(6)) and nb == 6
    b, c, nb = orc.cyclades_batches([3, 1], 2)  # a sample with no internal edge: one batch
    assert list(b) == [0, 0] and nb == 1


def _check_schedule(prob, order, B, batch_of, comp_of, nb):
    g = _graph(prob)
    m = len(order)
    base = 0
    for k0 in range(0, m, B):
        k1 = min(m, k0 + B)
        sample = order[k0:k1]
        comps = list(nx.connected_components(g.subgraph(sample.tolist())))
        pos = {int(s): k0 + i for i, s in enumerate(sample)}
        # components as networkx finds them, each labelled by its first member's position
        mine = {}
        for i in range(k0, k1):
            mine.setdefault(int(comp_of[i]), set()).add(int(order[i]))
        assert sorted(map(sorted, mine.values())) == sorted(map(sorted, comps))
        for lab, members in mine.items():
            assert lab == min(pos[s] for s in members)
            ranks = sorted(pos[s] for s in members)
            assert [batch_of[p] - base for p in ranks] == list(range(len(members)))
        rounds = max(len(c) for c in comps)
        assert set(batch_of[k0:k1].tolist()) == set(range(base, base + rounds))
        base += rounds
    assert nb == base
    # every batch is conflict-free
    for t in range(nb):
        members = order[batch_of == t]
        assert g.subgraph(members.tolist()).number_of_edges() == 0


@pytest.mark.parametrize("B", [1, 3, 8, 64, 100])
def test_oracle_schedule_matches_networkx(crowded, B):
    orc = Oracle(crowded)
    rng = np.random.default_rng(40 + B)
    for _ in range(3):
        order = rng.permutation(crowded.n_src).astype(np.int32)
        b, c, nb = orc.cyclades_batches(order, B)
        _check_schedule(crowded, order, B, b, c, nb)


def test_oracle_schedule_of_a_subset(crowded):
    orc = Oracle(crowded)
    order = np.random.default_rng(5).choice(crowded.n_src, 20, replace=False).astype(np.int32)
    b, c, nb = orc.cyclades_batches(order, 7)
    _check_schedule(crowded, order, 7, b, c, nb)


@pytest.mark.parametrize("B", [1, 2, 5, 16, 64, 1000])
def test_library_scheduler_matches_oracle(crowded, B):
    from paper_1801_10277_gb300 import celeste
    orc = Oracle(crowded)
    rng = np.random.default_rng(90 + B)
    for m in (crowded.n_src, 17, 0):
        order = rng.choice(crowded.n_src, m, replace=False).astype(np.int32)
        lb, lc, lnb = celeste.cyclades_batches(crowded.nbr_offsets, crowded.nbrs, order, B)
        ob, oc, onb = orc.cyclades_batches(order, B)
        assert lnb == onb
        np.testing.assert_array_equal(lb, ob)
        np.testing.assert_array_equal(lc, oc)


def test_library_scheduler_rejects_bad_orders(crowded):
    from paper_1801_10277_gb300 import celeste
    with pytest.raises(celeste.CelesteError) as e:
        celeste.cyclades_batches(crowded.nbr_offsets, crowded.nbrs, [0, 1, 0], 4)
    assert e.value.status == celeste.ERR_ARG
    with pytest.raises(celeste.CelesteError):
        celeste.cyclades_batches(crowded.nbr_offsets, crowded.nbrs, [0, crowded.n_src], 4)
    with pytest.raises(celeste.CelesteError):
        celeste.cyclades_batches(crowded.nbr_offsets, crowded.nbrs, [0, 1], 0)


def test_oracle_cyclades_fit_reduces_to_colouring():
    """Two overlapping sources, order (0, 1) every sweep, samples of 2: the batches are
    {0} then {1}, exactly the two colour classes, so the fits agree bit for bit.  The
    reverse order follows another path: an accepted step raises ELBO_s, and ELBO_s holds
    every term that theta_s changes, so each sweep can only raise the total."""
    prob = synth.config(0)
    orc = Oracle(prob)
    col, nc = orc.colouring()
    assert nc == 2 and list(col) == [0, 1]
    kw = dict(max_sweeps=6, sweep_tol=1e-12)
    th0, it0, st0, el0, _ = orc.fit(prob.theta, **kw)
    th1, it1, st1, el1, _ = orc.fit(prob.theta, order=np.tile([0, 1], (6, 1)), sample_size=2, **kw)
    np.testing.assert_array_equal(th0, th1)
    np.testing.assert_array_equal(it0, it1)
    assert el0 == el1
    start, _ = orc.elbo(prob.theta)
    prev = start
    th = prob.theta
    for sweep in range(3):
        th, _, _, el, _ = orc.fit(th, order=np.array([[1, 0]]), sample_size=2, max_sweeps=1)
        assert el >= prev
        prev = el
    assert prev > start


def test_oracle_cyclades_fit_of_an_independent_set_is_schedule_free(crowded):
    """Sources that never overlap see the same fixed neighbours whatever the schedule."""
    chosen = []
    for s in range(0, crowded.n_src, 3):
        nb = set(crowded.nbrs[crowded.nbr_offsets[s]:crowded.nbr_offsets[s + 1]].tolist())
        if not nb & set(chosen):
            chosen.append(s)
        if len(chosen) == 5:
            break
    which = np.array(chosen, np.int32)
    orc = Oracle(crowded)
    kw = dict(which=which, max_sweeps=1)
    th0, it0, _, _, _ = orc.fit(crowded.theta, **kw)
    order = np.random.default_rng(3).permutation(which)[None, :].astype(np.int32)
    th1, it1, _, _, _ = orc.fit(crowded.theta, order=order, sample_size=2, **kw)
    np.testing.assert_array_equal(th0, th1)
    np.testing.assert_array_equal(it0, it1)


def test_oracle_cyclades_fit_is_serially_equivalent(crowded):
    """For one order, samples of one (strictly sequential block-coordinate ascent) and
    samples of two whose members do not touch (so they move together) give the same fit
    bit for bit: a conflicting pair is always updated in order."""
    g = _graph(crowded)
    seen = [0]
    for s in seen:
        seen += [o for o in g.neighbors(s) if o not in seen][:5 - len(seen)]
        if len(seen) == 5:
            break
    # an order whose first sample is a non-adjacent pair
    pair = next((a, b) for a in seen for b in seen if a < b and not g.has_edge(a, b))
    rest = [s for s in seen if s not in pair]
    order = np.array([list(pair) + rest], np.int32)
    orc = Oracle(crowded)
    b2, _, _ = orc.cyclades_batches(order[0], 2)
    assert b2[0] == b2[1] == 0   # the pair shares a batch
    which = np.sort(order[0])
    a = orc.fit(crowded.theta, which=which, order=order, sample_size=1, max_sweeps=1)
    b = orc.fit(crowded.theta, which=which, order=order, sample_size=2, max_sweeps=1)
    np.testing.assert_array_equal(a[0], b[0])
    assert a[3] == b[3]


def _geometric_graph(n, side, radius, seed):
    """Sources at uniform positions in a side x side box; two conflict when closer than
    radius (the shape of a patch-overlap graph of equal-sized patches)."""
    rng = np.random.default_rng(seed)
    p = rng.uniform(0, side, (n, 2))
    cell = np.floor(p / radius).astype(np.int64)
    buckets = {}
    for i, c in enumerate(map(tuple, cell)):
        buckets.setdefault(c, []).append(i)
    edges = []
    for (cx, cy), members in buckets.items():
        near = [j for dx in (-1, 0, 1) for dy in (-1, 0, 1) for j in buckets.get((cx + dx, cy + dy), [])]
        for i in members:
            for j in near:
                if j > i and np.sum((p[i] - p[j]) ** 2) < radius * radius:
                    edges.append((i, j))
    return _Graph(n, edges)


@pytest.mark.parametrize("B", [7, 256, 5000])
def test_library_scheduler_on_a_large_random_graph(B):
    """6,000 sources, about five conflicts each: the library's batches equal the oracle's
    and, checked against networkx, are the connected components of each sample in rounds,
    every batch conflict-free."""
    from paper_1801_10277_gb300 import celeste
    g = _geometric_graph(6000, 1000.0, 16.3, 7)
    deg = np.diff(g.nbr_offsets)
    assert 3.5 < deg.mean() < 6.5
    orc = Oracle(g)
    order = np.random.default_rng(B).permutation(g.n_src).astype(np.int32)
    lb, lc, lnb = celeste.cyclades_batches(g.nbr_offsets, g.nbrs, order, B)
    ob, oc, onb = orc.cyclades_batches(order, B)
    assert lnb == onb
    np.testing.assert_array_equal(lb, ob)
    np.testing.assert_array_equal(lc, oc)
    _check_schedule(g, order, B, lb, lc, lnb)
    if B == 5000:
        assert lnb > 5   # samples large enough for long components: several rounds
