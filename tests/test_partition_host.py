"""Re-partitioning of G_tau on the host (gsp2_partition, gsp2_partition_cost), checked on the
CPU: the Eq. 5 cost against the paper's worked example (Fig. 2: 189 and 243) and the
oracle's core/halo sets, the block partition against the sizes of Section 2.3, and the
automatic choice against every method's cost."""

import os

import numpy as np
import pytest

import oracle
from synth import make_workload
from synth.tb import ORBS_PER_SITE, _csr_from_coo

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def g():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1801_10016_gb300 import gsp2
    return gsp2


def _fig2():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "fig2_core_halo.txt")) if l.strip() and not l.startswith("#")]
    names = rows[0][1:]
    idx = {v: i for i, v in enumerate(names)}
    edges = [(idx[r[1]], idx[r[2]]) for r in rows if r[0] == "edge"]
    parts, expect = {}, {}
    for r in rows:
        if r[0] == "partition":
            bar = r.index("|")
            parts[r[1]] = r[bar + 1:]
        if r[0] == "expect":
            expect[r[1]] = dict(sizes=[int(r[3]), int(r[4])], cost=int(r[9]))
    e = np.array(edges + [(b, a) for a, b in edges])
    rp, ci, _ = _csr_from_coo(len(names), e[:, 0].astype(np.int64), e[:, 1].astype(np.int64), None)
    return names, idx, rp, ci, parts, expect


@pytest.mark.parametrize("case", ["a", "b"])
def test_cost_of_the_fig2_partitions(g, case):
    names, idx, rp, ci, parts, expect = _fig2()
    part = np.zeros(len(names), np.int32)
    for v in parts[case]:
        part[idx[v]] = 1
    cost, sizes = g.partition_cost(rp, ci, part, 2)
    assert sizes.tolist() == expect[case]["sizes"]
    assert cost == expect[case]["cost"]


def test_block_partition_of_section_2_3(g):
    kv = {l.split()[0]: l.split()[1:] for l in open(os.path.join(GOLDEN, "block_partition_polyalanine.txt"))
          if l.strip() and not l.startswith("#")}
    n, nparts = int(kv["n"][0]), int(kv["nparts"][0])
    # a chain graph: the block partition does not look at the edges
    a = np.arange(n - 1, dtype=np.int64)
    rp, ci, _ = _csr_from_coo(n, np.concatenate([a, a + 1]), np.concatenate([a + 1, a]), None)
    part, method, cost = g.partition(rp, ci, nparts, "block")
    assert method == "block"
    counts = np.bincount(part, minlength=nparts)
    c35, c34 = int(kv["count35"][0]), int(kv["count34"][0])
    assert counts[:c35].tolist() == [35] * c35 and counts[c35:].tolist() == [34] * c34
    assert np.all(np.diff(part) >= 0)  # consecutive indices


def test_cost_matches_the_oracle_core_halo(g):
    s = make_workload("tb512")
    cost, sizes = g.partition_cost(s.g_rowptr, s.g_colind, s.part, s.nparts)
    ch = oracle.core_halo(s.g_rowptr, s.g_colind, s.part, s.nparts)
    want = [len(c) + len(h) for c, h in ch]
    assert sizes.tolist() == want
    assert cost == oracle.ch_cost(want)


def test_automatic_choice_takes_the_smallest_cost(g):
    s = make_workload("tb4k")
    xyz = np.repeat(s.coords, ORBS_PER_SITE, axis=0)
    costs = {}
    for m in ("block", "graph_order", "rcb"):
        part, method, cost = g.partition(s.g_rowptr, s.g_colind, s.nparts, m, coords=xyz)
        assert method == m
        counts = np.bincount(part, minlength=s.nparts)
        assert counts.min() >= 1 and counts.sum() == s.n
        if m != "rcb":
            assert counts.max() - counts.min() <= 1
        assert g.partition_cost(s.g_rowptr, s.g_colind, part, s.nparts)[0] == cost
        costs[m] = cost
    part, method, cost = g.partition(s.g_rowptr, s.g_colind, s.nparts, "auto", coords=xyz)
    assert cost == min(costs.values()) and method == min(costs, key=lambda k: (costs[k], list(costs).index(k)))
    # sites in random index order: blocks of indices are scattered in space, so both the graph
    # order and the bisection beat the plain block partition by far
    assert costs["graph_order"] < 0.5 * costs["block"] and costs["rcb"] < 0.5 * costs["block"]
    # without coordinates the choice is among the graph-only methods
    part2, method2, cost2 = g.partition(s.g_rowptr, s.g_colind, s.nparts, "auto")
    assert method2 in ("block", "graph_order") and cost2 == min(costs["block"], costs["graph_order"])
    # deterministic
    assert np.array_equal(g.partition(s.g_rowptr, s.g_colind, s.nparts, "auto", coords=xyz)[0], part)


def test_graph_order_recovers_a_shuffled_chain(g):
    n, nparts = 1000, 10
    rng = np.random.default_rng(1)
    lab = rng.permutation(n)  # chain 0-1-2-... under random labels
    a = lab[:-1].astype(np.int64)
    b = lab[1:].astype(np.int64)
    rp, ci, _ = _csr_from_coo(n, np.concatenate([a, b]), np.concatenate([b, a]), None)
    part, _, cost = g.partition(rp, ci, nparts, "graph_order")
    # each part is a contiguous stretch of the chain: halo of at most 2, s <= 102
    _, sizes = g.partition_cost(rp, ci, part, nparts)
    assert sizes.max() <= n // nparts + 2
    assert cost < g.partition(rp, ci, nparts, "block")[2]


def test_partition_errors(g):
    s = make_workload("tb512")
    with pytest.raises(g.GSP2Error):
        g.partition(s.g_rowptr, s.g_colind, s.n + 1, "block")
    with pytest.raises(g.GSP2Error):
        g.partition(s.g_rowptr, s.g_colind, 4, "rcb")  # no coordinates
    bad = s.part.copy()
    bad[0] = s.nparts
    with pytest.raises(g.GSP2Error):
        g.partition_cost(s.g_rowptr, s.g_colind, bad, s.nparts)
