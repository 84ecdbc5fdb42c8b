"""The steps either side of the path in an SCF or MD loop: reuse of the recorded branch
sequence while it gives the right trace (Section 2.1), and the dependency graph G_tau
rebuilt from the thresholded P for the next plan (Section 2.2)."""

import numpy as np
import pytest

import oracle
from synth import make_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1801_10016_gb300 import gsp2
    return gsp2


def plan_for(g, s, **kw):
    return g.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind, device="cuda:0",
                  ckpt_every=0, **kw)


@pytest.mark.parametrize("prec", ["fp64", "fp64e"])
def test_sequence_reuse_replays_and_recomputes(g, prec):
    import torch
    s = make_workload("tb512")
    plan = plan_for(g, s, precision=prec)
    h = torch.from_numpy(s.vals).to("cuda:0")
    p_ref = plan.density(h).clone()
    ref_alphas = plan.history()["alphas"]
    alpha = torch.zeros(plan.alpha_len, dtype=torch.int8, device="cuda:0")
    # first call: nothing to replay, the sequence is recorded
    p1, n1, rec1, st1 = plan.density_reuse(h, alpha, 0)
    assert rec1 and st1 == 0 and n1 == len(ref_alphas)
    assert torch.equal(p1, p_ref)
    assert alpha[:n1].cpu().numpy().tolist() == ref_alphas
    # the same H again: the replay gives the right trace and bitwise the same P
    p2, n2, rec2, st2 = plan.density_reuse(h, alpha, n1)
    assert not rec2 and st2 == 0 and n2 == n1 and torch.equal(p2, p_ref)
    # a sequence that no longer fits (first branch flipped): wrong trace, recorded afresh
    alpha[0] = -alpha[0]
    p3, n3, rec3, st3 = plan.density_reuse(h, alpha, n1)
    assert rec3 and st3 == 0 and n3 == n1 and torch.equal(p3, p_ref)
    assert alpha[:n3].cpu().numpy().tolist() == ref_alphas


def test_threshold_graph_and_replan(g):
    import torch
    s = make_workload("tb512")
    plan = plan_for(g, s)
    p = plan.density(plan_h := torch.from_numpy(s.vals).to("cuda:0"))
    tau = 1e-5
    rp, ci = plan.threshold_graph(p, tau)
    # the same graph from the stored values on the host
    pv = p.cpu().numpy()
    cols = np.repeat(np.arange(s.n), np.diff(plan.p_colptr))
    keep = (np.abs(pv) > tau) & (plan.p_rowind != cols)
    r, c = plan.p_rowind[keep].astype(np.int64), cols[keep]
    rows = np.concatenate([r, c, np.arange(s.n)])
    cc = np.concatenate([c, r, np.arange(s.n)])
    pairs = np.unique(rows * s.n + cc)
    want_rp = np.searchsorted(pairs // s.n, np.arange(s.n + 1))
    np.testing.assert_array_equal(rp, want_rp)
    np.testing.assert_array_equal(ci, (pairs % s.n).astype(np.int32))
    # the next plan on the refreshed graph, against the oracle on the same graph
    nxt = g.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, rp, ci, device="cuda:0", ckpt_every=0)
    pn = nxt.density(plan_h).cpu().numpy()
    st, _ = nxt.status()
    assert st == 0
    ref = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, rp, ci)
    err = float(np.max(np.abs(pn - ref.p_on_pattern(nxt.p_colptr, nxt.p_rowind))))
    print(f"refreshed graph: {len(ci)} entries (was {len(s.g_colind)}), sizes {nxt.part_sizes.min()}-"
          f"{nxt.part_sizes.max()}, max|dP| vs oracle {err:.3e}")
    assert err <= 1e-10


def test_refresh_repartitions_by_the_eq5_cost_and_replans(g):
    """Section 1.1 / Fig. 1: after P, G_tau is rebuilt from it and re-partitioned before the
    next plan.  The partition is the one of smallest Eq. 5 cost among the block partition
    of Section 2.3, blocks over a graph order and coordinate bisection; the plan built on
    the refreshed graph and the new partition matches the oracle on the same graph and
    partition."""
    import torch
    from synth.tb import ORBS_PER_SITE
    s = make_workload("tb4k")
    plan = plan_for(g, s)
    h = torch.from_numpy(s.vals).to("cuda:0")
    p = plan.density(h)
    rp, ci = plan.threshold_graph(p, 1e-4)
    xyz = np.repeat(s.coords, ORBS_PER_SITE, axis=0)
    costs = {m: g.partition(rp, ci, s.nparts, m, coords=xyz)[2] for m in ("block", "graph_order", "rcb")}
    part, method, cost = g.partition(rp, ci, s.nparts, "auto", coords=xyz)
    assert cost == min(costs.values()) and costs[method] == cost
    assert g.partition_cost(rp, ci, part, s.nparts)[0] == cost
    assert np.bincount(part, minlength=s.nparts).min() >= 1
    nxt = g.GSP2(s.n, s.rowptr, s.colind, s.nocc, part, s.nparts, rp, ci, device="cuda:0", ckpt_every=0,
                 precision="fp64e")
    pn = nxt.density(h).cpu().numpy()
    st, _ = nxt.status()
    assert st == 0
    ref = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, part, s.nparts, rp, ci)
    err = float(np.max(np.abs(pn - ref.p_on_pattern(nxt.p_colptr, nxt.p_rowind))))
    print(f"re-partitioned ({method}): Eq. 5 costs {costs}, sizes {nxt.part_sizes.min()}-{nxt.part_sizes.max()}, "
          f"max|dP| vs oracle {err:.3e}")
    assert err <= 1e-10
