"""Shard plans on the GPU, through the C ABI.

* One rank holding every part: the exchange is the identity, and P, the branch sequence and
  the trace history are bitwise those of the fused path (the step kernels' partial sums go
  through the exchange slot and the decide kernel instead of being used in place).
* Two and three ranks emulated on one GPU: every shard plan runs its own launches, driven
  in lockstep from one thread; the exchange between them is a host-side stack of their
  16-byte partials on the same stream (no kernel waits for another).  The union of their
  core columns is P: the same branch sequence as one plan and the same P bit for bit (a
  part's arithmetic does not depend on which plan runs it), within 1e-10 of the oracle;
  the shards' Hbar shares add up to the one-plan adjoint."""

import numpy as np
import pytest

import oracle
from synth import make_workload
from synth.tb import make_tb_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1801_10016_gb300 import gsp2, shard
    return gsp2, shard


def _args(s):
    return (s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind)


def run_lockstep(plans, h, mode="record", nsteps=0, alpha=None):
    """Drive shard plans (all on cuda:0) through one density call, exchanging in rank order."""
    import torch
    outs = [torch.empty(p.nnz_p, dtype=torch.float64, device="cuda:0") for p in plans]
    sends = [torch.empty(2, dtype=torch.float64, device="cuda:0") for _ in plans]
    count = plans[0].exchanges(mode, nsteps)
    assert all(p.exchanges(mode, nsteps) == count for p in plans)
    for p, o, sd in zip(plans, outs, sends):
        p.begin(h, o, sd, alpha, mode, nsteps)
    for x in range(count):
        recv = torch.stack(sends)
        for p in plans:
            p.decide(x, recv)
        if x + 1 < count:
            for p, sd in zip(plans, sends):
                p.step(x + 1, sd)
    for p in plans:
        p.end()
    return outs


@pytest.mark.parametrize("prec", ["fp64", "fp64e", "fp16x3", "tf32x3"])
def test_one_rank_shard_is_the_fused_path_bitwise(lib, prec):
    import torch
    gsp2, shard = lib
    s = make_workload("tb512")
    full = gsp2.GSP2(*_args(s), device="cuda:0", precision=prec)
    h = torch.from_numpy(s.vals).to("cuda:0")
    p_full = full.density(h)
    hist_full = full.history()
    one = shard.ShardPlan(*_args(s), np.zeros(s.nparts, np.int32), 0, device="cuda:0", precision=prec)
    p_one = one.density(h, exchange=lambda send: send.view(1, 2))
    hist_one = one.history()
    assert hist_full["status"] == 0 and hist_one["status"] == 0
    assert hist_one["alphas"] == hist_full["alphas"]
    assert np.array_equal(hist_one["traces"], hist_full["traces"])
    assert np.array_equal(hist_one["idem"], hist_full["idem"])
    assert np.array_equal(one.p_colptr, full.p_colptr)
    assert torch.equal(p_one, p_full)


@pytest.mark.parametrize("prec,nranks,case", [("fp64", 2, "tb512"), ("fp64e", 2, "tb512"), ("fp64e", 3, "tb4k"),
                                              ("fp16x3", 2, "tb512")])
def test_shards_in_lockstep_match_one_plan(lib, prec, nranks, case):
    import torch
    gsp2, shard = lib
    s = make_workload(case)
    full = gsp2.GSP2(*_args(s), device="cuda:0", precision=prec)
    h = torch.from_numpy(s.vals).to("cuda:0")
    p_full = full.density(h)
    hist_full = full.history()
    pr, _ = shard.assign_parts(full.part_sizes, nranks)
    plans = [shard.ShardPlan(*_args(s), pr, r, device="cuda:0", precision=prec) for r in range(nranks)]
    outs = run_lockstep(plans, h)
    hists = [p.history() for p in plans]
    for hs in hists:
        assert hs["status"] == 0
        assert hs["alphas"] == hist_full["alphas"]
        # traces summed in another order: equal to rounding
        np.testing.assert_allclose(hs["traces"], hist_full["traces"], rtol=0, atol=1e-10)
    assert all(hs["traces"].tolist() == hists[0]["traces"].tolist() for hs in hists)
    cp, ri, pos = shard.merge_patterns([p.p_colptr for p in plans], [p.p_rowind for p in plans])
    assert np.array_equal(cp, full.p_colptr) and np.array_equal(ri, full.p_rowind)
    p = torch.empty_like(p_full)
    for q, o in zip(pos, outs):
        p[torch.from_numpy(q).to("cuda:0")] = o
    assert torch.equal(p, p_full)
    if prec.startswith("fp64") and case == "tb512":
        ref = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind)
        assert np.max(np.abs(p.cpu().numpy() - ref.p_on_pattern(cp, ri))) <= 1e-10


@pytest.mark.parametrize("prec", ["fp64", "fp64e"])
def test_shard_adjoint_shares_add_up(lib, prec):
    import torch
    gsp2, shard = lib
    s = make_tb_system(60, 6, 3.5, seed=31)
    full = gsp2.GSP2(*_args(s), device="cuda:0", precision=prec)
    h = torch.from_numpy(s.vals).to("cuda:0")
    full.density(h)
    rng = np.random.default_rng(2)
    pb = torch.from_numpy(rng.standard_normal(full.nnz_p)).to("cuda:0")
    hb_full = full.backward(pb)
    pr, _ = shard.assign_parts(full.part_sizes, 2)
    plans = [shard.ShardPlan(*_args(s), pr, r, device="cuda:0", precision=prec) for r in range(2)]
    run_lockstep(plans, h)
    _, _, pos = shard.merge_patterns([p.p_colptr for p in plans], [p.p_rowind for p in plans])
    hb = sum(p.backward(pb[torch.from_numpy(q).to("cuda:0")]) for p, q in zip(plans, pos))
    scale = float(hb_full.abs().max())
    assert float((hb - hb_full).abs().max()) <= 1e-12 * scale


def test_shard_replay_and_call_order(lib):
    import torch
    gsp2, shard = lib
    s = make_workload("tb512")
    full = gsp2.GSP2(*_args(s), device="cuda:0")
    h = torch.from_numpy(s.vals).to("cuda:0")
    alpha = torch.zeros(full.alpha_len, dtype=torch.int8, device="cuda:0")
    p_full = full.density(h, alpha=alpha)
    n = full.history()["report"]["steps"]
    pr, _ = shard.assign_parts(full.part_sizes, 2)
    plans = [shard.ShardPlan(*_args(s), pr, r, device="cuda:0") for r in range(2)]
    outs = run_lockstep(plans, h, mode="replay", nsteps=n, alpha=alpha)
    _, _, pos = shard.merge_patterns([p.p_colptr for p in plans], [p.p_rowind for p in plans])
    p = torch.empty_like(p_full)
    for q, o in zip(pos, outs):
        p[torch.from_numpy(q).to("cuda:0")] = o
    assert torch.equal(p, p_full)
    assert all(pl.status()[0] == 0 for pl in plans)
    # out of order: a step before its decision, a fused density call on a shard plan
    pl = plans[0]
    out = torch.empty(pl.nnz_p, dtype=torch.float64, device="cuda:0")
    send = torch.empty(2, dtype=torch.float64, device="cuda:0")
    pl.begin(h, out, send)
    with pytest.raises(gsp2.GSP2Error) as e:
        pl.step(1, send)
    assert e.value.status == gsp2.E_STATE
    with pytest.raises(gsp2.GSP2Error) as e:
        pl.end()
    assert e.value.status == gsp2.E_STATE
    with pytest.raises(gsp2.GSP2Error) as e:
        gsp2.GSP2.density(pl, h)
    assert e.value.status == gsp2.E_STATE
