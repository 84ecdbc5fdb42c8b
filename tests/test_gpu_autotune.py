"""The schedule autotuner and the tile orders it chooses between: every tile order, and the
static deal or claimed tiles, computes bitwise the same P (a tile's arithmetic does not
depend on the CTA that runs it), split-K work items the same P to the last bits, and the
autotuner keeps a candidate it timed."""

import numpy as np
import pytest

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


def run(g, s, **opt):
    import torch
    plan = g.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind, device="cuda:0",
                  ckpt_every=0, **opt)
    h = torch.from_numpy(s.vals).to("cuda:0")
    p = plan.density(h)
    st, _ = plan.status()
    assert st == 0
    return plan, h, p.cpu().numpy()


@pytest.mark.parametrize("prec", ["tf32x3", "fp16x3", "fp64e"])
def test_tile_orders_give_bitwise_equal_p(g, prec):
    s = make_workload("tb4k")  # more 128-tiles than SMs: the second order differs
    _, _, p0 = run(g, s, precision=prec, tile_order=0)
    _, _, p1 = run(g, s, precision=prec, tile_order=1)
    _, _, p2 = run(g, s, precision=prec, tile_order=2)
    assert np.array_equal(p0, p1) and np.array_equal(p0, p2)
    # the static deal against claimed tiles (the default)
    pl, _, p3 = run(g, s, precision=prec, tile_order=1, tile_claim=0)
    assert pl.info.tile_claim == 0
    assert np.array_equal(p0, p3)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "tf32", "bf16", "fp16x3"])
def test_tile_shapes_give_bitwise_equal_p(g, prec):
    """128 x 256 work items (two upper tiles per N = 256 MMA) compute every element as the
    128 x 128 tiles do."""
    s = make_workload("tb4k")
    _, _, p0 = run(g, s, precision=prec, tile_shape=0)
    _, _, p1 = run(g, s, precision=prec, tile_shape=1)
    _, _, p2 = run(g, s, precision=prec, tile_shape=1, tile_order=1)
    assert np.array_equal(p0, p1) and np.array_equal(p0, p2)


@pytest.mark.parametrize("prec", ["tf32x3", "fp16x3", "fp64e", "fp64"])
def test_autotune_keeps_a_timed_candidate(g, prec):
    s = make_workload("tb4k")
    plan, h, p0 = run(g, s, precision=prec)
    rep = plan.autotune(h, trials=2)
    cands = rep["candidates"]
    # tensor-core steps: orders 0 and 1 with claimed tiles and with the static deal, the
    # 128 x 256 tiles in either order, one CTA per tile; fp64e on this plan (193 tiles, parts
    # above 128 orbitals): the three tile orders with claimed tiles, the first two with
    # split-K work items, order 2 with the static deal
    assert len(cands) == {"tf32x3": 7, "fp16x3": 7, "fp64e": 6, "fp64": 1}[prec]
    assert all(c["ms"] > 0 for c in cands)
    best = cands[rep["chosen"]]
    assert best["ms"] == min(c["ms"] for c in cands)
    assert (plan.info.tc_schedule, plan.info.tile_order, plan.info.tile_shape, plan.info.split_k,
            plan.info.tile_claim) == (best["tc_schedule"], best["tile_order"], best["tile_shape"], best["split_k"],
                                      best["tile_claim"])
    p1 = plan.density(h).cpu().numpy()
    if best["split_k"] == 1:  # the default of this plan: bitwise the same
        assert np.array_equal(p0, p1)
    else:
        assert np.max(np.abs(p0 - p1)) <= 1e-14
    print(prec, rep)


def test_split_k_items_of_the_emulated_steps(g):
    """Split-K work items (each tile's K stages in two halves whose 64-bit partials the
    second to finish adds) against one item per tile: the same branch sequence and P to the
    last bits (only the FP32 rounding of the low-order digit groups can differ), both tile
    orders bitwise equal within each setting; plans with a part of 128 orbitals or fewer
    never split."""
    s = make_workload("tb4k")
    pa, _, p_split = run(g, s, precision="fp64e", split_k=1)
    pb, _, p_one = run(g, s, precision="fp64e", split_k=0)
    assert pa.info.split_k == 1 and pb.info.split_k == 0
    assert pa.history()["alphas"] == pb.history()["alphas"]
    assert np.max(np.abs(p_split - p_one)) <= 1e-14
    _, _, p_split0 = run(g, s, precision="fp64e", split_k=1, tile_order=0)
    assert np.array_equal(p_split, p_split0)
    # split items dealt statically: the same bits as claimed ones
    _, _, p_split_static = run(g, s, precision="fp64e", split_k=1, tile_claim=0)
    assert np.array_equal(p_split, p_split_static)
    from synth.tb import make_tb_system
    small = make_tb_system(33, 5, 3.2, seed=133)  # parts of fewer than 128 orbitals
    pc, _, _ = run(g, small, precision="fp64e", split_k=1)
    assert pc.info.split_k == 0
