"""CPU-only checks of the C ABI: the library builds and exports every declared symbol,
and gsp2_create (host-only planning) validates its inputs and builds the halos, the
layout and the pattern of P as Section 2.2 defines them.  No CUDA call is made."""

import ctypes as C
import os

import numpy as np
import pytest

import oracle
from synth import make_workload
from synth.tb import _csr_from_coo, make_tb_system

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def g():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1801_10016_gb300 import gsp2
    return gsp2


def test_library_exports_every_declared_symbol(g):
    names = g.header_functions()
    assert "gsp2_create" in names and "gsp2_density" in names and "gsp2_backward" in names
    lib = C.CDLL(g.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def _plan(g, s, **kw):
    return g.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind, bind=False, **kw)


def test_default_options(g):
    o = g.default_options()
    assert o.max_steps == 45 and o.precision == 0 and o.use_graph == 1 and o.ckpt_every == -1
    assert o.idem_tol == 1e-3 and o.fp64_tail_steps == -1 and o.lp_tail_steps == 0 and o.tc_schedule == 0
    # "-1" resolves to no tail for FP64 (the paper's method) and two FP64 steps otherwise
    s = make_workload("tb512")
    assert _plan(g, s).info.fp64_tail_steps == 0
    assert _plan(g, s, precision="tf32x3").info.fp64_tail_steps == 2
    assert _plan(g, s, fp64_tail_steps=3).info.fp64_tail_steps == 3


def test_halos_and_p_pattern_match_section_2_2(g):
    s = make_workload("tb512")
    plan = _plan(g, s)
    ch = oracle.core_halo(s.g_rowptr, s.g_colind, s.part, s.nparts)
    sizes = [len(c) + len(h) for c, h in ch]
    assert plan.part_sizes.tolist() == sizes
    assert plan.part_cores.tolist() == [len(c) for c, _ in ch]
    assert plan.nnz_p == sum(len(c) * (len(c) + len(h)) for c, h in ch)
    # column g of P holds sorted(S_part(g))
    for k, (c, h) in enumerate(ch):
        want = np.sort(np.concatenate([c, h]))
        for gcol in c[:3]:
            rows = plan.p_rowind[plan.p_colptr[gcol]:plan.p_colptr[gcol + 1]]
            np.testing.assert_array_equal(rows, want)
    assert plan.info.sum_s3 == float(oracle.ch_cost(sizes))
    assert plan.info.ntiles == sum((-(-sz // 64)) * (-(-sz // 64) + 1) // 2 for sz in sizes)


def test_fig2_through_the_library(g):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "fig2_core_halo.txt")) if l.strip() and not l.startswith("#")]
    names = rows[0][1:]
    idx = {v: i for i, v in enumerate(names)}
    edges = [(idx[r[1]], idx[r[2]]) for r in rows if r[0] == "edge"]
    e = np.array(edges + [(b, a) for a, b in edges] + [(i, i) for i in range(len(names))])
    rp, ci, _ = _csr_from_coo(len(names), e[:, 0].astype(np.int64), e[:, 1].astype(np.int64), None)
    for case, want, cost in (("a", [4, 5], 189), ("b", [6, 3], 243)):
        r = [r for r in rows if r[0] == "partition" and r[1] == case][0]
        bar = r.index("|")
        part = np.zeros(len(names), np.int32)
        for v in r[bar + 1:]:
            part[idx[v]] = 1
        plan = g.GSP2(len(names), rp, ci, 3, part, 2, bind=False)
        assert plan.part_sizes.tolist() == want
        assert plan.info.sum_s3 == cost


@pytest.mark.parametrize("bad", ["unsorted", "nodiag", "asym", "range", "part", "empty", "nocc", "graph_half"])
def test_create_rejects_bad_input(g, bad):
    s = make_tb_system(16, 2, 3.0, seed=5)
    rp, ci, part = s.rowptr.copy(), s.colind.copy(), s.part.copy()
    grp, gci = s.g_rowptr, s.g_colind
    nocc, nparts = s.nocc, s.nparts
    if bad == "unsorted":
        ci[rp[3]], ci[rp[3] + 1] = ci[rp[3] + 1], ci[rp[3]]
    elif bad == "nodiag":
        keep = np.ones(len(ci), bool)
        row0 = np.arange(rp[0], rp[1])
        keep[row0[ci[row0] == 0]] = False
        rows = np.repeat(np.arange(s.n), np.diff(rp))[keep]
        rp, ci, _ = _csr_from_coo(s.n, rows.astype(np.int64), ci[keep].astype(np.int64), None)
    elif bad == "asym":
        rows = np.repeat(np.arange(s.n), np.diff(rp))
        drop = np.nonzero((rows == 0) & (ci != 0))[0][0]
        keep = np.ones(len(ci), bool)
        keep[drop] = False
        rp, ci, _ = _csr_from_coo(s.n, rows[keep].astype(np.int64), ci[keep].astype(np.int64), None)
    elif bad == "range":
        ci[-1] = s.n
    elif bad == "part":
        part[0] = nparts
    elif bad == "empty":
        nparts = 3
    elif bad == "nocc":
        nocc = s.n + 1
    elif bad == "graph_half":
        gci = None
    with pytest.raises(g.GSP2Error) as ei:
        g.GSP2(s.n, rp, ci, nocc, part, nparts, grp, gci, bind=False)
    assert ei.value.status == g.E_ARG
    assert str(ei.value)


def test_options_rejected(g):
    s = make_tb_system(16, 2, 3.0, seed=5)
    for kw in (dict(max_steps=0), dict(max_steps=5000), dict(idem_tol=-1.0), dict(ckpt_every=-2)):
        with pytest.raises(g.GSP2Error):
            _plan(g, s, **kw)


def test_workspace_size_covers_two_arenas(g):
    s = make_workload("tb512")
    plan = _plan(g, s)
    assert plan.workspace_bytes >= 2 * 8 * plan.info.arena_elems
    # padded leading dimensions: every part padded to the 128 multiple
    ld = -(-plan.part_sizes // 128) * 128
    assert plan.info.arena_elems == int(np.sum(ld.astype(np.int64) ** 2))


def test_tile_order_option(g):
    s = make_tb_system(16, 2, 3.0, seed=5)
    assert g.default_options().tile_order == 1
    for bad in (-1, 3):
        with pytest.raises(g.GSP2Error):
            _plan(g, s, tile_order=bad)
    p = _plan(g, s, precision="tf32x3", tile_order=1, tc_schedule=1)
    assert p.info.tile_order == 1 and p.info.tc_schedule == 1
    assert g.default_options().tile_shape == 0
    for bad in (-1, 2):
        with pytest.raises(g.GSP2Error):
            _plan(g, s, tile_shape=bad)
    assert _plan(g, s, precision="tf32x3", tile_shape=1).info.tile_shape == 1
    assert g.default_options().tile_claim == 1
    for bad in (-1, 2):
        with pytest.raises(g.GSP2Error):
            _plan(g, s, tile_claim=bad)
    assert _plan(g, s, precision="fp16x3", tile_claim=0).info.tile_claim == 0


def test_low_precision_adjoint_layout(g):
    """ckpt_every = -1 keeps FP64 iterates every 8 steps for FP64 plans and none for the
    low-precision ones; an explicit k adds FP32 checkpoints, and excludes low-precision
    tail steps."""
    s = make_workload("tb512")
    base = _plan(g, s, precision="tf32x3").workspace_bytes
    k4 = _plan(g, s, precision="tf32x3", ckpt_every=4).workspace_bytes
    af = 4 * _plan(g, s).info.arena_elems
    # 45 // 4 + 1 checkpoints, 3 segments, 2 Xbar, 2 tail iterates, FP32 each
    assert k4 - base >= (45 // 4 + 1 + 3 + 2 + 2) * af
    assert _plan(g, s).workspace_bytes > _plan(g, s, ckpt_every=0).workspace_bytes
    with pytest.raises(g.GSP2Error):
        _plan(g, s, precision="tf32x3", ckpt_every=4, lp_tail_steps=2, fp64_tail_steps=0)
