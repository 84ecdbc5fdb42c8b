"""Host logic of shard plans (one G-SP2 problem's parts split over several GPUs), checked on
the CPU: the longest-processing-time assignment of parts to ranks by the Eq. 5 cost s^3,
the disjoint core columns of the shards' patterns, and a two-rank gloo run in which every
rank purifies its own parts (with the oracle's arithmetic) and takes each step's branch
from the rank-order sum of the partial traces exchanged by the library's exchange
function (Section 2.1: one branch for all parts from the global trace)."""

import itertools
import os
import socket

import numpy as np
import pytest

import oracle
from synth import make_workload
from synth.tb import make_tb_system


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1801_10016_gb300 import gsp2, shard
    return gsp2, shard


def test_lpt_assignment_is_balanced_and_deterministic(lib):
    gsp2, shard = lib
    rng = np.random.default_rng(5)
    for nparts, nranks in [(7, 3), (8, 2), (9, 4), (6, 6)]:
        sizes = rng.integers(50, 400, nparts).astype(np.int32)
        pr, cost = shard.assign_parts(sizes, nranks)
        pr2, _ = shard.assign_parts(sizes, nranks)
        assert np.array_equal(pr, pr2)
        assert set(pr.tolist()) == set(range(nranks))  # every rank gets a part
        c3 = sizes.astype(np.float64) ** 3
        np.testing.assert_allclose(cost, [c3[pr == r].sum() for r in range(nranks)])
        # against the optimum by brute force: LPT's bound is 4/3 - 1/(3m) of it
        best = min(max(c3[np.array(a) == r].sum() for r in range(nranks))
                   for a in itertools.product(range(nranks), repeat=nparts))
        assert cost.max() <= (4.0 / 3.0 - 1.0 / (3 * nranks)) * best * (1 + 1e-12)
    with pytest.raises(gsp2.GSP2Error):
        shard.assign_parts(np.array([10, 20], np.int32), 3)


@pytest.mark.parametrize("nranks", [1, 2, 3, 8])
def test_shard_patterns_cover_p_once(lib, nranks):
    gsp2, shard = lib
    s = make_workload("tb512")
    args = (s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind)
    full = gsp2.GSP2(*args, bind=False)
    pr, _ = shard.assign_parts(full.part_sizes, nranks)
    plans = [shard.ShardPlan(*args, pr, r, bind=False) for r in range(nranks)]
    cp, ri, pos = shard.merge_patterns([p.p_colptr for p in plans], [p.p_rowind for p in plans])
    np.testing.assert_array_equal(cp, full.p_colptr)
    np.testing.assert_array_equal(ri, full.p_rowind)
    assert np.array_equal(np.sort(np.concatenate(pos)), np.arange(full.nnz_p))
    for r, p in enumerate(plans):
        assert np.array_equal(p.part_ids, np.nonzero(pr == r)[0])
        np.testing.assert_array_equal(p.part_sizes, full.part_sizes[p.part_ids])
        np.testing.assert_array_equal(p.part_cores, full.part_cores[p.part_ids])
        # a rank's columns are the cores of its parts
        owned = np.isin(s.part, p.part_ids)
        assert np.array_equal(np.diff(p.p_colptr) > 0, owned)
    with pytest.raises(gsp2.GSP2Error):  # a rank with no part
        shard.ShardPlan(*args, np.zeros(s.nparts, np.int32), 1, bind=False)


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1801_10016_gb300 import shard
    s = make_tb_system(40, 5, 3.2, seed=77)
    args = (s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind)
    sizes = shard.part_sizes(*args)
    pr, _ = shard.assign_parts(sizes, world)
    plan = shard.ShardPlan(*args, pr, rank, bind=False)
    # this rank's parts, purified with the oracle's arithmetic; the branch of every step from
    # the exchanged partial traces summed in rank order
    bounds = oracle.gershgorin_bounds(s.n, s.rowptr, s.colind, s.vals)
    ch = oracle.core_halo(s.g_rowptr, s.g_colind, s.part, s.nparts, which=[int(k) for k in plan.part_ids])
    import scipy.sparse as sp
    Hs = sp.csr_matrix((s.vals, s.colind, s.rowptr), shape=(s.n, s.n))
    S = [np.concatenate([c, h]) for c, h in ch]
    nc = [len(c) for c, _ in ch]
    X = [oracle.initial_guess(Hs[Sk][:, Sk].toarray(), *bounds) for Sk in S]
    exchange = shard.dist_exchange()

    def total(t, y):
        recv = exchange(torch.tensor([t, y], dtype=torch.float64))
        assert recv.shape == (world, 2)
        return float(recv[:, 0].sum()), float(recv[:, 1].sum()), recv.clone()

    T, _, first = total(sum(float(np.trace(x[:c, :c])) for x, c in zip(X, nc)), 0.0)
    traces, idem, alphas, seen = [T], [], [], [first]
    for i in range(1, 46):
        a = oracle.branch_alpha(traces[-1], s.nocc)
        y = sum(float(np.einsum("ij,ji->", x[:c, :], x[:, :c])) for x, c in zip(X, nc))
        X = [oracle.sp2_step(x, a) for x in X]
        t, ysum, recv = total(sum(float(np.trace(x[:c, :c])) for x, c in zip(X, nc)), y)
        seen.append(recv)
        alphas.append(a)
        idem.append(traces[-1] - ysum)
        traces.append(t)
        if oracle.stop_now(idem, i, 1e-3):
            break
    vals = np.empty(plan.nnz_p)
    for Sk, c, x in zip(S, nc, X):
        loc = {int(g): q for q, g in enumerate(Sk)}
        for j in range(c):
            g = int(Sk[j])
            rows = plan.p_rowind[plan.p_colptr[g]:plan.p_colptr[g + 1]]
            vals[plan.p_colptr[g]:plan.p_colptr[g + 1]] = x[[loc[int(r)] for r in rows], j]
    p = plan.gather_p(torch.from_numpy(vals))
    out[rank] = dict(alphas=alphas, traces=traces, recv=[r.numpy().tolist() for r in seen], p=p.numpy(),
                     colptr=plan.full_colptr, rowind=plan.full_rowind, parts=plan.part_ids.tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_global_branch_sequence():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        r0, r1 = dict(out[0]), dict(out[1])
    # the parts are split, both ranks received the same partials in the same (rank) order
    assert set(r0["parts"]).isdisjoint(r1["parts"]) and sorted(r0["parts"] + r1["parts"]) == list(range(5))
    assert r0["recv"] == r1["recv"] and r0["alphas"] == r1["alphas"] and r0["traces"] == r1["traces"]
    # against the oracle's G-SP2 of the whole problem: the same branches and the same P on
    # the same pattern (the trace sums differ only by the order of addition)
    s = make_tb_system(40, 5, 3.2, seed=77)
    ref = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind)
    assert r0["alphas"] == ref.alphas
    np.testing.assert_allclose(r0["traces"], ref.traces, rtol=0, atol=1e-10)
    want = ref.p_on_pattern(r0["colptr"], r0["rowind"])
    assert np.max(np.abs(r0["p"] - want)) <= 1e-12
    assert np.array_equal(r0["p"], r1["p"])
