"""The 120,000-orbital, 1,024-part workload: TF32 split squarings with two FP64 tail steps,
autotuned schedule, the whole loop in one CUDA graph, FP32 adjoint from checkpoints every 8
steps, all inside 180 GB.  The oracle cannot run the whole problem in test time, so values
are checked where it can compute them one by one: P on sampled parts (each part's
polynomial of its own submatrix, the GPU's bounds and branch sequence) and dL/dH on sampled
rows (the sum over the parts holding each entry)."""

import numpy as np
import pytest
import scipy.sparse as sp

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


def test_tb120k_forward_and_adjoint_on_samples(g):
    import torch
    s = make_workload("tb120k")
    plan = g.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind, device="cuda:0",
                  precision="tf32x3", ckpt_every=8)
    assert plan.workspace_bytes <= 180e9
    h = torch.from_numpy(s.vals).to("cuda:0")
    tune = plan.autotune(h, trials=1)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record()
    p = plan.density(h)
    e[1].record()
    hist = plan.history()
    rep = hist["report"]
    assert hist["status"] == 0 and rep["fp64_steps"] == 2
    # the Gershgorin bounds are the oracle's own (they are cheap at any size)
    bounds = oracle.gershgorin_bounds(s.n, s.rowptr, s.colind, s.vals)
    assert rep["eps_min"] == pytest.approx(bounds[0], rel=1e-13, abs=1e-13)
    assert rep["eps_max"] == pytest.approx(bounds[1], rel=1e-13, abs=1e-13)
    alphas = hist["alphas"]
    Hs = sp.csr_matrix((s.vals, s.colind, s.rowptr), shape=(s.n, s.n))
    p_host = p.cpu().numpy()

    # P on the largest, the smallest and a middle part
    sizes = plan.part_sizes
    ks = [int(np.argmax(sizes)), int(np.argmin(sizes)), int(np.argsort(sizes)[len(sizes) // 2])]
    worst = 0.0
    for k, (c, hh) in zip(ks, oracle.core_halo(s.g_rowptr, s.g_colind, s.part, s.nparts, which=ks)):
        S = np.concatenate([c, hh])
        Xk, _ = oracle.sp2_dense(Hs[S][:, S].toarray(), s.nocc, bounds=bounds, alphas=alphas)
        loc = {int(v): t for t, v in enumerate(S)}
        for j in range(len(c)):
            gcol = int(S[j])
            a, b = plan.p_colptr[gcol], plan.p_colptr[gcol + 1]
            rows = plan.p_rowind[a:b]
            worst = max(worst, float(np.max(np.abs(p_host[a:b] - Xk[[loc[int(r)] for r in rows], j]))))
    print(f"tb120k tf32x3: steps={rep['steps']} sampled parts {ks} max|dP|={worst:.3e}")
    assert worst <= 3e-6, worst

    # dL/dH for L = sum pbar .* P, pbar random on a sparse subset of P's pattern
    rng = np.random.default_rng(11)
    pb = np.zeros(plan.nnz_p)
    pb[rng.choice(plan.nnz_p, 200000, replace=False)] = rng.standard_normal(200000)
    pbt = torch.from_numpy(pb).to("cuda:0")
    e[2].record()
    hb = plan.backward(pbt)
    e[3].record()
    torch.cuda.synchronize()
    hb = hb.cpu().numpy()
    fwd_ms, bwd_ms = e[0].elapsed_time(e[1]), e[2].elapsed_time(e[3])
    print(f"tb120k: forward {fwd_ms:.1f} ms, backward {bwd_ms:.1f} ms, workspace "
          f"{plan.workspace_bytes / 1e9:.1f} GB, schedule {tune['candidates'][tune['chosen']]}")
    errs = []
    for r in (int(s.n // 3), int(2 * s.n // 3)):
        nb = s.g_colind[s.g_rowptr[r]:s.g_rowptr[r + 1]]
        ks_r = sorted({int(s.part[r])} | {int(s.part[v]) for v in nb})
        q0, q1 = s.rowptr[r], s.rowptr[r + 1]
        want = np.zeros(q1 - q0)
        for k, (c, hh) in zip(ks_r, oracle.core_halo(s.g_rowptr, s.g_colind, s.part, s.nparts, which=ks_r)):
            S = np.concatenate([c, hh])
            loc = {int(v): t for t, v in enumerate(S)}
            if r not in loc:
                continue
            seed = oracle.seed_on_pattern(S, len(c), pb, plan.p_colptr, plan.p_rowind)
            Gk = oracle.part_adjoint(Hs[S][:, S].toarray(), alphas, bounds, seed)
            for t, col in enumerate(s.colind[q0:q1]):
                if int(col) in loc:
                    want[t] += Gk[loc[int(r)], loc[int(col)]]
        errs.append(float(np.max(np.abs(hb[q0:q1] - want))) / max(1e-30, float(np.max(np.abs(want)))))
    print(f"tb120k FP32 adjoint: sampled rows relative max|dHbar| = {max(errs):.3e}")
    assert max(errs) <= 4e-5, errs
