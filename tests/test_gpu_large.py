"""The 120,000-orbital, 1,024-part workload with uneven cores (part sizes from about 200 to
2,000, the spread of subproblem sizes Fig. 3 shows), held to the oracle's own full G-SP2:

* the FP64-accurate emulated path: every value of P within 1e-10 of the oracle, the oracle's
  Gershgorin bounds and its branch sequence on every step with a margin;
* TF32 split squarings with two FP64 tail steps, the autotuned schedule and the whole loop
  in one CUDA graph: every value of P within the 1e-6 gate of the oracle run with the same
  two tail steps, inside 180 GB with the FP32 adjoint's checkpoints every 8 steps;
* the FP32 adjoint of that forward on sampled rows of dL/dH (the sum over the parts
  holding each entry), through the branch sequence the forward recorded (the adjoint
  differentiates the recorded polynomial)."""

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


@pytest.fixture(scope="module")
def tb120k():
    return make_workload("tb120k")


@pytest.fixture(scope="module")
def ref(tb120k):
    s = tb120k
    return oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind)


def _args(s):
    return (s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind)


def test_tb120k_sizes_span_the_configuration(g, tb120k):
    plan = g.GSP2(*_args(tb120k), bind=False)
    sz = plan.part_sizes
    assert tb120k.nparts == 1024 and tb120k.n == 120000
    assert np.percentile(sz, 1) >= 150 and np.percentile(sz, 1) <= 250
    assert sz.max() >= 1800 and sz.max() <= 2000


def test_tb120k_emulated_fp64_matches_the_oracle(g, tb120k, ref):
    import torch
    s = tb120k
    plan = g.GSP2(*_args(s), device="cuda:0", precision="fp64e", ckpt_every=0)
    h = torch.from_numpy(s.vals).to("cuda:0")
    p = plan.density(h)
    hist = plan.history()
    rep = hist["report"]
    assert hist["status"] == 0
    assert rep["eps_min"] == pytest.approx(ref.bounds[0], rel=1e-13, abs=1e-13)
    assert rep["eps_max"] == pytest.approx(ref.bounds[1], rel=1e-13, abs=1e-13)
    margin = 1e-9 * s.n
    for i in range(min(len(ref.alphas), len(hist["alphas"]))):
        if abs(ref.traces[i] - s.nocc) > margin:
            assert hist["alphas"][i] == ref.alphas[i], i
    assert len(hist["alphas"]) == len(ref.alphas)
    want = ref.p_on_pattern(plan.p_colptr, plan.p_rowind)
    err = float(np.max(np.abs(p.cpu().numpy() - want)))
    print(f"tb120k fp64e: steps={rep['steps']} max|dP|={err:.3e}")
    assert err <= 1e-10, err


def test_tb120k_tf32x3_gate_and_adjoint(g, tb120k, ref):
    import torch
    s = tb120k
    plan = g.GSP2(*_args(s), device="cuda:0", precision="tf32x3", ckpt_every=8)
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
    bounds = ref.bounds
    assert rep["eps_min"] == pytest.approx(bounds[0], rel=1e-13, abs=1e-13)
    assert rep["eps_max"] == pytest.approx(bounds[1], rel=1e-13, abs=1e-13)
    # the gate, against the oracle with the same two alternating FP64 tail steps
    ref2 = oracle.gsp2_tail(ref, s.nocc, 2)
    want = ref2.p_on_pattern(plan.p_colptr, plan.p_rowind)
    err = float(np.max(np.abs(p.cpu().numpy() - want)))
    print(f"tb120k tf32x3: steps={rep['steps']} max|dP| vs oracle with the same tail = {err:.3e}")
    assert err <= 1e-6, err
    del ref2, want

    # dL/dH for L = sum pbar .* P, pbar random on a sparse subset of P's pattern
    alphas = hist["alphas"]
    Hs = sp.csr_matrix((s.vals, s.colind, s.rowptr), shape=(s.n, s.n))
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
