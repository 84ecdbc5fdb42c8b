"""GPU checks of the low-precision purification paths (TF32/BF16/FP16 on tcgen05 tensor
cores, FP32 on CUDA cores) against the FP64 oracle.

* one step, element by element, inside the rounding bound of the arithmetic:
  operands rounded to the format's unit roundoff u, FP32 accumulation over K terms;
* a full run with the FP64 tail, reported against the oracle's P with the accuracy
  gates max|dP|, part idempotency and |Tr P - Nocc|.
"""

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from synth import make_workload
from synth.tb import make_tb_system

pytestmark = pytest.mark.gpu

# unit roundoff of one operand, and of one product of the split (x3) forms
U_OPERAND = {"tf32": 2.0 ** -11, "bf16": 2.0 ** -8, "tf32x3": 2.0 ** -21, "bf16x3": 2.0 ** -15, "fp32": 2.0 ** -24,
             "fp16x3": 2.0 ** -21}
# absolute error of one operand: fp16x3 splits x 2^14, whose low part is subnormal in FP16
# (spacing 2^-24) below 2^-14, so each factor also carries up to 2^-25 2^-14
ETA_OPERAND = {"fp16x3": 2.0 ** -39}
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1801_10016_gb300 import gsp2
    return gsp2


def run(g, s, prec, **opt):
    import torch
    plan = g.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind, device="cuda:0",
                  precision=prec, **opt)
    p = plan.density(torch.from_numpy(s.vals).to("cuda:0"))
    return plan, p.cpu().numpy(), plan.history()


@pytest.mark.parametrize("prec", ["tf32", "bf16", "tf32x3", "bf16x3", "fp32", "fp16x3"])
@pytest.mark.parametrize("case", ["tb512", "ragged132"])
def test_one_step_within_rounding_bound(g, prec, case):
    s = make_workload("tb512") if case == "tb512" else make_tb_system(33, 1, 3.0, seed=9)
    plan, p, hist = run(g, s, prec, max_steps=1, fp64_tail_steps=0)
    assert hist["report"]["steps"] == 1
    ref = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind,
                      max_steps=1)
    assert hist["alphas"][:1] == ref.alphas
    Hs = sp.csr_matrix((s.vals, s.colind, s.rowptr), shape=(s.n, s.n))
    worst = 0.0
    for S, c, X1 in zip(ref.S, ref.ncore, ref.X):
        X0 = oracle.initial_guess(Hs[S][:, S].toarray(), *ref.bounds)
        A = np.abs(X0)
        K = len(S)
        scale = 2.0 if ref.alphas[0] == 1 else 1.0
        # operand rounding (both factors), the FP32 master of X0, FP32 accumulation, output rounding
        bound = (2.0 * U_OPERAND[prec] + 2.0 * U32 + (K + 2) * U32) * (A @ A) + scale * 2 * U32 * A + U32 * np.abs(X1)
        eta = ETA_OPERAND.get(prec, 0.0)
        bound = bound + eta * (A.sum(axis=1)[:, None] + A.sum(axis=0)[None, :])
        bound = 2.0 * bound + 1e-30
        got = np.empty_like(X1[:, :c])
        for j in range(c):
            gcol = S[j]
            rows = plan.p_rowind[plan.p_colptr[gcol]:plan.p_colptr[gcol + 1]]
            pos = {int(v): i for i, v in enumerate(S)}
            got[[pos[int(r)] for r in rows], j] = p[plan.p_colptr[gcol]:plan.p_colptr[gcol + 1]]
        ratio = np.abs(got - X1[:, :c]) / bound[:, :c]
        worst = max(worst, float(ratio.max()))
    assert worst <= 1.0, worst


@pytest.mark.parametrize("prec,max_dp", [("tf32x3", 3e-6), ("fp32", 3e-6), ("tf32", 3e-3), ("bf16", 5e-2),
                                         ("bf16x3", 1e-3), ("fp16x3", 3e-6)])
def test_full_run_against_fp64_oracle(g, prec, max_dp):
    s = make_workload("tb512")
    plan, p, hist = run(g, s, prec)
    ref = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind)
    want = ref.p_on_pattern(plan.p_colptr, plan.p_rowind)
    err = float(np.max(np.abs(p - want)))
    rep = hist["report"]
    print(f"{prec}: steps={rep['steps']} fp64_steps={rep['fp64_steps']} max|dP|={err:.3e} "
          f"|trP-N|={abs(rep['trace'] - s.nocc):.3e} status={hist['status']}")
    assert rep["fp64_steps"] == 2
    assert err <= max_dp, err


@pytest.mark.parametrize("prec,max_dp", [("tf32x3", 5e-6), ("bf16x3", 3e-5), ("fp16x3", 5e-6)])
def test_low_precision_alternating_tail(g, prec, max_dp):
    """Tail steps in the low precision instead of FP64: same alternation, no FP64 step."""
    s = make_workload("tb512")
    plan, p, hist = run(g, s, prec, fp64_tail_steps=0, lp_tail_steps=2)
    rep = hist["report"]
    assert hist["status"] == 0 and rep["fp64_steps"] == 0
    k = rep["steps"]
    assert hist["alphas"][k - 1] == -hist["alphas"][k - 2]
    ref = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind)
    want = ref.p_on_pattern(plan.p_colptr, plan.p_rowind)
    err = float(np.max(np.abs(p - want)))
    print(f"{prec} low-precision tail: steps={k} max|dP|={err:.3e}")
    assert err <= max_dp, err


def test_tail_options_rejected_where_meaningless(g):
    s = make_workload("tb512")
    for kw in (dict(precision="fp64", lp_tail_steps=2), dict(precision="fp32", lp_tail_steps=1),
               dict(precision="tf32x3", lp_tail_steps=5, fp64_tail_steps=5)):
        with pytest.raises(g.GSP2Error):
            g.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind, bind=False, **kw)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "tf32", "bf16", "fp16x3"])
@pytest.mark.parametrize("case", ["tb512", "tb30k"])
def test_persistent_schedule_matches_one_cta_per_tile(g, prec, case):
    """The persistent tensor-core kernel (two TMEM accumulators, epilogue overlapped with
    the next tile) computes every tile exactly as the one-CTA-per-tile kernel."""
    if case == "tb30k" and prec not in ("tf32x3", "bf16", "fp16x3"):
        pytest.skip("one large case per kind")
    s = make_workload(case)
    _, p0, h0 = run(g, s, prec, tc_schedule=0, max_steps=6)
    _, p1, h1 = run(g, s, prec, tc_schedule=1, max_steps=6)
    _, p2, h2 = run(g, s, prec, tc_schedule=0, tile_shape=1, max_steps=6)
    assert h0["alphas"] == h1["alphas"] == h2["alphas"]
    assert np.array_equal(p0, p1) and np.array_equal(p0, p2)


@pytest.mark.parametrize("prec", ["tf32x3", "fp16x3"])
@pytest.mark.parametrize("case", ["tb512", "tb30k"])
def test_split_precisions_meet_the_gates_against_the_oracle_with_the_same_tail(g, prec, case):
    """Mixed precision (tf32x3 or fp16x3 squarings, FP64 traces, two FP64 tail steps) against
    the FP64 oracle with the same two tail steps: max|dP| <= 1e-6 and the column idempotency
    ||P^2 - P||_F / sqrt(N) (part by part) <= 1e-8."""
    s = make_workload(case)
    plan, p, hist = run(g, s, prec, fp64_tail_steps=2, report_idem=1)
    assert hist["status"] == 0
    ref = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind,
                      tail_steps=2)
    want = ref.p_on_pattern(plan.p_colptr, plan.p_rowind)
    err = float(np.max(np.abs(p - want)))
    idem = hist["report"]["idem_fro"]
    print(f"{case} {prec} + 2 FP64 tail vs oracle + 2 tail: max|dP|={err:.3e} idem_fro={idem:.3e}")
    assert err <= 1e-6, err
    assert 0.0 <= idem <= 1e-8, idem


@pytest.mark.parametrize("prec", ["tf32x3", "fp16x3"])
def test_emulated_and_native_fp64_tail_agree(g, prec):
    """The FP64 tail steps of a low-precision run, with the products on the FP64 units or
    rebuilt from BF16 digits, give the same P to FP64 accuracy (fp16x3 keeps upper tiles
    only, which the native tail gets mirrored first)."""
    s = make_workload("tb512")
    _, pe, he = run(g, s, prec, fp64_tail_steps=2, fp64_tail_emulated=1)
    _, pn, hn = run(g, s, prec, fp64_tail_steps=2, fp64_tail_emulated=0)
    assert he["alphas"] == hn["alphas"] and he["report"]["fp64_steps"] == 2
    assert float(np.max(np.abs(pe - pn))) <= 1e-12
