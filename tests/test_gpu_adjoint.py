"""GPU parity of the hand-written adjoint (gsp2_backward) against the oracle's
reverse-mode adjoint, which the CPU suite pins to finite differences and to the
Daleckii-Krein divided differences of the same SP2 polynomial."""

import numpy as np
import pytest

import oracle
from synth import make_workload, dense_from_csr, random_symmetric_on_pattern
from synth.tb import make_tb_system

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


def pbar_for_trace_loss(s, plan):
    """L = tr(P A) with A a seeded symmetric Gaussian matrix on H's pattern:
    dL/dP_ij = A_ji = A_ij on the pattern of P."""
    A = dense_from_csr(s.n, s.rowptr, s.colind, random_symmetric_on_pattern(s.rowptr, s.colind, 5678))
    cols = np.repeat(np.arange(s.n), np.diff(plan.p_colptr))
    pb = A[plan.p_rowind, cols]
    Pbar = np.zeros((s.n, s.n))
    Pbar[plan.p_rowind, cols] = pb
    return pb, Pbar


def run_adjoint(g, s, **opt):
    import torch
    plan = g.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind, device="cuda:0", **opt)
    h = torch.from_numpy(s.vals).to("cuda:0")
    plan.density(h)
    hist = plan.history()
    pb, Pbar = pbar_for_trace_loss(s, plan)
    hb = plan.backward(torch.from_numpy(pb).to("cuda:0"))
    return plan, h, hist, pb, Pbar, hb


@pytest.mark.parametrize("case", ["small", "tb512", "tb4k"])
def test_adjoint_matches_oracle(g, case):
    s = {"small": lambda: make_tb_system(48, 4, 3.0, seed=21), "tb512": lambda: make_workload("tb512"),
         "tb4k": lambda: make_workload("tb4k")}[case]()
    plan, h, hist, pb, Pbar, hb = run_adjoint(g, s)
    assert hist["status"] == 0
    ref = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind)
    assert hist["alphas"] == ref.alphas  # same polynomial on both sides
    want = oracle.gsp2_adjoint(s.n, s.rowptr, s.colind, s.vals, ref, Pbar)
    got = hb.cpu().numpy()
    scale = max(1.0, np.max(np.abs(want)))
    assert np.max(np.abs(got - want)) <= 1e-9 * scale, np.max(np.abs(got - want))


@pytest.mark.parametrize("k", [1, 3, 45])
def test_checkpoint_interval_does_not_change_the_gradient(g, k):
    import torch
    s = make_tb_system(48, 4, 3.0, seed=21)
    _, _, _, _, _, hb8 = run_adjoint(g, s)
    _, _, _, _, _, hbk = run_adjoint(g, s, ckpt_every=k)
    assert torch.equal(hb8, hbk)


def test_autograd_function_uses_the_adjoint(g):
    import torch
    s = make_tb_system(48, 4, 3.0, seed=21)
    plan = g.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind, device="cuda:0")
    pb, _ = pbar_for_trace_loss(s, plan)
    pbt = torch.from_numpy(pb).to("cuda:0")
    h = torch.from_numpy(s.vals).to("cuda:0").requires_grad_(True)
    P = g.gsp2_density(h, plan)
    loss = (P * pbt).sum()
    loss.backward()
    direct = plan.backward(pbt)
    assert torch.equal(h.grad, direct)


def test_autograd_refuses_a_forward_replaced_by_a_later_call(g):
    """The library keeps the adjoint state of a plan's last density call only: a backward
    through an earlier forward on the same plan must raise instead of returning the
    gradient at the later H."""
    import torch
    s = make_tb_system(48, 4, 3.0, seed=21)
    plan = g.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind, device="cuda:0")
    pb, _ = pbar_for_trace_loss(s, plan)
    pbt = torch.from_numpy(pb).to("cuda:0")
    h1 = torch.from_numpy(s.vals).to("cuda:0").requires_grad_(True)
    h2 = (torch.from_numpy(s.vals) * 1.01).to("cuda:0").requires_grad_(True)
    P1 = g.gsp2_density(h1, plan)
    P2 = g.gsp2_density(h2, plan)
    with pytest.raises(RuntimeError, match="another density call"):
        (P1 * pbt).sum().backward()
    # the live (last) forward still differentiates, and a plain density call also
    # invalidates it
    (P2 * pbt).sum().backward()
    assert torch.equal(h2.grad, plan.backward(pbt))
    P3 = g.gsp2_density(h1.detach().requires_grad_(True), plan)
    plan.density(h2.detach())
    with pytest.raises(RuntimeError, match="another density call"):
        (P3 * pbt).sum().backward()


def test_backward_state_errors(g):
    import torch
    s = make_tb_system(20, 2, 3.0, seed=4)
    plan = g.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind, device="cuda:0")
    with pytest.raises(g.GSP2Error) as e:
        plan.backward(torch.zeros(plan.nnz_p, dtype=torch.float64, device="cuda:0"))
    assert e.value.status == g.E_STATE
    plan0 = g.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind, device="cuda:0",
                   ckpt_every=0)
    plan0.density(torch.from_numpy(s.vals).to("cuda:0"))
    with pytest.raises(g.GSP2Error) as e:
        plan0.backward(torch.zeros(plan0.nnz_p, dtype=torch.float64, device="cuda:0"))
    assert e.value.status == g.E_STATE


@pytest.mark.parametrize("prec", ["fp64", "fp64e"])
def test_adjoint_through_tail_steps(g, prec):
    s = make_tb_system(48, 4, 3.0, seed=21)
    plan, h, hist, pb, Pbar, hb = run_adjoint(g, s, precision=prec, fp64_tail_steps=2, ckpt_every=3)
    ref = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind,
                      tail_steps=2)
    assert hist["alphas"] == ref.alphas
    want = oracle.gsp2_adjoint(s.n, s.rowptr, s.colind, s.vals, ref, Pbar)
    got = hb.cpu().numpy()
    assert np.max(np.abs(got - want)) <= 1e-9 * max(1.0, np.max(np.abs(want)))


@pytest.mark.parametrize("prec,tail,case,tol", [("fp32", 0, "small", 2e-5), ("fp32", 0, "tb4k", 2e-5),
                                                ("fp32", 2, "tb4k", 2e-5), ("tf32x3", 2, "tb4k", 2e-5),
                                                ("tf32x3", 2, "small", 2e-5), ("fp32", 3, "tb512", 2e-5),
                                                ("fp16x3", 2, "tb4k", 2e-5), ("bf16x3", 1, "tb512", 1e-4)])
def test_low_precision_adjoint_matches_oracle_on_the_same_sequence(g, prec, tail, case, tol):
    """FP32 adjoint (FP16 hi + lo products on the tensor cores, Xbar's scaled per part) of a
    low-precision forward against the oracle's FP64 adjoint of the same polynomial (the
    GPU's own branch sequence, tail steps included).  The sweep rebuilds its iterates from
    the forward's checkpoints, so a bf16x3 forward (16-bit operands, outside the 1e-6 gate on
    P) bounds it at 1e-4."""
    s = make_tb_system(48, 4, 3.0, seed=21) if case == "small" else make_workload(case)
    plan, h, hist, pb, Pbar, hb = run_adjoint(g, s, precision=prec, fp64_tail_steps=tail, ckpt_every=4)
    assert hist["status"] == 0 and hist["report"]["fp64_steps"] == tail
    ref = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind,
                      alphas=hist["alphas"])
    assert ref.alphas == hist["alphas"]
    want = oracle.gsp2_adjoint(s.n, s.rowptr, s.colind, s.vals, ref, Pbar)
    got = hb.cpu().numpy()
    err = float(np.max(np.abs(got - want))) / max(1.0, float(np.max(np.abs(want))))
    print(f"{prec} tail={tail} {case}: steps={hist['report']['steps']} relative max|dHbar|={err:.3e}")
    assert err <= tol, err


@pytest.mark.parametrize("prec,tail", [("fp32", 2), ("tf32x3", 2), ("fp16x3", 2), ("fp64e", 2), ("fp64", 0)])
def test_density_after_backward_is_unchanged(g, prec, tail):
    """A backward shares scratch arenas with the forward (the FP32 adjoint keeps Xbar's
    operands in the FP64 tail arenas): a density call after it gives bitwise the same P,
    branch sequence and idempotency report as before it."""
    import torch
    s = make_tb_system(48, 4, 3.0, seed=21)
    plan = g.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind, device="cuda:0",
                  precision=prec, fp64_tail_steps=tail, ckpt_every=3, report_idem=1)
    h = torch.from_numpy(s.vals).to("cuda:0")
    p0 = plan.density(h).clone()
    r0 = plan.history()
    pb, _ = pbar_for_trace_loss(s, plan)
    hb = plan.backward(torch.from_numpy(pb).to("cuda:0"))
    assert torch.isfinite(hb).all()
    p1 = plan.density(h)
    r1 = plan.history()
    assert torch.equal(p0, p1)
    assert r0["alphas"] == r1["alphas"] and r0["report"]["idem_fro"] == r1["report"]["idem_fro"]


@pytest.mark.parametrize("case,k", [("small", 1), ("small", 3), ("small", 45), ("tb512", 5)])
def test_fp16x3_checkpoint_interval_does_not_change_the_gradient(g, case, k):
    """The FP32 adjoint rebuilds iterates with the fp16x3 step's own tensor-core arithmetic
    from the same FP16 operand split, so for fp16x3 plans every rebuilt iterate equals the
    forward's bit for bit: the same gradient whatever the checkpoint interval."""
    import torch
    s = make_tb_system(48, 4, 3.0, seed=21) if case == "small" else make_workload("tb512")
    _, _, _, _, _, hb4 = run_adjoint(g, s, precision="fp16x3", fp64_tail_steps=0, ckpt_every=4)
    _, _, _, _, _, hbk = run_adjoint(g, s, precision="fp16x3", fp64_tail_steps=0, ckpt_every=k)
    assert torch.equal(hb4, hbk)


def test_fp16_adjoint_is_exact_under_power_of_two_scaling(g):
    """Xbar's FP16 operands carry a per-part power-of-two scale taken from its largest entry:
    Pbar scaled by 2^e gives Hbar scaled by 2^e exactly, far beyond FP16's own range."""
    import torch
    s = make_workload("tb512")
    plan = g.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind, device="cuda:0",
                  precision="fp16x3", fp64_tail_steps=2, ckpt_every=4)
    plan.density(torch.from_numpy(s.vals).to("cuda:0"))
    pb, _ = pbar_for_trace_loss(s, plan)
    pbt = torch.from_numpy(pb).to("cuda:0")
    hb = plan.backward(pbt).clone()
    assert torch.isfinite(hb).all()
    for e in (-40, 40):
        assert torch.equal(plan.backward(pbt * 2.0 ** e), hb * 2.0 ** e), e


@pytest.mark.parametrize("case,k", [("small", 3), ("tb512", 8), ("tb4k", 3), ("tb4k", 8)])
def test_adjoint_of_the_emulated_fp64_forward(g, case, k):
    """Emulated FP64 adjoint (reverse steps and rebuilt iterates from BF16 digit products,
    Xbar digits scaled per part) against the oracle's adjoint on the same branch sequence."""
    s = {"small": lambda: make_tb_system(48, 4, 3.0, seed=21), "tb512": lambda: make_workload("tb512"),
         "tb4k": lambda: make_workload("tb4k")}[case]()
    plan, h, hist, pb, Pbar, hb = run_adjoint(g, s, precision="fp64e", ckpt_every=k)
    assert hist["status"] == 0
    ref = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind)
    assert hist["alphas"] == ref.alphas
    want = oracle.gsp2_adjoint(s.n, s.rowptr, s.colind, s.vals, ref, Pbar)
    err = float(np.max(np.abs(hb.cpu().numpy() - want)))
    assert err <= 1e-9 * max(1.0, float(np.max(np.abs(want)))), err
    st, _ = plan.status()
    assert st == 0


def test_emulated_adjoint_is_exact_under_power_of_two_scaling(g):
    """Xbar's digits carry a per-part power-of-two scale taken from its row norms, so scaling
    Pbar by 2^e scales every step's scale exponent by e and Hbar exactly by 2^e, far outside
    the range a fixed scale would hold."""
    import torch
    s = make_workload("tb512")
    plan = g.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind, device="cuda:0",
                  precision="fp64e", ckpt_every=4)
    plan.density(torch.from_numpy(s.vals).to("cuda:0"))
    pb, _ = pbar_for_trace_loss(s, plan)
    pbt = torch.from_numpy(pb).to("cuda:0")
    hb = plan.backward(pbt).clone()
    for e in (-300, -60, 60, 300):
        hbe = plan.backward(pbt * 2.0 ** e)
        assert torch.equal(hbe, hb * 2.0 ** e), e


def test_emulated_adjoint_propagates_nonfinite_like_the_fp64_adjoint(g):
    """A NaN in Pbar makes every Hbar entry that draws on its part NaN, in the emulated adjoint
    (the part's scale marks it) as in the FP64 one (through the arithmetic)."""
    import torch
    s = make_workload("tb512")
    out = {}
    for prec in ("fp64", "fp64e"):
        plan = g.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind, device="cuda:0",
                      precision=prec, ckpt_every=8)
        plan.density(torch.from_numpy(s.vals).to("cuda:0"))
        pb, _ = pbar_for_trace_loss(s, plan)
        pb[len(pb) // 3] = np.nan
        out[prec] = plan.backward(torch.from_numpy(pb).to("cuda:0")).cpu().numpy()
    nan64, nan_e = np.isnan(out["fp64"]), np.isnan(out["fp64e"])
    assert nan64.any() and not nan64.all()
    assert np.array_equal(nan64, nan_e)
    ok = ~nan64
    assert np.max(np.abs(out["fp64"][ok] - out["fp64e"][ok])) <= 1e-9 * max(1.0, np.max(np.abs(out["fp64"][ok])))


@pytest.mark.parametrize("case", ["tb512", "tb4k"])
def test_emulated_adjoint_split_k_matches_one_item_per_tile(g, case):
    """Split K (each reverse step's tile as two work items, its Xbar X and X Xbar halves,
    added as 64-bit integers) against one item per tile: the same gradient up to the FP32
    rounding of the low-order digit groups (far below the 1e-9 adjoint bar), both within
    1e-9 of the oracle's adjoint."""
    s = make_workload(case)
    plan1, h, hist, pb, Pbar, hb1 = run_adjoint(g, s, precision="fp64e", split_k=1)
    plan0, _, _, _, _, hb0 = run_adjoint(g, s, precision="fp64e", split_k=0)
    assert plan1.info.split_k == 1 and plan0.info.split_k == 0
    a, b = hb1.cpu().numpy(), hb0.cpu().numpy()
    scale = max(1.0, float(np.max(np.abs(b))))
    assert np.max(np.abs(a - b)) <= 1e-13 * scale
    ref = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind)
    want = oracle.gsp2_adjoint(s.n, s.rowptr, s.colind, s.vals, ref, Pbar)
    assert np.max(np.abs(a - want)) <= 1e-9 * max(1.0, float(np.max(np.abs(want))))
    # a second backward on the same plan (the per-tile counters are left at zero) repeats it
    hb2 = plan1.backward(torch_from(pb))
    assert np.array_equal(hb2.cpu().numpy(), a)


def torch_from(x):
    import torch
    return torch.from_numpy(x).to("cuda:0")


@pytest.mark.parametrize("prec", ["fp64e", "fp16x3"])
def test_adjoint_claimed_tiles_match_the_static_deal(g, prec):
    """Reverse steps whose CTAs claim their tiles from a counter against the static deal: a
    tile's arithmetic does not depend on the CTA that runs it, so the same Hbar bit for bit,
    also on a second backward (the counter is left at zero)."""
    s = make_workload("tb4k")
    kw = dict(precision=prec, ckpt_every=8, split_k=0)
    plan1, _, _, pb, _, hb1 = run_adjoint(g, s, tile_claim=1, **kw)
    plan0, _, _, _, _, hb0 = run_adjoint(g, s, tile_claim=0, **kw)
    assert plan1.info.tile_claim == 1 and plan0.info.tile_claim == 0
    a = hb1.cpu().numpy()
    assert np.array_equal(a, hb0.cpu().numpy())
    assert np.array_equal(plan1.backward(torch_from(pb)).cpu().numpy(), a)


@pytest.mark.parametrize("prec", ["fp64", "fp64e", "fp16x3"])
def test_adjoint_after_a_status_read_is_the_same(g, prec):
    """Once gsp2_sync_status has read the applied step count, the adjoint schedules only those
    steps (the launches for steps beyond it return at once otherwise): bitwise the same Hbar,
    and a later density call falls back to the full schedule until its status is read."""
    import torch
    s = make_tb_system(48, 4, 3.0, seed=21)
    kw = dict(precision=prec, ckpt_every=3)
    if prec == "fp16x3":
        kw["fp64_tail_steps"] = 2
    plan = g.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind, device="cuda:0", **kw)
    h = torch.from_numpy(s.vals).to("cuda:0")
    pb, _ = pbar_for_trace_loss(s, plan)
    pbt = torch.from_numpy(pb).to("cuda:0")
    plan.density(h)
    full = plan.backward(pbt).clone()      # step count not read: every step launch scheduled
    assert plan.status()[0] == 0
    exact = plan.backward(pbt).clone()     # only the applied steps
    assert torch.equal(full, exact)
    plan.density(h * 1.001)
    again = plan.backward(pbt)             # a new forward: the full schedule again
    plan.status()
    assert torch.equal(again, plan.backward(pbt))
