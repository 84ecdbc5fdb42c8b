"""GPU parity of the FP64 G-SP2 forward path (through the C ABI) against the CPU
oracle: every P value within 1e-10, the same branch sequence on every step whose
trace is not within 1e-9 N of Nocc, the same Gershgorin bounds, plus edge cases."""

import numpy as np
import pytest

import oracle
from synth import make_workload, block_partition
from synth.tb import make_tb_system, _csr_from_coo

pytestmark = pytest.mark.gpu

TOL_P = 1e-10


@pytest.fixture(scope="module")
def g():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1801_10016_gb300 import gsp2
    return gsp2


def run_gpu(g, s_or_args, **opt):
    import torch
    s = s_or_args
    plan = g.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind, device="cuda:0", **opt)
    h = torch.from_numpy(s.vals).to("cuda:0")
    alpha = torch.zeros(plan.alpha_len, dtype=torch.int8, device="cuda:0")
    p = plan.density(h, alpha=alpha)
    hist = plan.history()
    return plan, h, p, alpha, hist


def check_against_oracle(plan, p, hist, s, ref=None):
    if ref is None:
        ref = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind)
    want = ref.p_on_pattern(plan.p_colptr, plan.p_rowind)
    got = p.cpu().numpy()
    err = np.max(np.abs(got - want)) if want.size else 0.0
    assert err <= TOL_P, err
    rep = hist["report"]
    assert rep["eps_min"] == pytest.approx(ref.bounds[0], rel=1e-13, abs=1e-13)
    assert rep["eps_max"] == pytest.approx(ref.bounds[1], rel=1e-13, abs=1e-13)
    # branch sequence: identical wherever the decision has a margin
    margin = 1e-9 * s.n
    common = min(len(ref.alphas), len(hist["alphas"]))
    for i in range(common):
        if abs(ref.traces[i] - s.nocc) > margin:
            assert hist["alphas"][i] == ref.alphas[i], (i, hist["alphas"][:common], ref.alphas[:common])
            np.testing.assert_allclose(hist["traces"][i], ref.traces[i], rtol=0, atol=margin)
    assert abs(len(ref.alphas) - len(hist["alphas"])) <= 2
    return err


def test_tb512_matches_oracle(g):
    s = make_workload("tb512")
    plan, h, p, alpha, hist = run_gpu(g, s)
    assert hist["status"] == 0
    check_against_oracle(plan, p, hist, s)
    # alpha tensor written in RECORD mode: the applied sequence then zeros
    a = alpha.cpu().numpy()
    k = hist["report"]["steps"]
    assert a[:k].tolist() == hist["alphas"] and not np.any(a[k:])


@pytest.mark.parametrize("n_sites,nparts,radius", [(9, 3, 3.0), (33, 5, 3.2), (70, 4, 4.0), (40, 1, 3.0)])
def test_ragged_part_sizes(g, n_sites, nparts, radius):
    s = make_tb_system(n_sites, nparts, radius, seed=100 + n_sites)
    plan, h, p, alpha, hist = run_gpu(g, s)
    # sizes that are not multiples of the 64 tile or the 16 K slice
    assert np.any(plan.part_sizes % 64 != 0)
    check_against_oracle(plan, p, hist, s)


def test_single_orbital_parts_without_halo(g):
    """s_k = 1 for every part (empty graph): each part is a scalar SP2 sharing the
    global branch."""
    s = make_tb_system(6, 1, 3.0, seed=77)
    s.part = block_partition(s.n, s.n)
    s.nparts = s.n
    s.g_rowptr = np.zeros(s.n + 1, np.int64)
    s.g_colind = np.zeros(0, np.int32)
    plan, h, p, alpha, hist = run_gpu(g, s)
    assert plan.part_sizes.tolist() == [1] * s.n
    check_against_oracle(plan, p, hist, s)


def test_one_part_of_ragged_size(g):
    s = make_tb_system(33, 1, 3.0, seed=9)  # 132 orbitals: 3 tiles, the last one ragged
    plan, h, p, alpha, hist = run_gpu(g, s)
    assert plan.part_sizes.tolist() == [132]
    check_against_oracle(plan, p, hist, s)
    from synth import dense_from_csr
    H = dense_from_csr(s.n, s.rowptr, s.colind, s.vals)
    assert np.max(np.abs(plan.dense_p(p) - oracle.eig_projector(H, s.nocc))) <= 1e-9


def test_replay_reproduces_record_bitwise(g):
    import torch
    s = make_workload("tb512")
    plan, h, p, alpha, hist = run_gpu(g, s)
    k = hist["report"]["steps"]
    p2 = plan.density(h, alpha=alpha, mode="replay", nsteps=k)
    st, rep = plan.status()
    assert st == 0 and rep["steps"] == k
    assert torch.equal(p, p2)


def test_replay_with_wrong_sequence_reports_trace_error(g):
    """Section 2.1: a wrong multiplication sequence ends with the wrong trace."""
    s = make_workload("tb512")
    plan, h, p, alpha, hist = run_gpu(g, s)
    k = hist["report"]["steps"]
    bad = alpha.clone()
    bad[2] = -bad[2]
    plan.density(h, alpha=bad, mode="replay", nsteps=k)
    st, rep = plan.status()
    assert st == g.E_TRACE
    assert abs(rep["trace"] - s.nocc) > 0.5


def test_nonfinite_h_is_reported(g):
    import torch
    s = make_workload("tb512")
    plan, h, p, alpha, hist = run_gpu(g, s)
    h2 = h.clone()
    h2[17] = float("nan")
    plan.density(h2)
    st, rep = plan.status()
    assert st == g.E_NONFINITE
    # the plan stays usable
    p3 = plan.density(h)
    assert plan.status()[0] == 0
    assert torch.equal(p3, p)


def test_graph_and_direct_launch_agree(g):
    import torch
    s = make_workload("tb512")
    plan1, h, p1, _, _ = run_gpu(g, s, use_graph=1)
    plan0, _, p0, _, _ = run_gpu(g, s, use_graph=0)
    assert torch.equal(p0, p1)
    # repeated calls reuse the captured graph and are deterministic
    p2 = plan1.density(h)
    assert torch.equal(p2, p1)


@pytest.mark.parametrize("prec", ["fp64e", "fp16x3"])
def test_alternating_buffer_pairs_replay_their_graphs(g, prec):
    """The plan keeps a graph for each of the two most recent (H, P) buffer pairs: calls that
    alternate two pairs (as a caller overlapping copies with compute does) and a third pair
    that evicts one all give bitwise the same P."""
    import torch
    s = make_workload("tb512")
    plan = g.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind, device="cuda:0",
                  precision=prec)
    hs = [torch.from_numpy(s.vals).to("cuda:0") for _ in range(3)]
    ps = [torch.full((plan.nnz_p,), float("nan"), dtype=torch.float64, device="cuda:0") for _ in range(3)]
    ref = plan.density(hs[0], out=ps[0]).clone()
    for i in (1, 0, 1, 2, 0, 2, 1):
        ps[i].fill_(float("nan"))
        plan.density(hs[i], out=ps[i])
        assert torch.equal(ps[i], ref), i


def test_max_steps_cap_reports_not_converged(g):
    s = make_workload("tb512")
    plan, h, p, alpha, hist = run_gpu(g, s, max_steps=6)
    assert hist["status"] == g.E_NOT_CONVERGED
    assert hist["report"]["steps"] == 6
    ref = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind,
                      max_steps=6)
    want = ref.p_on_pattern(plan.p_colptr, plan.p_rowind)
    assert np.max(np.abs(p.cpu().numpy() - want)) <= TOL_P


def test_tb30k_full_size_matches_oracle(g):
    """The 30,000-orbital, 256-part workload in the benchmark's launch configuration:
    every value of P against the oracle."""
    s = make_workload("tb30k")
    plan, h, p, alpha, hist = run_gpu(g, s)
    assert hist["status"] == 0
    assert plan.nparts == 256 and plan.part_sizes.min() >= 300 and plan.part_sizes.max() <= 1300
    check_against_oracle(plan, p, hist, s)


def test_step_times_recorded_in_graph_mode(g):
    s = make_workload("tb512")
    plan, h, p, alpha, hist = run_gpu(g, s, time_steps=1)
    ms = plan.step_times()
    k = hist["report"]["steps"]
    assert np.all(ms[:k] > 0.0)
    assert np.all(np.isfinite(ms))


def test_idempotency_report_matches_oracle(g):
    """report_idem: sqrt(sum_k ||(X_k^2 - X_k)[:, cores]||_F^2 / N) of the final iterates."""
    s = make_workload("tb512")
    plan, h, p, alpha, hist = run_gpu(g, s, report_idem=1)
    ref = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind)
    want = np.sqrt(sum(np.linalg.norm((X @ X - X)[:, :c]) ** 2 for X, c in zip(ref.X, ref.ncore)) / s.n)
    got = hist["report"]["idem_fro"]
    assert got == pytest.approx(want, rel=1e-6, abs=1e-15)
    plan2, _, _, _, hist2 = run_gpu(g, s)
    assert hist2["report"]["idem_fro"] == -1.0


def test_fp64_tail_matches_oracle_tail(g):
    """fp64_tail_steps = 2 on the FP64 path: the loop continues past the stopping test
    with two alternating steps, as the oracle's tail."""
    s = make_workload("tb512")
    plan, h, p, alpha, hist = run_gpu(g, s, fp64_tail_steps=2, report_idem=1)
    assert hist["status"] == 0
    ref = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind,
                      tail_steps=2)
    check_against_oracle(plan, p, hist, s, ref=ref)
    assert hist["alphas"] == ref.alphas and hist["alphas"][-1] == -hist["alphas"][-2]
    assert hist["report"]["idem_fro"] < 1e-10
    # replaying the recorded sequence (tail included) reproduces P bitwise
    import torch
    k = hist["report"]["steps"]
    p2 = plan.density(h, alpha=alpha, mode="replay", nsteps=k)
    assert plan.status()[0] == 0 and torch.equal(p, p2)


# ---------------------------------------------------------------- FP64 from BF16 digits

@pytest.mark.parametrize("case", ["tb512", "ragged36", "ragged132", "ragged280", "tb30k"])
def test_fp64_emulated_matches_oracle(g, case):
    """precision fp64e: X X rebuilt from 8 BF16 digits on the tensor cores, FP64 master and
    bookkeeping; held to the FP64 parity bar (1e-10) against the oracle."""
    s = {"tb512": lambda: make_workload("tb512"), "ragged36": lambda: make_tb_system(9, 3, 3.0, seed=109),
         "ragged132": lambda: make_tb_system(33, 1, 3.0, seed=9), "ragged280": lambda: make_tb_system(70, 4, 4.0, seed=170),
         "tb30k": lambda: make_workload("tb30k")}[case]()
    plan, h, p, alpha, hist = run_gpu(g, s, precision="fp64e")
    assert hist["status"] == 0
    err = check_against_oracle(plan, p, hist, s)
    print(f"fp64e {case}: steps={hist['report']['steps']} max|dP|={err:.3e}")


def test_fp64_emulated_one_step_error(g):
    """One emulated step against the FP64 product, element by element: the digit expansion
    truncates below 2^-56 and drops products of order 2^{-7 (d+2)} for d >= 8."""
    s = make_workload("tb512")
    plan, h, p, alpha, hist = run_gpu(g, s, precision="fp64e", max_steps=1)
    ref = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind,
                      max_steps=1)
    want = ref.p_on_pattern(plan.p_colptr, plan.p_rowind)
    err = float(np.max(np.abs(p.cpu().numpy() - want)))
    print(f"fp64e one step: max|dY|={err:.3e}")
    assert err <= 1e-13
