"""One dense part whose iterates spread every row over all of its columns: the case that
presses hardest on the bounds under which the emulated FP64 step keeps its leading digit
groups exact in FP32 (sum_k |x_ik x_kj| <= 1, and sum_k |x_ik| up to sqrt(K) ||x_i||_2 for the
group that shares an accumulator; K = s for a forward step and 2 s for an adjoint step).

H = Q diag(lambda) Q^T with Q a seeded Haar-random orthogonal matrix and a gap around the
Fermi level, so that P = Q_occ Q_occ^T has entries of size 1/sqrt(n) everywhere and the
rows of the late iterates reach row 1-norms of about sqrt(2 n / pi) ||x_i||_2.  Both sides
run the paper's G-SP2 (Section 2.1) on the single part; the oracle runs its own bounds and
branch sequence.  Once X is idempotent to rounding its trace equals N_occ to the last bit
(the oracle's last two traces differ from N_occ by exactly 0.0), so the branch rule takes
either side there and the stopping test, which asks whether the idempotency error still
falls, may end a step or two apart: the branches are compared where the trace is more than
1e-9 from N_occ (the GPU's traces carry about 1e-12), P against the oracle's own run and
against the oracle replaying the GPU's sequence."""

import numpy as np
import pytest

import oracle
from synth import TBSystem, csr_from_dense, dense_from_csr, random_symmetric_on_pattern

pytestmark = pytest.mark.gpu

N = 2048  # K = 2048 forward, 4096 (the limit of the exactness bounds) in the adjoint


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
def dense():
    rng = np.random.default_rng(20240611)
    q, r = np.linalg.qr(rng.standard_normal((N, N)))
    q *= np.sign(np.diag(r))
    nocc = N // 2
    lam = np.concatenate([rng.uniform(-1.0, -0.2, nocc), rng.uniform(0.2, 1.0, N - nocc)])
    H = (q * lam) @ q.T
    H = 0.5 * (H + H.T)
    rowptr, colind, vals = csr_from_dense(H)
    assert rowptr[-1] == N * N
    # one part holding every orbital: no halo, so the dependency graph can stay empty
    return TBSystem(name="dense2048", n_sites=N // 4, n=N, nocc=nocc, rowptr=rowptr, colind=colind, vals=vals,
                    coords=np.zeros((N // 4, 3)), part=np.zeros(N, dtype=np.int32), nparts=1,
                    g_rowptr=np.zeros(N + 1, dtype=np.int64), g_colind=np.zeros(0, dtype=np.int32))


@pytest.fixture(scope="module")
def ref(dense):
    s = dense
    return oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind)


def test_dense_part_rows_reach_the_one_norm_bound(dense, ref):
    """The converged P spreads each row: its row 1-norms come within a factor 2 of the
    Cauchy-Schwarz limit sqrt(K) ||p_i||_2 that the exactness bound allows for."""
    P = ref.dense_p()
    one = np.abs(P).sum(axis=1)
    two = np.sqrt((P * P).sum(axis=1))
    assert np.min(one / (np.sqrt(N) * two)) > 0.5


def test_dense_part_emulated_forward_matches_the_oracle(g, dense, ref):
    import torch
    s = dense
    plan = g.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind, device="cuda:0",
                  precision="fp64e", ckpt_every=0)
    p = plan.density(torch.from_numpy(s.vals).to("cuda:0"))
    hist = plan.history()
    assert hist["status"] == 0
    assert hist["report"]["eps_min"] == pytest.approx(ref.bounds[0], rel=1e-13, abs=1e-13)
    assert hist["report"]["eps_max"] == pytest.approx(ref.bounds[1], rel=1e-13, abs=1e-13)
    ga = hist["alphas"]
    for i in range(min(len(ga), len(ref.alphas))):
        if abs(ref.traces[i] - s.nocc) > 1e-9:
            assert ga[i] == ref.alphas[i], i
    assert abs(len(ga) - len(ref.alphas)) <= 2
    got = p.cpu().numpy()
    err = float(np.max(np.abs(got - ref.p_on_pattern(plan.p_colptr, plan.p_rowind))))
    rep_ = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind,
                       alphas=ga)
    err_r = float(np.max(np.abs(got - rep_.p_on_pattern(plan.p_colptr, plan.p_rowind))))
    print(f"dense part n={N}: steps={len(ga)} (oracle {len(ref.alphas)}) fp64e max|dP|={err:.3e}, "
          f"against the replayed sequence {err_r:.3e}")
    assert err <= 1e-10, err
    assert err_r <= 1e-10, err_r


def test_dense_part_emulated_adjoint_matches_the_oracle(g, dense, ref):
    import torch
    s = dense
    plan = g.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind, device="cuda:0",
                  precision="fp64e", ckpt_every=8)
    plan.density(torch.from_numpy(s.vals).to("cuda:0"))
    # the adjoint differentiates the polynomial the forward applied: the oracle replays it
    rep_ = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind,
                       alphas=plan.history()["alphas"])
    A = dense_from_csr(s.n, s.rowptr, s.colind, random_symmetric_on_pattern(s.rowptr, s.colind, 5678))
    cols = np.repeat(np.arange(s.n), np.diff(plan.p_colptr))
    pb = A[plan.p_rowind, cols]
    Pbar = np.zeros((s.n, s.n))
    Pbar[plan.p_rowind, cols] = pb
    got = plan.backward(torch.from_numpy(pb).to("cuda:0")).cpu().numpy()
    want = oracle.gsp2_adjoint(s.n, s.rowptr, s.colind, s.vals, rep_, Pbar)
    scale = max(1.0, float(np.max(np.abs(want))))
    err = float(np.max(np.abs(got - want)))
    print(f"dense part n={N}: fp64e adjoint max|dHbar|={err:.3e} (scale {scale:.3e})")
    assert err <= 1e-9 * scale, err
