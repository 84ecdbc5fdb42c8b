"""Second workload, shaped like a dense molecular crystal (the paper's urea case): sites
twice as dense as the solvated-protein stand-in, so each core carries a halo several times
its size.  FP64 and FP64-accurate emulated paths against the oracle on every value of P."""

import numpy as np
import pytest

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


@pytest.mark.parametrize("case,prec", [("crystal512", "fp64"), ("crystal512", "fp64e"), ("crystal8k", "fp64e")])
def test_crystal_matches_oracle(g, case, prec):
    import torch
    s = make_workload(case)
    plan = g.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind, device="cuda:0",
                  precision=prec, ckpt_every=0)
    p = plan.density(torch.from_numpy(s.vals).to("cuda:0")).cpu().numpy()
    hist = plan.history()
    assert hist["status"] == 0
    ref = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind)
    assert hist["alphas"] == ref.alphas
    err = float(np.max(np.abs(p - ref.p_on_pattern(plan.p_colptr, plan.p_rowind))))
    print(f"{case} {prec}: sizes {plan.part_sizes.min()}-{plan.part_sizes.max()} steps={len(ref.alphas)} "
          f"max|dP|={err:.3e}")
    assert err <= 1e-10
