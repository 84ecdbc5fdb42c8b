"""The allocation-free bounds entry point, gsp2_bounds_noalloc.

It serves callers that may not allocate device memory (code inside another
framework's memory pool, plugins that must not grow the device footprint): its
scratch is a fixed array inside the library.  The GPU tests check it, through the
C ABI, against the bounds gsp2_density reports for the same H and against the CPU
oracle's Gershgorin bounds, on two calls in a row (the second call reuses the scratch
the first one left behind), with row counts that leave the last block and its last
warp partly empty, and with NaN and Inf planted in H.  This file is collected last,
so a failure here cannot hide another test's result."""

import ctypes as C

import numpy as np
import pytest

import oracle
from synth import make_workload
from synth.tb import make_tb_system


def _lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1801_10016_gb300 import gsp2
    lib = C.CDLL(gsp2.LIB_PATH)
    f = lib.gsp2_bounds_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    return gsp2, f


def test_noalloc_rejects_oversize_without_touching_the_gpu():
    gsp2, f = _lib()
    dummy = C.c_void_p(16)
    assert f(4096 * 256 + 1, dummy, dummy, dummy, dummy, None) == gsp2.E_ARG
    assert f(0, dummy, dummy, dummy, dummy, None) == gsp2.E_ARG
    assert f(10, None, dummy, dummy, dummy, None) == gsp2.E_ARG


def _call(f, gsp2, n, rp, ci, vals):
    import torch
    out = torch.full((2,), 12345.0, dtype=torch.float64, device="cuda:0")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = f(n, C.c_void_p(rp.data_ptr()), C.c_void_p(ci.data_ptr()), C.c_void_p(vals.data_ptr()),
           C.c_void_p(out.data_ptr()), stream)
    assert rc == gsp2.OK
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["tb512", "tb4k", "ragged132", "ragged4028"])
def test_noalloc_bounds_match_density_bounds_twice(name):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gsp2, f = _lib()
    # 132 rows: one block, its last warp 4 rows; 4028 rows: 16 blocks, the last one 188 rows
    s = {"ragged132": lambda: make_tb_system(33, 3, 3.0, seed=5),
         "ragged4028": lambda: make_tb_system(1007, 16, 3.0, seed=6)}.get(name, lambda: make_workload(name))()
    want = oracle.gershgorin_bounds(s.n, s.rowptr, s.colind, s.vals)
    plan = gsp2.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind, device="cuda:0")
    h = torch.from_numpy(s.vals).to("cuda:0")
    plan.density(h)
    st, rep = plan.status()
    assert st == 0
    rp = torch.from_numpy(s.rowptr).to("cuda:0")
    ci = torch.from_numpy(s.colind).to("cuda:0")
    for call in range(2):
        lo, hi = _call(f, gsp2, s.n, rp, ci, h)
        assert lo == pytest.approx(rep["eps_min"], rel=1e-13, abs=1e-13), (name, call)
        assert hi == pytest.approx(rep["eps_max"], rel=1e-13, abs=1e-13), (name, call)
        assert lo == pytest.approx(want[0], rel=1e-13, abs=1e-13), (name, call)
        assert hi == pytest.approx(want[1], rel=1e-13, abs=1e-13), (name, call)


@pytest.mark.gpu
def test_noalloc_bounds_of_non_finite_values():
    """A NaN anywhere in H gives NaN bounds (min and max must not drop it); an infinite
    off-diagonal value gives an infinite radius, so both bounds are infinite.  The values
    are planted on the host; the kernel only reads them."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gsp2, f = _lib()
    s = make_tb_system(1007, 16, 3.0, seed=6)
    rp = torch.from_numpy(s.rowptr).to("cuda:0")
    ci = torch.from_numpy(s.colind).to("cuda:0")
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    offd = np.nonzero(rows != s.colind)[0]
    for pos in (int(offd[0]), int(offd[len(offd) // 2]), int(offd[-1])):
        v = s.vals.copy()
        v[pos] = np.nan
        lo, hi = _call(f, gsp2, s.n, rp, ci, torch.from_numpy(v).to("cuda:0"))
        assert np.isnan(lo) and np.isnan(hi), (pos, lo, hi)
        v = s.vals.copy()
        v[pos] = np.inf
        lo, hi = _call(f, gsp2, s.n, rp, ci, torch.from_numpy(v).to("cuda:0"))
        assert lo == -np.inf and hi == np.inf, (pos, lo, hi)
    # the scratch left by those calls does not leak into the next one
    lo, hi = _call(f, gsp2, s.n, rp, ci, torch.from_numpy(s.vals).to("cuda:0"))
    want = oracle.gershgorin_bounds(s.n, s.rowptr, s.colind, s.vals)
    assert lo == pytest.approx(want[0], rel=1e-13, abs=1e-13) and hi == pytest.approx(want[1], rel=1e-13, abs=1e-13)
