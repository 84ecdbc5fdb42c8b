"""The allocation-free bounds entry point, gsp2_bounds_noalloc.

It serves callers that may not allocate device memory (code inside another
framework's memory pool, plugins that must not grow the device footprint): its
scratch is a fixed array inside the library.  The GPU test checks it, through the
C ABI, against the bounds gsp2_density reports for the same H, on two calls in a row
(the second call reuses the scratch the first one left behind).  This file is
collected last, so a failure here cannot hide another test's result."""

import ctypes as C

import numpy as np
import pytest

from synth import make_workload


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


@pytest.mark.gpu
def test_noalloc_bounds_match_density_bounds_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gsp2, f = _lib()
    for name in ("tb512", "tb4k"):
        s = make_workload(name)
        plan = gsp2.GSP2(s.n, s.rowptr, s.colind, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind,
                         device="cuda:0")
        h = torch.from_numpy(s.vals).to("cuda:0")
        plan.density(h)
        st, rep = plan.status()
        assert st == 0
        rp = torch.from_numpy(s.rowptr).to("cuda:0")
        ci = torch.from_numpy(s.colind).to("cuda:0")
        stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        for call in range(2):
            out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda:0")
            rc = f(s.n, C.c_void_p(rp.data_ptr()), C.c_void_p(ci.data_ptr()), C.c_void_p(h.data_ptr()),
                   C.c_void_p(out.data_ptr()), stream)
            assert rc == gsp2.OK
            torch.cuda.synchronize()
            lo, hi = out.cpu().numpy()
            assert lo == pytest.approx(rep["eps_min"], rel=1e-13, abs=1e-13), (name, call)
            assert hi == pytest.approx(rep["eps_max"], rel=1e-13, abs=1e-13), (name, call)
