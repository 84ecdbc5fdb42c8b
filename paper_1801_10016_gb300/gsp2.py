"""Python binding of libgsp2.so (ctypes).  Argument marshalling only: every step of
the density-matrix path runs in the library's CUDA kernels.  PyTorch provides the
device memory (workspace, H and P values) and the stream.

    plan = GSP2(n, rowptr, colind, nocc, part, nparts, g_rowptr, g_colind)
    p = plan.density(h_vals)            # torch.float64 on cuda, P on plan.p_colptr/p_rowind
    p = gsp2_density(h_vals, plan)      # same, differentiable (adjoint through the library)
"""

from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgsp2.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "gsp2.h")

OK, E_ARG, E_OOM, E_STATE, E_CUDA, E_NOT_CONVERGED, E_TRACE, E_NONFINITE, E_WORKSPACE, E_TIMEOUT = range(10)
STATUS_NAMES = {0: "OK", 1: "E_ARG", 2: "E_OOM", 3: "E_STATE", 4: "E_CUDA", 5: "E_NOT_CONVERGED",
                6: "E_TRACE", 7: "E_NONFINITE", 8: "E_WORKSPACE", 9: "E_TIMEOUT"}
PRECISIONS = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3, "bf16x3": 4, "tf32x3": 5, "fp64e": 6, "fp16x3": 7}
MODES = {"record": 0, "replay": 1}


class GSP2Error(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"gsp2 {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Options(C.Structure):
    _fields_ = [("max_steps", C.c_int32), ("idem_tol", C.c_double), ("trace_tol", C.c_double),
                ("precision", C.c_int32), ("fp64_tail_steps", C.c_int32), ("ckpt_every", C.c_int32),
                ("use_graph", C.c_int32), ("time_steps", C.c_int32), ("lp_tail_steps", C.c_int32),
                ("tc_schedule", C.c_int32), ("report_idem", C.c_int32), ("fp64_tail_emulated", C.c_int32),
                ("tile_order", C.c_int32), ("tile_shape", C.c_int32), ("split_k", C.c_int32),
                ("tile_claim", C.c_int32)]


class Report(C.Structure):
    _fields_ = [("status", C.c_int32), ("steps", C.c_int32), ("stopped", C.c_int32), ("fp64_steps", C.c_int32),
                ("eps_min", C.c_double), ("eps_max", C.c_double), ("trace", C.c_double), ("idem", C.c_double),
                ("idem_fro", C.c_double)]


class PlanInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("nocc", C.c_int64), ("nparts", C.c_int32), ("max_s", C.c_int32),
                ("sum_s", C.c_int64), ("sum_s2", C.c_double), ("sum_s3", C.c_double), ("nnz_h", C.c_int64),
                ("nnz_p", C.c_int64), ("arena_elems", C.c_int64), ("ntiles", C.c_int64), ("tile", C.c_int32),
                ("ld_pad", C.c_int32), ("step_launches", C.c_int32), ("fp64_tail_steps", C.c_int32),
                ("tc_schedule", C.c_int32), ("tile_order", C.c_int32), ("tile_shape", C.c_int32),
                ("split_k", C.c_int32), ("tile_claim", C.c_int32)]


class TuneReport(C.Structure):
    _fields_ = [("ncand", C.c_int32), ("chosen", C.c_int32), ("tc_schedule", C.c_int32 * 8),
                ("tile_order", C.c_int32 * 8), ("tile_shape", C.c_int32 * 8), ("ms", C.c_double * 8),
                ("split_k", C.c_int32 * 8), ("tile_claim", C.c_int32 * 8)]


_lib = None
_P = C.c_void_p


def header_functions() -> list[str]:
    """Names of the functions declared in include/gsp2.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gsp2_\w+)\s*\(", txt)))


def load(path: str = LIB_PATH):
    """Load libgsp2.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(the CUDA library is required; there is no CPU path)")
    L = C.CDLL(path)
    sig = {
        "gsp2_default_options": (None, [C.POINTER(Options)]),
        "gsp2_create": (C.c_int, [C.c_int64, _P, _P, C.c_int64, _P, C.c_int32, _P, _P, C.POINTER(Options),
                                  C.POINTER(_P)]),
        "gsp2_workspace_bytes": (C.c_int, [_P, C.POINTER(C.c_size_t)]),
        "gsp2_bind_workspace": (C.c_int, [_P, _P, C.c_size_t, _P]),
        "gsp2_p_pattern": (C.c_int, [_P, _P, _P, C.POINTER(C.c_int64)]),
        "gsp2_plan_query": (C.c_int, [_P, C.POINTER(PlanInfo), _P, _P]),
        "gsp2_density": (C.c_int, [_P, _P, _P, _P, C.c_int32, C.c_int32, _P]),
        "gsp2_sync_status": (C.c_int, [_P, C.POINTER(Report)]),
        "gsp2_history": (C.c_int, [_P, _P, _P, _P, C.c_int32]),
        "gsp2_step_times": (C.c_int, [_P, _P, C.c_int32]),
        "gsp2_backward": (C.c_int, [_P, _P, _P, _P]),
        "gsp2_autotune": (C.c_int, [_P, _P, _P, C.c_int32, _P, C.POINTER(TuneReport)]),
        "gsp2_density_reuse": (C.c_int, [_P, _P, _P, _P, C.POINTER(C.c_int32), _P, C.POINTER(C.c_int32)]),
        "gsp2_threshold_graph": (C.c_int, [_P, _P, C.c_double, _P, _P, _P, C.c_int64, C.POINTER(C.c_int64)]),
        "gsp2_create_shard": (C.c_int, [C.c_int64, _P, _P, C.c_int64, _P, C.c_int32, _P, _P, _P, C.c_int32,
                                        C.POINTER(Options), C.POINTER(_P)]),
        "gsp2_assign_parts": (C.c_int, [_P, C.c_int32, C.c_int32, _P, _P]),
        "gsp2_shard_info": (C.c_int, [_P, _P, _P, _P]),
        "gsp2_shard_exchanges": (C.c_int, [_P, C.c_int32, C.c_int32, C.POINTER(C.c_int32)]),
        "gsp2_shard_begin": (C.c_int, [_P, _P, _P, _P, C.c_int32, C.c_int32, _P, _P]),
        "gsp2_shard_decide": (C.c_int, [_P, C.c_int32, _P, C.c_int32, _P]),
        "gsp2_shard_step": (C.c_int, [_P, C.c_int32, _P, _P]),
        "gsp2_shard_end": (C.c_int, [_P, _P]),
        "gsp2_partition_cost": (C.c_int, [C.c_int64, _P, _P, _P, C.c_int32, C.POINTER(C.c_double), _P]),
        "gsp2_partition": (C.c_int, [C.c_int64, _P, _P, C.c_int32, C.c_int32, _P, _P, C.POINTER(C.c_int32),
                                     C.POINTER(C.c_double)]),
        "gsp2_last_error": (C.c_char_p, [_P]),
        "gsp2_destroy": (None, [_P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def default_options() -> Options:
    o = Options()
    load().gsp2_default_options(C.byref(o))
    return o


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_P) if a is not None else None


def _tptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


PARTITION_METHODS = {"auto": -1, "block": 0, "graph_order": 1, "rcb": 2}


def partition_cost(g_rowptr, g_colind, part, nparts):
    """Eq. 5 cost sum_i (c_i + h_i)^3 of a partition of G_tau, and the sizes c_i + h_i
    (gsp2_partition_cost)."""
    L = load()
    rp = np.ascontiguousarray(g_rowptr, np.int64)
    ci = np.ascontiguousarray(g_colind, np.int32)
    pa = np.ascontiguousarray(part, np.int32)
    sizes = np.empty(int(nparts), np.int32)
    cost = C.c_double()
    st = L.gsp2_partition_cost(rp.size - 1, _ptr(rp), _ptr(ci), _ptr(pa), int(nparts), C.byref(cost), _ptr(sizes))
    if st != OK:
        raise GSP2Error(st, "gsp2_partition_cost: bad graph or part ids")
    return cost.value, sizes


def partition(g_rowptr, g_colind, nparts, method="auto", coords=None):
    """A partition of G_tau into nparts parts (gsp2_partition): block (Section 2.3), block over a
    breadth-first graph order, or coordinate bisection (coords [n, 3]); "auto" keeps the one
    with the smallest Eq. 5 cost.  Returns (part int32[n], method name, cost)."""
    L = load()
    rp = np.ascontiguousarray(g_rowptr, np.int64)
    ci = np.ascontiguousarray(g_colind, np.int32)
    n = rp.size - 1
    xyz = None if coords is None else np.ascontiguousarray(coords, np.float64).reshape(n, 3)
    part = np.empty(n, np.int32)
    chosen = C.c_int32()
    cost = C.c_double()
    st = L.gsp2_partition(n, _ptr(rp), _ptr(ci), int(nparts), PARTITION_METHODS[method], _ptr(xyz), _ptr(part),
                          C.byref(chosen), C.byref(cost))
    if st != OK:
        raise GSP2Error(st, "gsp2_partition: bad graph, nparts or coordinates")
    names = {v: k for k, v in PARTITION_METHODS.items()}
    return part, names[chosen.value], cost.value


class GSP2:
    """A G-SP2 plan: pattern of H, partition and graph fixed; H values change per call."""

    def __init__(self, n, rowptr, colind, nocc, part, nparts, g_rowptr=None, g_colind=None,
                 device=None, bind=True, **options):
        L = load()
        self._lib = L
        self.n = int(n)
        self.nocc = int(nocc)
        self.nparts = int(nparts)
        o = default_options()
        for k, v in options.items():
            if k == "precision" and isinstance(v, str):
                v = PRECISIONS[v]
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        self.options = o
        self._keep = [np.ascontiguousarray(rowptr, np.int64), np.ascontiguousarray(colind, np.int32),
                      np.ascontiguousarray(part, np.int32)]
        grp = None if g_rowptr is None else np.ascontiguousarray(g_rowptr, np.int64)
        gci = None if g_colind is None else np.ascontiguousarray(g_colind, np.int32)
        h = _P()
        st = self._create(L, grp, gci, o, h)
        if st != OK:
            raise GSP2Error(st, L.gsp2_last_error(None).decode())
        self._h = h
        self.nnz_h = int(self._keep[0][-1])
        info = PlanInfo()
        self._check(L.gsp2_plan_query(h, C.byref(info), None, None))
        s = np.empty(info.nparts, np.int32)
        c = np.empty(info.nparts, np.int32)
        self._check(L.gsp2_plan_query(h, C.byref(info), _ptr(s), _ptr(c)))
        self.info = info
        self.part_sizes, self.part_cores = s, c
        nnz = C.c_int64()
        self._check(L.gsp2_p_pattern(h, None, None, C.byref(nnz)))
        self.nnz_p = nnz.value
        self.p_colptr = np.empty(self.n + 1, np.int64)
        self.p_rowind = np.empty(self.nnz_p, np.int32)
        self._check(L.gsp2_p_pattern(h, _ptr(self.p_colptr), _ptr(self.p_rowind), C.byref(nnz)))
        b = C.c_size_t()
        self._check(L.gsp2_workspace_bytes(h, C.byref(b)))
        self.workspace_bytes = b.value
        self.workspace = None
        # density calls made through this plan; gsp2_backward differentiates the last one,
        # so the autograd function checks that no other call came in between
        self.forward_count = 0
        if bind:
            self.bind(device)

    # -- plumbing
    def _create(self, L, grp, gci, o, h):
        return L.gsp2_create(self.n, _ptr(self._keep[0]), _ptr(self._keep[1]), self.nocc, _ptr(self._keep[2]),
                             self.nparts, _ptr(grp), _ptr(gci), C.byref(o), C.byref(h))

    def _check(self, st):
        if st != OK:
            raise GSP2Error(st, self._lib.gsp2_last_error(self._h).decode())

    def bind(self, device=None):
        import torch
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        with torch.cuda.device(dev):
            self.workspace = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device=dev)
            base = self.workspace.data_ptr()
            off = (-base) % 256
            self._check(self._lib.gsp2_bind_workspace(self._h, C.c_void_p(base + off), self.workspace_bytes,
                                                      _stream_ptr()))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gsp2_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- calls
    def density(self, h_vals, out=None, alpha=None, mode="record", nsteps=0, stream=None):
        """P values (torch float64, on the pattern p_colptr/p_rowind) for H values h_vals
        (torch float64 [nnz_h] on the plan's device).  `alpha` (int8 device tensor of
        max_steps) receives (record) or supplies (replay) the branch sequence."""
        import torch
        if h_vals.dtype != torch.float64 or not h_vals.is_cuda or h_vals.numel() != self.nnz_h:
            raise ValueError("h_vals must be a CUDA float64 tensor of nnz(H) values")
        h_vals = h_vals.contiguous()
        if out is None:
            out = torch.empty(self.nnz_p, dtype=torch.float64, device=h_vals.device)
        if alpha is not None and (alpha.dtype != torch.int8 or not alpha.is_cuda):
            raise ValueError("alpha must be a CUDA int8 tensor")
        self._check(self._lib.gsp2_density(self._h, _tptr(h_vals), _tptr(out), _tptr(alpha), MODES[mode],
                                           int(nsteps), _stream_ptr(stream)))
        self.forward_count += 1
        return out

    def autotune(self, h_vals, trials=3, stream=None):
        """Time every schedule candidate of the plan's precision on whole density calls and
        keep the fastest (gsp2_autotune); returns the candidates and their median times."""
        import torch
        if h_vals.dtype != torch.float64 or not h_vals.is_cuda or h_vals.numel() != self.nnz_h:
            raise ValueError("h_vals must be a CUDA float64 tensor of nnz(H) values")
        out = torch.empty(self.nnz_p, dtype=torch.float64, device=h_vals.device)
        r = TuneReport()
        self.forward_count += 1  # the candidates' density calls replace the last forward
        self._check(self._lib.gsp2_autotune(self._h, _tptr(h_vals.contiguous()), _tptr(out), int(trials),
                                            _stream_ptr(stream), C.byref(r)))
        self._refresh_info()
        cands = [dict(tc_schedule=r.tc_schedule[i], tile_order=r.tile_order[i], tile_shape=r.tile_shape[i],
                      split_k=r.split_k[i], tile_claim=r.tile_claim[i], ms=r.ms[i]) for i in range(r.ncand)]
        return dict(chosen=r.chosen, candidates=cands)

    def density_reuse(self, h_vals, alpha, nsteps, out=None, stream=None):
        """Density for the next H of an SCF/MD sequence (gsp2_density_reuse): replays the
        `nsteps` branches in `alpha` (int8 CUDA tensor of alpha_len) and records a new
        sequence when they give the wrong trace.  Returns (P, nsteps, recomputed, status)."""
        import torch
        if h_vals.dtype != torch.float64 or not h_vals.is_cuda or h_vals.numel() != self.nnz_h:
            raise ValueError("h_vals must be a CUDA float64 tensor of nnz(H) values")
        if alpha.dtype != torch.int8 or not alpha.is_cuda or alpha.numel() < self.alpha_len:
            raise ValueError("alpha must be a CUDA int8 tensor of alpha_len entries")
        if out is None:
            out = torch.empty(self.nnz_p, dtype=torch.float64, device=h_vals.device)
        n = C.c_int32(int(nsteps))
        rec = C.c_int32(0)
        self.forward_count += 1
        st = self._lib.gsp2_density_reuse(self._h, _tptr(h_vals.contiguous()), _tptr(out), _tptr(alpha), C.byref(n),
                                          _stream_ptr(stream), C.byref(rec))
        if st in (E_ARG, E_STATE, E_CUDA, E_TIMEOUT):
            self._check(st)
        return out, n.value, bool(rec.value), st

    def threshold_graph(self, p_vals, tau, stream=None):
        """G_tau from P (gsp2_threshold_graph): (g_rowptr int64[n+1], g_colind int32[nnz]),
        symmetric with the diagonal, ready for a new plan."""
        rp = np.empty(self.n + 1, np.int64)
        nnz = C.c_int64(0)
        self._check(self._lib.gsp2_threshold_graph(self._h, _tptr(p_vals), float(tau), _stream_ptr(stream), _ptr(rp),
                                                   None, 0, C.byref(nnz)))
        ci = np.empty(nnz.value, np.int32)
        self._check(self._lib.gsp2_threshold_graph(self._h, _tptr(p_vals), float(tau), _stream_ptr(stream), _ptr(rp),
                                                   _ptr(ci), nnz.value, C.byref(nnz)))
        return rp, ci

    def _refresh_info(self):
        info = PlanInfo()
        self._check(self._lib.gsp2_plan_query(self._h, C.byref(info), None, None))
        self.info = info
        self.options.tc_schedule = info.tc_schedule
        self.options.tile_order = info.tile_order
        self.options.tile_shape = info.tile_shape
        self.options.tile_claim = info.tile_claim

    def status(self):
        """(status code, report dict) of the last density call; waits for it."""
        r = Report()
        st = self._lib.gsp2_sync_status(self._h, C.byref(r))
        if st in (E_ARG, E_STATE, E_CUDA, E_TIMEOUT):
            self._check(st)
        return st, {f: getattr(r, f) for f, _ in Report._fields_}

    def history(self):
        m = self.options.max_steps + 9
        tr = np.zeros(m)
        e = np.zeros(m)
        a = np.zeros(m, np.int8)
        self._check(self._lib.gsp2_history(self._h, _ptr(tr), _ptr(e), _ptr(a), m))
        st, rep = self.status()
        k = rep["steps"]
        return dict(traces=tr[:k + 1], idem=e[:k], alphas=a[:k].astype(int).tolist(), report=rep, status=st)

    @property
    def alpha_len(self):
        """Length of the branch-sequence buffer a density call may fill (max_steps + 8)."""
        return self.options.max_steps + 8

    def step_times(self):
        """Per-step device milliseconds of the last density call (needs time_steps=1)."""
        ms = np.zeros(self.info.step_launches, np.float32)
        self._check(self._lib.gsp2_step_times(self._h, _ptr(ms), len(ms)))
        return ms

    def backward(self, p_bar, out=None, stream=None):
        import torch
        if p_bar.dtype != torch.float64 or not p_bar.is_cuda or p_bar.numel() != self.nnz_p:
            raise ValueError("p_bar must be a CUDA float64 tensor on the pattern of P")
        p_bar = p_bar.contiguous()
        if out is None:
            out = torch.empty(self.nnz_h, dtype=torch.float64, device=p_bar.device)
        self._check(self._lib.gsp2_backward(self._h, _tptr(p_bar), _tptr(out), _stream_ptr(stream)))
        return out

    # -- helpers for users
    def dense_p(self, p_vals):
        """Dense N x N numpy copy of P (small problems)."""
        P = np.zeros((self.n, self.n))
        cols = np.repeat(np.arange(self.n), np.diff(self.p_colptr))
        P[self.p_rowind, cols] = p_vals.detach().cpu().numpy() if hasattr(p_vals, "detach") else p_vals
        return P

    def flops_per_step(self):
        """dgemm-equivalent flops of one purification step, sum_k 2 s_k^3 (Eq. 5 cost)."""
        return 2.0 * self.info.sum_s3


def _make_function():
    import torch

    class GSP2Density(torch.autograd.Function):
        """P(H) through the library, with the hand-written adjoint as its backward."""

        @staticmethod
        def forward(ctx, h_vals, plan):
            ctx.plan = plan
            p = plan.density(h_vals)
            ctx.forward_id = plan.forward_count
            return p

        @staticmethod
        def backward(ctx, p_bar):
            # the library keeps the checkpoints and branch sequence of the plan's last density
            # call only: a later call on the same plan has replaced this forward's
            if ctx.plan.forward_count != ctx.forward_id:
                raise RuntimeError("gsp2_density: the plan ran another density call after this forward; its "
                                   "adjoint state is gone (use one plan per live forward)")
            return ctx.plan.backward(p_bar.contiguous()), None

    return GSP2Density


_fn = None


def gsp2_density(h_vals, plan: GSP2):
    global _fn
    if _fn is None:
        _fn = _make_function()
    return _fn.apply(h_vals, plan)
