"""Shard plans: the parts of one G-SP2 problem split over several GPUs, one process each.

Parts are independent except through the one branch every step takes for all of them,
chosen from the trace of the whole iterate (Section 2.1), in G-SP2 the sum of every
part's core diagonal (Section 2.2).  So each rank purifies its own parts and, once per
step, the ranks exchange 16 bytes each (their partial core traces of X and of X^2); the
library adds the gathered partials in rank order on the device, so that every rank takes
bitwise the same branch.  P's core columns are disjoint between ranks.

    sizes = part_sizes(n, rowptr, colind, nocc, part, nparts, g_rowptr, g_colind)
    part_rank, _ = assign_parts(sizes, world)          # LPT on the Eq. 5 cost s_k^3
    plan = ShardPlan(n, rowptr, colind, nocc, part, nparts, g_rowptr, g_colind, part_rank, rank)
    p_local = plan.density(h_vals, exchange=dist_exchange())   # P on this rank's columns
    p = plan.gather_p(p_local)                                 # all of P, on every rank

Argument marshalling and the collective only: the steps, the rank-order sum and the
branch decision run in the library's kernels (gsp2_shard_* in gsp2.h).  The gradient of
a shard plan (GSP2.backward) is this rank's share of dL/dH; the sum over ranks is dL/dH.
"""

from __future__ import annotations

import ctypes as C

import numpy as np

from .gsp2 import GSP2, MODES, OK, GSP2Error, _P, _ptr, _stream_ptr, _tptr, load


def part_sizes(n, rowptr, colind, nocc, part, nparts, g_rowptr=None, g_colind=None) -> np.ndarray:
    """Core + halo size s_k of every part (a host-only plan, no workspace)."""
    return GSP2(n, rowptr, colind, nocc, part, nparts, g_rowptr, g_colind, bind=False).part_sizes.copy()


def assign_parts(sizes, nranks: int):
    """Part -> rank by longest processing time first on s_k^3 (gsp2_assign_parts); the same
    on every rank for the same sizes.  Returns (part_rank int32[nparts], cost per rank)."""
    L = load()
    s = np.ascontiguousarray(sizes, np.int32)
    pr = np.empty(s.size, np.int32)
    cost = np.empty(int(nranks), np.float64)
    st = L.gsp2_assign_parts(_ptr(s), int(s.size), int(nranks), _ptr(pr), _ptr(cost))
    if st != OK:
        raise GSP2Error(st, "gsp2_assign_parts: need 1 <= nranks <= nparts and sizes >= 1")
    return pr, cost


def merge_patterns(colptrs, rowinds):
    """The pattern of the whole P from the shards' patterns (each a core-column CSC over all
    n columns, empty where another shard owns the column), and for each shard the positions
    of its values in it.  Every column must belong to exactly one shard."""
    cnts = [np.diff(np.asarray(cp, np.int64)) for cp in colptrs]
    owners = sum((c > 0).astype(np.int64) for c in cnts)
    if np.any(owners != 1):
        raise ValueError("the shards' columns must cover every column exactly once")
    counts = sum(cnts)
    colptr = np.zeros(counts.size + 1, np.int64)
    np.cumsum(counts, out=colptr[1:])
    rowind = np.empty(int(colptr[-1]), np.int32)
    positions = []
    for cp, ri, c in zip(colptrs, rowinds, cnts):
        cp = np.asarray(cp, np.int64)
        pos = np.arange(int(cp[-1]), dtype=np.int64) + np.repeat(colptr[:-1] - cp[:-1], c)
        rowind[pos] = ri
        positions.append(pos)
    return colptr, rowind, positions


def dist_exchange(group=None):
    """The exchange of a multi-process run: all-gather of every rank's 16-byte partial into
    a [world, 2] tensor in rank order (torch.distributed; NCCL for CUDA tensors, gloo for
    CPU tensors), queued on the current stream."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    buf = {}

    def exchange(send):
        recv = buf.get(send.device)
        if recv is None:
            recv = buf[send.device] = torch.empty((world, 2), dtype=send.dtype, device=send.device)
        dist.all_gather(list(recv.unbind(0)), send, group=group)
        return recv

    return exchange


class ShardPlan(GSP2):
    """The parts `part_rank` gives to `rank`, with the steps' branch taken from the partial
    traces of all ranks (gsp2_create_shard)."""

    def __init__(self, n, rowptr, colind, nocc, part, nparts, g_rowptr, g_colind, part_rank, rank, device=None,
                 bind=True, **options):
        self.part_rank = np.ascontiguousarray(part_rank, np.int32)
        self.rank = int(rank)
        self.nranks = int(self.part_rank.max()) + 1
        super().__init__(n, rowptr, colind, nocc, part, nparts, g_rowptr, g_colind, device=device, bind=bind,
                         **options)
        ids = np.empty(self.info.nparts, np.int32)
        self._check(self._lib.gsp2_shard_info(self._h, None, None, _ptr(ids)))
        self.part_ids = ids  # global id of each local part

    def _create(self, L, grp, gci, o, h):
        return L.gsp2_create_shard(self.n, _ptr(self._keep[0]), _ptr(self._keep[1]), self.nocc, _ptr(self._keep[2]),
                                   self.nparts, _ptr(grp), _ptr(gci), _ptr(self.part_rank), self.rank, C.byref(o),
                                   C.byref(h))

    # -- the exchange sequence, one call each (several shard plans can be driven in lockstep
    #    from one thread with these)
    def exchanges(self, mode="record", nsteps=0) -> int:
        n = C.c_int32()
        self._check(self._lib.gsp2_shard_exchanges(self._h, MODES[mode], int(nsteps), C.byref(n)))
        return n.value

    def begin(self, h_vals, out, send, alpha=None, mode="record", nsteps=0, stream=None):
        import torch
        if h_vals.dtype != torch.float64 or not h_vals.is_cuda or h_vals.numel() != self.nnz_h:
            raise ValueError("h_vals must be a CUDA float64 tensor of nnz(H) values")
        if out.dtype != torch.float64 or out.numel() != self.nnz_p:
            raise ValueError("out must be a float64 tensor of nnz_p values")
        self._call_args = (h_vals, out, alpha, send)  # kept alive until end()
        self._check(self._lib.gsp2_shard_begin(self._h, _tptr(h_vals), _tptr(out), _tptr(alpha), MODES[mode],
                                               int(nsteps), _tptr(send), _stream_ptr(stream)))

    def decide(self, x, recv, stream=None):
        import torch
        if recv.dtype != torch.float64 or recv.dim() != 2 or recv.shape[1] != 2 or not recv.is_contiguous():
            raise ValueError("recv must be a contiguous float64 tensor [nranks, 2]")
        self._check(self._lib.gsp2_shard_decide(self._h, int(x), _tptr(recv), int(recv.shape[0]),
                                                _stream_ptr(stream)))

    def step(self, x, send, stream=None):
        self._check(self._lib.gsp2_shard_step(self._h, int(x), _tptr(send), _stream_ptr(stream)))

    def end(self, stream=None):
        self._check(self._lib.gsp2_shard_end(self._h, _stream_ptr(stream)))
        self._call_args = None
        self.forward_count += 1

    def density(self, h_vals, exchange, out=None, alpha=None, mode="record", nsteps=0, stream=None):
        """P on this rank's columns (the pattern p_colptr/p_rowind).  `exchange(send)` takes
        this rank's partial (float64 [2] on the device) and returns every rank's, [nranks, 2]
        in rank order, queued on the current stream (dist_exchange() under torch.distributed)."""
        import torch
        if out is None:
            out = torch.empty(self.nnz_p, dtype=torch.float64, device=h_vals.device)
        send = torch.empty(2, dtype=torch.float64, device=h_vals.device)
        count = self.exchanges(mode, nsteps)
        self.begin(h_vals, out, send, alpha, mode, nsteps, stream)
        for x in range(count):
            recv = exchange(send)
            self.decide(x, recv.contiguous(), stream)
            if x + 1 < count:
                self.step(x + 1, send, stream)
        self.end(stream)
        return out

    def gather_p(self, p_local, group=None):
        """All of P (on the merged pattern, self.full_colptr / self.full_rowind) on every rank,
        from each rank's values (torch.distributed all-gathers)."""
        import torch
        import torch.distributed as dist
        world = dist.get_world_size(group)
        if getattr(self, "_merged", None) is None:
            pats = [None] * world
            dist.all_gather_object(pats, (self.p_colptr, self.p_rowind), group=group)
            cp, ri, pos = merge_patterns([p[0] for p in pats], [p[1] for p in pats])
            self.full_colptr, self.full_rowind = cp, ri
            self._merged = [torch.from_numpy(q).to(p_local.device) for q in pos]
        sizes = [int(q.numel()) for q in self._merged]
        buf = torch.zeros((world, max(sizes)), dtype=p_local.dtype, device=p_local.device)
        mine = torch.zeros(max(sizes), dtype=p_local.dtype, device=p_local.device)
        mine[:p_local.numel()] = p_local
        dist.all_gather(list(buf.unbind(0)), mine, group=group)
        p = torch.empty(int(self.full_colptr[-1]), dtype=p_local.dtype, device=p_local.device)
        for r in range(world):
            p[self._merged[r]] = buf[r, :sizes[r]]
        return p
