"""Seeded gapped tight-binding Hamiltonians, partitions and dependency graphs.

The paper's own test systems (water, a solvated protein, polyalanine 289, urea;
Sections 3.1-3.2) are not available, so every workload here is synthetic:

* sites uniform in a non-periodic cube at 0.1 sites per cubic Angstrom;
* four orbitals per site, two low (onsite -8 eV + U[-0.5, 0.5]) and two high
  (onsite +2 eV + U[-0.5, 0.5]); filling the low band (Nocc = 2 per site) gives
  an insulator with a gap of several eV;
* hopping between sites closer than 6 Angstrom:
  H_ab = -exp(-r / 1.5 Angstrom) * B_ab with B_ab = (R + R^T)/2, R ~ U[-1, 1]^{4x4},
  H_ba = H_ab^T; intra-site off-diagonal elements are zero;
* recursive coordinate bisection of the sites into parts (all four orbitals of a
  site share a part), standing in for the METIS partitions of Section 2.2; median splits
  give equal cores, weighted splits uneven ones (the spread of subproblem sizes Fig. 3
  shows);
* the dependency graph G_tau (Section 2.2) is built from locality: orbitals are
  adjacent when their sites are closer than a radius R_g, the localisation-radius
  construction mentioned at the end of Section 2.2.  R_g is chosen per workload so
  that core+halo sizes span the ranges the workloads call for.

Everything is drawn from numpy's Philox generator with fixed seeds, so a workload
is identical on every machine.  No part of the density-matrix method is computed
here.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

ORBS_PER_SITE = 4


@dataclass
class TBSystem:
    """A tight-binding Hamiltonian (full symmetric CSR) plus partition and graph."""

    name: str
    n_sites: int
    n: int
    nocc: int
    rowptr: np.ndarray  # int64 [n+1]
    colind: np.ndarray  # int32 [nnz], ascending within each row
    vals: np.ndarray  # float64 [nnz]
    coords: np.ndarray  # float64 [n_sites, 3] (Angstrom)
    part: np.ndarray  # int32 [n], orbital -> part id
    nparts: int
    g_rowptr: np.ndarray  # int64 [n+1], dependency graph G_tau (no self loops)
    g_colind: np.ndarray  # int32
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


def _pairs_within(coords: np.ndarray, radius: float) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """All site pairs a < b with distance < radius, lexicographically sorted.

    A cell list keeps this O(n); distances are recomputed here so the cut is decided
    by one fixed formula on every machine.
    """
    n = coords.shape[0]
    if n < 2:
        e = np.zeros(0, np.int64)
        return e, e, np.zeros(0)
    lo = coords.min(axis=0)
    cell = np.floor((coords - lo) / radius).astype(np.int64)
    dims = cell.max(axis=0) + 1
    key = (cell[:, 0] * dims[1] + cell[:, 1]) * dims[2] + cell[:, 2]
    order = np.argsort(key, kind="stable")
    skey = key[order]
    starts = np.searchsorted(skey, np.arange(dims.prod() + 1), side="left")
    out_a, out_b = [], []
    offsets = [(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)]
    for dx, dy, dz in offsets:
        nc = cell + np.array([dx, dy, dz])
        ok = np.all((nc >= 0) & (nc < dims), axis=1)
        idx_a = np.nonzero(ok)[0]
        nkey = (nc[idx_a, 0] * dims[1] + nc[idx_a, 1]) * dims[2] + nc[idx_a, 2]
        s = starts[nkey]
        e = starts[nkey + 1]
        cnt = e - s
        if cnt.sum() == 0:
            continue
        rep_a = np.repeat(idx_a, cnt)
        base = np.repeat(s - np.concatenate(([0], np.cumsum(cnt)[:-1])), cnt)
        pos = np.arange(cnt.sum()) + base
        b = order[pos]
        m = rep_a < b
        out_a.append(rep_a[m])
        out_b.append(b[m])
    a = np.concatenate(out_a)
    b = np.concatenate(out_b)
    d = coords[a] - coords[b]
    r = np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2])
    m = r < radius
    a, b, r = a[m], b[m], r[m]
    o = np.lexsort((b, a))
    return a[o], b[o], r[o]


def _csr_from_coo(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray | None):
    o = np.lexsort((cols, rows))
    rows = rows[o]
    cols = cols[o].astype(np.int32)
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return rowptr, cols, (None if vals is None else vals[o].astype(np.float64))


def make_hamiltonian(n_sites: int, seed: int = 1234, density: float = 0.1,
                     cutoff: float = 6.0, decay: float = 1.5):
    """Coordinates and the full symmetric CSR Hamiltonian of the generator above."""
    rng = np.random.Generator(np.random.Philox(seed))
    side = (n_sites / density) ** (1.0 / 3.0)
    coords = rng.uniform(0.0, side, size=(n_sites, 3))
    onsite = np.empty((n_sites, ORBS_PER_SITE))
    onsite[:, :2] = -8.0 + rng.uniform(-0.5, 0.5, size=(n_sites, 2))
    onsite[:, 2:] = 2.0 + rng.uniform(-0.5, 0.5, size=(n_sites, 2))
    a, b, r = _pairs_within(coords, cutoff)
    npair = a.shape[0]
    R = rng.uniform(-1.0, 1.0, size=(npair, ORBS_PER_SITE, ORBS_PER_SITE))
    blocks = -np.exp(-r / decay)[:, None, None] * 0.5 * (R + R.transpose(0, 2, 1))
    p = np.arange(ORBS_PER_SITE)
    # off-diagonal blocks (a, b) and their transposes (b, a)
    ra = (ORBS_PER_SITE * a[:, None, None] + p[None, :, None]) + 0 * p[None, None, :]
    cb = (ORBS_PER_SITE * b[:, None, None] + p[None, None, :]) + 0 * p[None, :, None]
    rows = np.concatenate([ra.ravel(), cb.ravel(), np.arange(n_sites * ORBS_PER_SITE)])
    cols = np.concatenate([cb.ravel(), ra.ravel(), np.arange(n_sites * ORBS_PER_SITE)])
    vals = np.concatenate([blocks.ravel(), blocks.ravel(), onsite.ravel()])
    n = n_sites * ORBS_PER_SITE
    rowptr, colind, v = _csr_from_coo(n, rows.astype(np.int64), cols.astype(np.int64), vals)
    return coords, rowptr, colind, v


def rcb_partition(coords: np.ndarray, nparts: int, weights: np.ndarray | None = None) -> np.ndarray:
    """Recursive coordinate bisection of sites: split along the longest extent at the
    (count-proportional) median, ties broken by site index.  With `weights` (one positive
    number per part) each split gives the two sides sites in proportion to the summed
    weights of their parts, so part k gets about weights[k] / sum(weights) of the sites
    (uneven cores).  Returns site -> part."""
    n_sites = coords.shape[0]
    if nparts < 1 or nparts > n_sites:
        raise ValueError("nparts must be in [1, n_sites]")
    wcum = None
    if weights is not None:
        w = np.asarray(weights, np.float64)
        if w.shape != (nparts,) or np.any(~(w > 0)):
            raise ValueError("weights must be nparts positive numbers")
        wcum = np.concatenate([[0.0], np.cumsum(w)])
    site_part = np.empty(n_sites, np.int32)
    stack = [(np.arange(n_sites), 0, nparts)]
    while stack:
        idx, p0, npp = stack.pop()
        if npp == 1:
            site_part[idx] = p0
            continue
        pts = coords[idx]
        ext = pts.max(axis=0) - pts.min(axis=0)
        ax = int(np.argmax(ext))
        order = np.lexsort((idx, pts[:, ax]))
        nl = npp // 2
        frac = nl / npp if wcum is None else (wcum[p0 + nl] - wcum[p0]) / (wcum[p0 + npp] - wcum[p0])
        nleft = int(round(len(idx) * frac))
        nleft = min(max(nleft, nl), len(idx) - (npp - nl))
        stack.append((idx[order[nleft:]], p0 + nl, npp - nl))
        stack.append((idx[order[:nleft]], p0, nl))
    return site_part


def block_partition(n: int, nparts: int) -> np.ndarray:
    """Block partitioning of Section 2.3: consecutive indices, sizes differing by at most
    one (the larger parts first).  Returns vertex -> part."""
    if nparts < 1 or nparts > n:
        raise ValueError("nparts must be in [1, n]")
    base, extra = divmod(n, nparts)
    sizes = np.full(nparts, base, np.int64)
    sizes[:extra] += 1
    return np.repeat(np.arange(nparts, dtype=np.int32), sizes)


def locality_graph(coords: np.ndarray, radius: float):
    """Orbital adjacency: u ~ v (u != v) when their sites are closer than `radius`
    (orbitals of one site are always adjacent).  Returns CSR (rowptr, colind)."""
    n_sites = coords.shape[0]
    a, b, _ = _pairs_within(coords, radius)
    p = np.arange(ORBS_PER_SITE)
    sa = np.concatenate([a, b, np.arange(n_sites)])
    sb = np.concatenate([b, a, np.arange(n_sites)])
    rows = (ORBS_PER_SITE * sa[:, None, None] + p[None, :, None] + 0 * p[None, None, :]).ravel()
    cols = (ORBS_PER_SITE * sb[:, None, None] + p[None, None, :] + 0 * p[None, :, None]).ravel()
    keep = rows != cols
    n = n_sites * ORBS_PER_SITE
    rowptr, colind, _ = _csr_from_coo(n, rows[keep].astype(np.int64), cols[keep].astype(np.int64), None)
    return rowptr, colind


def graph_from_dense_threshold(M: np.ndarray, tau: float):
    """G_tau of Section 2.2 from a dense symmetric matrix: u ~ v iff |M_uv| > tau, u != v."""
    A = np.abs(M) > tau
    A = A | A.T
    np.fill_diagonal(A, False)
    rows, cols = np.nonzero(A)
    return _csr_from_coo(M.shape[0], rows.astype(np.int64), cols.astype(np.int64), None)[:2]


def dense_from_csr(n: int, rowptr, colind, vals) -> np.ndarray:
    M = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    M[rows, colind] = vals
    return M


def csr_from_dense(M: np.ndarray, keep_diagonal: bool = True):
    A = M != 0
    if keep_diagonal:
        np.fill_diagonal(A, True)
    rows, cols = np.nonzero(A)
    rowptr, colind, _ = _csr_from_coo(M.shape[0], rows.astype(np.int64), cols.astype(np.int64), None)
    rows2 = np.repeat(np.arange(M.shape[0]), np.diff(rowptr))
    return rowptr, colind, M[rows2, colind].astype(np.float64)


def random_symmetric_on_pattern(rowptr, colind, seed: int = 5678) -> np.ndarray:
    """Seeded symmetric Gaussian values on a symmetric CSR pattern (A_ij = A_ji)."""
    n = rowptr.shape[0] - 1
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    cols = colind.astype(np.int64)
    keys = rows * n + cols
    upper = rows <= cols
    rng = np.random.Generator(np.random.Philox(seed))
    out = np.empty(keys.shape[0])
    out[upper] = rng.standard_normal(int(upper.sum()))
    lo = np.nonzero(~upper)[0]
    tpos = np.searchsorted(keys, cols[lo] * n + rows[lo])
    if np.any(keys[tpos] != cols[lo] * n + rows[lo]):
        raise ValueError("pattern is not symmetric")
    out[lo] = out[tpos]
    return out


# Workloads: (n_sites, nparts, graph radius in Angstrom).  The radius is set so that the
# core+halo sizes fall in the range each workload calls for.
WORKLOADS = {
    # 512 orbitals, 8 parts, sizes ~100-250: the case the oracle runs in seconds
    "tb512": dict(n_sites=128, nparts=8, graph_radius=3.5),
    # 30,000 orbitals, 256 uneven parts, sizes ~300-1,200
    "tb30k": dict(n_sites=7500, nparts=256, graph_radius=5.0),
    # 4,096 orbitals, 32 parts, sizes ~200-500 (adjoint workload)
    "tb4k": dict(n_sites=1024, nparts=32, graph_radius=3.0),
    # 8,000 orbitals, 64 parts, the part sizes of tb30k on a quarter of the volume (arenas
    # still larger than L2): the case kernel profiles are taken on
    "tb8k": dict(n_sites=2000, nparts=64, graph_radius=5.0),
    # dense molecular crystal (the paper's urea case stands behind it): sites twice as dense,
    # so each core carries a halo about twice as large; 8,000 orbitals, 64 parts
    "crystal8k": dict(n_sites=2000, nparts=64, graph_radius=5.0, density=0.2),
    # the same at 512 orbitals, for the oracle
    "crystal512": dict(n_sites=128, nparts=8, graph_radius=3.5, density=0.2),
    # 120,000 orbitals, 1,024 parts of uneven cores (weights 4 + 76 u^2, u ~ U[0, 1]), sizes
    # ~200-2,000 (152-1,960; 1st percentile 197)
    "tb120k": dict(n_sites=30000, nparts=1024, graph_radius=5.0, core_weights=(4321, 4.0, 76.0)),
}


def core_weights(nparts: int, seed: int, lo: float, span: float) -> np.ndarray:
    """Seeded part weights lo + span u^2, u ~ U[0, 1] (Philox): many small cores and a tail of
    large ones, for the uneven-size workloads."""
    rng = np.random.Generator(np.random.Philox(seed))
    return lo + span * rng.uniform(0.0, 1.0, nparts) ** 2


def make_tb_system(n_sites: int, nparts: int, graph_radius: float, seed: int = 1234,
                   name: str = "custom", density: float = 0.1, weights: np.ndarray | None = None) -> TBSystem:
    coords, rowptr, colind, vals = make_hamiltonian(n_sites, seed=seed, density=density)
    site_part = rcb_partition(coords, nparts, weights)
    part = np.repeat(site_part, ORBS_PER_SITE).astype(np.int32)
    g_rowptr, g_colind = locality_graph(coords, graph_radius)
    n = n_sites * ORBS_PER_SITE
    return TBSystem(name=name, n_sites=n_sites, n=n, nocc=2 * n_sites, rowptr=rowptr,
                    colind=colind, vals=vals, coords=coords, part=part, nparts=nparts,
                    g_rowptr=g_rowptr, g_colind=g_colind,
                    meta=dict(seed=seed, graph_radius=graph_radius, density=density,
                              uneven=weights is not None))


def make_workload(name: str, seed: int = 1234) -> TBSystem:
    w = WORKLOADS[name]
    cw = w.get("core_weights")
    weights = None if cw is None else core_weights(w["nparts"], *cw)
    return make_tb_system(w["n_sites"], w["nparts"], w["graph_radius"], seed=seed, name=name,
                          density=w.get("density", 0.1), weights=weights)
