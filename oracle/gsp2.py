"""Plain FP64 CPU oracle for SP2 and graph-partitioned SP2 (G-SP2).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the library.  It shares no code with the CUDA
path.  Everything is float64 and written in the order the paper states the method,
with numpy/scipy library calls (matmul, eigh, sparse slicing) as single steps:

* Gershgorin bounds of H                       -- Section 2.1 (text after Eq. 1)
* X0 = (eps_max I - H) / (eps_max - eps_min)     -- Eq. 1
* X_i = [I + alpha_i (I - X_{i-1})] X_{i-1}      -- Eq. 2
* alpha_i = +1 iff 2 Tr[X] <= N_el, else -1     -- Section 2.1 (text after Eq. 2)
* P = lim X_i, checked by idempotency           -- Eq. 3 and the text after it
* core and halo vertices, s_i = c_i + h_i        -- Section 2.2
* CH-partitioning cost sum (c_i + h_i)^3         -- Eq. 5
* G-SP2: every part purified with one global alpha sequence from the summed core
  traces, core columns assembled into P         -- Section 1.1 (Fig. 1), Section 2.2

Readings where the paper is silent or garbled (each also listed in the design notes):

* the branch test uses the trace of the iterate the step is applied to, X_{i-1}
  (the paper's index reads "X_i", the output of the same step);
* closed shell: N_el = 2 Nocc, so the test is Tr[X_{i-1}] <= Nocc, and a tie takes
  alpha = +1 ("<=");
* spectral bounds are global (Gershgorin over every row of the full H), so every part
  is mapped by the same affine map and purified by the same polynomial;
* halo = one hop in G_tau from any core vertex; S_k lists the cores in ascending
  global order, then the halo in ascending global order;
* P is assembled from core columns only: P[S_k, j] = X_k[:, j] for core j of part k.
  It is not symmetrised;
* in G-SP2 the trace for the branch is the sum over parts of the core diagonal
  entries of each part's iterate (part order, then core order);
* stopping (the paper asks for idempotency "within given error bounds" after Eq. 3):
  with e_i = Tr[X_i] - Tr[X_i^2] (core entries only in G-SP2), step i computes
  e_{i-1} alongside X_i, and the iteration stops after step i when i >= 2,
  |e_{i-1}| <= idem_tol and either e_{i-1} < 0 or e_{i-1} >= e_{i-2}.  In exact
  arithmetic e >= 0 (the spectrum of X0 lies in [0, 1], which both maps keep) and, once
  every eigenvalue is close to 0 or 1, e falls at every step; so a small e that is
  negative or no longer falls marks the point where only rounding (or, in G-SP2, the
  drift caused by a core trace that cannot reach Nocc exactly) is left.  Continuing
  past that point is harmful: 0 is an unstable fixed point of 2x - x^2 and 1 of x^2,
  so each further step doubles such errors.  max_steps caps the count.  A replayed
  alpha sequence runs exactly its length.
* optional tail (not in the paper): after the stopping test, `tail_steps` more steps
  whose first branch follows the trace rule and each further one the opposite.  A pair
  X^2, 2X - X^2 (either order) maps 1 - d to 1 - O(d^2) and d to O(d^2), so the pair
  purifies the eigenvalues the trace rule leaves drifting when the G-SP2 core trace
  cannot reach Nocc.

The adjoint functions (reverse mode through the recorded alpha sequence, the
Daleckii-Krein form and the finite-difference probe) differentiate
L = sum_ij Pbar_ij P_ij with the spectral bounds and the alpha sequence held fixed.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


# --------------------------------------------------------------------------------------
# Section 2.1: spectral bounds, initial guess, purification step, branch rule
# --------------------------------------------------------------------------------------

def gershgorin_bounds(n, rowptr, colind, vals):
    """(eps_min, eps_max) from the Gershgorin circle theorem over every row of H
    (Section 2.1): eps_min = min_i (H_ii - R_i), eps_max = max_i (H_ii + R_i), with
    R_i = sum_{j != i} |H_ij|."""
    rowptr = np.asarray(rowptr)
    colind = np.asarray(colind)
    vals = np.asarray(vals, dtype=np.float64)
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    on_diag = rows == colind
    centre = np.zeros(n)
    centre[rows[on_diag]] = vals[on_diag]
    radius = np.zeros(n)
    np.add.at(radius, rows[~on_diag], np.abs(vals[~on_diag]))
    return float(np.min(centre - radius)), float(np.max(centre + radius))


def initial_guess(H, eps_min, eps_max):
    """Eq. 1: X0 = (eps_max I - H) / (eps_max - eps_min) for a dense symmetric H."""
    s = H.shape[0]
    return (eps_max * np.eye(s) - H) / (eps_max - eps_min)


def sp2_step(X, alpha):
    """Eq. 2: X_i = [I + alpha (I - X)] X.  Expanded, alpha = +1 gives 2X - X^2 and
    alpha = -1 gives X^2; the two cases are written out so each is one matmul."""
    X2 = X @ X
    if alpha == 1:
        return 2.0 * X - X2
    if alpha == -1:
        return X2
    raise ValueError("alpha must be +1 or -1")


def branch_alpha(trace, nocc):
    """Branch rule of Section 2.1: alpha = +1 iff 2 Tr[X] <= N_el (N_el = 2 Nocc for a
    closed shell), else -1.  The trace is that of the iterate the step acts on."""
    return 1 if 2.0 * trace <= 2.0 * nocc else -1


# --------------------------------------------------------------------------------------
# Plain (global, dense) SP2: Section 2.1, Eqs. 1-3
# --------------------------------------------------------------------------------------

def stop_now(idem, i, idem_tol):
    """Stopping test after step i (see the module notes): i >= 2, |e_{i-1}| <= idem_tol
    and (e_{i-1} < 0 or e_{i-1} >= e_{i-2}).  `idem` holds e_0 .. e_{i-1}."""
    e = idem[i - 1]
    return i >= 2 and abs(e) <= idem_tol and (e < 0 or e >= idem[i - 2])


def tail_alpha(t, trace, prev_alpha, nocc):
    """Branch of the t-th purification step after the stopping test (t = 0, 1, ...):
    the first follows the trace rule, each further one is the opposite of the previous,
    so that eigenvalues near 0 and near 1 are both purified (see the module notes)."""
    return branch_alpha(trace, nocc) if t == 0 else -prev_alpha


def sp2_dense(H, nocc, max_steps=45, bounds=None, alphas=None, keep_iterates=False,
              idem_tol=1e-3, tail_steps=0):
    """Plain SP2 on a dense symmetric H.  Returns (X_final, record) where record holds
    the alpha sequence, the traces T_0..T_n of the iterates and the idempotency
    errors e_i = Tr[X_i] - Tr[X_i^2] (Eq. 3's convergence check).  `tail_steps`
    alternating steps follow the stopping test (not with a replayed sequence)."""
    H = np.asarray(H, dtype=np.float64)
    n = H.shape[0]
    if bounds is None:
        # Gershgorin discs of the dense rows (Section 2.1)
        centre = np.diag(H)
        radius = np.sum(np.abs(H), axis=1) - np.abs(centre)
        bounds = (float(np.min(centre - radius)), float(np.max(centre + radius)))
    eps_min, eps_max = bounds
    X = initial_guess(H, eps_min, eps_max)
    rec = dict(alphas=[], traces=[float(np.trace(X))], idem=[], bounds=(eps_min, eps_max))
    its = [X] if keep_iterates else None
    nsteps = max_steps if alphas is None else len(alphas)
    tail = 0 if alphas is not None else tail_steps
    t = -1  # index of the current tail step, -1 before the stopping test
    i = 0
    while True:
        i += 1
        if t >= 0:
            a = tail_alpha(t, rec["traces"][-1], rec["alphas"][-1], nocc)
        else:
            a = branch_alpha(rec["traces"][-1], nocc) if alphas is None else int(alphas[i - 1])
        rec["idem"].append(float(np.trace(X) - np.trace(X @ X)))
        X = sp2_step(X, a)
        rec["alphas"].append(a)
        rec["traces"].append(float(np.trace(X)))
        if keep_iterates:
            its.append(X)
        if t >= 0:
            t += 1
            if t == tail:
                break
        elif (alphas is None and stop_now(rec["idem"], i, idem_tol)) or i == nsteps:
            if tail == 0:
                break
            t = 0
    if keep_iterates:
        rec["iterates"] = its
    return X, rec


# --------------------------------------------------------------------------------------
# Section 2.2: core and halo vertices, Eq. 5
# --------------------------------------------------------------------------------------

def core_halo(g_rowptr, g_colind, part, nparts, which=None):
    """Per part k: (core_k, halo_k).  core_k = vertices with part == k, ascending;
    halo_k = vertices outside part k adjacent in G_tau to some core vertex, ascending
    (Section 2.2).  The subproblem's vertex list is S_k = core_k followed by halo_k.
    `which` lists the parts to build (default all, in order)."""
    part = np.asarray(part)
    g_colind = np.asarray(g_colind)
    out = []
    for k in (range(nparts) if which is None else which):
        core = np.nonzero(part == k)[0]
        if core.size == 0:
            raise ValueError(f"part {k} is empty")
        # every neighbour of every core vertex, once (np.unique sorts them)
        nbrs = np.unique(np.concatenate([g_colind[g_rowptr[u]:g_rowptr[u + 1]] for u in core]))
        halo = nbrs[part[nbrs] != k].astype(np.int64)
        out.append((core.astype(np.int64), halo))
    return out


def ch_cost(sizes):
    """Eq. 5: C = sum_i (c_i + h_i)^3, given the subproblem sizes s_i = c_i + h_i."""
    return int(sum(int(s) ** 3 for s in sizes))


# --------------------------------------------------------------------------------------
# G-SP2
# --------------------------------------------------------------------------------------

@dataclass
class GSP2Result:
    n: int
    S: list  # per part: int64 vertex list, cores first
    ncore: list  # per part: c_k
    X: list  # per part: final dense iterate X_k (s_k x s_k)
    alphas: list
    traces: list  # T_0..T_n, global core traces
    idem: list  # e_0..e_{n-1}: T_i - Tr_core[X_i^2], e_{i-1} computed during step i
    bounds: tuple
    iterates: list = field(default=None)  # per part, list of X_k^(0..n) (optional)

    def dense_p(self):
        """P as a dense N x N array: P[S_k, core_j] = X_k[:, j] (core columns)."""
        P = np.zeros((self.n, self.n))
        for S, c, X in zip(self.S, self.ncore, self.X):
            P[np.ix_(S, S[:c])] = X[:, :c]
        return P

    def p_on_pattern(self, colptr, rowind):
        """P values in the core-column CSC layout given by (colptr, rowind): column g = S_k[j]
        (core j of part k) at stored row r holds X_k[t, j], t the position of r in S_k."""
        vals = np.empty(int(colptr[-1]))
        rowind = np.asarray(rowind)
        loc = np.full(self.n, -1, np.int64)  # global vertex -> position in the current S_k
        for S, c, X in zip(self.S, self.ncore, self.X):
            loc[S] = np.arange(len(S))
            for j in range(c):
                g = int(S[j])
                t = loc[rowind[colptr[g]:colptr[g + 1]]]
                if np.any(t < 0):
                    raise ValueError(f"column {g}: a stored row lies outside S_k")
                vals[colptr[g]:colptr[g + 1]] = X[t, j]
            loc[S] = -1
        return vals


def _h_sparse(n, rowptr, colind, vals):
    return sp.csr_matrix((np.asarray(vals, np.float64), np.asarray(colind), np.asarray(rowptr)),
                         shape=(n, n))


def gsp2(n, rowptr, colind, vals, nocc, part, nparts, g_rowptr=None, g_colind=None,
         max_steps=45, alphas=None, bounds=None, keep_iterates=False, idem_tol=1e-3, tail_steps=0):
    """Graph-partitioned SP2 (Section 1.1, Fig. 1; Section 2.2).

    Each part k gets the dense submatrix H[S_k, S_k], is mapped by Eq. 1 with the
    global Gershgorin bounds, and is purified by Eq. 2.  Every step takes one alpha
    for all parts, from the global trace T = sum_k sum_{j core} X_k[j, j] of the
    iterates the step acts on.  Passing `alphas` replays a recorded sequence
    (Section 2.1's reuse of the multiplication sequence) for exactly its length;
    otherwise the stopping test of the module notes ends the loop, followed by
    `tail_steps` alternating steps.  Without a graph, the pattern of H is used as G_tau."""
    if g_rowptr is None:
        g_rowptr, g_colind = rowptr, colind
    if bounds is None:
        bounds = gershgorin_bounds(n, rowptr, colind, vals)
    eps_min, eps_max = bounds
    Hs = _h_sparse(n, rowptr, colind, vals)
    parts = core_halo(g_rowptr, g_colind, part, nparts)
    S = [np.concatenate([c, h]) for c, h in parts]
    ncore = [len(c) for c, _ in parts]
    X = [initial_guess(Hs[Sk][:, Sk].toarray(), eps_min, eps_max) for Sk in S]
    its = [[x] for x in X] if keep_iterates else None

    def core_trace(mats):
        return float(sum(float(np.sum(np.diag(m)[:c])) for m, c in zip(mats, ncore)))

    def core_trace_sq(mats):
        return float(sum(float(np.sum(np.einsum("ij,ji->i", m[:c, :], m[:, :c])))
                         for m, c in zip(mats, ncore)))

    traces = [core_trace(X)]
    idem, used = [], []
    nsteps = max_steps if alphas is None else len(alphas)
    tail = 0 if alphas is not None else tail_steps
    t = -1  # index of the current tail step, -1 before the stopping test
    i = 0
    while True:
        i += 1
        if t >= 0:
            a = tail_alpha(t, traces[-1], used[-1], nocc)
        else:
            a = branch_alpha(traces[-1], nocc) if alphas is None else int(alphas[i - 1])
        idem.append(traces[-1] - core_trace_sq(X))
        X = [sp2_step(x, a) for x in X]
        used.append(a)
        traces.append(core_trace(X))
        if keep_iterates:
            for lst, x in zip(its, X):
                lst.append(x)
        if t >= 0:
            t += 1
            if t == tail:
                break
        elif (alphas is None and stop_now(idem, i, idem_tol)) or i == nsteps:
            if tail == 0:
                break
            t = 0
    return GSP2Result(n=n, S=S, ncore=ncore, X=X, alphas=used, traces=traces, idem=idem,
                      bounds=(eps_min, eps_max), iterates=its)


def gsp2_tail(res: GSP2Result, nocc, tail_steps):
    """The optional alternating tail (module notes) applied to a finished G-SP2 run without
    one: `tail_steps` more steps on every part, the first branch from the trace rule on the
    last global core trace, each further one the opposite.  Gives what gsp2(...,
    tail_steps=tail_steps) gives, without repeating the loop; `res` is left unchanged."""
    X = list(res.X)
    traces, idem, used = list(res.traces), list(res.idem), list(res.alphas)
    for t in range(tail_steps):
        a = tail_alpha(t, traces[-1], used[-1], nocc)
        idem.append(traces[-1] - float(sum(float(np.sum(np.einsum("ij,ji->i", m[:c, :], m[:, :c])))
                                           for m, c in zip(X, res.ncore))))
        X = [sp2_step(x, a) for x in X]
        used.append(a)
        traces.append(float(sum(float(np.sum(np.diag(m)[:c])) for m, c in zip(X, res.ncore))))
    return GSP2Result(n=res.n, S=res.S, ncore=res.ncore, X=X, alphas=used, traces=traces, idem=idem,
                      bounds=res.bounds)


# --------------------------------------------------------------------------------------
# Brute-force checks: eigendecomposition
# --------------------------------------------------------------------------------------

def eig_projector(H, nocc):
    """Exact density matrix of a gapped closed-shell H: projector on the Nocc lowest
    eigenvectors, from numpy.linalg.eigh (the O(N^3) route SP2 replaces, Section 1)."""
    w, V = np.linalg.eigh(np.asarray(H, dtype=np.float64))
    Vo = V[:, :nocc]
    return Vo @ Vo.T


def sp2_map_on_spectrum(H, alphas, bounds):
    """The SP2 polynomial of a recorded alpha sequence applied to the spectrum of H:
    V F(Lambda) V^T with x0 = (eps_max - lambda)/(eps_max - eps_min) and
    x <- x^2 (alpha = -1) or 2x - x^2 (alpha = +1), step by step on each eigenvalue."""
    eps_min, eps_max = bounds
    w, V = np.linalg.eigh(np.asarray(H, dtype=np.float64))
    x = (eps_max - w) / (eps_max - eps_min)
    for a in alphas:
        x = x * x if a == -1 else 2.0 * x - x * x
    return (V * x) @ V.T


# --------------------------------------------------------------------------------------
# Adjoint of P(H): L = sum_ij Pbar_ij P_ij, bounds and alpha sequence held fixed
# --------------------------------------------------------------------------------------

def _seed(Pbar_dense, S, c):
    """dL/dX_k is Pbar[S_k, core_k] in the core columns, zero in halo columns; X_k is a
    symmetric function of a symmetric argument, so the symmetric part is used."""
    s = len(S)
    M = np.zeros((s, s))
    M[:, :c] = Pbar_dense[np.ix_(S, S[:c])]
    return 0.5 * (M + M.T)


def _hbar_on_pattern(n, rowptr, colind, parts_grad):
    """Sum per-part gradients G_k (s_k x s_k, w.r.t. H[S_k, S_k]) onto H's pattern."""
    G = np.zeros((n, n))
    for S, Gk in parts_grad:
        G[np.ix_(S, S)] += Gk
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    return G[rows, np.asarray(colind)]


def seed_on_pattern(S, c, pbar, colptr, rowind):
    """The seed of _seed from dL/dP given on P's core-column pattern (values `pbar`,
    column g holding rows rowind[colptr[g]:colptr[g+1]]) instead of a dense N x N array."""
    s = len(S)
    loc = {int(g): t for t, g in enumerate(S)}
    M = np.zeros((s, s))
    for j in range(c):
        g = int(S[j])
        rows = rowind[colptr[g]:colptr[g + 1]]
        M[[loc[int(r)] for r in rows], j] = pbar[colptr[g]:colptr[g + 1]]
    return 0.5 * (M + M.T)


def part_adjoint(Hk, alphas, bounds, Xbar):
    """One part's reverse mode through the recorded alpha sequence (parts are independent
    once alpha is fixed), from the symmetric seed Xbar = dL/dX_n.  For the step X_i = X^2
    the adjoint is Xbar <- Xbar X + X Xbar; for X_i = 2X - X^2 it is
    Xbar <- 2 Xbar - Xbar X - X Xbar, with X the iterate the step acted on.  Finally
    dX0/dH = -1/(eps_max - eps_min) (Eq. 1).  Returns dL/dH[S_k, S_k]."""
    eps_min, eps_max = bounds
    X = initial_guess(Hk, eps_min, eps_max)
    its = [X]
    for a in alphas:
        X = sp2_step(X, a)
        its.append(X)
    Xb = Xbar
    for i in range(len(alphas), 0, -1):
        Xp = its[i - 1]
        if alphas[i - 1] == -1:
            Xb = Xb @ Xp + Xp @ Xb
        else:
            Xb = 2.0 * Xb - Xb @ Xp - Xp @ Xb
    return -Xb / (eps_max - eps_min)


def gsp2_adjoint(n, rowptr, colind, vals, res: GSP2Result, Pbar_dense):
    """Reverse mode through the recorded alpha sequence (part_adjoint for every part),
    summed onto H's CSR pattern (a symmetric array of values)."""
    Hs = _h_sparse(n, rowptr, colind, vals)
    grads = [(S, part_adjoint(Hs[S][:, S].toarray(), res.alphas, res.bounds, _seed(Pbar_dense, S, c)))
             for S, c in zip(res.S, res.ncore)]
    return _hbar_on_pattern(n, rowptr, colind, grads)


def dk_adjoint(n, rowptr, colind, vals, res: GSP2Result, Pbar_dense):
    """Daleckii-Krein form of the same gradient.  Per part, with H_k = V diag(lambda) V^T
    and F the composed SP2 polynomial (x0 from Eq. 1 then the recorded steps),
    dL/dH_k = V (F^[1] o (V^T Mbar V)) V^T where F^[1](a, b) is the first divided
    difference.  It is built by the chain rule for divided differences, step by step:
    start d = -1/(eps_max - eps_min) for Eq. 1, then d <- d (a + b) for x -> x^2 and
    d <- d (2 - a - b) for x -> 2x - x^2, carrying (a, b) to their images."""
    eps_min, eps_max = res.bounds
    Hs = _h_sparse(n, rowptr, colind, vals)
    grads = []
    for S, c in zip(res.S, res.ncore):
        w, V = np.linalg.eigh(Hs[S][:, S].toarray())
        x = (eps_max - w) / (eps_max - eps_min)
        A = x[:, None] + 0.0 * x[None, :]
        B = x[None, :] + 0.0 * x[:, None]
        D = np.full(A.shape, -1.0 / (eps_max - eps_min))
        for a in res.alphas:
            if a == -1:
                D = D * (A + B)
                A, B = A * A, B * B
            else:
                D = D * (2.0 - A - B)
                A, B = 2.0 * A - A * A, 2.0 * B - B * B
        Mb = _seed(Pbar_dense, S, c)
        grads.append((S, V @ (D * (V.T @ Mb @ V)) @ V.T))
    return _hbar_on_pattern(n, rowptr, colind, grads)


def fd_directional(n, rowptr, colind, vals, nocc, part, nparts, g_rowptr, g_colind,
                   res: GSP2Result, Pbar_dense, entries, h=1e-6):
    """Central finite differences of L = sum Pbar * P with the alpha sequence and the
    bounds frozen at those of `res`.  For each (i, j) in `entries` the stored values
    H_ij and H_ji are both moved by +-h (one value if i == j); returns dL/dh."""
    vals = np.asarray(vals, dtype=np.float64)
    out = []
    for (i, j) in entries:
        pos = [int(rowptr[i] + np.searchsorted(colind[rowptr[i]:rowptr[i + 1]], j))]
        if i != j:
            pos.append(int(rowptr[j] + np.searchsorted(colind[rowptr[j]:rowptr[j + 1]], i)))
        Ls = []
        for sgn in (1.0, -1.0):
            v = vals.copy()
            v[pos] += sgn * h
            r = gsp2(n, rowptr, colind, v, nocc, part, nparts, g_rowptr, g_colind,
                     alphas=res.alphas, bounds=res.bounds)
            Ls.append(float(np.sum(Pbar_dense * r.dense_p())))
        out.append((Ls[0] - Ls[1]) / (2.0 * h))
    return np.array(out)
