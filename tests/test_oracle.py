"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each check is a worked value from the
paper (tests/golden), a closed form, an invariant of the exact density matrix, a
brute-force eigendecomposition, or a special case in which G-SP2 reduces exactly to
plain SP2.
"""

import os

import numpy as np
import pytest

import oracle
from synth import make_workload, dense_from_csr, csr_from_dense, block_partition
from synth.tb import graph_from_dense_threshold, make_tb_system, _csr_from_coo

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def tb512():
    return make_workload("tb512")


@pytest.fixture(scope="module")
def tb512_dense(tb512):
    return dense_from_csr(tb512.n, tb512.rowptr, tb512.colind, tb512.vals)


# ---------------------------------------------------------------- Gershgorin (Sec. 2.1)

def test_gershgorin_worked_example():
    lines = [l.split() for l in open(os.path.join(GOLDEN, "gershgorin_3x3.txt"))
             if l.strip() and not l.startswith("#")]
    i = [l[0] for l in lines].index("matrix")
    M = np.array([[float(x) for x in lines[i + r]] for r in (1, 2, 3)])
    want = {l[0]: float(l[1]) for l in lines if l[0] in ("eps_min", "eps_max")}
    rp, ci, v = csr_from_dense(M)
    lo, hi = oracle.gershgorin_bounds(3, rp, ci, v)
    assert lo == want["eps_min"] and hi == want["eps_max"]


def test_gershgorin_encloses_spectrum(tb512, tb512_dense):
    lo, hi = oracle.gershgorin_bounds(tb512.n, tb512.rowptr, tb512.colind, tb512.vals)
    w = np.linalg.eigvalsh(tb512_dense)
    assert lo <= w[0] and w[-1] <= hi
    # the bound is attained by some row: it is not looser than the widest disc
    d = np.diag(tb512_dense)
    r = np.abs(tb512_dense).sum(1) - np.abs(d)
    assert lo == pytest.approx(np.min(d - r), rel=1e-14) and hi == pytest.approx(np.max(d + r), rel=1e-14)


# ---------------------------------------------------------------- SP2 (Eqs. 1-3)

def test_initial_guess_maps_spectrum_reversed(tb512_dense):
    H = tb512_dense
    d = np.diag(H)
    r = np.abs(H).sum(1) - np.abs(d)
    lo, hi = float(np.min(d - r)), float(np.max(d + r))
    X0 = oracle.initial_guess(H, lo, hi)
    wh = np.linalg.eigvalsh(H)
    wx = np.linalg.eigvalsh(X0)
    assert wx.min() >= -1e-12 and wx.max() <= 1 + 1e-12
    # reversed order: the lowest eigenvalue of H maps to the largest of X0
    np.testing.assert_allclose(wx[::-1], (hi - wh) / (hi - lo), atol=1e-12)


def test_sp2_matches_eigendecomposition(tb512, tb512_dense):
    H = tb512_dense
    P, rec = oracle.sp2_dense(H, tb512.nocc, 45)
    Pex = oracle.eig_projector(H, tb512.nocc)
    assert np.max(np.abs(P - Pex)) <= 1e-10
    assert abs(np.trace(P) - tb512.nocc) <= 1e-9
    assert np.max(np.abs(P @ P - P)) <= 1e-10
    assert np.max(np.abs(H @ P - P @ H)) <= 1e-9
    # idempotency error e_i = Tr X - Tr X^2 >= 0 and vanishes at convergence (Eq. 3 check)
    e = np.array(rec["idem"])
    assert np.all(e >= -1e-9) and e[0] > 1.0 and e[-1] <= 1e-9


def test_sp2_diagonal_is_exact_step_function():
    rng = np.random.default_rng(7)
    lo_band = -8.0 + rng.uniform(-0.5, 0.5, 20)
    hi_band = 2.0 + rng.uniform(-0.5, 0.5, 20)
    eps = rng.permutation(np.concatenate([lo_band, hi_band]))
    H = np.diag(eps)
    P, _ = oracle.sp2_dense(H, 20, 45)
    want = np.diag((eps < -3.0).astype(float))
    assert np.max(np.abs(P - want)) <= 1e-14


def test_sp2_equals_polynomial_on_spectrum(tb512_dense, tb512):
    H = tb512_dense
    P, rec = oracle.sp2_dense(H, tb512.nocc, 30)
    Q = oracle.sp2_map_on_spectrum(H, rec["alphas"], rec["bounds"])
    assert np.max(np.abs(P - Q)) <= 1e-11


def test_sp2_step_single_cases():
    X = np.array([[0.3, 0.1], [0.1, 0.6]])
    # x^2 and 2x - x^2 of Eq. 2 on a 2x2, worked by hand
    sq = np.array([[0.09 + 0.01, 0.03 + 0.06], [0.03 + 0.06, 0.01 + 0.36]])
    np.testing.assert_allclose(oracle.sp2_step(X, -1), sq, atol=1e-15)
    np.testing.assert_allclose(oracle.sp2_step(X, 1), 2 * X - sq, atol=1e-15)
    assert oracle.branch_alpha(3.0, 3) == 1  # tie takes "<="
    assert oracle.branch_alpha(3.0 + 1e-9, 3) == -1
    assert oracle.branch_alpha(2.5, 3) == 1


def test_wrong_alpha_sequence_gives_wrong_trace(tb512, tb512_dense):
    """Section 2.1: with a wrong multiplication sequence the iteration ends with the
    wrong trace."""
    P, rec = oracle.sp2_dense(tb512_dense, tb512.nocc, 45)
    bad = list(rec["alphas"])
    bad[2] = -bad[2]
    Pb, _ = oracle.sp2_dense(tb512_dense, tb512.nocc, 45, alphas=bad)
    assert abs(np.trace(Pb) - tb512.nocc) >= 0.5


# ---------------------------------------------------------------- core/halo, Eq. 5

def _fig2():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "fig2_core_halo.txt"))
            if l.strip() and not l.startswith("#")]
    names = rows[0][1:]
    idx = {v: i for i, v in enumerate(names)}
    edges = [(idx[r[1]], idx[r[2]]) for r in rows if r[0] == "edge"]
    parts, expect = {}, {}
    for r in rows:
        if r[0] == "partition":
            bar = r.index("|")
            parts[r[1]] = (r[2:bar], r[bar + 1:])
        if r[0] == "expect":
            expect[r[1]] = dict(sizes=[int(r[3]), int(r[4])], halo=[int(r[6]), int(r[7])],
                                cost=int(r[9]), cut=int(r[11]))
    return names, idx, edges, parts, expect


@pytest.mark.parametrize("case", ["a", "b"])
def test_fig2_core_halo_and_cost(case):
    names, idx, edges, parts, expect = _fig2()
    n = len(names)
    e = np.array(edges + [(b, a) for a, b in edges])
    rp, ci, _ = _csr_from_coo(n, e[:, 0].astype(np.int64), e[:, 1].astype(np.int64), None)
    part = np.zeros(n, np.int32)
    for v in parts[case][1]:
        part[idx[v]] = 1
    ch = oracle.core_halo(rp, ci, part, 2)
    sizes = [len(c) + len(h) for c, h in ch]
    assert sizes == expect[case]["sizes"]
    assert [len(h) for _, h in ch] == expect[case]["halo"]
    assert oracle.ch_cost(sizes) == expect[case]["cost"]
    cut = sum(1 for a, b in edges if part[a] != part[b])
    assert cut == expect[case]["cut"]


def test_block_partition_sizes():
    kv = {l.split()[0]: l.split()[1:] for l in open(os.path.join(GOLDEN, "block_partition_polyalanine.txt"))
          if l.strip() and not l.startswith("#")}
    p = block_partition(int(kv["n"][0]), int(kv["nparts"][0]))
    counts = np.bincount(p)
    assert set(counts.tolist()) == {34, 35}
    assert int((counts == 35).sum()) == int(kv["count35"][0])
    assert int((counts == 34).sum()) == int(kv["count34"][0])


# ---------------------------------------------------------------- G-SP2 reductions

def test_gsp2_one_part_is_plain_sp2(tb512, tb512_dense):
    n = tb512.n
    r = oracle.gsp2(n, tb512.rowptr, tb512.colind, tb512.vals, tb512.nocc, np.zeros(n, np.int32), 1,
                    tb512.g_rowptr, tb512.g_colind, max_steps=45)
    P, rec = oracle.sp2_dense(tb512_dense, tb512.nocc, 45)
    assert r.alphas == rec["alphas"]
    assert np.max(np.abs(r.dense_p() - P)) <= 1e-13


def test_gsp2_complete_graph_is_plain_sp2(tb512, tb512_dense):
    n = tb512.n
    A = np.ones((n, n)) - np.eye(n)
    grp, gci = graph_from_dense_threshold(A, 0.5)
    r = oracle.gsp2(n, tb512.rowptr, tb512.colind, tb512.vals, tb512.nocc, tb512.part, tb512.nparts,
                    grp, gci, max_steps=45)
    assert all(len(S) == n for S in r.S)
    P, rec = oracle.sp2_dense(tb512_dense, tb512.nocc, 45)
    assert np.max(np.abs(r.dense_p() - P)) <= 1e-11


def test_gsp2_block_diagonal_has_no_halo():
    a = make_tb_system(40, 1, 3.0, seed=11)
    b = make_tb_system(56, 1, 3.0, seed=12)
    Ha = dense_from_csr(a.n, a.rowptr, a.colind, a.vals)
    Hb = dense_from_csr(b.n, b.rowptr, b.colind, b.vals)
    H = np.zeros((a.n + b.n, a.n + b.n))
    H[:a.n, :a.n] = Ha
    H[a.n:, a.n:] = Hb
    rp, ci, v = csr_from_dense(H)
    part = np.concatenate([np.zeros(a.n, np.int32), np.ones(b.n, np.int32)])
    nocc = a.nocc + b.nocc
    r = oracle.gsp2(H.shape[0], rp, ci, v, nocc, part, 2, rp, ci, max_steps=45)
    assert [len(S) for S in r.S] == [a.n, b.n]
    P, _ = oracle.sp2_dense(H, nocc, 45)
    assert np.max(np.abs(r.dense_p() - P)) <= 1e-12
    assert np.max(np.abs(P - oracle.eig_projector(H, nocc))) <= 1e-10


def test_gsp2_error_shrinks_with_threshold(tb512, tb512_dense):
    """Halos from G_tau (Section 2.2) with tau taken from the exact P: the truncation
    error of G-SP2 falls as tau falls."""
    Pex = oracle.eig_projector(tb512_dense, tb512.nocc)
    errs = []
    for tau in (1e-2, 1e-3, 1e-4, 1e-5):
        grp, gci = graph_from_dense_threshold(Pex, tau)
        r = oracle.gsp2(tb512.n, tb512.rowptr, tb512.colind, tb512.vals, tb512.nocc, tb512.part,
                        tb512.nparts, grp, gci, max_steps=45)
        errs.append(np.max(np.abs(r.dense_p() - Pex)))
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1)), errs
    assert errs[-1] <= 1e-4


def test_gsp2_parts_follow_shared_polynomial(tb512):
    """Every part is the same SP2 polynomial (one alpha sequence, global bounds)
    applied to its own submatrix: X_k = V_k F(Lambda_k) V_k^T."""
    r = oracle.gsp2(tb512.n, tb512.rowptr, tb512.colind, tb512.vals, tb512.nocc, tb512.part,
                    tb512.nparts, tb512.g_rowptr, tb512.g_colind, max_steps=45)
    H = dense_from_csr(tb512.n, tb512.rowptr, tb512.colind, tb512.vals)
    for S, X in zip(r.S, r.X):
        Q = oracle.sp2_map_on_spectrum(H[np.ix_(S, S)], r.alphas, r.bounds)
        assert np.max(np.abs(X - Q)) <= 1e-10
    # the core-diagonal trace reaches Nocc up to the halo truncation of G_tau (each part
    # converges to a projector of its own submatrix), and it is the trace of P
    assert abs(r.traces[-1] - tb512.nocc) <= 1e-3
    P = r.dense_p()
    assert abs(np.trace(P) - r.traces[-1]) <= 1e-9


# ---------------------------------------------------------------- adjoint

@pytest.fixture(scope="module")
def small_adj():
    s = make_tb_system(48, 4, 3.0, seed=21)
    r = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind,
                    max_steps=40)
    from synth import random_symmetric_on_pattern
    A = dense_from_csr(s.n, s.rowptr, s.colind, random_symmetric_on_pattern(s.rowptr, s.colind, 5678))
    return s, r, A


def test_adjoint_matches_daleckii_krein(small_adj):
    s, r, A = small_adj
    g = oracle.gsp2_adjoint(s.n, s.rowptr, s.colind, s.vals, r, A)
    d = oracle.dk_adjoint(s.n, s.rowptr, s.colind, s.vals, r, A)
    assert np.max(np.abs(g - d)) <= 1e-10 * max(1.0, np.max(np.abs(d)))
    # symmetric gradient on a symmetric pattern
    G = dense_from_csr(s.n, s.rowptr, s.colind, g)
    assert np.max(np.abs(G - G.T)) <= 1e-12 * max(1.0, np.max(np.abs(G)))


def test_adjoint_matches_finite_differences(small_adj):
    s, r, A = small_adj
    g = oracle.gsp2_adjoint(s.n, s.rowptr, s.colind, s.vals, r, A)
    G = dense_from_csr(s.n, s.rowptr, s.colind, g)
    rng = np.random.default_rng(3)
    rows = np.repeat(np.arange(s.n), np.diff(s.rowptr))
    pick = rng.choice(len(rows), 8, replace=False)
    entries = [(int(rows[p]), int(s.colind[p])) for p in pick] + [(5, 5)]
    fd = oracle.fd_directional(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts,
                               s.g_rowptr, s.g_colind, r, A, entries, h=1e-6)
    an = np.array([G[i, j] + G[j, i] if i != j else G[i, i] for i, j in entries])
    scale = max(1e-3, np.max(np.abs(an)))
    assert np.max(np.abs(fd - an)) <= 1e-6 * scale, (fd, an)


def test_gsp2_assembles_core_columns(tb512):
    """Section 1.1 / Fig. 1: P is reassembled from the parts; a core vertex j of part k
    owns column j, filled on the rows S_k (cores and halo of part k) and zero elsewhere."""
    r = oracle.gsp2(tb512.n, tb512.rowptr, tb512.colind, tb512.vals, tb512.nocc, tb512.part,
                    tb512.nparts, tb512.g_rowptr, tb512.g_colind, max_steps=45)
    P = r.dense_p()
    for S, c, X in zip(r.S, r.ncore, r.X):
        outside = np.ones(tb512.n, bool)
        outside[S] = False
        for j in range(c):
            g = S[j]
            assert not np.any(P[outside, g])
            np.testing.assert_array_equal(P[S, g], X[:, j])
    # halos are non-empty, so some entries of P lie outside the diagonal blocks
    assert any(len(S) > c for S, c in zip(r.S, r.ncore))


# ---------------------------------------------------------------- optional tail

def test_tail_steps_alternate_and_purify(tb512, tb512_dense):
    """Plain SP2 with a tail stays on the exact projector; in G-SP2 the alternating tail
    removes the drift left by a core trace that cannot reach Nocc."""
    P0, r0 = oracle.sp2_dense(tb512_dense, tb512.nocc, 45)
    P2, r2 = oracle.sp2_dense(tb512_dense, tb512.nocc, 45, tail_steps=2)
    assert r2["alphas"][:len(r0["alphas"])] == r0["alphas"] and len(r2["alphas"]) == len(r0["alphas"]) + 2
    assert r2["alphas"][-1] == -r2["alphas"][-2]
    assert np.max(np.abs(P2 - oracle.eig_projector(tb512_dense, tb512.nocc))) <= 1e-10
    # the recorded sequence, tail included, is one SP2 polynomial
    assert np.max(np.abs(P2 - oracle.sp2_map_on_spectrum(tb512_dense, r2["alphas"], r2["bounds"]))) <= 1e-11
    kw = dict(max_steps=45)
    args = (tb512.n, tb512.rowptr, tb512.colind, tb512.vals, tb512.nocc, tb512.part, tb512.nparts,
            tb512.g_rowptr, tb512.g_colind)
    g0 = oracle.gsp2(*args, **kw)
    g2 = oracle.gsp2(*args, tail_steps=2, **kw)
    assert g2.alphas[:len(g0.alphas)] == g0.alphas and g2.alphas[-1] == -g2.alphas[-2]

    def part_idem(r):
        return np.sqrt(sum(np.linalg.norm(X @ X - X) ** 2 for X in r.X) / tb512.n)
    assert part_idem(g0) > 1e-8 and part_idem(g2) < 1e-10
    # a replayed sequence runs exactly its length (the tail is part of it)
    g3 = oracle.gsp2(*args, alphas=g2.alphas, tail_steps=5)
    assert g3.alphas == g2.alphas and np.array_equal(g3.dense_p(), g2.dense_p())


def test_tail_continuation_equals_a_run_with_the_tail(tb512):
    """gsp2_tail appends the alternating tail to a finished run: the same branches, traces,
    idempotency history and iterates as one run with tail_steps (the large-size checks
    use it to get both results from one loop)."""
    args = (tb512.n, tb512.rowptr, tb512.colind, tb512.vals, tb512.nocc, tb512.part, tb512.nparts,
            tb512.g_rowptr, tb512.g_colind)
    g0 = oracle.gsp2(*args)
    for tail in (1, 2, 3):
        g2 = oracle.gsp2(*args, tail_steps=tail)
        c2 = oracle.gsp2_tail(g0, tb512.nocc, tail)
        assert c2.alphas == g2.alphas and c2.traces == g2.traces and c2.idem == g2.idem
        for a, b in zip(c2.X, g2.X):
            np.testing.assert_array_equal(a, b)
    assert len(g0.alphas) == len(oracle.gsp2_tail(g0, tb512.nocc, 2).alphas) - 2  # g0 untouched


def test_seed_on_pattern_and_core_halo_subset_agree_with_the_dense_forms():
    """The pattern-based seed equals the dense-Pbar seed, and core_halo for a subset of
    parts equals those entries of the full list (the forms the large-size checks use)."""
    from oracle.gsp2 import _seed
    s = make_workload("tb512")
    res = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind)
    # pattern of P from the oracle's own lists (sorted rows S_part(g) per core column g)
    colptr = np.zeros(s.n + 1, np.int64)
    rows_of = {}
    for S, c in zip(res.S, res.ncore):
        for j in range(c):
            rows_of[int(S[j])] = np.sort(S)
    for g in range(s.n):
        colptr[g + 1] = colptr[g] + len(rows_of[g])
    rowind = np.concatenate([rows_of[g] for g in range(s.n)])
    rng = np.random.default_rng(3)
    pbar = rng.standard_normal(int(colptr[-1]))
    dense = np.zeros((s.n, s.n))
    cols = np.repeat(np.arange(s.n), np.diff(colptr))
    dense[rowind, cols] = pbar
    for S, c in zip(res.S, res.ncore):
        np.testing.assert_array_equal(oracle.seed_on_pattern(S, c, pbar, colptr, rowind), _seed(dense, S, c))
    full = oracle.core_halo(s.g_rowptr, s.g_colind, s.part, s.nparts)
    sub = oracle.core_halo(s.g_rowptr, s.g_colind, s.part, s.nparts, which=[5, 2])
    for k, (c, h) in zip([5, 2], sub):
        np.testing.assert_array_equal(c, full[k][0])
        np.testing.assert_array_equal(h, full[k][1])


@pytest.mark.parametrize("case", ["tb512", "ragged"])
def test_p_on_pattern_is_dense_p_read_on_the_pattern(case):
    """Every GPU parity test reads the oracle's P through p_on_pattern: it must give, for
    each stored (row, column) of a core-column pattern, the entry of the assembled P that
    dense_p() holds there (dense_p itself is pinned by the core-column test above), in
    whatever row order a column lists its rows."""
    s = make_workload("tb512") if case == "tb512" else make_tb_system(33, 5, 3.2, seed=133)
    res = oracle.gsp2(s.n, s.rowptr, s.colind, s.vals, s.nocc, s.part, s.nparts, s.g_rowptr, s.g_colind)
    P = res.dense_p()
    rows_of = {}
    for S, c in zip(res.S, res.ncore):
        for j in range(c):
            rows_of[int(S[j])] = np.sort(S)
    assert sorted(rows_of) == list(range(s.n))
    rng = np.random.default_rng(7)
    for order in ("ascending", "shuffled"):
        lists = [rows_of[g] if order == "ascending" else rng.permutation(rows_of[g]) for g in range(s.n)]
        colptr = np.zeros(s.n + 1, np.int64)
        colptr[1:] = np.cumsum([len(r) for r in lists])
        rowind = np.concatenate(lists).astype(np.int32)
        cols = np.repeat(np.arange(s.n), np.diff(colptr))
        got = res.p_on_pattern(colptr, rowind)
        np.testing.assert_array_equal(got, P[rowind, cols])
    # the pattern holds every nonzero of P (nothing of P lies off the core-column pattern)
    mask = np.zeros((s.n, s.n), bool)
    mask[rowind, cols] = True
    assert not np.any(P[~mask])
