"""Magnitudes of the digit-product groups on which the emulated FP64 step rests.

The step writes every entry of X (||X||_2 <= 1) as balanced base-2^7 digits,
x ~ sum_t S_t 2^{-7(t+1)}, and sums the products S_a S_b of each group d = a + b in FP32;
a group's sum is exact while every partial sum stays below 2^24 in its own units.  G_0 and
G_1 share one accumulator, G_0 + 2^-7 G_1, whose terms are multiples of 2^-7: exact while
the magnitudes of the terms of 2^7 G_0 + G_1 sum to less than 2^23, which the bound
2^21 + 3 2^13 (sum_k |x_ik| + |x_kj|) + 2^8 K guarantees for K <= 4096.  Groups 2-4 have no
such bound; these tests measure them on the two kinds of extreme input at K = 4096: a dense
projector (rows spread over all columns) and a scaled Hadamard matrix (every entry of one
magnitude, so that the digit products are coherent wherever the signs are).

The digits here are written from their definition, independently of the kernels."""

import numpy as np
import pytest

T = 7


def balanced_digits(X):
    """S_0 .. S_{T-1} with w = round(x 2^{7T}) = sum_t S_t 2^{7(T-1-t)}, S_t in [-64, 63]
    for t >= 1 and S_0 the rest."""
    w = np.rint(np.asarray(X) * 2.0 ** (7 * T)).astype(np.int64)
    S = [None] * T
    r = w
    for t in range(T - 1, 0, -1):
        d = ((r + 64) % 128) - 64
        S[t] = d
        r = (r - d) // 128
    S[0] = r
    return S


def sylvester_hadamard(K):
    H = np.ones((1, 1))
    while H.shape[0] < K:
        H = np.block([[H, H], [H, -H]])
    return H


def group_terms(S, rows):
    """For the given rows i and every column j: the sums over k of the magnitudes of the
    terms of 2^7 G_0 + G_1, and of G_2, G_3, G_4."""
    A = [np.abs(s).astype(np.float64) for s in S]
    merged = np.stack([2.0 ** 7 * A[0][i] @ A[0] + A[0][i] @ A[1] + A[1][i] @ A[0] for i in rows])
    groups = {d: np.stack([sum(A[a][i] @ A[d - a] for a in range(d + 1)) for i in rows]) for d in (2, 3, 4)}
    return merged, groups


def merged_bound(X, rows):
    K = X.shape[0]
    one = np.abs(X).sum(axis=1)
    return np.stack([2.0 ** 21 + 3 * 2.0 ** 13 * (one[i] + one) + 2.0 ** 8 * K for i in rows])


def test_balanced_digits_reconstruct_and_stay_in_range():
    rng = np.random.default_rng(3)
    x = rng.uniform(-1.0, 1.0, 20000)
    S = balanced_digits(x)
    w = sum(S[t] * 2 ** (7 * (T - 1 - t)) for t in range(T))
    assert np.array_equal(w, np.rint(x * 2.0 ** (7 * T)).astype(np.int64))
    for t in range(1, T):
        assert S[t].min() >= -64 and S[t].max() <= 63
    assert np.all(np.abs(S[0]) <= 2 ** 7 * np.abs(x) + 1)


@pytest.fixture(scope="module")
def projector():
    K = 4096
    rng = np.random.default_rng(11)
    q, _ = np.linalg.qr(rng.standard_normal((K, K)))
    return q[:, : K // 2] @ q[:, : K // 2].T


def test_groups_of_a_dense_projector_at_k_4096(projector):
    X = projector
    rows = [0, 1, 2048, 4095]
    S = balanced_digits(X)
    merged, groups = group_terms(S, rows)
    assert np.all(merged <= merged_bound(X, rows))
    assert merged.max() < 2.0 ** 23
    for d, g in groups.items():
        assert g.max() < 2.0 ** 24, (d, np.log2(g.max()))
    # the coherent part of the even groups: the diagonal's sums of squares
    S1sq = float((S[1][0].astype(np.float64) ** 2).sum())
    assert 2.0 ** 21 < S1sq < 2.0 ** 23


def test_groups_of_a_scaled_hadamard_matrix_at_k_4096():
    K = 4096
    X = 0.987654321 * sylvester_hadamard(K) / np.sqrt(K)
    assert np.linalg.norm(X[:64] @ X.T[:, :64] - 0.987654321 ** 2 * np.eye(64)) < 1e-12
    rows = [0, 1]
    S = balanced_digits(X)
    merged, groups = group_terms(S, rows)
    assert np.all(merged <= merged_bound(X, rows))
    assert merged.max() < 2.0 ** 23
    for d, g in groups.items():
        assert g.max() < 2.0 ** 23, (d, np.log2(g.max()))
