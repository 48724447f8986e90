"""Pins of the TT-rSI oracle (Alg. 4, subspace iteration) and of TT-rSVD
(Alg. 2 = TT-rBKI with q = 0), against facts fixed outside the oracle."""
import numpy as np
import pytest

import oracle
from oracle import tt_oracle as O
from paper_2308_01480_gb300 import workloads as W


def rand_tt(dims, ranks, seed):
    rng = np.random.default_rng(seed)
    return W.dense_from_cores(W.random_tt_cores(dims, ranks, rng))


def rand_matrix(m, n, ratio, seed):
    rng = np.random.default_rng(seed)
    k = min(m, n)
    U, _ = np.linalg.qr(rng.standard_normal((m, k)))
    V, _ = np.linalg.qr(rng.standard_normal((n, k)))
    return (U * ratio ** np.arange(k)) @ V.T


def projector_gap(Q1, Q2):
    return float(np.linalg.norm(Q1 @ Q1.T - Q2 @ Q2.T, 2))


@pytest.mark.parametrize("m,n,b,q", [(30, 200, 4, 2), (25, 120, 3, 3), (40, 90, 6, 1)])
def test_subspace_basis_spans_the_power(m, n, b, q):
    """span(Q) = span((C C^T)^q C W): the power built naively (normalising
    columns between products) and orthonormalised by Householder QR."""
    C = rand_matrix(m, n, 0.9, 7)
    Om = np.random.default_rng(8).standard_normal((n, b))
    Q = O.subspace_basis(C, Om, q)
    Y = C @ Om
    for _ in range(q):
        Y = Y / np.linalg.norm(Y, axis=0)
        Y = C @ (C.T @ Y)
    QK, _ = np.linalg.qr(Y)
    assert Q.shape == QK.shape == (m, b)
    assert projector_gap(Q, QK) < 1e-8
    assert np.max(np.abs(Q.T @ Q - np.eye(b))) < 1e-13


def test_q0_rsi_equals_rsvd():
    """Without iterations Alg. 4 is Alg. 2 (TT-rSVD): the same range finder."""
    A = W.add_noise(rand_tt((9, 10, 11, 8), (3, 4, 3), 4), 0.05, np.random.default_rng(5))
    a = oracle.tt_rsi(A, (3, 4, 3), 3, 0, seed=7)
    b = oracle.tt_rbki(A, (3, 4, 3), 3, 0, seed=7)
    assert oracle.tt_distance(a, b) < 1e-12


@pytest.mark.parametrize("dims,ranks,p,q", [((16, 16, 16, 16), (4, 4, 4), 5, 2), ((6, 7, 8, 5), (3, 4, 2), 2, 1),
                                            ((3, 50), (2,), 0, 3)])
def test_rsi_exact_recovery(dims, ranks, p, q):
    A = rand_tt(dims, ranks, 11)
    assert oracle.tt_error(A, oracle.tt_rsi(A, ranks, p, q, seed=3)) < 1e-12


def test_rsi_exhaustion_equals_tt_svd():
    """With r + p covering every unfolding's rank the subspace is range(C):
    the result is TT-SVD's."""
    B = np.random.default_rng(5).standard_normal((8, 8, 8))
    assert oracle.tt_distance(oracle.tt_rsi(B, (4, 4), 4, 2, seed=9), oracle.tt_svd(B, ranks=(4, 4))) < 1e-12


def test_rbki_subspace_contains_rsi_subspace():
    """span((C C^T)^q C W) lies in the block Krylov space of Alg. 3 with the
    same W, so Rayleigh-Ritz over the Krylov space captures at least as much
    energy of the first unfolding (optimality over nested subspaces)."""
    A = W.add_noise(rand_tt((12, 10, 9, 8), (4, 4, 4), 6), 0.2, np.random.default_rng(1))
    C = A.reshape(12, -1)
    Om = np.random.default_rng(2).standard_normal((C.shape[1], 6))
    Qs = O.subspace_basis(C, Om, 2)
    Qk = O.krylov_basis(C, Om, 2)
    assert np.linalg.norm(Qs - Qk @ (Qk.T @ Qs)) < 1e-10
    Us, _, _ = O.rsi_mode(C, 4, Om, 2)
    Uk, _, _ = O.rbki_mode(C, 4, Om, 2)
    assert np.linalg.norm(Uk.T @ C) >= np.linalg.norm(Us.T @ C) - 1e-12


def test_rsi_mutation_missing_transpose_fails_span_pin(monkeypatch):
    """A subspace step that applies C instead of C^T on the right breaks the
    span pin (the power would be (C C)^q, not (C C^T)^q)."""
    def wrong(C, Omega, q):
        m, n = C.shape
        b = Omega.shape[1]
        Q = O.orth_top(C @ Omega, min(b, m, n))
        for _ in range(q):
            Qh, _ = np.linalg.qr(C[:, :m].T @ Q)        # mistake: wrong operand
            Q = O.orth_top(C[:, :m] @ Qh, Q.shape[1])
        return Q
    monkeypatch.setattr(O, "subspace_basis", wrong)
    with pytest.raises(AssertionError):
        test_subspace_basis_spans_the_power(30, 200, 4, 2)
