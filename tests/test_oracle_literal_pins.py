"""Pins of the literal forms of Alg. 2-4 in the oracle (the paper's
right-side Krylov matrix with the first-r truncation of an unpivoted QR).

The leading columns of a QR span the leading columns of its input, so the
literal truncation of Alg. 3 equals an orthonormal basis of
(C C^T) C W(:, 1:r): U(:, 1:r) spans C^T C W(:, 1:r), and Y(:, 1:r) = C U(:, 1:r).
Likewise Alg. 2 gives span C W(:, 1:r) and Alg. 4 span (C C^T)^q C W(:, 1:r).
These closed forms are computed here independently (one QR of the product),
and compared as projectors."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.filterwarnings("ignore")


def _proj(Q):
    return Q @ Q.T


def _case(m, n, rank, seed, decay=0.7):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, rank)))
    V, _ = np.linalg.qr(rng.standard_normal((n, rank)))
    s = decay ** np.arange(rank)
    return (U * s) @ V.T


@pytest.mark.parametrize("m,n,r,b,seed", [(20, 300, 4, 7, 1), (35, 120, 6, 9, 2), (12, 400, 3, 3, 3)])
def test_literal_rbki_span_is_one_power_of_first_r_columns(m, n, r, b, seed):
    C = _case(m, n, min(m, n) // 2, seed)
    Om = np.random.default_rng(seed + 10).standard_normal((n, b))
    for q in (1, 2, 3):
        Q, R, _ = oracle.literal_rbki_mode(C, r, Om, q)
        ref, _ = np.linalg.qr(C @ (C.T @ (C @ Om[:, :r])))
        assert Q.shape == (m, r)
        assert np.max(np.abs(_proj(Q) - _proj(ref))) < 1e-9
        assert np.max(np.abs(Q.T @ Q - np.eye(r))) < 1e-12
        assert np.max(np.abs(R - Q.T @ C)) < 1e-12


def test_literal_rbki_pin_catches_a_dropped_power():
    """Planted mistake: K built from W instead of C^T C W (the first power
    dropped) spans C W(:, 1:r), which differs from the closed form."""
    C = _case(30, 200, 15, 4)
    Om = np.random.default_rng(14).standard_normal((200, 8))
    r = 5
    wrong_U, _ = np.linalg.qr(np.hstack([Om, C.T @ (C @ Om)]))
    wrong, _ = np.linalg.qr(C @ wrong_U)
    ref, _ = np.linalg.qr(C @ (C.T @ (C @ Om[:, :r])))
    assert np.max(np.abs(_proj(wrong[:, :r]) - _proj(ref))) > 1e-3


@pytest.mark.parametrize("q", [0, 1, 2])
def test_literal_rsi_and_rsvd_spans(q):
    C = _case(25, 250, 12, 5)
    Om = np.random.default_rng(15).standard_normal((250, 9))
    r = 4
    Q, _, _ = oracle.literal_rsi_mode(C, r, Om, q)
    X = C @ Om[:, :r]
    for _ in range(q):
        X = C @ (C.T @ X)
    ref, _ = np.linalg.qr(X)
    assert np.max(np.abs(_proj(Q) - _proj(ref))) < 1e-9
    if q == 0:   # Alg. 2 taken literally is also the q = 0 form of Alg. 3
        Q2, _, _ = oracle.literal_rbki_mode(C, r, Om, 0)
        assert np.max(np.abs(_proj(Q2) - _proj(ref))) < 1e-12


def test_literal_exact_recovery_of_low_tt_rank():
    """Target ranks at least the TT ranks: every unfolding has rank <= r, the
    first-r sketch spans its range with probability one, and the literal
    decomposition reproduces the tensor."""
    rng = np.random.default_rng(6)
    dims, ranks = (7, 8, 6, 5), (3, 4, 2)
    cores = [rng.standard_normal((a, I, b)) for a, I, b in zip((1,) + ranks, dims, ranks + (1,))]
    A = oracle.tt_full(cores)
    for q in (0, 1, 2):
        got = oracle.tt_rbki_literal(A, ranks, 2, q, seed=3)
        assert oracle.tt_error(A, got) < 1e-12
        got = oracle.tt_rsi_literal(A, ranks, 2, q, seed=3)
        assert oracle.tt_error(A, got) < 1e-12


def test_literal_cores_left_orthogonal_and_projection_identity():
    rng = np.random.default_rng(7)
    A = rng.standard_normal((6, 7, 8, 5))
    got = oracle.tt_rbki_literal(A, (3, 4, 3), 2, 2, seed=1)
    for G in got[:-1]:
        assert oracle.left_orthogonality_defect(G) < 1e-12
    # orthogonal projections: ||A||^2 = ||A_hat||^2 + ||A - A_hat||^2
    Ah = oracle.tt_full(got)
    lhs = np.sum(A ** 2)
    rhs = np.sum(Ah ** 2) + np.sum((A - Ah) ** 2)
    assert abs(lhs - rhs) < 1e-10 * lhs
