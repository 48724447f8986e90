"""Pins of the FP64 oracle against things other than itself.

Each test checks the oracle against a closed form, a library routine on a
special case, a published known-answer vector, brute force, or an invariant
that the mathematics fixes.  The mutation tests at the end plant plausible
mistakes in the oracle (on the CPU) and check that some pin catches each.
"""
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.stats

import oracle
from oracle import tt_oracle as O
from oracle.philox import omega_from_seed, philox4x32_10
from paper_2308_01480_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_tt(dims, ranks, seed, decay=0.0):
    rng = np.random.default_rng(seed)
    return W.dense_from_cores(W.random_tt_cores(dims, ranks, rng, decay))


def rand_matrix(m, n, ratio, seed):
    """m x n matrix with singular values ratio**j (j = 0..min-1)."""
    rng = np.random.default_rng(seed)
    k = min(m, n)
    U, _ = np.linalg.qr(rng.standard_normal((m, k)))
    V, _ = np.linalg.qr(rng.standard_normal((n, k)))
    return (U * ratio ** np.arange(k)) @ V.T


def projector_gap(Q1, Q2):
    return float(np.linalg.norm(Q1 @ Q1.T - Q2 @ Q2.T, 2))


# ---------------------------------------------------------------- exact recovery
@pytest.mark.parametrize("dims,ranks", [
    ((16, 16, 16, 16), (4, 4, 4)),
    ((6, 7, 8, 5), (3, 4, 2)),
    ((5, 6, 7), (2, 3)),
    ((3, 50), (2,)),
])
@pytest.mark.parametrize("p,q", [(5, 2), (0, 0), (2, 1)])
def test_exact_recovery_from_tt_cores(dims, ranks, p, q):
    """A tensor of TT rank r is recovered exactly at target rank r: range(C W)
    = range(C) with probability one (Alg. 3 with rank(C) <= r' + p)."""
    A = rand_tt(dims, ranks, 11)
    cores = oracle.tt_rbki(A, ranks, p, q, seed=3)
    assert oracle.tt_error(A, cores) < 1e-12
    assert oracle.tt_error(A, oracle.tt_svd(A, ranks=ranks)) < 1e-12


def test_exact_recovery_config1_noise_free():
    w = W.CONFIGS[1]
    A = rand_tt(w.dims, w.tt_ranks, w.tensor_seed)
    cores = oracle.tt_rbki(A, w.ranks, w.oversample, w.q, seed=w.omega_seed)
    assert oracle.tt_error(A, cores) < 1e-12


# ---------------------------------------------------------------- exhaustion
@pytest.mark.parametrize("dims,ranks,p,q", [
    ((8, 8, 8), (4, 4), 4, 1),       # every mode exhausted by the first block
    ((10, 9, 8), (3, 3), 1, 5),      # mode 1 needs a capped third block
    ((10, 4, 7), (10, 2), 1, 3),     # mode 2: D = n < m, last block truncated to 1
    ((12, 5, 3), (3, 3), 2, 4),      # mode 2: first block truncated to rank(C)
])
def test_exhaustion_equals_tt_svd(dims, ranks, p, q):
    """When the Krylov basis reaches D = min(m, n) columns, Rayleigh-Ritz on it
    is the exact truncated SVD, so TT-rBKI equals TT-SVD (Alg. 1)."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal(dims)
    cores = oracle.tt_rbki(A, ranks, p, q, seed=9)
    ref = oracle.tt_svd(A, ranks=ranks)
    assert oracle.tt_distance(cores, ref) < 1e-12


def test_tt_svd_order2_is_lapack_truncated_svd():
    """d = 2: TT-SVD is the rank-r truncated SVD (Eckart-Young); compare with
    LAPACK's gesvd driver, a different SVD algorithm than numpy's gesdd."""
    rng = np.random.default_rng(1)
    M = rng.standard_normal((30, 45))
    cores = oracle.tt_svd(M, ranks=(7,))
    U, s, Vt = scipy.linalg.svd(M, full_matrices=False, lapack_driver="gesvd")
    ref = (U[:, :7] * s[:7]) @ Vt[:7]
    assert np.max(np.abs(oracle.tt_full(cores) - ref)) < 1e-12
    # and the error equals the tail energy tau_8 (Def. 3)
    err = np.linalg.norm(M - oracle.tt_full(cores))
    assert abs(err ** 2 - np.sum(s[7:] ** 2)) < 1e-10 * np.sum(s ** 2)


def test_tt_svd_eps_truncation():
    """Alg. 1 with accuracy eps: ||A - B|| <= eps ||A||, and each rank is the
    smallest meeting delta = eps ||A|| / sqrt(d-1) on its unfolding."""
    A = rand_tt((7, 8, 9, 6), (3, 5, 2), 4)
    A = W.add_noise(A, 0.02, np.random.default_rng(2))
    for eps in (0.5, 0.1, 0.03):
        cores = oracle.tt_svd(A, eps=eps)
        assert oracle.tt_error(A, cores) <= eps * (1 + 1e-12)
    # tight case: eps below the noise forces near-full ranks at the first mode
    cores = oracle.tt_svd(A, eps=1e-3)
    assert cores[0].shape[2] == 7


# ---------------------------------------------------------------- bounds
def _unfolding_tails(A, ranks):
    dims = A.shape
    out = []
    for k, r in enumerate(ranks):
        M = A.reshape(int(np.prod(dims[:k + 1])), -1)
        out.append(oracle.tail_energy(M, r + 1))
    return out


def test_theorem1_and_eckart_young_bounds():
    """Thm 1: ||A - B_svd|| <= sqrt(sum_k tau_{r_k+1}^2(A_k)); and any TT of
    ranks r has error >= max_k tau_{r_k+1}(A_k) (Def. 3)."""
    A = rand_tt((9, 8, 7, 6), (3, 4, 3), 21)
    A = W.add_noise(A, 0.05, np.random.default_rng(3))
    ranks = (3, 4, 3)
    taus = _unfolding_tails(A, ranks)
    nA = np.linalg.norm(A)
    e_svd = oracle.tt_error(A, oracle.tt_svd(A, ranks=ranks)) * nA
    assert e_svd <= np.sqrt(sum(taus)) * (1 + 1e-12)
    assert e_svd >= np.sqrt(max(taus)) * (1 - 1e-12)
    for q in (0, 1, 3):
        e = oracle.tt_error(A, oracle.tt_rbki(A, ranks, 3, q, seed=q)) * nA
        assert e >= np.sqrt(max(taus)) * (1 - 1e-12)


def test_tail_energy_closed_form():
    s = np.array([5.0, 3.0, 2.0, 1.0, 0.5])
    M = rand_matrix(5, 9, 1.0, 0)           # orthonormal-ish frame
    U, _, Vt = np.linalg.svd(M, full_matrices=False)
    X = (U * s) @ Vt
    assert abs(oracle.tail_energy(X, 3) - (4 + 1 + 0.25)) < 1e-12
    assert abs(oracle.tail_energy(X, 1) - np.sum(s ** 2)) < 1e-12


# ---------------------------------------------------------------- Krylov basis
@pytest.mark.parametrize("m,n,b,q,ratio", [(30, 200, 4, 2, 0.9), (25, 120, 3, 3, 0.85)])
def test_krylov_span_matches_raw_powers(m, n, b, q, ratio):
    """span(Q) equals the span of the raw block Krylov matrix
    [C W, (C C^T) C W, ..., (C C^T)^q C W], built naively and orthonormalised
    by Householder QR instead of the oracle's recurrence."""
    C = rand_matrix(m, n, ratio, 7)
    Omega = np.random.default_rng(8).standard_normal((n, b))
    Q = O.krylov_basis(C, Omega, q)
    blocks = []
    Y = C @ Omega
    for _ in range(q + 1):
        blocks.append(Y / np.linalg.norm(Y, axis=0))
        Y = C @ (C.T @ Y)
    QK, _ = np.linalg.qr(np.hstack(blocks))
    assert Q.shape == QK.shape
    assert projector_gap(Q, QK) < 1e-8
    assert np.max(np.abs(Q.T @ Q - np.eye(Q.shape[1]))) < 1e-13


def test_q0_is_randomized_range_finder():
    """q = 0 reduces to Halko et al. Alg. 4.1 (Q = qr(C W)) followed by
    Alg. 5.1 (SVD of Q^T C), written here with Householder QR."""
    C = rand_matrix(40, 300, 0.8, 3)
    r, b = 5, 9
    Omega = np.random.default_rng(4).standard_normal((300, b))
    U, R, _ = O.rbki_mode(C, r, Omega, 0)
    Qh, _ = np.linalg.qr(C @ Omega)
    Ub, _, _ = np.linalg.svd(Qh.T @ C)
    Uh = Qh @ Ub[:, :r]
    assert projector_gap(U, Uh) < 1e-10
    assert np.max(np.abs(U @ R - Uh @ (Uh.T @ C))) < 1e-12


# ---------------------------------------------------------------- invariants
def _noisy(dims, ranks, seed, level):
    A = rand_tt(dims, ranks, seed)
    return W.add_noise(A, level, np.random.default_rng(seed + 1))


def test_left_orthogonal_cores_and_projection_identity():
    """Cores 1..d-1 are left-orthogonal, so A_hat is an orthogonal projection
    of A and ||A||^2 - ||A_hat||^2 = ||A - A_hat||^2 (proof of Thm 3)."""
    A = _noisy((10, 9, 8, 7), (4, 5, 3), 31, 0.1)
    for q in (0, 2):
        cores = oracle.tt_rbki(A, (4, 5, 3), 3, q, seed=5)
        for G in cores[:-1]:
            assert oracle.left_orthogonality_defect(G) < 1e-13
        Ah = oracle.tt_full(cores)
        lhs = np.sum(A ** 2) - np.sum(Ah ** 2)
        rhs = np.sum((A - Ah) ** 2)
        assert abs(lhs - rhs) < 1e-10 * np.sum(A ** 2)


def test_captured_energy_monotone_in_q_and_p():
    """Rayleigh-Ritz picks the best rank-r subspace of span(Q); spans are
    nested in q, and in p for column-nested Omega, so the captured energy
    ||U^T C||^2 cannot decrease."""
    C = rand_matrix(60, 400, 0.93, 12) + 0.02 * np.random.default_rng(1).standard_normal((60, 400))
    r = 6
    prev = -1.0
    for q in range(5):
        U, R, _ = O.rbki_mode(C, r, omega_from_seed(17, 0, 400, r + 3), q)
        e = np.sum(R ** 2)
        assert e >= prev * (1 - 1e-13)
        prev = e
    prev = -1.0
    for p in range(0, 8):
        U, R, _ = O.rbki_mode(C, r, omega_from_seed(17, 0, 400, r + p), 1)
        e = np.sum(R ** 2)
        assert e >= prev * (1 - 1e-13)
        prev = e
    # and never above the optimum (Eckart-Young)
    s = np.linalg.svd(C, compute_uv=False)
    assert prev <= np.sum(s[:r] ** 2) * (1 + 1e-12)


def test_tt_full_matches_generator_contraction():
    rng = np.random.default_rng(6)
    cores = W.random_tt_cores((4, 5, 6, 3), (2, 3, 2), rng)
    assert np.max(np.abs(oracle.tt_full(cores) - W.dense_from_cores(cores))) < 1e-12
    A = rng.standard_normal((4, 5, 6, 3))
    brute = np.linalg.norm(A - W.dense_from_cores(cores)) / np.linalg.norm(A)
    assert abs(oracle.tt_error(A, cores) - brute) < 1e-14
    cores2 = W.random_tt_cores((4, 5, 6, 3), (3, 2, 2), rng)
    full2 = W.dense_from_cores(cores2)
    brute2 = np.linalg.norm(W.dense_from_cores(cores) - full2) / np.linalg.norm(full2)
    assert abs(oracle.tt_distance(cores, cores2) - brute2) < 1e-14


@pytest.mark.parametrize("dims,ranks,want", [
    ((1, 5, 6, 4), (3, 3, 2), [1, 1, 3, 2, 1]),    # first mode of size one
    ((5, 1, 6, 4), (2, 2, 3), [1, 2, 2, 3, 1]),    # a middle mode of size one
    ((4, 5, 1), (3, 1), [1, 3, 1, 1]),             # last mode of size one
    ((7, 8, 9), (1, 1), [1, 1, 1, 1]),             # rank one
])
def test_exact_recovery_degenerate_shapes(dims, ranks, want):
    """Modes of size one and rank one.  Def. 2's clamp bounds each bond by
    the product of the modes on either side (r_1' = 1 next to a first mode
    of size one, whatever r_1 asks for).  A tensor of that TT rank is
    recovered exactly, with no oversampling and no power as well as with
    both, and every core has the clamped shape."""
    A = rand_tt(dims, want[1:-1], 11)
    for p, q in ((0, 0), (2, 1)):
        cores = oracle.tt_rbki(A, ranks, p, q, seed=4)
        assert [c.shape for c in cores] == [(want[k], dims[k], want[k + 1]) for k in range(len(dims))]
        assert oracle.tt_error(A, cores) < 1e-12


def test_clamp_ranks():
    assert oracle.clamp_ranks((16, 16, 16, 16), (4, 4, 4)) == [1, 4, 4, 4, 1]
    assert oracle.clamp_ranks((3, 5, 4), (10, 10)) == [1, 3, 4, 1]
    assert oracle.clamp_ranks((256, 256, 64, 32), (30, 30, 30)) == [1, 30, 30, 30, 1]
    assert oracle.clamp_ranks((2, 2, 2, 2), (9, 9, 9)) == [1, 2, 4, 2, 1]


# ---------------------------------------------------------------- Omega generator
def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(t, 16) for t in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = philox4x32_10(r[0:4], r[4:6])
        assert [int(v) for v in out] == r[6:10]


def test_omega_is_standard_gaussian_and_nested():
    n = 50000
    Om = omega_from_seed(123, 2, n, 7)
    x = Om.ravel()
    assert abs(x.mean()) < 0.01 and abs(x.var() - 1) < 0.01
    assert scipy.stats.kstest(x, "norm").pvalue > 1e-3
    corr = np.corrcoef(Om.T)
    assert np.max(np.abs(corr - np.eye(7))) < 0.03
    # column nesting in b, row slicing, determinism, per-mode independence
    assert np.array_equal(omega_from_seed(123, 2, n, 5), Om[:, :5])
    assert np.array_equal(omega_from_seed(123, 2, n, 7, 1000, 1200), Om[1000:1200])
    assert np.array_equal(omega_from_seed(123, 2, n, 7), Om)
    assert np.max(np.abs(np.corrcoef(Om[:, 0], omega_from_seed(123, 3, n, 1)[:, 0])[0, 1])) < 0.03
    assert not np.array_equal(omega_from_seed(124, 2, 100, 7), Om[:100])


def test_omega_uniforms_exact_in_binary32():
    """u(x) = ((x >> 9) + 1/2) 2^-23 has at most 24 significant bits."""
    x = np.array([0, 1, 511, 512, 2 ** 32 - 1, 123456789], dtype=np.uint64)
    u = ((x >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)
    assert np.all((u > 0) & (u < 1))


# ---------------------------------------------------------------- statistical sanity
def test_config1_close_to_tt_svd():
    """Configuration 1 (16^4, TT ranks 4, 1e-3 noise): TT-rBKI reaches the
    TT-SVD error to a fraction of a percent (Sec. 4 observations)."""
    w = W.CONFIGS[1]
    A = W.make_tensor(w)
    e = oracle.tt_error(A, oracle.tt_rbki(A, w.ranks, w.oversample, w.q, seed=w.omega_seed))
    e_svd = oracle.tt_error(A, oracle.tt_svd(A, ranks=w.ranks))
    assert e_svd <= e <= 1.001 * e_svd
    assert 5e-4 < e < 2e-3


# ---------------------------------------------------------------- planted mistakes
def _pins_fail(monkeypatch_target=None):
    """Run a small pin battery; return the names of pins that fail."""
    failed = []
    A = rand_tt((6, 7, 8, 5), (3, 4, 2), 11)
    try:
        if oracle.tt_error(A, O.tt_rbki(A, (3, 4, 2), 2, 1, seed=3)) > 1e-12:
            failed.append("exact")
    except Exception:
        failed.append("exact")
    C = rand_matrix(30, 200, 0.9, 7)
    Om = np.random.default_rng(8).standard_normal((200, 4))
    try:
        Q = O.krylov_basis(C, Om, 2)
        blocks, Y = [], C @ Om
        for _ in range(3):
            blocks.append(Y / np.linalg.norm(Y, axis=0))
            Y = C @ (C.T @ Y)
        QK, _ = np.linalg.qr(np.hstack(blocks))
        if Q.shape != QK.shape or projector_gap(Q, QK) > 1e-8 or \
                np.max(np.abs(Q.T @ Q - np.eye(Q.shape[1]))) > 1e-13:
            failed.append("krylov")
    except Exception:
        failed.append("krylov")
    B = np.random.default_rng(5).standard_normal((8, 8, 8))
    try:
        if oracle.tt_distance(O.tt_rbki(B, (4, 4), 4, 1, seed=9), oracle.tt_svd(B, ranks=(4, 4))) > 1e-12:
            failed.append("exhaustion")
    except Exception:
        failed.append("exhaustion")
    return failed


def test_pins_pass_unmutated():
    assert _pins_fail() == []


def test_mutation_bottom_singular_vectors(monkeypatch):
    real = O.orth_top

    def wrong(Z, c):
        U, _, _ = np.linalg.svd(Z, full_matrices=False)
        return U[:, U.shape[1] - c:]
    monkeypatch.setattr(O, "orth_top", wrong)
    assert _pins_fail() != []
    monkeypatch.setattr(O, "orth_top", real)


def test_mutation_dropped_power(monkeypatch):
    """A Krylov step that forgets the C C^T factor (Z = X)."""
    def krylov_no_power(C, Omega, q):
        m, n = C.shape
        b = Omega.shape[1]
        D = min(m, n)
        X = O.orth_top(C @ Omega, min(b, D))
        Q = X
        for _ in range(q):
            if Q.shape[1] >= D:
                break
            Z = C @ (C.T @ Omega[:, :X.shape[1]])     # mistake: restarts from Omega
            for _ in range(2):
                Z = Z - Q @ (Q.T @ Z)
            X = O.orth_top(Z, min(b, D - Q.shape[1]))
            Q = np.hstack([Q, X])
        return Q
    monkeypatch.setattr(O, "krylov_basis", krylov_no_power)
    assert "krylov" in _pins_fail()


def test_mutation_projection_sign(monkeypatch):
    """Block Gram-Schmidt with the wrong sign."""
    def krylov_plus(C, Omega, q):
        m, n = C.shape
        b = Omega.shape[1]
        D = min(m, n)
        X = O.orth_top(C @ Omega, min(b, D))
        Q = X
        for _ in range(q):
            if Q.shape[1] >= D:
                break
            Z = C @ (C.T @ X)
            for _ in range(2):
                Z = Z + Q @ (Q.T @ Z)
            X = O.orth_top(Z, min(b, D - Q.shape[1]))
            Q = np.hstack([Q, X])
        return Q
    monkeypatch.setattr(O, "krylov_basis", krylov_plus)
    assert "krylov" in _pins_fail()


def test_mutation_transposed_remainder(monkeypatch):
    """Remainder taken from the wrong side of the unfolding."""
    real = O.rbki_mode

    def wrong(C, r, Omega, q):
        U, R, s = real(C, r, Omega, q)
        return U, (U.T @ C)[:, ::-1].copy(), s
    monkeypatch.setattr(O, "rbki_mode", wrong)
    assert "exact" in _pins_fail()
