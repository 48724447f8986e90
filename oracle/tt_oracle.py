"""Plain float64 restatement of TT-SVD (Alg. 1), TT-rBKI (Alg. 3) and
TT-rSI (Alg. 4); TT-rSVD (Alg. 2) is TT-rBKI with q = 0.

TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline leg and reference arm (both time it on the host
cores).  Never imported by the CUDA library.

Notation follows the paper: a tensor A of order d with mode sizes I_1..I_d,
TT ranks r_0 = r_d = 1 (Def. 2).  Tensors are row-major with i_1 the slowest
index, so the unfolding at mode k is the free view
    C = reshape(R, [r_{k-1} I_k, I_{k+1} ... I_d])
(Alg. 3 step 2).  MATLAB's column-major reshape differs only by a row and
column permutation of C, which leaves singular values and the reconstructed
tensor unchanged.

Readings of the paper taken here (each also listed in the design notes):
  * Krylov side: Alg. 3 step 4 builds K from A^T A on the right.  Here the
    left form K = [C W, (C C^T) C W, ..., (C C^T)^q C W] is used (W = Omega),
    whose span contains span(A U) of Alg. 3 steps 5-6 and keeps the basis at
    r_{k-1} I_k rows.
  * Truncation: Alg. 3 steps 7-8 keep the first r_k columns of an unpivoted
    QR.  Here the block is truncated by Rayleigh-Ritz: the top-r_k left
    singular vectors of Q^T C (Musco & Musco's block Krylov method, which the
    paper builds on in Sec. 2.3).
  * Infeasible ranks are clamped, r_k' = min(r_k, r_{k-1}' I_k, prod_{j>k} I_j).
  * Krylov exhaustion: once the basis spans D = min(m, n) directions no
    further block is added; a block that would overshoot D keeps only the
    top (D - cols) left singular directions of the projected block.
  * Gaussian Omega is drawn fresh per mode with r_k' + p columns (Alg. 3
    step 3); the seeded form uses philox.omega_from_seed.

Every step below uses numpy's matmul and LAPACK SVD as library primitives,
with no blocking, fusion or reordering beyond the algorithm's own steps.
"""
import numpy as np

from .philox import omega_from_seed


def clamp_ranks(dims, ranks):
    """Feasible TT ranks [r_0', r_1', ..., r_d'] with r_0' = r_d' = 1.

    r_k' = min(r_k, r_{k-1}' I_k, I_{k+1} ... I_d)  (Def. 2; Alg. 3 input).
    """
    d = len(dims)
    if len(ranks) != d - 1:
        raise ValueError("need d-1 ranks")
    out = [1]
    for k in range(d - 1):
        m = out[-1] * int(dims[k])
        n = int(np.prod([int(x) for x in dims[k + 1:]], dtype=np.int64))
        out.append(int(min(int(ranks[k]), m, n)))
    out.append(1)
    return out


def unfold(R, m):
    """Alg. 3 step 2: reshape the remainder to m rows (row-major view)."""
    return np.reshape(R, (m, -1))


def orth_top(Z, c):
    """Orthonormal basis of the top-c left singular directions of Z.

    When c equals the column count of a full-rank Z this is just an
    orthonormal basis of its column span (the economy QR of Alg. 3 step 5).
    """
    U, _, _ = np.linalg.svd(Z, full_matrices=False)
    return U[:, :c]


def krylov_basis(C, Omega, q):
    """Orthonormal basis Q of the left block Krylov space of C.

    span(Q) = span[C W, (C C^T) C W, ..., (C C^T)^q C W]   (Alg. 3 step 4,
    left reading), built block by block: each new block is C (C^T X_{j-1})
    with the previous blocks projected out twice, then orthonormalised,
    projected once more and orthonormalised again.
    The loop stops once the basis has D = min(m, n) columns.
    Returns Q with min(D, (q+1) b) columns.
    """
    m, n = C.shape
    b = Omega.shape[1]
    D = min(m, n)
    Y = C @ Omega                       # Alg. 3 step 3-4: sketch C W
    X = orth_top(Y, min(b, D))
    Q = X
    for _ in range(q):
        if Q.shape[1] >= D:
            break
        Z = C @ (C.T @ X)               # one more power of C C^T
        for _ in range(2):              # block Gram-Schmidt, twice
            Z = Z - Q @ (Q.T @ Z)
        c = min(b, D - Q.shape[1])
        X = orth_top(Z, c)
        # Once more on the normalised block: when Z was pure cancellation
        # (range(C) already inside span(Q), e.g. exact-rank inputs) it is
        # orthogonal to Q only relative to its own tiny norm.
        X = orth_top(X - Q @ (Q.T @ X), c)
        Q = np.hstack([Q, X])
    return Q


def rbki_mode(C, r, Omega, q):
    """One mode of TT-rBKI on the unfolding C (m x n).

    Returns (U, R, sigma): U (m x r) the left factor that becomes core k
    (Alg. 3 step 9), R = U^T C (r x n) the next remainder (Alg. 3 step 10),
    and sigma the Ritz singular values of Q^T C in descending order.
    """
    Q = krylov_basis(C, Omega, q)
    B = Q.T @ C                         # Rayleigh-Ritz: project C on span(Q)
    Ub, sigma, _ = np.linalg.svd(B, full_matrices=False)
    U = Q @ Ub[:, :r]
    R = U.T @ C
    return U, R, sigma


def _tt_randomized(A, ranks, oversample, q, omegas, seed, mode_fn):
    """The mode loop shared by Alg. 3 and Alg. 4: unfold, draw Omega, run
    mode_fn(C, r, Omega, q) -> (U, R, sigma), store U as the core, carry R."""
    A = np.asarray(A, dtype=np.float64)
    dims = A.shape
    d = len(dims)
    if d < 2:
        raise ValueError("order must be >= 2")
    rr = clamp_ranks(dims, ranks)
    R = A
    cores = []
    for k in range(d - 1):
        m = rr[k] * dims[k]
        C = unfold(R, m)
        n = C.shape[1]
        b = rr[k + 1] + int(oversample)
        if omegas is not None:
            Omega = np.asarray(omegas[k], dtype=np.float64)
        else:
            Omega = omega_from_seed(seed, k, n, b)
        if Omega.shape != (n, b):
            raise ValueError(f"omega {k} has shape {Omega.shape}, want {(n, b)}")
        U, R, _ = mode_fn(C, rr[k + 1], Omega, q)
        cores.append(U.reshape(rr[k], dims[k], rr[k + 1]))
    cores.append(np.reshape(R, (rr[d - 1], dims[d - 1], 1)))
    return cores


def tt_rbki(A, ranks, oversample, q, omegas=None, seed=None):
    """TT-rBKI (Alg. 3) in float64.

    A        : ndarray of order d >= 2 (converted to float64).
    ranks    : target TT ranks r_1..r_{d-1}; clamped as in clamp_ranks.
    oversample, q : the paper's p and q.
    omegas   : optional list of d-1 Gaussian matrices, omegas[k] of shape
               (I_{k+1}...I_d, r_k' + p); otherwise drawn from ``seed`` with
               omega_from_seed(seed, k, n, b).
    Returns the list of d cores, core k of shape (r_{k-1}', I_k, r_k').
    With q = 0 this is TT-rSVD (Alg. 2) under the Rayleigh-Ritz reading.
    """
    return _tt_randomized(A, ranks, oversample, q, omegas, seed, rbki_mode)


def subspace_basis(C, Omega, q):
    """Orthonormal basis of the subspace iteration of Alg. 4 (steps 4-11):
    Y = C W, Q_0 = qr(Y); then q times Yhat = C^T Q, Qhat = qr(Yhat),
    Y = C Qhat, Q = qr(Y).  Its span is that of (C C^T)^q C W.  Under the
    Krylov dimension cap the left factors keep min(b, D) columns (the top
    singular directions), D = min(m, n); once Q spans D columns further
    steps cannot change its span and are skipped.
    """
    m, n = C.shape
    b = Omega.shape[1]
    D = min(m, n)
    c = min(b, D)
    Q = orth_top(C @ Omega, c)              # steps 4-5
    for _ in range(q):
        if c >= D:
            break
        Qh, _ = np.linalg.qr(C.T @ Q)       # steps 7-8
        Q = orth_top(C @ Qh, c)             # steps 9-10
    return Q


def rsi_mode(C, r, Omega, q):
    """One mode of TT-rSI (Alg. 4) on the unfolding C: the subspace basis,
    then the top-r left singular vectors of Q^T C (Rayleigh-Ritz, the same
    reading of step 12 as for Alg. 3).  Returns (U, R = U^T C, sigma)."""
    Q = subspace_basis(C, Omega, q)
    B = Q.T @ C
    Ub, sigma, _ = np.linalg.svd(B, full_matrices=False)
    U = Q @ Ub[:, :r]
    R = U.T @ C
    return U, R, sigma


def tt_rsi(A, ranks, oversample, q, omegas=None, seed=None):
    """TT-rSI (Alg. 4) in float64; arguments and result as tt_rbki."""
    return _tt_randomized(A, ranks, oversample, q, omegas, seed, rsi_mode)


def literal_rbki_mode(C, r, Omega, q):
    """One mode of Alg. 3 taken literally (the right-side Krylov matrix and
    the first-r truncation of steps 7-8; a study option beside the
    Rayleigh-Ritz reading used by rbki_mode):
        K = [C^T C W, (C^T C)^2 W, ..., (C^T C)^q W]     step 4
        U = qr(K, 0)                                      step 5
        Y = C U                                           step 6
        Q = qr(Y, 0)(:, 1:r)                              steps 7-8
    With q = 0 the matrix K is empty; that case is Alg. 2 (TT-rSVD) taken
    literally, Y = C W (steps 4-6 of Alg. 2).  numpy's QR is Householder
    based (LAPACK geqrf), the economy form of MATLAB's qr(., 0).
    Returns (Q, R = Q^T C, None)."""
    if q == 0:
        Y = C @ Omega
    else:
        blocks = []
        B = Omega
        for _ in range(q):
            B = C.T @ (C @ B)               # (C^T C)^j W
            blocks.append(B)
        K = np.hstack(blocks)
        U, _ = np.linalg.qr(K)              # economy QR
        Y = C @ U
    Qy, _ = np.linalg.qr(Y)
    Q = Qy[:, :r]
    return Q, Q.T @ C, None


def literal_rsi_mode(C, r, Omega, q):
    """One mode of Alg. 4 taken literally: Q_0 = qr(C W) (steps 4-5); q times
    Yhat = C^T Q, Qhat = qr(Yhat), Y = C Qhat, Q = qr(Y) (steps 6-11); then
    Q = Q(:, 1:r) (step 12).  Returns (Q, R = Q^T C, None)."""
    Q, _ = np.linalg.qr(C @ Omega)
    for _ in range(q):
        Qh, _ = np.linalg.qr(C.T @ Q)
        Q, _ = np.linalg.qr(C @ Qh)
    Q = Q[:, :r]
    return Q, Q.T @ C, None


def tt_rbki_literal(A, ranks, oversample, q, omegas=None, seed=None):
    """TT-rBKI with Alg. 3 steps 4-8 taken literally (literal_rbki_mode);
    arguments and result as tt_rbki.  q = 0 is Alg. 2 taken literally."""
    return _tt_randomized(A, ranks, oversample, q, omegas, seed, literal_rbki_mode)


def tt_rsi_literal(A, ranks, oversample, q, omegas=None, seed=None):
    """TT-rSI with Alg. 4 taken literally (literal_rsi_mode)."""
    return _tt_randomized(A, ranks, oversample, q, omegas, seed, literal_rsi_mode)


def tt_svd(A, ranks=None, eps=None):
    """TT-SVD (Alg. 1) in float64.

    Either fixed ``ranks`` (clamped as in clamp_ranks) or the prescribed
    accuracy ``eps``: each unfolding is truncated to the smallest rank whose
    discarded tail has norm <= delta = eps ||A|| / sqrt(d-1) (Alg. 1 step 1,
    step 4).
    """
    A = np.asarray(A, dtype=np.float64)
    dims = A.shape
    d = len(dims)
    if (ranks is None) == (eps is None):
        raise ValueError("give exactly one of ranks, eps")
    delta = None
    if eps is not None:
        delta = eps / np.sqrt(d - 1) * np.linalg.norm(A)
    R = A
    r_prev = 1
    cores = []
    for k in range(d - 1):
        C = unfold(R, r_prev * dims[k])
        U, s, Vt = np.linalg.svd(C, full_matrices=False)
        if ranks is not None:
            r = int(min(int(ranks[k]), s.size))
        else:
            tails = np.sqrt(np.cumsum((s ** 2)[::-1])[::-1])   # tails[j] = ||s[j:]||
            ok = np.nonzero(np.append(tails, 0.0)[1:] <= delta)[0]
            r = max(1, int(ok[0]) + 1)
        cores.append(U[:, :r].reshape(r_prev, dims[k], r))
        R = s[:r, None] * Vt[:r]          # carry S V^T forward (Alg. 1 step 6)
        r_prev = r
    cores.append(np.reshape(R, (r_prev, dims[d - 1], 1)))
    return cores


def _right_matrix(cores):
    """Contract cores[1:] into a matrix of shape (r_1, I_2 ... I_d)."""
    M = np.asarray(cores[-1], dtype=np.float64).reshape(cores[-1].shape[0], -1)
    for G in reversed(cores[1:-1]):
        G = np.asarray(G, dtype=np.float64)
        ra, I, rb = G.shape
        M = (G.reshape(ra * I, rb) @ M).reshape(ra, -1)
    return M


def tt_full(cores):
    """Dense tensor of a TT (Def. 2): Q_1 x_3^1 Q_2 x_3^1 ... x_3^1 Q_d."""
    dims = tuple(G.shape[1] for G in cores)
    G1 = np.asarray(cores[0], dtype=np.float64).reshape(dims[0], -1)
    return (G1 @ _right_matrix(cores)).reshape(dims)


def _chunked_diff_norms(first_a, right_a, first_b, right_b, chunk=64):
    """||Fa Ra - Fb Rb||^2 and ||Fb Rb||^2 by row chunks of the first mode."""
    num = 0.0
    den = 0.0
    for s in range(0, first_a.shape[0], chunk):
        xa = first_a[s:s + chunk] @ right_a if right_a is not None else first_a[s:s + chunk]
        xb = first_b[s:s + chunk] @ right_b
        num += float(np.sum((xa - xb) ** 2))
        den += float(np.sum(xb ** 2))
    return num, den


def tt_error(A, cores):
    """Relative error ||A - A_hat||_F / ||A||_F of Sec. 4, A_hat from cores.

    Evaluated directly on the dense difference, chunked over i_1, in float64,
    always against the given (float64) A.
    """
    A = np.asarray(A, dtype=np.float64)
    I1 = A.shape[0]
    Am = A.reshape(I1, -1)
    F = np.asarray(cores[0], dtype=np.float64).reshape(I1, -1)
    Rm = _right_matrix(cores)
    num, den = _chunked_diff_norms(Am, None, F, Rm)
    # _chunked_diff_norms measured ||A - A_hat||^2 and ||A_hat||^2
    return float(np.sqrt(num) / np.linalg.norm(Am))


def tt_distance(cores_a, cores_b):
    """Relative TT distance ||A_a - A_b||_F / ||A_b||_F (dense, chunked)."""
    I1 = cores_b[0].shape[1]
    Fa = np.asarray(cores_a[0], dtype=np.float64).reshape(I1, -1)
    Fb = np.asarray(cores_b[0], dtype=np.float64).reshape(I1, -1)
    num, den = _chunked_diff_norms(Fa, _right_matrix(cores_a), Fb, _right_matrix(cores_b))
    return float(np.sqrt(num / den)) if den > 0 else float(np.sqrt(num))


def tail_energy(X, j):
    """Def. 3: tau_j^2(X) = sum_{i >= j} sigma_i(X)^2 (j is 1-based)."""
    s = np.linalg.svd(np.asarray(X, dtype=np.float64), compute_uv=False)
    return float(np.sum(s[j - 1:] ** 2))


def left_orthogonality_defect(core):
    """max |U^T U - I| for U = reshape(core, [r_{k-1} I_k, r_k])."""
    ra, I, rb = core.shape
    U = np.asarray(core, dtype=np.float64).reshape(ra * I, rb)
    return float(np.max(np.abs(U.T @ U - np.eye(rb))))


def psnr(A, A_hat):
    """Peak signal-to-noise ratio of Sec. 4: 10 log10(N ||A_hat||_max^2 /
    ||A - A_hat||_F^2) with N the number of entries (the paper prints the
    third-order case I_1 I_2 I_3; the product of all mode sizes is the
    reading for any order) and ||A_hat||_max the largest absolute entry of
    the reconstruction, as printed.  Dense float64."""
    A = np.asarray(A, dtype=np.float64)
    A_hat = np.asarray(A_hat, dtype=np.float64)
    err2 = float(np.sum((A - A_hat) ** 2))
    peak = float(np.max(np.abs(A_hat)))
    return 10.0 * np.log10(A.size * peak * peak / err2)
