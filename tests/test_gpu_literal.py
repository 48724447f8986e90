"""The paper's steps taken literally (option paper_literal): Alg. 3 with its
right-side Krylov matrix and the first-r truncation of an unpivoted QR,
Alg. 4 likewise, Alg. 2 for q = 0; against the oracle's literal forms
(oracle.tt_rbki_literal / tt_rsi_literal) with the same Omega.  FP32 form
within relative TT distance 1e-4, BF16 form within the error criterion."""
import numpy as np
import pytest

import oracle
from paper_2308_01480_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    # dims, generating ranks, target ranks, p, noise
    ((16, 16, 16, 16), (4, 4, 4), (4, 4, 4), 5, 1e-2),
    ((37, 29, 41), (5, 6), (5, 6), 3, 0.05),
    ((5, 4, 6, 3, 7, 4), (3, 4, 5, 4, 3), (3, 4, 5, 4, 3), 2, 0.02),
    ((20, 30, 40, 10), (15, 15, 5), (15, 15, 5), 4, 0.03),
    ((24, 32, 40, 16), (6, 8, 4), (6, 8, 4), 4, 0.03),
]


@pytest.fixture(scope="module")
def tt():
    import paper_2308_01480_gb300 as tt
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    tt._native.lib()
    return tt


def _tensor(dims, gr, seed, noise):
    rng = np.random.default_rng(seed)
    A = W.dense_from_cores(W.random_tt_cores(dims, gr, rng))
    return W.add_noise(A, noise, rng)


def _run(tt, A, ranks, p, q, method, storage, omegas=None, seed=0):
    t = torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32)).cuda()
    code = tt.TT_F32
    if storage == "bf16":
        t = t.to(torch.bfloat16)
        code = tt.TT_BF16
    opts = tt.options(storage=code, method=method, paper_literal=True)
    om = [torch.from_numpy(o).cuda() for o in omegas] if omegas is not None else None
    cores, rr = tt.decompose(t, ranks, p, q, omega_seed=seed, omegas=om, opts=opts)
    torch.cuda.synchronize()
    assert tt.device_status(tt.decompose.last_workspace) == 0
    return [c.cpu().double().numpy() for c in cores], rr


def _oracle(method):
    import paper_2308_01480_gb300 as tt
    return oracle.tt_rsi_literal if method == tt.TT_METHOD_RSI else oracle.tt_rbki_literal


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("q", [0, 1, 2])
@pytest.mark.parametrize("rsi", [False, True])
def test_literal_fp32_matches_oracle(tt, case, q, rsi):
    dims, gr, ranks, p, noise = case
    method = tt.TT_METHOD_RSI if rsi else tt.TT_METHOD_RBKI
    A = _tensor(dims, gr, 61, noise)
    rr = oracle.clamp_ranks(dims, ranks)
    om = W.explicit_omegas(dims, rr, p, 67)
    ref = _oracle(method)(A.astype(np.float32), ranks, p, q, omegas=om)
    got, rr_gpu = _run(tt, A, ranks, p, q, method, "f32", omegas=om)
    assert rr_gpu == rr
    assert oracle.tt_distance(got, ref) <= 1e-4
    for G in got[:-1]:
        assert oracle.left_orthogonality_defect(G) < 1e-4


@pytest.mark.parametrize("case", CASES)
def test_literal_bf16_error_criterion(tt, case):
    dims, gr, ranks, p, noise = case
    A = _tensor(dims, gr, 71, noise)
    eps_ref = oracle.tt_error(A, oracle.tt_rbki_literal(A, ranks, p, 1, seed=9))
    got, _ = _run(tt, A, ranks, p, 1, tt.TT_METHOD_RBKI, "bf16", seed=9)
    assert oracle.tt_error(A, got) <= 1.05 * eps_ref + 1e-4


def test_literal_exact_recovery(tt):
    """Target ranks equal to the TT ranks.  Without oversampling the first-r
    sketch (C C^T)^s C W(:, 1:r) carries the spread of C's r singular values
    (cubed for one power) times the conditioning of a square Gaussian sketch,
    and its FP32 orthonormalisation resolves the weakest direction only to
    about u times that condition number: FP32 recovery to 5e-4 (the FP64
    oracle's literal forms reach 1e-12 on the same tensors)."""
    rng = np.random.default_rng(8)
    dims, ranks = (12, 10, 9, 8), (3, 4, 2)
    A = W.dense_from_cores(W.random_tt_cores(dims, ranks, rng))
    for q in (0, 1, 2):
        got, _ = _run(tt, A, ranks, 3, q, tt.TT_METHOD_RBKI, "f32", seed=4)
        assert oracle.tt_error(A, got) < 5e-4, q
        assert oracle.tt_error(A, oracle.tt_rbki_literal(A, ranks, 3, q, seed=4)) < 1e-12
