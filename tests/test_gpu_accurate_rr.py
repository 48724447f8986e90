"""Option accurate_rr: Rayleigh-Ritz through the singular vectors of
B = Q^T C (Alg. 3 steps 6-8) with the compensated Gram, FP64 Cholesky and
one-sided Jacobi of rr_svd.cu.  FP32 form against the oracle (same Omega)
within relative TT distance 1e-4; BF16 form within the error criterion; on
a power-function tensor whose rank-12 truncation error (4.6e-5) lies below
what an FP32 eigendecomposition of the squared Gram resolves, the option
reaches the FP64 oracle's error."""
import numpy as np
import pytest

import oracle
from paper_2308_01480_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    # dims, generating ranks, target ranks, p, q, noise
    ((16, 16, 16, 16), (4, 4, 4), (4, 4, 4), 5, 2, 1e-3),
    ((37, 29, 41), (5, 6), (5, 6), 3, 3, 0.05),
    ((5, 4, 6, 3, 7, 4), (3, 4, 5, 4, 3), (3, 4, 5, 4, 3), 2, 1, 0.02),
    ((20, 30, 40, 10), (15, 15, 5), (15, 15, 5), 4, 2, 0.03),
    ((1100, 6, 5, 4), (8, 6, 4), (8, 6, 4), 4, 2, 0.05),
]


@pytest.fixture(scope="module")
def tt():
    import paper_2308_01480_gb300 as tt
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    tt._native.lib()
    return tt


def _noisy(dims, gr, seed, noise):
    rng = np.random.default_rng(seed)
    A = W.dense_from_cores(W.random_tt_cores(dims, gr, rng))
    return W.add_noise(A, noise, rng)


def _run(tt, A, ranks, p, q, storage="f32", omegas=None, seed=0, method=None, **kw):
    t = torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32)).cuda()
    code = tt.TT_F32
    if storage == "bf16":
        t = t.to(torch.bfloat16)
        code = tt.TT_BF16
    opts = tt.options(storage=code, method=tt.TT_METHOD_RBKI if method is None else method, **kw)
    om = [torch.from_numpy(o).cuda() for o in omegas] if omegas is not None else None
    cores, _ = tt.decompose(t, ranks, p, q, omega_seed=seed, omegas=om, opts=opts)
    torch.cuda.synchronize()
    assert tt.device_status(tt.decompose.last_workspace) == 0
    return [c.cpu().double().numpy() for c in cores]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("exhaust", [True, False])
def test_accurate_fp32_matches_oracle(tt, case, exhaust):
    dims, gr, ranks, p, q, noise = case
    A = _noisy(dims, gr, 17, noise)
    rr = oracle.clamp_ranks(dims, ranks)
    om = W.explicit_omegas(dims, rr, p, 23)
    ref = oracle.tt_rbki(A.astype(np.float32), ranks, p, q, omegas=om)
    tt.profile_begin(event_timing=False)
    got = _run(tt, A, ranks, p, q, omegas=om, exhaust_gram=exhaust, accurate_rr=True)
    fams = tt.profile_end()
    assert "rr_svd" in fams and "gram_df" in fams
    assert oracle.tt_distance(got, ref) <= 1e-4
    for G in got[:-1]:
        assert oracle.left_orthogonality_defect(G) < 1e-4


def test_accurate_rsi_matches_oracle(tt):
    dims, gr, ranks, p, q, noise = CASES[3]
    A = _noisy(dims, gr, 19, noise)
    rr = oracle.clamp_ranks(dims, ranks)
    om = W.explicit_omegas(dims, rr, p, 29)
    ref = oracle.tt_rsi(A.astype(np.float32), ranks, p, q, omegas=om)
    got = _run(tt, A, ranks, p, q, omegas=om, method=tt.TT_METHOD_RSI, accurate_rr=True)
    assert oracle.tt_distance(got, ref) <= 1e-4


@pytest.mark.parametrize("case", CASES[:4])
def test_accurate_bf16_error_criterion(tt, case):
    dims, gr, ranks, p, q, noise = case
    A = _noisy(dims, gr, 31, noise)
    eps_ref = oracle.tt_error(A, oracle.tt_rbki(A, ranks, p, q, seed=3))
    got = _run(tt, A, ranks, p, q, storage="bf16", seed=3, remainder=tt.TT_F32, accurate_rr=True)
    assert oracle.tt_error(A, got) <= 1.05 * eps_ref + 1e-4


def test_accurate_rr_below_fp32_floor(tt):
    """30^4 power function (h = 5), r = 12, p = 2, q = 2: the FP64 oracle's
    error is 4.6e-5, the singular values at the cut ~1e-5 of the largest.
    The first mode's Gram C C^T (30 x 30) is singular to FP64 accuracy
    (condition ~1e23), so this case also checks that the Cholesky of the
    Gram pivots and stops at its numerical rank: unpivoted, rounding-size
    pivots scatter the error between 1.0 and 1.25 times the oracle's."""
    A = W.power_tensor_h((30, 30, 30, 30), 5.0)
    ranks = (12, 12, 12)
    eps_ref = oracle.tt_error(A, oracle.tt_rbki(A, ranks, 2, 2, seed=1))
    got = _run(tt, A, ranks, 2, 2, seed=1, accurate_rr=True)
    assert oracle.tt_error(A, got) <= 1.02 * eps_ref


def test_accurate_rank_deficient_stays_orthonormal(tt):
    """Target ranks above the TT ranks: B is numerically rank-deficient, the
    wanted vectors past its rank are completed orthonormally."""
    A = _noisy((12, 10, 9, 8), (3, 4, 2), 8, 0.0)
    got = _run(tt, A, (6, 6, 6), 3, 2, seed=4, accurate_rr=True)
    assert oracle.tt_error(A, got) < 2e-5
    for G in got[:-1]:
        assert oracle.left_orthogonality_defect(G) < 1e-4
