"""Whole-decomposition parity of the GPU path against the FP64 oracle.

FP32 form: the reconstructed TT must match the oracle's to relative
Frobenius distance 1e-4 when both get the same Omega.  BF16 form: the TT
relative error against the FP64 tensor must satisfy
eps_gpu <= 1.05 eps_oracle + 1e-4.
"""
import numpy as np
import pytest

import oracle
from paper_2308_01480_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4
# kernel families that only the Gram-power route launches: the Gram of a
# tall-enough unfolding, the power through it, the one-launch Krylov loop
GRAM_POWER_FAMILIES = {"gram_tc_tiled", "gram_simt_tiled", "gram_power", "krylov_cluster"}


@pytest.fixture(scope="module")
def tt():
    import paper_2308_01480_gb300 as tt
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    tt._native.lib()
    return tt


def gpu_decompose(tt, A, ranks, p, q, storage="f32", omegas=None, seed=0, exhaust=True, remainder=None,
                  gram_power=True):
    t = torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32)).cuda()
    code = tt.TT_F32
    if storage == "bf16":
        t = t.to(torch.bfloat16)
        code = tt.TT_BF16
    rem = None if remainder is None else (tt.TT_BF16 if remainder == "bf16" else tt.TT_F32)
    opts = tt.options(storage=code, remainder=rem, exhaust_gram=exhaust, gram_power=gram_power)
    om = [torch.from_numpy(o).cuda() for o in omegas] if omegas is not None else None
    cores, rr = tt.decompose(t, ranks, p, q, omega_seed=seed, omegas=om, opts=opts)
    torch.cuda.synchronize()
    assert tt.device_status(tt.decompose.last_workspace) == 0
    return [c.cpu().double().numpy() for c in cores], rr


def noisy_tt(dims, ranks, seed, level, kind="gaussian"):
    rng = np.random.default_rng(seed)
    A = W.dense_from_cores(W.random_tt_cores(dims, ranks, rng))
    return W.add_noise(A, level, rng, kind)


CASES = [
    # dims, generating ranks, target ranks, p, q, noise
    ((16, 16, 16, 16), (4, 4, 4), (4, 4, 4), 5, 2, 1e-3),
    ((6, 7, 8, 5), (3, 4, 2), (3, 4, 2), 2, 2, 0.05),
    ((37, 29, 41), (5, 6), (5, 6), 3, 3, 0.05),
    ((5, 4, 6, 3, 7, 4), (3, 4, 5, 4, 3), (3, 4, 5, 4, 3), 2, 1, 0.02),
    ((20, 30, 40, 10), (15, 15, 5), (15, 15, 5), 4, 2, 0.03),      # tall unfolding at mode 2
    ((64, 33, 65), (12, 9), (10, 8), 6, 3, 0.1),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("exhaust", [True, False])
def test_fp32_matches_oracle_explicit_omega(tt, case, exhaust):
    dims, gr, ranks, p, q, noise = case
    A = noisy_tt(dims, gr, 17, noise)
    rr = oracle.clamp_ranks(dims, ranks)
    om = W.explicit_omegas(dims, rr, p, 23)
    ref = oracle.tt_rbki(A.astype(np.float32), ranks, p, q, omegas=om)
    got, rr_gpu = gpu_decompose(tt, A, ranks, p, q, omegas=om, exhaust=exhaust)
    assert rr_gpu == rr
    assert [g.shape for g in got] == [r.shape for r in ref]
    assert oracle.tt_distance(got, ref) <= FP32_TOL
    for G in got[:-1]:
        assert oracle.left_orthogonality_defect(G) < 1e-4


@pytest.mark.parametrize("case", CASES[:4])
def test_fp32_matches_oracle_seed_form(tt, case):
    """Omega drawn on the device from the seed versus the oracle's own
    Philox4x32-10 / Box-Muller evaluation of the same definition."""
    dims, gr, ranks, p, q, noise = case
    A = noisy_tt(dims, gr, 5, noise)
    ref = oracle.tt_rbki(A.astype(np.float32), ranks, p, q, seed=77)
    got, _ = gpu_decompose(tt, A, ranks, p, q, seed=77)
    assert oracle.tt_distance(got, ref) <= FP32_TOL


@pytest.mark.parametrize("dims,ranks", [((16, 16, 16, 16), (4, 4, 4)), ((9, 10, 11, 12), (3, 5, 4)),
                                        ((3, 50), (2,))])
def test_exact_recovery_fp32(tt, dims, ranks):
    A = noisy_tt(dims, ranks, 9, 0.0)
    got, _ = gpu_decompose(tt, A, ranks, 3, 2, seed=1)
    # FP32 working accuracy: Gram-type products square the conditioning of
    # the unfoldings, so the error is a few u kappa^2 rather than u.
    assert oracle.tt_error(A, got) < 2e-5


# shapes whose unfoldings take the tensor-core passes in BF16 (n % 8 == 0)
CASES_TC = [
    ((24, 32, 40, 16), (6, 8, 4), (6, 8, 4), 4, 3, 0.03),
    ((48, 64, 64), (10, 12), (10, 12), 6, 2, 0.05),
    ((20, 40, 40, 32), (15, 15, 5), (15, 15, 5), 5, 2, 0.02),       # m = 600 at mode 2 (two-pass power)
    ((40, 40, 40, 40), (20, 20, 20), (20, 20, 20), 10, 4, 0.05),
]


@pytest.mark.parametrize("case", CASES + CASES_TC)
def test_bf16_error_criterion(tt, case):
    dims, gr, ranks, p, q, noise = case
    A = noisy_tt(dims, gr, 31, noise)
    eps_ref = oracle.tt_error(A, oracle.tt_rbki(A, ranks, p, q, seed=3))
    for rem in ("f32", "bf16"):
        if rem == "bf16" and noise < 0.01:
            # a BF16 remainder is rounded inside the retained subspace
            # (relative 2^-9 per entry), which exceeds a 1e-3 noise floor
            continue
        got, _ = gpu_decompose(tt, A, ranks, p, q, storage="bf16", seed=3, remainder=rem)
        eps = oracle.tt_error(A, got)
        assert eps <= 1.05 * eps_ref + 1e-4, (rem, eps, eps_ref)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("gram_power", [True, False])
def test_fp32_power_routes_match_oracle(tt, case, gram_power):
    """Both ways of applying (C C^T)^j: through the m x m Gram matrix formed
    once, and through alternating projections with C and C^T."""
    dims, gr, ranks, p, q, noise = case
    A = noisy_tt(dims, gr, 41, noise)
    rr = oracle.clamp_ranks(dims, ranks)
    om = W.explicit_omegas(dims, rr, p, 43)
    ref = oracle.tt_rbki(A.astype(np.float32), ranks, p, q, omegas=om)
    tt.profile_begin(event_timing=False)
    got, _ = gpu_decompose(tt, A, ranks, p, q, omegas=om, exhaust=False, gram_power=gram_power)
    fams = tt.profile_end()
    assert oracle.tt_distance(got, ref) <= FP32_TOL
    if not gram_power:
        assert not set(fams) & GRAM_POWER_FAMILIES


@pytest.mark.parametrize("case", CASES_TC)
@pytest.mark.parametrize("gram_power", [True, False])
def test_bf16_power_routes_error_criterion(tt, case, gram_power):
    dims, gr, ranks, p, q, noise = case
    A = noisy_tt(dims, gr, 47, noise)
    eps_ref = oracle.tt_error(A, oracle.tt_rbki(A, ranks, p, q, seed=5))
    tt.profile_begin(event_timing=False)
    got, _ = gpu_decompose(tt, A, ranks, p, q, storage="bf16", seed=5, gram_power=gram_power)
    fams = tt.profile_end()
    eps = oracle.tt_error(A, got)
    assert eps <= 1.05 * eps_ref + 1e-4, (gram_power, eps, eps_ref)
    # the 40^4 case applies q = 4 powers to an 800 x 1600 unfolding at mode 2
    if dims == (40, 40, 40, 40):
        assert bool(set(fams) & GRAM_POWER_FAMILIES) == gram_power


def test_nonfinite_input_flagged(tt):
    A = noisy_tt((8, 9, 10), (3, 3), 2, 0.01).astype(np.float32)
    A[3, 4, 5] = np.nan
    t = torch.from_numpy(A).cuda()
    cores, _ = tt.decompose(t, (3, 3), 2, 1, omega_seed=1)
    torch.cuda.synchronize()
    assert tt.device_status(tt.decompose.last_workspace) == tt._native.TT_ENONFINITE


def test_two_runs_bitwise_identical(tt):
    """Fixed-order reductions: the same call twice gives identical bits."""
    A = noisy_tt((40, 30, 20, 10), (6, 6, 6), 4, 0.05)
    a, _ = gpu_decompose(tt, A, (6, 6, 6), 4, 3, seed=11)
    b, _ = gpu_decompose(tt, A, (6, 6, 6), 4, 3, seed=11)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_rank_clamp_and_order2(tt):
    A = noisy_tt((3, 5, 4), (3, 4), 1, 0.1)
    got, rr = gpu_decompose(tt, A, (10, 10), 2, 2, seed=2)
    assert rr == [1, 3, 4, 1]
    assert oracle.tt_error(A, got) < 1e-5        # full ranks: exact
    B = np.random.default_rng(0).standard_normal((50, 70))
    got, rr = gpu_decompose(tt, B, (6,), 4, 2, seed=5)
    ref = oracle.tt_rbki(B.astype(np.float32), (6,), 4, 2, seed=5)
    assert oracle.tt_distance(got, ref) <= FP32_TOL


# unfoldings with more rows than one thread-block cluster holds (m > 1024):
# the block orthonormalisation runs over all CTAs of a cooperative launch
CASES_TALL = [
    # dims, generating ranks, target ranks, p, q, noise
    ((1100, 6, 5, 4), (8, 6, 4), (8, 6, 4), 4, 2, 0.05),             # m = 1100 at mode 1
    ((20, 60, 30, 24), (20, 16, 10), (20, 16, 10), 4, 2, 0.03),      # m = 1200 at mode 2
    ((2050, 16, 16), (12, 6), (12, 6), 5, 3, 0.02),                  # m = 2050, n = 256
]


@pytest.mark.parametrize("case", CASES_TALL)
def test_tall_blocks_fp32_match_oracle(tt, case):
    dims, gr, ranks, p, q, noise = case
    A = noisy_tt(dims, gr, 53, noise)
    rr = oracle.clamp_ranks(dims, ranks)
    om = W.explicit_omegas(dims, rr, p, 59)
    ref = oracle.tt_rbki(A.astype(np.float32), ranks, p, q, omegas=om)
    tt.profile_begin(event_timing=False)
    got, rr_gpu = gpu_decompose(tt, A, ranks, p, q, omegas=om, exhaust=False, gram_power=False)
    fams = tt.profile_end()
    assert "orth_grid" in fams
    assert rr_gpu == rr
    assert oracle.tt_distance(got, ref) <= FP32_TOL
    for G in got[:-1]:
        assert oracle.left_orthogonality_defect(G) < 1e-4


@pytest.mark.parametrize("case", CASES_TALL)
def test_tall_blocks_bf16_error_criterion(tt, case):
    dims, gr, ranks, p, q, noise = case
    A = noisy_tt(dims, gr, 61, noise)
    eps_ref = oracle.tt_error(A, oracle.tt_rbki(A, ranks, p, q, seed=7))
    got, _ = gpu_decompose(tt, A, ranks, p, q, storage="bf16", seed=7)
    assert oracle.tt_error(A, got) <= 1.05 * eps_ref + 1e-4


def test_tall_rank_deficient_blocks_repaired(tt):
    """Target ranks above the TT ranks of an exact low-rank tensor: from the
    second Krylov block on, the blocks of the 1500-row unfolding are
    numerically inside the span of the basis; their columns are replaced
    inside the launch by pseudo-random vectors, the cores stay orthonormal
    and the tensor is recovered exactly (to FP32 working accuracy)."""
    dims = (1500, 8, 6, 5)
    A = noisy_tt(dims, (3, 3, 2), 67, 0.0)
    tt.profile_begin(event_timing=False)
    got, _ = gpu_decompose(tt, A, (10, 8, 5), 3, 2, seed=9, exhaust=False, gram_power=False)
    fams = tt.profile_end()
    assert "orth_grid" in fams and "orth_block" not in fams
    assert oracle.tt_error(A, got) < 2e-5
    for G in got[:-1]:
        assert oracle.left_orthogonality_defect(G) < 1e-4
