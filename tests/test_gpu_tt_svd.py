"""TT-SVD (Alg. 1) on the GPU against the float64 oracle's TT-SVD.

  * prescribed accuracy: on tensors whose singular-value gaps make the
    delta-truncation unambiguous (delta^2 far above the FP32 Gram's
    rounding, far below the smallest kept squared singular value), the
    ranks equal the oracle's and the
    cores reconstruct the same tensor (relative TT distance <= 1e-4, FP32);
  * fixed ranks (eps = 0 with rank caps): the relative error matches the
    oracle's to 1e-4 relative, the BF16 form meets eps_gpu <= 1.05
    eps_oracle + 1e-4;
  * caps below the delta-rank win; order 2 is the truncated matrix SVD;
    invalid arguments are rejected.
"""
import numpy as np
import pytest

import oracle
from paper_2308_01480_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tt():
    import paper_2308_01480_gb300 as tt
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    tt._native.lib()
    return tt


def _noisy_tt(dims, ranks, seed, level):
    rng = np.random.default_rng(seed)
    A = W.dense_from_cores(W.random_tt_cores(dims, ranks, rng))
    return W.add_noise(A, level, rng) if level > 0 else A


def _host(cores):
    return [c.cpu().double().numpy() for c in cores]


# caps that do not bind keep the workspace (sized for the caps) small where
# full ranks would give a 32768-row unfolding
@pytest.mark.parametrize("dims,ranks,caps", [((12, 10, 14, 8), (3, 4, 3), None),
                                             ((32, 32, 32, 32), (8, 8, 8), (32, 64, 32)),
                                             ((6, 5, 7, 4, 6), (2, 3, 3, 2), None), ((50, 300), (7,), None)])
def test_delta_truncation_matches_oracle(tt, dims, ranks, caps):
    A = _noisy_tt(dims, ranks, 3, 1e-5)
    eps = 1e-2
    ref = oracle.tt_svd(A, eps=eps)
    ref_ranks = [1] + [c.shape[2] for c in ref]
    cores, rr = tt.tt_svd(torch.from_numpy(A.astype(np.float32)).cuda(), eps=eps, max_ranks=caps)
    assert rr == ref_ranks
    assert list(rr[1:-1]) == list(ranks)
    got = _host(cores)
    assert oracle.tt_distance(got, ref) <= 1e-4
    assert oracle.tt_error(A, got) <= eps


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_fixed_ranks_error_matches_oracle(tt, storage):
    dims, gen_ranks, caps = (16, 12, 14, 10), (5, 6, 4), (3, 4, 3)
    A = _noisy_tt(dims, gen_ranks, 8, 0.05)
    ref = oracle.tt_svd(A, ranks=caps)
    eps_ref = oracle.tt_error(A, ref)
    t = torch.from_numpy(A.astype(np.float32)).cuda()
    if storage == "bf16":
        t = t.to(torch.bfloat16)
    cores, rr = tt.tt_svd(t, eps=0.0, max_ranks=caps)
    assert rr == [1, 3, 4, 3, 1]
    eps_gpu = oracle.tt_error(A, _host(cores))
    if storage == "f32":
        assert abs(eps_gpu - eps_ref) <= 1e-4 * eps_ref
    else:
        assert eps_gpu <= 1.05 * eps_ref + 1e-4


def test_caps_below_delta_rank(tt):
    A = _noisy_tt((10, 12, 9), (4, 5), 5, 1e-5)
    cores, rr = tt.tt_svd(torch.from_numpy(A.astype(np.float32)).cuda(), eps=1e-2, max_ranks=(2, 3))
    assert rr == [1, 2, 3, 1]
    for k, c in enumerate(cores):
        assert tuple(c.shape) == (rr[k], A.shape[k], rr[k + 1])


def test_large_eps_gives_rank_one(tt):
    A = _noisy_tt((8, 9, 10), (3, 3), 6, 0.0)
    cores, rr = tt.tt_svd(torch.from_numpy(A.astype(np.float32)).cuda(), eps=10.0)
    assert rr == [1, 1, 1, 1]


def test_rejects_bad_arguments(tt):
    x = torch.ones((4, 5, 6), device="cuda")
    with pytest.raises(tt.TTError):
        tt.tt_svd(x, eps=-1.0)
    with pytest.raises(tt.TTError):
        tt.tt_svd(x, eps=0.1, max_ranks=(0, 2))
