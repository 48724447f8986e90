"""Parity at the full workload sizes, in the configuration the benchmark
times (seeded Omega on the device, default options, one call per
decomposition).

  * 32^5 FP32 form (Student-t noise): relative TT distance to the float64
    oracle with the same seed <= 1e-4.
  * 40^5 (the benchmark workload): BF16 form eps <= 1.05 eps_oracle + 1e-4
    against the float64 tensor, FP32 form within TT distance 1e-4.
  * 256 x 256 x 64 x 32 power function, BF16 form: the BF16 criterion.
The oracle runs on the host in float64 (tens of seconds in total).
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


def _gpu(tt, A, w, storage):
    t = torch.from_numpy(A.astype(np.float32)).cuda()
    if storage == "bf16":
        t = tt.permute_convert(t, dst_dtype=torch.bfloat16)
        opts = tt.options(storage=tt.TT_BF16, remainder=tt.TT_BF16)
    else:
        opts = tt.options(storage=tt.TT_F32, remainder=tt.TT_F32)
    cores, rr = tt.decompose(t, w.ranks, w.oversample, w.q, omega_seed=w.omega_seed, opts=opts)
    torch.cuda.synchronize()
    assert tt.device_status(tt.decompose.last_workspace) == 0
    assert rr == oracle.clamp_ranks(w.dims, w.ranks)
    out = [c.cpu().double().numpy() for c in cores]
    del t
    torch.cuda.empty_cache()
    return out


@pytest.fixture(scope="module")
def config3():
    w = W.CONFIGS[3]
    A = W.make_tensor(w)
    ref = oracle.tt_rbki(A, w.ranks, w.oversample, w.q, seed=w.omega_seed)
    return w, A, ref, oracle.tt_error(A, ref)


def test_config2_fp32_matches_oracle(tt):
    w = W.CONFIGS[2]
    A = W.make_tensor(w)
    A32 = A.astype(np.float32).astype(np.float64)
    ref = oracle.tt_rbki(A32, w.ranks, w.oversample, w.q, seed=w.omega_seed)
    got = _gpu(tt, A, w, "f32")
    assert oracle.tt_distance(got, ref) <= 1e-4
    for G in got[:-1]:
        assert oracle.left_orthogonality_defect(G) < 1e-4


def test_config3_bf16_error_criterion(tt, config3):
    w, A, ref, eps_ref = config3
    got = _gpu(tt, A, w, "bf16")
    eps = oracle.tt_error(A, got)
    assert eps <= 1.05 * eps_ref + 1e-4, (eps, eps_ref)


def test_config3_fp32_matches_oracle(tt, config3):
    w, A, _, _ = config3
    A32 = A.astype(np.float32).astype(np.float64)
    ref32 = oracle.tt_rbki(A32, w.ranks, w.oversample, w.q, seed=w.omega_seed)
    got = _gpu(tt, A, w, "f32")
    assert oracle.tt_distance(got, ref32) <= 1e-4


def test_config4_bf16_error_criterion(tt):
    w = W.CONFIGS[4]
    A = W.make_tensor(w)
    ref = oracle.tt_rbki(A, w.ranks, w.oversample, w.q, seed=w.omega_seed)
    eps_ref = oracle.tt_error(A, ref)
    got = _gpu(tt, A, w, "bf16")
    eps = oracle.tt_error(A, got)
    assert eps <= 1.05 * eps_ref + 1e-4, (eps, eps_ref)
