"""The synthetic accuracy study (Sec. 4.1, 4.2) on the GPU against the
float64 oracle, on reduced sizes of its tensors: for the h = 5 power
function (E2), the same with 5 dB white noise (E6) and the decaying-spectrum
diagonal tensor (E1), each method's cores meet the FP32 parity bar
(TT-rBKI with either Rayleigh-Ritz, TT-rSI, TT-rSVD: relative TT distance <= 1e-4 to the oracle with
the same seed; for E6, whose spectrum is nearly flat at the truncation
rank, relative errors equal to 1e-4 relative and distance <= 1e-3; TT-SVD:
relative error within 1e-4 relative of the oracle's), and
the study's device-side relative error and PSNR equal the oracle's metrics
of the same cores to 1e-9 relative."""
import numpy as np
import pytest

import oracle
from paper_2308_01480_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def study():
    from paper_2308_01480_gb300 import accuracy_study as S
    import paper_2308_01480_gb300 as tt
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    tt._native.lib()
    return S


def _tensors():
    rng = np.random.default_rng(11)
    e2 = W.power_tensor_h((18,) * 5, 5.0)
    e6 = W.add_noise_snr(e2, 5.0, rng)
    e1 = W.decaying_diag_tensor(60, 10, 1.0)
    return {"e2": e2, "e6": e6, "e1": e1}


@pytest.mark.parametrize("name,r", [("e2", 3), ("e2", 6), ("e6", 5), ("e1", 8)])
def test_study_case_matches_oracle(study, name, r):
    import paper_2308_01480_gb300 as tt
    A = _tensors()[name]
    d = A.ndim
    ranks = (r,) * (d - 1)
    p, q, seed = 2, 2, 4242 + r
    res = study.run_case(A, ranks, p, q, seed)
    A32 = A.astype(np.float32).astype(np.float64)
    t32 = torch.from_numpy(A.astype(np.float32)).cuda()
    refs = {"tt_rbki": oracle.tt_rbki(A32, ranks, p, q, seed=seed),
            "tt_rsi": oracle.tt_rsi(A32, ranks, p, q, seed=seed),
            "tt_rsvd": oracle.tt_rbki(A32, ranks, p, 0, seed=seed)}
    refs["tt_rbki_acc"] = refs["tt_rbki"]       # the same method, Rayleigh-Ritz without squaring
    for m, ref in refs.items():
        method = tt.TT_METHOD_RSI if m == "tt_rsi" else tt.TT_METHOD_RBKI
        cores, _ = tt.decompose(t32, ranks, p, 0 if m == "tt_rsvd" else q, omega_seed=seed,
                                opts=tt.options(storage=tt.TT_F32, method=method, accurate_rr=(m == "tt_rbki_acc")))
        got = [c.cpu().double().numpy() for c in cores]
        Ahat = oracle.tt_full(got)
        eps_o, psnr_o = oracle.tt_error(A, got), oracle.psnr(A, Ahat)
        if name == "e6":
            # at 5 dB the spectrum around rank r is nearly flat (noise norm
            # 0.56 of the signal's), so the rank-r subspace is fixed only to
            # the size of those gaps: the errors are compared
            eps_ref = oracle.tt_error(A, ref)
            assert abs(eps_o - eps_ref) <= 1e-4 * eps_ref, m
            assert oracle.tt_distance(got, ref) <= 1e-3, m
        else:
            assert oracle.tt_distance(got, ref) <= 1e-4, m
        assert abs(res[m]["eps"] - eps_o) <= 1e-9 * eps_o + 1e-15, m
        assert abs(res[m]["psnr"] - psnr_o) <= 1e-9 * abs(psnr_o), m
    eps_svd = oracle.tt_error(A, oracle.tt_svd(A32, ranks=ranks))
    assert abs(res["tt_svd"]["eps"] - eps_svd) <= 1e-4 * eps_svd + 1e-7
    for m in study.METHODS:
        assert np.isfinite(res[m]["ms"]) and res[m]["ms"] > 0
