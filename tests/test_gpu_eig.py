"""The Rayleigh-Ritz eigensolver (Alg. 3 steps 6-8) against LAPACK.

For symmetric H with random, graded, clustered, rank-deficient spectra and
a cluster of eigenvalues far below FP32 resolution
the r largest eigenvalues must match numpy.linalg.eigh to 1e-5 ||H|| and
the eigenvectors must be orthonormal with residual ||H v - lam v|| below
2e-5 ||H||; for eigenvalues separated from the rest by a gap g, the
computed vector must match LAPACK's up to sign within 1e-5 ||H|| / g.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tt():
    import paper_2308_01480_gb300 as tt
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    tt._native.lib()
    return tt


def _sym(k, spectrum, seed):
    rng = np.random.default_rng(seed)
    Qm, _ = np.linalg.qr(rng.standard_normal((k, k)))
    return (Qm * spectrum) @ Qm.T


def _spectra(k, seed):
    rng = np.random.default_rng(seed)
    out = {
        "random": rng.standard_normal(k),
        "graded": 10.0 ** (-8 * np.arange(k) / max(1, k - 1)),
        "psd_decay": np.sort(rng.random(k) ** 4)[::-1],
        "clustered": np.concatenate([np.full(k // 3, 1.0) + 1e-7 * rng.standard_normal(k // 3),
                                     rng.random(k - k // 3) * 0.5]),
        "rank_deficient": np.concatenate([rng.random(max(1, k // 4)) + 1.0, np.zeros(k - max(1, k // 4))]),
        # a few large eigenvalues, the rest a cluster far below FP32
        # resolution (Rayleigh-Ritz on an exactly low-rank unfolding): the
        # wanted vectors inside the cluster must still come out orthonormal
        "tiny_cluster": np.concatenate([rng.random(max(1, k // 16)) + 1.0,
                                        1e-10 * rng.random(k - max(1, k // 16))]),
    }
    return out


SIZES = [(1, 1), (2, 1), (3, 2), (17, 5), (32, 20), (33, 32), (40, 20), (64, 30), (96, 25), (150, 20),
         (130, 31), (160, 30), (160, 32), (161, 20), (200, 30), (224, 10)]


@pytest.mark.parametrize("k,r", SIZES)
def test_eig_top_matches_lapack(tt, k, r):
    for name, lam in _spectra(k, 7 + k).items():
        H = _sym(k, lam, 11 + k)
        Hd = torch.from_numpy(H.astype(np.float32)).cuda()
        V, ev = tt.sym_eig_top(Hd, r)
        torch.cuda.synchronize()
        V = V.cpu().double().numpy()
        ev = ev.cpu().double().numpy()
        H32 = H.astype(np.float32).astype(np.float64)
        w, U = np.linalg.eigh(0.5 * (H32 + H32.T))
        w, U = w[::-1], U[:, ::-1]
        nrm = max(np.abs(w).max(), 1e-30)
        assert np.all(np.isfinite(V)) and np.all(np.isfinite(ev)), name
        assert np.max(np.abs(ev - w[:r])) <= 1e-5 * nrm, (name, np.max(np.abs(ev - w[:r])) / nrm)
        assert np.max(np.abs(V.T @ V - np.eye(r))) <= 2e-5, (name, np.max(np.abs(V.T @ V - np.eye(r))))
        res = np.linalg.norm(H32 @ V - V * ev, axis=0)
        assert res.max() <= 2e-5 * nrm * np.sqrt(k), (name, res.max() / nrm)
        # well-separated eigenvalues: vectors agree with LAPACK up to sign
        for j in range(r):
            gap = min(abs(w[j] - w[i]) for i in range(k) if i != j) if k > 1 else nrm
            if gap > 1e-2 * nrm:
                c = abs(float(V[:, j] @ U[:, j]))
                assert 1.0 - c <= 1e-5 * nrm / gap + 1e-6, (name, j, 1.0 - c)


def test_eig_top_rejects_bad_arguments(tt):
    H = torch.zeros((8, 8), device="cuda")
    with pytest.raises(tt.TTError):
        tt.sym_eig_top(H, 9)
    with pytest.raises(tt.TTError):
        tt.sym_eig_top(torch.zeros((225, 225), device="cuda"), 4)
