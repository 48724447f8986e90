"""Pins of the accuracy-study pieces of the oracle and of the study inputs:
the PSNR of Sec. 4 against hand-computed values, and the synthetic tensors
of Sec. 4.1 against their printed formulas at a few entries (no GPU)."""
import numpy as np

import oracle
from paper_2308_01480_gb300 import workloads as W


def test_psnr_single_entry_error():
    A = np.ones((2, 3, 4))
    B = A.copy()
    B[1, 2, 3] += 0.5
    # N = 24 entries, peak |B| = 1.5, error norm^2 = 0.25
    assert np.isclose(oracle.psnr(A, B), 10 * np.log10(24 * 1.5 ** 2 / 0.25), rtol=0, atol=1e-12)


def test_psnr_uses_reconstruction_peak_and_all_modes():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((3, 4, 5, 2))
    B = A + 1e-3 * rng.standard_normal(A.shape)
    expect = 10 * np.log10(A.size * np.abs(B).max() ** 2 / np.sum((A - B) ** 2))
    assert np.isclose(oracle.psnr(A, B), expect, rtol=1e-14)
    # scaling the error by 10 lowers the PSNR by 20 dB when the peak is kept
    C = A + 10 * (B - A)
    C_peak_fixed = oracle.psnr(A, C) - 20 * np.log10(np.abs(C).max() / np.abs(B).max())
    assert np.isclose(oracle.psnr(A, B) - C_peak_fixed, 20.0, atol=1e-9)


def test_power_function_entries():
    X = W.power_tensor_h((4, 3, 5, 2, 3), 5.0)
    for idx in [(0, 0, 0, 0, 0), (3, 2, 4, 1, 2), (1, 0, 2, 1, 0)]:
        i = np.array(idx) + 1            # printed with 1-based indices
        assert np.isclose(X[idx], np.sum(i ** 5.0) ** (-1 / 5), rtol=1e-15)


def test_decaying_diag_slices():
    X = W.decaying_diag_tensor(8, 3, 1.0)
    for j in range(1, 9):
        S = X[:, :, j - 1]
        t = min(3, j)
        expect = np.concatenate([np.ones(t), 10.0 ** -np.arange(1, 8 - t + 1)])
        assert np.allclose(np.diag(S), expect, rtol=1e-15, atol=0)
        assert np.count_nonzero(S - np.diag(np.diag(S))) == 0


def test_snr_noise_is_measured():
    rng = np.random.default_rng(3)
    X = W.power_tensor_h((6, 5, 4), 5.0)
    Y = W.add_noise_snr(X, 5.0, rng)
    assert np.isclose(np.linalg.norm(Y - X) / np.linalg.norm(X), 10 ** (-5 / 20), rtol=1e-12)
