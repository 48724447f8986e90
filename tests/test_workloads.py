"""The input recipe: the seeded generators every test, the benchmark and the
oracle draw their tensors from.

These check the generators against the properties the recipe states: noise
scaled to an exact relative norm, geometric right-slice scales of the
generating cores, the power function's values, the workload table, and the
batched form's sampling limits.
"""
import numpy as np
import pytest

from paper_2308_01480_gb300 import workloads as W


@pytest.mark.parametrize("kind", ["gaussian", "student_t"])
@pytest.mark.parametrize("level", [1e-3, 0.05, 0.1])
def test_noise_has_the_exact_relative_norm(kind, level):
    rng = np.random.default_rng(1)
    X = W.dense_from_cores(W.random_tt_cores((6, 7, 8), (3, 4), rng))
    Y = W.add_noise(X, level, np.random.default_rng(2), kind)
    assert np.linalg.norm(Y - X) == pytest.approx(level * np.linalg.norm(X), rel=1e-12)
    assert W.add_noise(X, 0.0, np.random.default_rng(2)) is X


def test_slice_decay_scales_right_rank_slices():
    """Right-rank slice j of every core but the last is scaled by a**j; the
    last core is left as drawn."""
    dims, ranks, a = (5, 6, 7, 4), (3, 4, 2), 0.8
    plain = W.random_tt_cores(dims, ranks, np.random.default_rng(9))
    scaled = W.random_tt_cores(dims, ranks, np.random.default_rng(9), slice_decay=a)
    for k, (G, H) in enumerate(zip(plain, scaled)):
        if k < len(dims) - 1:
            for j in range(G.shape[2]):
                assert np.allclose(H[:, :, j], G[:, :, j] * a ** j, rtol=1e-15, atol=0)
        else:
            assert np.array_equal(H, G)


def test_dense_from_cores_is_the_tt_contraction():
    rng = np.random.default_rng(4)
    cores = W.random_tt_cores((3, 4, 2, 5), (2, 3, 2), rng)
    want = np.einsum("ia,ajb,bkc,cl->ijkl", cores[0][0], cores[1], cores[2], cores[3][:, :, 0])
    assert np.allclose(W.dense_from_cores(cores), want, rtol=1e-14, atol=1e-14)


def test_power_function_values():
    """f(i) = 1 / (i_1 + ... + i_d + 1) with 0-based indices."""
    dims = (7, 5, 6, 3)
    X = W.power_tensor(dims)
    assert X.shape == dims and X[0, 0, 0, 0] == 1.0
    rng = np.random.default_rng(0)
    for _ in range(20):
        i = tuple(int(rng.integers(0, n)) for n in dims)
        assert X[i] == 1.0 / (sum(i) + 1)


def test_workload_table():
    want = {
        1: ((16, 16, 16, 16), (4, 4, 4), 5, 2, "tt", 1e-3),
        2: ((32,) * 5, (10,) * 4, 5, 3, "tt", 0.10),
        3: ((40,) * 5, (20,) * 4, 10, 4, "tt", 0.05),
        4: ((256, 256, 64, 32), (30, 30, 30), 10, 3, "power", 0.01),
    }
    for cfg, (dims, ranks, p, q, family, noise) in want.items():
        w = W.CONFIGS[cfg]
        assert (w.dims, w.ranks, w.oversample, w.q, w.family, w.noise) == (dims, ranks, p, q, family, noise)
        assert w.tensor_seed == 20230803 + cfg and w.omega_seed == 7 + cfg
    assert W.CONFIGS[2].noise_kind == "student_t" and W.CONFIGS[3].slice_decay == 0.8
    assert W.CONFIGS[3].numel == 40 ** 5


def test_make_tensor_is_deterministic():
    w = W.CONFIGS[1]
    A, B = W.make_tensor(w), W.make_tensor(w)
    assert A.dtype == np.float64 and A.shape == w.dims and np.array_equal(A, B)


def test_batch_sampling_limits():
    """256 problems of order 3..6, modes 8..64, every tensor at most 2^24
    entries, TT ranks 2..16 (target = generating), p = 5, q = 2, 5% noise;
    2,700,934,876 bytes in BF16 in all."""
    ws = W.batch_workloads()
    assert len(ws) == 256
    for i, w in enumerate(ws):
        assert 3 <= len(w.dims) <= 6 and all(8 <= n <= 64 for n in w.dims)
        assert w.numel <= W.BATCH_ENTRY_CAP == 1 << 24
        assert len(w.ranks) == len(w.dims) - 1 and all(2 <= r <= 16 for r in w.ranks)
        assert w.tt_ranks == w.ranks and (w.oversample, w.q, w.noise) == (5, 2, 0.05)
        assert w.tensor_seed == (20230803 + 5) * 1000 + i and w.omega_seed == (7 + 5) * 1000 + i
    assert sum(w.numel for w in ws) * 2 == 2_700_934_876
    assert {len(w.dims) for w in ws} == {3, 4, 5, 6}
