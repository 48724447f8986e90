"""Seeded synthetic inputs shaped like the paper's workloads.

This module only builds inputs.  It holds none of the decomposition's
arithmetic and imports neither the CUDA binding nor the oracle, so tests,
the benchmark and the oracle all draw identical inputs from it.

Families (the paper's public datasets are not available, so these stand in
for them):
  * low TT rank plus noise, the structure of the paper's noisy experiments
    (Sec. 4.2): Gaussian TT cores of given ranks contracted to a dense tensor,
    then a noise tensor E scaled so that ||E|| = level * ||X|| exactly for
    the realised sample (Gaussian or heavy-tailed Student-t);
  * the smooth power-function tensor of Sec. 4.1, f(i) = 1 / (sum_k i_k + 1)
    with 0-based indices (h = 1), plus Gaussian noise.

Every generator is keyed by an integer seed through numpy's PCG64, which is
platform independent.
"""
from dataclasses import dataclass, field

import numpy as np

TENSOR_SEED_BASE = 20230803
OMEGA_SEED_BASE = 7


@dataclass
class Workload:
    """One decomposition problem: tensor recipe plus TT-rBKI parameters."""
    name: str
    dims: tuple
    ranks: tuple              # target r_1..r_{d-1}
    oversample: int           # p
    q: int                    # Krylov depth
    storage: str              # "f32" or "bf16" on the GPU
    tensor_seed: int
    omega_seed: int
    family: str = "tt"        # "tt" or "power"
    tt_ranks: tuple = ()      # ranks of the generating TT (family "tt")
    slice_decay: float = 0.0  # right-slice scale ratio (0 = none)
    noise: float = 0.0        # relative noise level
    noise_kind: str = "gaussian"
    notes: str = field(default="")

    @property
    def numel(self):
        return int(np.prod(self.dims, dtype=np.int64))


def random_tt_cores(dims, tt_ranks, rng, slice_decay=0.0):
    """Gaussian cores G_k of shape (r_{k-1}, I_k, r_k), r_0 = r_d = 1.

    With slice_decay = a > 0, the j-th right-rank slice of every core but the
    last is scaled by a**j, which gives geometrically decaying spectra.
    """
    d = len(dims)
    rs = [1] + list(tt_ranks) + [1]
    cores = []
    for k in range(d):
        G = rng.standard_normal((rs[k], dims[k], rs[k + 1]))
        if slice_decay and k < d - 1:
            G *= slice_decay ** np.arange(rs[k + 1])[None, None, :]
        cores.append(G)
    return cores


def dense_from_cores(cores):
    """Dense float64 tensor sum_{a} G_1[:, i1, a1] G_2[a1, i2, a2] ... ."""
    dims = tuple(G.shape[1] for G in cores)
    T = cores[0].reshape(dims[0], -1)
    for G in cores[1:]:
        ra, I, rb = G.shape
        T = (T @ G.reshape(ra, I * rb)).reshape(-1, rb)
    return T.reshape(dims)


def add_noise(X, level, rng, kind="gaussian", nu=2.0):
    """X + E with ||E||_F = level * ||X||_F exactly for this sample."""
    if level <= 0:
        return X
    if kind == "gaussian":
        E = rng.standard_normal(X.shape)
    elif kind == "student_t":
        E = rng.standard_t(nu, X.shape)
    else:
        raise ValueError(kind)
    E *= level * np.linalg.norm(X) / np.linalg.norm(E)
    return X + E


def power_tensor(dims):
    """f(i_1, ..., i_d) = 1 / (i_1 + ... + i_d + 1), 0-based indices."""
    s = np.zeros(dims, dtype=np.float64)
    for k, n in enumerate(dims):
        shape = [1] * len(dims)
        shape[k] = n
        s = s + np.arange(n, dtype=np.float64).reshape(shape)
    return 1.0 / (s + 1.0)


def power_tensor_h(dims, h):
    """The power function of Sec. 4.1, Eq. (5): x = (i_1^h + ... + i_d^h)^(-1/h)
    with 1-based indices i_k = 1 .. I_k, as printed."""
    s = np.zeros(dims, dtype=np.float64)
    for k, n in enumerate(dims):
        shape = [1] * len(dims)
        shape[k] = n
        s = s + (np.arange(1, n + 1, dtype=np.float64) ** h).reshape(shape)
    return s ** (-1.0 / h)


def decaying_diag_tensor(n, T, D, dtype=np.float64):
    """The spectrum-decaying tensor of Sec. 4.1: frontal slice j (1-based)
    is diag(1 x min(T, j), 10^-D, 10^-2D, ..., 10^-(n - min(T, j)) D),
    n x n; entries below the dtype's range are zero."""
    X = np.zeros((n, n, n), dtype=dtype)
    idx = np.arange(n)
    for j in range(1, n + 1):
        t = min(T, j)
        diag = np.ones(n, dtype=np.float64)
        diag[t:] = 10.0 ** (-D * np.arange(1, n - t + 1, dtype=np.float64))
        X[idx, idx, j - 1] = diag.astype(dtype)
    return X


def add_noise_snr(X, snr_db, rng):
    """Gaussian white noise at a measured SNR: ||E|| / ||X|| = 10^(-SNR/20)."""
    return add_noise(X, 10.0 ** (-snr_db / 20.0), rng)


def make_tensor(w: Workload):
    """Dense float64 tensor of workload w (deterministic in w.tensor_seed)."""
    rng = np.random.default_rng(w.tensor_seed)
    if w.family == "tt":
        X = dense_from_cores(random_tt_cores(w.dims, w.tt_ranks, rng, w.slice_decay))
    elif w.family == "power":
        X = power_tensor(w.dims)
    elif w.family == "power_h5":
        X = power_tensor_h(w.dims, 5.0)
    elif w.family == "decay_diag":
        X = decaying_diag_tensor(w.dims[0], 50, 1.0)
    else:
        raise ValueError(w.family)
    return add_noise(X, w.noise, rng, w.noise_kind)


def explicit_omegas(dims, ranks_clamped, oversample, seed):
    """Gaussian Omega_k (n_k x (r_k' + p)) rounded to float32, for the
    explicit-Omega entry point; ranks_clamped = [r_0', ..., r_d']."""
    rng = np.random.default_rng(seed)
    out = []
    d = len(dims)
    for k in range(d - 1):
        n = int(np.prod(dims[k + 1:], dtype=np.int64))
        b = ranks_clamped[k + 1] + oversample
        out.append(rng.standard_normal((n, b)).astype(np.float32))
    return out


CONFIGS = {
    1: Workload("tt16^4_r4_noise1e-3", (16, 16, 16, 16), (4, 4, 4), 5, 2, "f32",
                TENSOR_SEED_BASE + 1, OMEGA_SEED_BASE + 1, "tt", (4, 4, 4),
                noise=1e-3, notes="small case: order 4, 16^4, TT ranks 4"),
    2: Workload("tt32^5_r10_studentt10pct", (32,) * 5, (10,) * 4, 5, 3, "f32",
                TENSOR_SEED_BASE + 2, OMEGA_SEED_BASE + 2, "tt", (10,) * 4,
                noise=0.10, noise_kind="student_t",
                notes="32^5 (33.5M), TT ranks 10, Student-t nu=2 noise at 10%"),
    3: Workload("tt40^5_r20_decay0.8_noise5pct", (40,) * 5, (20,) * 4, 10, 4, "bf16",
                TENSOR_SEED_BASE + 3, OMEGA_SEED_BASE + 3, "tt", (20,) * 4,
                slice_decay=0.8, noise=0.05,
                notes="40^5 (102.4M), TT ranks 20 with 0.8^j slice scales, 5% noise"),
    4: Workload("power256x256x64x32_noise1pct", (256, 256, 64, 32), (30, 30, 30), 10, 3, "bf16",
                TENSOR_SEED_BASE + 4, OMEGA_SEED_BASE + 4, "power",
                noise=0.01, notes="f(i)=1/(i1+i2+i3+i4+1), 134.2M entries, 1% noise"),
}


# Batched form: each problem's mode vector is resampled until the tensor has
# at most this many entries (an unconstrained order-6 tensor with modes up to
# 64 would hold ~7e10 entries, far from "about 2 GB" for the whole batch).
BATCH_ENTRY_CAP = 1 << 24


def batch_workloads(count=256, seed=TENSOR_SEED_BASE + 5, omega_seed=OMEGA_SEED_BASE + 5):
    """Independent problems of the batched form: order uniform in 3..6,
    modes uniform in 8..64 (resampled until the entry count is at most
    BATCH_ENTRY_CAP), per-bond TT ranks uniform in 2..16 for both the
    generating cores and the target, 5% Gaussian noise, p = 5, q = 2, BF16
    storage.  Problem i gets tensor seed seed*1000 + i and Omega seed
    omega_seed*1000 + i."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        d = int(rng.integers(3, 7))
        while True:
            dims = tuple(int(x) for x in rng.integers(8, 65, size=d))
            if int(np.prod(dims, dtype=np.int64)) <= BATCH_ENTRY_CAP:
                break
        ranks = tuple(int(x) for x in rng.integers(2, 17, size=d - 1))
        out.append(Workload(f"batch{i}", dims, ranks, 5, 2, "bf16", seed * 1000 + i, omega_seed * 1000 + i,
                            "tt", ranks, noise=0.05))
    return out


# The paper's synthetic accuracy experiments (Sec. 4.1, 4.2), parameterised
# by the target rank r (all bonds r) and, for the noisy one, the SNR in dB.
# q is not stated for them; q = 2 is taken (the TT-rBKI depth of the
# paper's other experiments is small).
STUDY_SEED_BASE = 20230900


def study_workload(name, r, snr_db=5.0, q=2):
    if name == "e1":          # 500^3 decaying spectrum, T = 50, D = 1, p = 2
        return Workload(f"e1_decay500_r{r}", (500, 500, 500), (r, r), 2, q, "f32",
                        STUDY_SEED_BASE + 1, OMEGA_SEED_BASE + 100 + r, "decay_diag",
                        notes="500^3 diagonal slices, T=50, D=1")
    if name == "e2":          # 45^5 power function, h = 5, p = 2
        return Workload(f"e2_power45_r{r}", (45,) * 5, (r,) * 4, 2, q, "f32",
                        STUDY_SEED_BASE + 2, OMEGA_SEED_BASE + 200 + r, "power_h5",
                        notes="45^5 power function, h=5")
    if name == "e6":          # E2 plus white noise at snr_db (measured)
        return Workload(f"e6_power45_r{r}_snr{snr_db:g}", (45,) * 5, (r,) * 4, 2, q, "f32",
                        STUDY_SEED_BASE + 6, OMEGA_SEED_BASE + 600 + r, "power_h5",
                        noise=10.0 ** (-snr_db / 20.0),
                        notes=f"45^5 power function, h=5, white noise at {snr_db:g} dB")
    raise ValueError(name)
