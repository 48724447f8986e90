"""TT-rBKI and TT-rSI split over ranks by the last mode, on CPU (gloo,
world size 2).

Rank g holds the slab A[..., S_g] of the last mode.  Every unfolding of the
remainder then splits by columns, C = [C_g], because the last mode index is
part of every column index (it is the fastest one, so slab S_g owns the
columns j = j' I_d + i_d with i_d in S_g).  Alg. 3 then needs one sum over
the ranks per pass, of a block that does not depend on n:
  sketch          Y = sum_g C_g W_g                    (m x b)
  Krylov power    Z = sum_g C_g (C_g^T X)              (m x b)
  Rayleigh-Ritz   H = sum_g (Q^T C_g)(Q^T C_g)^T        (k x k; its top
                  eigenvectors are the top left singular vectors of Q^T C)
while the projection R_g = U^T C_g stays on its rank and is already that
rank's column slab of the next unfolding: nothing moves between modes.  The
last core is gathered.  Orthonormalisation and the small eigenproblem run
replicated on the reduced blocks.

Each rank's result must match the single-process oracle up to summation
order, and the replicated cores must be bit-identical across ranks.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2308_01480_gb300 import workloads as W  # noqa: E402

# dims, generating ranks, target ranks, p, q, noise
CASES = [
    ((6, 7, 8, 5), (3, 4, 2), (3, 4, 2), 2, 2, 0.05),
    ((9, 10, 11, 7), (3, 5, 4), (3, 5, 4), 3, 2, 0.02),
    ((5, 4, 6, 3, 7, 4), (3, 4, 5, 4, 3), (3, 4, 5, 4, 3), 2, 1, 0.02),   # Krylov exhaustion on small modes
    ((20, 12, 9), (6, 5), (4, 3), 3, 3, 0.1),
]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _tensor(case):
    dims, gr, _, _, _, noise = case
    rng = np.random.default_rng(101)
    A = W.dense_from_cores(W.random_tt_cores(dims, gr, rng))
    return W.add_noise(A, noise, rng, "gaussian")


def _slab(I_d, rank, world):
    """Contiguous slabs of the last mode; the first ones are one larger when
    I_d is not a multiple of the world size."""
    cuts = [(i * I_d + world - 1) // world for i in range(world + 1)]
    return np.arange(cuts[rank], cuts[rank + 1])


def _allreduce(a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
    dist.all_reduce(t)
    return t.numpy()


def _sharded_tt(A_g, dims, slab, ranks, p, q, omegas, method):
    """Alg. 3 (method "rbki") or Alg. 4 ("rsi") on this rank's slab; products
    with C summed over the ranks.  The subspace iteration takes each step as
    one power, Q <- orth(C (C^T Q)): the span of Alg. 4's two half steps."""
    d = len(dims)
    rr = oracle.clamp_ranks(dims, ranks)
    R_g = A_g
    cores = []
    for k in range(d - 1):
        m = rr[k] * dims[k]
        C_g = np.reshape(R_g, (m, -1))
        lead = int(np.prod(dims[k + 1:d - 1], dtype=np.int64))     # column index j = j' I_d + i_d
        cols = (np.arange(lead)[:, None] * dims[-1] + slab[None, :]).reshape(-1)
        assert C_g.shape[1] == cols.size
        n = lead * dims[-1]
        b = rr[k + 1] + p
        Om_g = np.asarray(omegas[k], dtype=np.float64)[cols]
        D = min(m, n)
        X = oracle.orth_top(_allreduce(C_g @ Om_g), min(b, D))
        Q = X
        for _ in range(q):
            if Q.shape[1] >= D:
                break
            Z = _allreduce(C_g @ (C_g.T @ X))
            if method == "rsi":
                X = Q = oracle.orth_top(Z, Q.shape[1])
                continue
            for _ in range(2):
                Z = Z - Q @ (Q.T @ Z)
            c = min(b, D - Q.shape[1])
            X = oracle.orth_top(Z, c)
            X = oracle.orth_top(X - Q @ (Q.T @ X), c)
            Q = np.hstack([Q, X])
        P_g = Q.T @ C_g
        evals, V = np.linalg.eigh(_allreduce(P_g @ P_g.T))
        U = Q @ V[:, ::-1][:, :rr[k + 1]]
        R_g = U.T @ C_g
        cores.append(U.reshape(rr[k], dims[k], rr[k + 1]))
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, R_g)
    cores.append(np.concatenate(parts, axis=1).reshape(rr[d - 1], dims[d - 1], 1))
    return cores


def _worker(rank, world, port, case, method, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dims, _, ranks, p, q, _ = case
        A = _tensor(case)
        rr = oracle.clamp_ranks(dims, ranks)
        om = W.explicit_omegas(dims, rr, p, 7)
        slab = _slab(dims[-1], rank, world)
        cores = _sharded_tt(np.ascontiguousarray(A[..., slab]), dims, slab, ranks, p, q, om, method)
        ref = (oracle.tt_rsi if method == "rsi" else oracle.tt_rbki)(A, ranks, p, q, omegas=om)
        mine = [c.tobytes() for c in cores]
        theirs = [None] * world
        dist.all_gather_object(theirs, mine)
        out[rank] = dict(distance=oracle.tt_distance(cores, ref),
                         replicated=all(t == mine for t in theirs),
                         shapes=[c.shape for c in cores] == [c.shape for c in ref],
                         slab=int(slab.size))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("method", ["rbki", "rsi"])
@pytest.mark.parametrize("case", CASES)
def test_sharded_matches_single_process_oracle(case, method):
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(2, _free_port(), case, method, out), nprocs=2, join=True,
                           start_method="spawn")
        res = dict(out)
    assert set(res) == {0, 1}
    assert res[0]["slab"] + res[1]["slab"] == case[0][-1] and res[1]["slab"] >= 1
    for r in res.values():
        assert r["shapes"] and r["replicated"]
        assert r["distance"] <= 1e-9, r["distance"]


def test_slabs_partition_the_last_mode():
    for I_d in (2, 3, 5, 7, 16):
        s0, s1 = _slab(I_d, 0, 2), _slab(I_d, 1, 2)
        assert np.array_equal(np.concatenate([s0, s1]), np.arange(I_d)) and s1.size >= 1
