"""The sharded form's host-side plan (tt_rbki_shard_plan) driving TT-rBKI and
TT-rSI split over ranks by the last mode, on CPU (gloo, world size 2).

Rank g holds the slab A[..., lo_g : lo_g + w_g] of the last mode that the
library's plan assigns it.  Every unfolding of the remainder then splits by
columns, C = [C_g], because the last mode index is part of every column
index (it is the fastest one).  Following the plan's route for each mode,
the ranks sum (gloo all-reduce) exactly the blocks the library's sharded
entry point sums through its callback:
  Krylov route      the sketch C W (m x b) and every power C (C^T X) (m x b)
  Gram-power route  the sketch and the Gram C C^T (m x m) once; the powers
                    G X are then local
  Gram-rows route   the Gram C C^T (m x m)
while the orthonormalisation, Rayleigh-Ritz on H = Q^T W and the cores run
replicated, and the projection R_g = U^T C_g stays on its rank as its slab
of the next unfolding.  The last core is gathered.  The steps are the
oracle's (plain float64 numpy); the library contributes the slabs, the
local column counts, the routes and the number of sums per mode, which
must agree with what the schedule performs.  This checks the reduction
scheme and the library's partitioning on CPU; the device path of the
sharded form is exercised on one GPU by tests/test_gpu_sharded.py.

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


def _allreduce(a, counter):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
    dist.all_reduce(t)
    counter[0] += 1
    return t.numpy()


def _sharded_tt(A_g, dims, lo, w, plan, ranks, p, q, omegas, method):
    """Alg. 3 (method "rbki") or Alg. 4 ("rsi") on this rank's slab, the
    sums over ranks where the plan's route puts them.  The subspace
    iteration takes each step as one power, Q <- orth(C (C^T Q)): the span
    of Alg. 4's two half steps."""
    d = len(dims)
    rr = oracle.clamp_ranks(dims, ranks)
    slab = np.arange(lo, lo + w)
    R_g = A_g
    cores, counts = [], []
    for k in range(d - 1):
        e = plan[k]
        m = rr[k] * dims[k]
        C_g = np.reshape(R_g, (m, -1))
        assert (e["m"], e["n_local"]) == C_g.shape
        lead = int(np.prod(dims[k + 1:d - 1], dtype=np.int64))     # column index j = j' I_d + i_d
        cols = (np.arange(lead)[:, None] * dims[-1] + slab[None, :]).reshape(-1)
        n = lead * dims[-1]
        assert e["n_global"] == n
        b = rr[k + 1] + p
        cnt = [0]
        if e["route"] == "gram_rows":
            G = _allreduce(C_g @ C_g.T, cnt)
            evals, V = np.linalg.eigh(G)
            U = V[:, ::-1][:, :rr[k + 1]]
        else:
            assert e["route"] in ("krylov", "gram_power")
            G = _allreduce(C_g @ C_g.T, cnt) if e["route"] == "gram_power" else None

            def power(X):
                return G @ X if G is not None else _allreduce(C_g @ (C_g.T @ X), cnt)

            Om_g = np.asarray(omegas[k], dtype=np.float64)[cols]
            D = min(m, n)
            X = oracle.orth_top(_allreduce(C_g @ Om_g, cnt), min(b, D))
            Q, Ws = X, []
            if method == "rsi":
                for it in range(q + 1):
                    Z = power(Q)
                    if it < q and Q.shape[1] < D:
                        Q = oracle.orth_top(Z, Q.shape[1])
                    else:
                        Ws = [Z]
                        break
            else:
                while True:
                    Z = power(X)
                    Ws.append(Z)
                    if Q.shape[1] >= D or len(Ws) > q:
                        break
                    for _ in range(2):
                        Z = Z - Q @ (Q.T @ Z)
                    c = min(b, D - Q.shape[1])
                    X = oracle.orth_top(Z, c)
                    X = oracle.orth_top(X - Q @ (Q.T @ X), c)
                    Q = np.hstack([Q, X])
            H = Q.T @ np.hstack(Ws)
            evals, V = np.linalg.eigh(0.5 * (H + H.T))
            U = Q @ V[:, ::-1][:, :rr[k + 1]]
        counts.append(cnt[0])
        R_g = U.T @ C_g
        cores.append(U.reshape(rr[k], dims[k], rr[k + 1]))
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, R_g)
    cores.append(np.concatenate(parts, axis=1).reshape(rr[d - 1], dims[d - 1], 1))
    return cores, counts


def _worker(rank, world, port, case, method, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_2308_01480_gb300 as tt
        dims, _, ranks, p, q, _ = case
        A = _tensor(case)
        rr = oracle.clamp_ranks(dims, ranks)
        om = W.explicit_omegas(dims, rr, p, 7)
        mcode = tt.TT_METHOD_RSI if method == "rsi" else tt.TT_METHOD_RBKI
        lo, w, plan = tt.shard_plan(dims, ranks, p, q, world, rank, tt.options(method=mcode))
        cores, counts = _sharded_tt(np.ascontiguousarray(A[..., lo:lo + w]), dims, lo, w, plan, ranks, p, q, om,
                                    method)
        ref = (oracle.tt_rsi if method == "rsi" else oracle.tt_rbki)(A, ranks, p, q, omegas=om)
        mine = [c.tobytes() for c in cores]
        theirs = [None] * world
        dist.all_gather_object(theirs, mine)
        out[rank] = dict(distance=oracle.tt_distance(cores, ref),
                         replicated=all(t == mine for t in theirs),
                         shapes=[c.shape for c in cores] == [c.shape for c in ref],
                         slab=int(w), lo=int(lo),
                         counts_match=counts == [e["allreduces"] for e in plan])
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
    assert res[0]["lo"] == 0 and res[1]["lo"] == res[0]["slab"]
    for r in res.values():
        assert r["shapes"] and r["replicated"] and r["counts_match"]
        assert r["distance"] <= 1e-9, r["distance"]


def test_plan_slabs_partition_the_last_mode():
    import paper_2308_01480_gb300 as tt
    for I_d in (2, 3, 5, 7, 16):
        for world in (1, 2, 3):
            if world > I_d:
                continue
            slabs = [tt.shard_plan((4, 3, I_d), (2, 2), 1, 1, world, g)[:2] for g in range(world)]
            cover = np.concatenate([np.arange(lo, lo + w) for lo, w in slabs])
            assert np.array_equal(cover, np.arange(I_d)) and min(w for _, w in slabs) >= 1


def test_plan_rejects_what_the_sharded_form_lacks():
    import paper_2308_01480_gb300 as tt
    with pytest.raises(tt.TTError):
        tt.shard_plan((4, 3, 2), (2, 2), 1, 1, 3, 0)               # more ranks than last-mode indices
    with pytest.raises(tt.TTError):
        tt.shard_plan((4, 3, 8), (2, 2), 1, 1, 2, 2)               # rank outside the world
    with pytest.raises(tt.TTError):
        tt.shard_plan((4, 3, 8), (2, 2), 1, 1, 2, 0, tt.options(accurate_rr=True))
    # the column-Gram exhaustion route (the 800 x 40 last unfolding of the
    # 40^5 workload alone) needs every rank's columns: the sharded plan takes
    # the Gram-power route there
    alone = tt.plan_modes((40,) * 5, (20,) * 4, 10, 4, tt.options(storage=tt.TT_BF16))
    _, _, sharded = tt.shard_plan((40,) * 5, (20,) * 4, 10, 4, 2, 1, tt.options(storage=tt.TT_BF16))
    assert alone[-1]["route"] == "gram_cols" and sharded[-1]["route"] == "gram_power"
    assert [e["n_local"] for e in sharded] == [1280000, 32000, 800, 20]
