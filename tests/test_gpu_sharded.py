"""The sharded form (tt_rbki_decompose_sharded) on one GPU.

World size 1: the same kernels and the same arithmetic as tt_rbki_decompose,
so the cores must be bit-identical.  World size 2: two ranks emulated by two
host threads, each on its own stream with its own slab of the last mode;
the sum callback synchronises its stream, exchanges the partial block with
the other thread on the host and writes the sum back (the same sum on both
ranks).  No kernel waits on another rank's kernel: the ranks meet only on
the host.  The replicated cores must be bit-identical across the ranks, the
gathered last core completes the TT, and the whole TT matches the oracle
(FP32, Omega drawn from the seed) within relative TT distance 1e-4, with as
many sums per mode as the library's plan states."""
import threading

import numpy as np
import pytest

import oracle
from paper_2308_01480_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    # dims, generating ranks, target ranks, p, q, noise
    ((6, 7, 8, 5), (3, 4, 2), (3, 4, 2), 2, 2, 0.05),
    ((9, 10, 11, 7), (3, 5, 4), (3, 5, 4), 3, 2, 0.02),
    ((20, 30, 40, 10), (15, 15, 5), (15, 15, 5), 4, 2, 0.03),
    ((24, 32, 40, 16), (6, 8, 4), (6, 8, 4), 4, 3, 0.03),
]


@pytest.fixture(scope="module")
def tt():
    import paper_2308_01480_gb300 as tt
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    tt._native.lib()
    return tt


def _tensor(case, seed=101):
    dims, gr, _, _, _, noise = case
    rng = np.random.default_rng(seed)
    A = W.dense_from_cores(W.random_tt_cores(dims, gr, rng))
    return W.add_noise(A, noise, rng)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_world_one_bit_identical(tt, case, storage):
    dims, _, ranks, p, q, _ = case
    A = _tensor(case)
    t = torch.from_numpy(A.astype(np.float32)).cuda()
    code = tt.TT_F32
    if storage == "bf16":
        t, code = t.to(torch.bfloat16), tt.TT_BF16
    opts = tt.options(storage=code)
    ref, _ = tt.decompose(t, ranks, p, q, omega_seed=5, opts=opts)
    got, _ = tt.decompose_sharded(t, dims, ranks, p, q, 1, 0, lambda buf: None, omega_seed=5, opts=opts)
    torch.cuda.synchronize()
    assert tt.device_status(tt.decompose_sharded.last_workspace) == 0
    for a, b in zip(ref, got):
        assert torch.equal(a, b)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("method", ["rbki", "rsi"])
def test_two_ranks_match_oracle(tt, case, method):
    dims, _, ranks, p, q, _ = case
    A = _tensor(case)
    world, seed = 2, 9
    mcode = tt.TT_METHOD_RSI if method == "rsi" else tt.TT_METHOD_RBKI
    opts = tt.options(storage=tt.TT_F32, method=mcode)
    barrier = threading.Barrier(world)
    shared = [None] * world
    calls = [[0] for _ in range(world)]
    out, errs = [None] * world, []

    def rank_main(g):
        try:
            lo, w, modes = tt.shard_plan(dims, ranks, p, q, world, g, opts)
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                local = torch.from_numpy(np.ascontiguousarray(A[..., lo:lo + w], dtype=np.float32)).cuda()

                def allreduce(buf):
                    torch.cuda.current_stream().synchronize()
                    shared[g] = buf.cpu()
                    barrier.wait()
                    total = shared[0] + shared[1]
                    barrier.wait()
                    buf.copy_(total.to(buf.device))
                    calls[g][0] += 1

                cores, _ = tt.decompose_sharded(local, dims, ranks, p, q, world, g, allreduce, omega_seed=seed,
                                                opts=opts)
                stream.synchronize()
                st = tt.device_status(tt.decompose_sharded.last_workspace)
            out[g] = (lo, w, modes, [c.cpu() for c in cores], st)
        except Exception as e:          # surfaced below
            errs.append(e)
            barrier.abort()

    th = [threading.Thread(target=rank_main, args=(g,)) for g in range(world)]
    for x in th:
        x.start()
    for x in th:
        x.join(timeout=300)
    assert not errs, errs
    assert all(o is not None for o in out)
    for g in range(world):
        assert out[g][4] == 0
        assert calls[g][0] == sum(e["allreduces"] for e in out[g][2])
    for a, b in zip(out[0][3][:-1], out[1][3][:-1]):
        assert torch.equal(a, b)                 # replicated cores
    cores = [c.double().numpy() for c in out[0][3][:-1]]
    cores.append(np.concatenate([out[g][3][-1].double().numpy() for g in range(world)], axis=1))
    ref = (oracle.tt_rsi if method == "rsi" else oracle.tt_rbki)(A.astype(np.float32), ranks, p, q, seed=seed)
    assert oracle.tt_distance(cores, ref) <= 1e-4
