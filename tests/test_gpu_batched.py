"""Batched form: many independent TT-rBKI problems of uneven order, mode
sizes and ranks in one call (direct enqueue and one CUDA-graph launch).

Every problem of a batch must equal, bit for bit, the single-problem
decomposition with the same options (the batch runs the same kernels on
the same inputs); sampled problems are also held to the oracle criteria.
The full batched workload (256 problems, 2.7 GB of BF16) is decomposed in
the launch configuration the benchmark uses.
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
    return W.add_noise(A, level, rng)


# uneven orders, ragged modes (tensor-core and SIMT passes), exhaustion and
# Krylov modes, rank clamping, blocks taller than a cluster
SMALL = [
    ((16, 16, 16, 16), (4, 4, 4), 5, 2),
    ((37, 29, 41), (5, 6), 3, 3),
    ((5, 4, 6, 3, 7, 4), (3, 4, 5, 4, 3), 2, 1),
    ((20, 30, 40, 10), (15, 15, 5), 4, 2),
    ((64, 33, 65), (10, 8), 6, 3),
    ((8, 64, 64, 16), (6, 12, 9), 5, 2),
    ((3, 200), (7,), 2, 1),
    ((12, 12, 12, 12, 12), (16, 16, 16, 16), 5, 2),
    ((1100, 6, 5, 4), (8, 6, 4), 4, 2),          # 1100-row blocks: cooperative-launch orthonormalisation
]


def _single(tt, t, ranks, p, q, seed, opts):
    cores, _ = tt.decompose(t, ranks, p, q, omega_seed=seed, opts=opts)
    return cores


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("streams", [1, 3, 0])
def test_batch_bitwise_equals_single(tt, storage, graph, streams):
    code = tt.TT_BF16 if storage == "bf16" else tt.TT_F32
    dt = torch.bfloat16 if storage == "bf16" else torch.float32
    opts = tt.options(storage=code, batch_streams=streams)
    tensors = [torch.from_numpy(_noisy_tt(dims, r, 100 + i, 0.05).astype(np.float32)).cuda().to(dt)
               for i, (dims, r, p, q) in enumerate(SMALL)]
    probs = [tt.Problem(t, r, p, q, 1000 + i) for i, (t, (dims, r, p, q)) in enumerate(zip(tensors, SMALL))]
    if graph:
        g = tt.BatchGraph(probs, opts)
        for c in (c for pb in probs for c in pb.cores):
            c.fill_(float("nan"))
        g.launch()
        torch.cuda.synchronize()
        statuses = g.device_status()
        g.close()
    else:
        ws = tt.decompose_batched(probs, opts)
        torch.cuda.synchronize()
        statuses = tt.batched_device_status(ws, len(probs))
    assert statuses == [0] * len(probs)
    for i, (pb, (dims, r, p, q)) in enumerate(zip(probs, SMALL)):
        ref = _single(tt, tensors[i], r, p, q, 1000 + i, tt.options(storage=code))
        assert pb.rr == oracle.clamp_ranks(dims, r)
        for a, b in zip(pb.cores, ref):
            assert torch.equal(a, b), f"problem {i} differs from the single-problem path"


def test_batch_fp32_matches_oracle(tt):
    """Sampled problems of an FP32 batch against the oracle with the same
    seeded Omega (relative TT distance 1e-4)."""
    opts = tt.options(storage=tt.TT_F32)
    As = [_noisy_tt(dims, r, 200 + i, 0.05) for i, (dims, r, p, q) in enumerate(SMALL)]
    probs = [tt.Problem(torch.from_numpy(A.astype(np.float32)).cuda(), r, p, q, 77 + i)
             for i, (A, (dims, r, p, q)) in enumerate(zip(As, SMALL))]
    ws = tt.decompose_batched(probs, opts)
    torch.cuda.synchronize()
    assert tt.batched_device_status(ws, len(probs)) == [0] * len(probs)
    for i in (0, 2, 4, 7):
        dims, r, p, q = SMALL[i]
        ref = oracle.tt_rbki(As[i].astype(np.float32), r, p, q, seed=77 + i)
        got = [c.cpu().double().numpy() for c in probs[i].cores]
        assert oracle.tt_distance(got, ref) <= 1e-4


def test_batch_rejects_invalid_problem_before_enqueue(tt):
    opts = tt.options(storage=tt.TT_F32)
    good = tt.Problem(torch.ones((8, 8, 8), device="cuda"), (2, 2), 2, 1, 1)
    bad = tt.Problem(torch.ones((8, 8, 8), device="cuda"), (2, 2), 2, 1, 2)
    bad.ranks = [0, 2]
    with pytest.raises(tt.TTError) as e:
        tt.decompose_batched([good, bad], opts)
    assert "problem 1" in str(e.value)
    with pytest.raises(tt.TTError):
        tt.decompose_batched([good], tt.options(storage=tt.TT_F32, batch_streams=65))


def test_batch_empty_is_noop(tt):
    ws = tt.decompose_batched([], tt.options(storage=tt.TT_BF16))
    torch.cuda.synchronize()
    assert ws.numel() >= 1


def test_full_batched_workload(tt):
    """The 256-problem batched workload (orders 3-6, modes 8-64, ranks 2-16,
    5% noise, BF16, p = 5, q = 2) as one graph launch: every status OK,
    every core finite, sampled problems bit-identical to the single path and
    within the BF16 criterion eps_gpu <= 1.05 eps_oracle + 1e-4."""
    ws_list = W.batch_workloads()
    opts = tt.options(storage=tt.TT_BF16)
    rng = np.random.default_rng(5)
    sample = sorted(set([0, int(np.argmax([w.numel for w in ws_list])), int(np.argmin([w.numel for w in ws_list]))]
                        + [int(x) for x in rng.choice(len(ws_list), 3, replace=False)]))
    host = {}
    probs = []
    for i, w in enumerate(ws_list):
        A = W.make_tensor(w)
        if i in sample:
            host[i] = A
        t = torch.from_numpy(A.astype(np.float32)).cuda().to(torch.bfloat16)
        probs.append(tt.Problem(t, w.ranks, w.oversample, w.q, w.omega_seed))
    g = tt.BatchGraph(probs, opts)
    g.launch()
    torch.cuda.synchronize()
    assert g.device_status() == [0] * len(probs)
    for pb in probs:
        for c in pb.cores:
            assert bool(torch.isfinite(c).all())
    for i in sample:
        w = ws_list[i]
        ref_single = _single(tt, probs[i].tensor, w.ranks, w.oversample, w.q, w.omega_seed, opts)
        for a, b in zip(probs[i].cores, ref_single):
            assert torch.equal(a, b)
        got = [c.cpu().double().numpy() for c in probs[i].cores]
        eps_gpu = oracle.tt_error(host[i], got)
        eps_ref = oracle.tt_error(host[i], oracle.tt_rbki(host[i], w.ranks, w.oversample, w.q, seed=w.omega_seed))
        assert eps_gpu <= 1.05 * eps_ref + 1e-4, (i, eps_gpu, eps_ref)
    g.close()
