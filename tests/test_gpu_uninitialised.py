"""No kernel may read memory it has not written: results must not depend on
what the workspace or shared memory held before the call.

Each case runs twice: once with a zeroed workspace, once with a workspace of
0xFF bytes (NaN as float32, negative NaN as bfloat16) after every SM's
shared memory has been filled with NaN.  The two results must be finite and
bit-identical.  (A memory-checking tool is not available, so this stands in
for its uninitialised-read check.)
"""
import numpy as np
import pytest

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


CASES = [
    ((16, 16, 16, 16), (4, 4, 4), 5, 2),
    ((37, 29, 41), (5, 6), 3, 3),
    ((5, 4, 6, 3, 7, 4), (3, 4, 5, 4, 3), 2, 1),
    ((20, 30, 40, 10), (15, 15, 5), 4, 2),
    ((64, 33, 65), (10, 8), 6, 3),
    ((8, 64, 64, 16), (6, 12, 9), 5, 2),
    ((3, 200), (7,), 2, 1),
    ((12, 12, 12, 12, 12), (16, 16, 16, 16), 5, 2),
    ((24, 24, 24, 24), (10, 10, 10), 10, 4),
    ((256, 16, 64), (30, 20), 10, 3),
]


def _run(tt, t, dims, r, p, q, seed, opts, poison):  # noqa: D401
    need = tt.workspace_size(dims, r, p, q, opts)
    ws = torch.full((need,), 255 if poison else 0, dtype=torch.uint8, device="cuda")
    rr, _ = tt.core_sizes(dims, r)
    cores = [torch.full((rr[k], dims[k], rr[k + 1]), float("nan") if poison else 0.0, device="cuda")
             for k in range(len(dims))]
    if poison:
        tt.debug_fill_shared()
    tt.decompose(t, r, p, q, omega_seed=seed, opts=opts, workspace=ws, cores=cores)
    torch.cuda.synchronize()
    assert tt.device_status(ws) == 0
    return cores


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("exhaust,method", [(True, 0), (False, 0), (True, 1)])
def test_decompose_ignores_prior_memory_contents(tt, case, storage, exhaust, method):
    dims, r, p, q = case
    code = tt.TT_BF16 if storage == "bf16" else tt.TT_F32
    dt = torch.bfloat16 if storage == "bf16" else torch.float32
    opts = tt.options(storage=code, exhaust_gram=exhaust, method=method)
    t = torch.from_numpy(_noisy_tt(dims, r, 31, 0.05).astype(np.float32)).cuda().to(dt)
    clean = _run(tt, t, dims, r, p, q, 5, opts, False)
    dirty = _run(tt, t, dims, r, p, q, 5, opts, True)
    for a, b in zip(clean, dirty):
        assert bool(torch.isfinite(a).all())
        assert torch.equal(a, b)


PASS_SHAPES = [(7, 31, 9), (40, 4104, 30), (300, 1024, 20), (129, 1000, 1), (200, 72, 33), (64, 1032, 64),
               (800, 2056, 30), (1536, 1024, 32)]


@pytest.mark.parametrize("m,n,b", PASS_SHAPES)
@pytest.mark.parametrize("op", ["sketch", "gramapply", "project"])
@pytest.mark.parametrize("bf16", [False, True])
def test_passes_ignore_prior_memory_contents(tt, m, n, b, op, bf16):
    code = {"sketch": tt.TT_PASS_SKETCH, "gramapply": tt.TT_PASS_GRAMAPPLY, "project": tt.TT_PASS_PROJECT}[op]
    g = torch.Generator(device="cpu").manual_seed(9)
    C = torch.randn(m, n, generator=g).cuda()
    if bf16:
        C = C.to(torch.bfloat16)
    x = torch.randn(n if op == "sketch" else m, b, generator=g).cuda()
    cdt = tt.TT_BF16 if bf16 else tt.TT_F32
    need = tt.pass_workspace_size(code, m, n, b, cdt)
    shape = (b, n) if op == "project" else (m, b)
    outs = []
    for poison in (False, True):
        ws = torch.full((need,), 255 if poison else 0, dtype=torch.uint8, device="cuda")
        out = torch.full(shape, float("nan") if poison else 0.0, device="cuda")
        if poison:
            tt.debug_fill_shared()
        y = tt.tt_pass(code, C, x=x, workspace=ws, out=out)
        torch.cuda.synchronize()
        outs.append(y)
    assert bool(torch.isfinite(outs[0].float()).all())
    assert torch.equal(outs[0], outs[1])
