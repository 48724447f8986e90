"""Launch shapes from the tuning table compute the same passes: every knob
value of every BF16 tensor-core pass against the FP64 reference of the same
inputs, with the tolerances of the built-in shapes (test_gpu_kernels.py),
on unfoldings with ragged tails; and the bench workload's decomposition
with the committed table agrees with the built-in shapes'."""
import os

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tt():
    import paper_2308_01480_gb300 as tt
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    tt._native.lib()
    yield tt
    if os.path.exists(tt._native.TUNE_TABLE):
        tt.tune_load(tt._native.TUNE_TABLE)
    else:
        tt.tune_clear()


def _data(m, n, b, seed, op, tt):
    g = np.random.default_rng(seed)
    C = torch.from_numpy(g.standard_normal((m, n)).astype(np.float32)).cuda().to(torch.bfloat16)
    if op == tt.TT_PASS_SKETCH:
        X = g.standard_normal((n, b)).astype(np.float32)
    elif op == tt.TT_PASS_GRAM:
        X = None
    else:
        X = g.standard_normal((m, b)).astype(np.float32)
    return C, X


def _bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).double().numpy()


def _check(tt, op, C, X):
    Ch = C.double().cpu().numpy()
    x = torch.from_numpy(X).cuda() if X is not None else None
    if op == tt.TT_PASS_GRAM:
        y = tt.tt_pass(op, C)
        ref, bound = Ch @ Ch.T, np.abs(Ch) @ np.abs(Ch).T
        tol = 1e-5
    elif op == tt.TT_PASS_SKETCH:
        y = tt.tt_pass(op, C, x=x)
        ref, bound = Ch @ _bf16(X), np.abs(Ch) @ np.abs(X.astype(np.float64))
        tol = 1e-5
    elif op == tt.TT_PASS_GRAMAPPLY:
        y = tt.tt_pass(op, C, x=x)
        ref = Ch @ _bf16(Ch.T @ _bf16(X))
        bound = np.abs(Ch) @ (np.abs(Ch).T @ np.abs(X.astype(np.float64)))
        tol = 2e-4
    else:
        y = tt.tt_pass(op, C, x=x)
        b = X.shape[1]
        Xr = _bf16(X) if b > 32 else X.astype(np.float64)
        ref, bound = Xr.T @ Ch, np.abs(X.astype(np.float64)).T @ np.abs(Ch)
        tol = 1e-5
    err = np.max(np.abs(y.double().cpu().numpy() - ref))
    assert err <= tol * np.max(bound), err
    return y


def _entries(tt, op, m):
    out = []
    for st in (2, 3, 5, 8):
        for per in (1, 2):
            if op == tt.TT_PASS_GRAM:
                out += [(st, per, kb, 0) for kb in (1, 2, 4, 8)]
            elif op == tt.TT_PASS_PROJECT and m > 128:
                out += [(st, per, 0, cr) for cr in (64, 128)]
            else:
                out.append((st, per, 0, 0))
    return out


CASES = [("gram", 40, 8200, 0), ("gram", 128, 4104, 0), ("gram", 17, 2056, 0),
         ("project", 40, 8200, 20), ("project", 300, 2056, 20), ("project", 800, 1032, 40),
         ("sketch", 300, 2056, 30), ("sketch", 40, 4104, 48),
         ("gram_apply", 256, 2056, 40), ("gram_apply", 897, 1032, 16)]


@pytest.mark.parametrize("name,m,n,b", CASES)
def test_tuned_shapes_compute_the_pass(tt, name, m, n, b):
    op = {"gram": tt.TT_PASS_GRAM, "project": tt.TT_PASS_PROJECT, "sketch": tt.TT_PASS_SKETCH,
          "gram_apply": tt.TT_PASS_GRAMAPPLY}[name]
    C, X = _data(m, n, b, 5 + m, op, tt)
    key = tt.tune_key(op, m, n, b)
    tt.tune_clear()
    y0 = _check(tt, op, C, X)
    differs = 0
    for e in _entries(tt, op, m):
        tt.tune_clear()
        tt.tune_set(key, *e)
        y = _check(tt, op, C, X)
        differs += int(not torch.equal(y, y0))
    tt.tune_clear()
    assert torch.equal(_check(tt, op, C, X), y0)      # the built-in shape again, bit for bit
    if op == tt.TT_PASS_GRAM:
        # other stage widths and grids regroup the FP32 partial sums: the
        # entries took effect
        assert differs > 0


def test_decompose_with_committed_table(tt):
    """The 40^5 BF16 bench workload (whose unfoldings the sweep tuned) with
    the committed table and with the built-in shapes: the same TT error to
    the order of FP32 partial sums, and orthonormal cores.  (The full-size
    tests compare it with the oracle; they run with the table loaded.)"""
    if not os.path.exists(tt._native.TUNE_TABLE):
        pytest.skip("no committed tuning table")
    from paper_2308_01480_gb300 import workloads as W
    w = W.CONFIGS[3]
    A = W.make_tensor(w)
    t = tt.permute_convert(torch.from_numpy(A.astype(np.float32)).cuda(), dst_dtype=torch.bfloat16)
    o = tt.options(storage=tt.TT_BF16, remainder=tt.TT_BF16)
    eps = []
    for table in (True, False):
        if table:
            tt.tune_load(tt._native.TUNE_TABLE)
            assert tt.tune_entries() > 0
        else:
            tt.tune_clear()
        cores, _ = tt.decompose(t, w.ranks, w.oversample, w.q, omega_seed=w.omega_seed, opts=o)
        torch.cuda.synchronize()
        assert tt.device_status(tt.decompose.last_workspace) == 0
        got = [c.cpu().double().numpy() for c in cores]
        for G in got[:-1]:
            assert oracle.left_orthogonality_defect(G) < 1e-4
        eps.append(oracle.tt_error(A, got))
    assert abs(eps[0] - eps[1]) <= 1e-3 * eps[1], eps
