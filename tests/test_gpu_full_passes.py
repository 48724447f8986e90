"""Element-wise parity of the streaming passes at the full unfolding shapes
the benchmark runs: 40 x 2,560,000 and 800 x 64,000 (modes 1 and 2 of the
40^5 workload) and 256 x 524,288 (mode 1 of the 256 x 256 x 64 x 32 one),
all BF16 on the tensor cores, each CTA working through hundreds of column
tiles and many wrap-arounds of its shared-memory ring.  Every output entry
is compared with an FP64 recomputation of the same stored operands on the
device (the same BF16 roundings the kernels apply by design), at the
tolerances of the small-shape pass tests."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FULL = [(40, 2_560_000), (800, 64_000), (256, 524_288)]


@pytest.fixture(scope="module")
def tt():
    import paper_2308_01480_gb300 as tt
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    tt._native.lib()
    return tt


def _c(m, n, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    return torch.randn(m, n, generator=g, device="cuda").to(torch.bfloat16)


def _x(rows, cols, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    return torch.randn(rows, cols, generator=g, device="cuda")


def _bf(t):
    return t.to(torch.bfloat16).double()


def _check(y, ref, bound, rel):
    err = (y.double() - ref).abs()
    lim = rel * bound.max().item()
    assert err.max().item() <= lim, (err.max().item(), lim, int((err > lim).sum()))


@pytest.mark.parametrize("m,n", FULL)
def test_full_sketch(tt, m, n):
    b = 30 if m != 256 else 40
    C = _c(m, n, 1)
    Wm = _x(n, b, 2)
    y = tt.tt_pass(tt.TT_PASS_SKETCH, C, x=Wm)
    c = C.double()
    _check(y, c @ _bf(Wm), c.abs() @ Wm.double().abs(), 1e-5)


@pytest.mark.parametrize("m,n", FULL)
def test_full_project(tt, m, n):
    b = 20 if m != 256 else 30
    C = _c(m, n, 3)
    X = _x(m, b, 4)
    c = C.double()
    ref = X.double().T @ c               # b <= 32: FP32-accurate hi + lo split
    bound = X.double().abs().T @ c.abs()
    _check(tt.tt_pass(tt.TT_PASS_PROJECT, C, x=X), ref, bound, 1e-5)
    yb = tt.tt_pass(tt.TT_PASS_PROJECT, C, x=X, y_dtype=torch.bfloat16)
    err = (yb.double() - ref).abs().max().item()
    assert err <= 2 ** -8 * ref.abs().max().item() + 1e-5 * bound.max().item()


@pytest.mark.parametrize("m,n", FULL)
def test_full_gram_apply(tt, m, n):
    b = 30 if m != 256 else 40
    C = _c(m, n, 5)
    X = _x(m, b, 6)
    y = tt.tt_pass(tt.TT_PASS_GRAMAPPLY, C, x=X)
    c = C.double()
    ref = c @ _bf(c.T @ _bf(X))          # X and T = C^T X rounded to BF16 by design
    bound = c.abs() @ (c.abs().T @ X.double().abs())
    _check(y, ref, bound, 2e-4)


@pytest.mark.parametrize("m,n", [(40, 2_560_000), (800, 64_000), (800, 1600)])
def test_full_gram(tt, m, n):
    """m = 40: the one-tile Gram pass of the exhaustion route; m = 800: the
    tiled tensor-core Gram of the Gram-power route at modes 2 and 3."""
    C = _c(m, n, 7)
    y = tt.tt_pass(tt.TT_PASS_GRAM, C)
    c = C.double()
    _check(y, c @ c.T, c.abs() @ c.abs().T, 1e-5)
    assert torch.equal(y, y.T)
