"""Kernel-level parity: each step-level entry point against the oracle or an
FP64 recomputation of the same inputs, on small odd shapes with ragged
tails.  Runs through the C ABI on the GPU."""
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
    return tt


@pytest.mark.parametrize("seed,k,n,b", [(7, 0, 1000, 9), (2 ** 40 + 5, 3, 4097, 30), (1, 1, 1, 1),
                                        (123, 2, 333, 40), (99, 0, 70001, 13)])
def test_omega_matches_oracle_generator(tt, seed, k, n, b):
    """Device Philox4x32-10 + Box-Muller equals the oracle's float64
    evaluation of the same definition to binary32 rounding of the transform."""
    g = tt.omega_generate(seed, k, n, b).cpu().double().numpy()
    ref = oracle.omega_from_seed(seed, k, n, b)
    assert g.shape == ref.shape
    assert np.max(np.abs(g - ref)) < 4e-6
    gb = tt.omega_generate(seed, k, n, b, dtype=torch.bfloat16).cpu().float()
    rb = torch.from_numpy(ref).float().to(torch.bfloat16).float()
    # identical except where the binary32 value sits on a bf16 rounding boundary
    diff = (gb - rb).abs()
    assert float(diff.max()) <= float(rb.abs().max()) * 2 ** -7
    assert float((diff > 0).float().mean()) < 1e-3


@pytest.mark.parametrize("shape,view_perm,perm", [
    ((5, 7, 3, 9), (2, 0, 3, 1), None),
    ((5, 7, 3, 9), (2, 0, 3, 1), (3, 1, 0, 2)),
    ((4, 1, 6, 5, 3), (0, 1, 2, 3, 4), (4, 3, 2, 1, 0)),
    ((33, 17), (1, 0), (1, 0)),
    ((2, 3, 4, 5, 6, 7), (5, 4, 3, 2, 1, 0), (1, 3, 5, 0, 2, 4)),
])
def test_permute_convert_bit_exact(tt, shape, view_perm, perm):
    g = torch.Generator(device="cpu").manual_seed(3)
    x = torch.randn(*shape, generator=g).cuda()
    xs = x.permute(*view_perm)            # a strided source
    ref = xs.permute(*perm).contiguous() if perm else xs.contiguous()
    out = tt.permute_convert(xs, perm)
    assert out.is_contiguous() and torch.equal(out, ref)
    outb = tt.permute_convert(xs, perm, dst_dtype=torch.bfloat16)
    assert torch.equal(outb, ref.to(torch.bfloat16))       # round-to-nearest-even
    xb = xs.to(torch.bfloat16)
    assert torch.equal(tt.permute_convert(xb, perm), ref.to(torch.bfloat16))
    assert torch.equal(tt.permute_convert(xb, perm, dst_dtype=torch.float32),
                       ref.to(torch.bfloat16).float())


def _rand(shape, seed, dtype=np.float32):
    return np.random.default_rng(seed).standard_normal(shape).astype(dtype)


def _as_dev(a, bf16):
    t = torch.from_numpy(a).cuda()
    return t.to(torch.bfloat16) if bf16 else t


def _host64(t):
    return t.float().cpu().double().numpy()


def _bf16(a):
    """Round-to-nearest-even to bfloat16, returned as float64."""
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).double().numpy()


def _tc_path(n, bf16):
    """BF16 unfoldings whose rows are 16-byte multiples take the tensor-core
    passes, which round the small operand (W, X, and C^T X inside a Krylov
    power) to BF16 by design; the projection keeps FP32 accuracy through a
    hi + lo split of X when b <= 32."""
    return bf16 and n % 8 == 0 and n >= 64


# Shapes with n a multiple of 8 (and n >= 64) take the tensor-core path for
# BF16 unfoldings; tails are ragged against the 64/128-column tiles.
SHAPES = [(1, 1, 1), (7, 31, 9), (40, 4097, 30), (129, 31, 1), (256, 2050, 40), (33, 1000, 15),
          (300, 777, 20), (7, 4097, 40),
          (40, 4104, 30), (256, 2048, 40), (300, 1024, 20), (7, 4104, 40), (129, 1000, 1),
          (800, 2056, 30), (64, 1032, 64), (128, 4096, 16), (1, 64, 8), (200, 72, 33),
          # tall Gram-apply: 128-row chunks, up to the 512-column TMEM limit
          # (1536 x 32 fills it; 1537 x 32 does not fit and falls back)
          (1536, 1024, 32), (897, 2048, 16), (640, 1032, 64), (1537, 1024, 32), (520, 8200, 48)]


@pytest.mark.parametrize("m,n,b", SHAPES)
@pytest.mark.parametrize("bf16", [False, True])
def test_pass_sketch(tt, m, n, b, bf16):
    C = _as_dev(_rand((m, n), 1), bf16)
    W = _rand((n, b), 2)
    y = tt.tt_pass(tt.TT_PASS_SKETCH, C, x=torch.from_numpy(W).cuda())
    Ch = _host64(C)
    Wr = _bf16(W) if _tc_path(n, bf16) else W.astype(np.float64)
    ref = Ch @ Wr
    bound = np.abs(Ch) @ np.abs(W.astype(np.float64))
    assert np.max(np.abs(_host64(y) - ref)) <= 1e-5 * np.max(bound)


@pytest.mark.parametrize("m,n,b", SHAPES)
@pytest.mark.parametrize("bf16", [False, True])
def test_pass_gram_apply(tt, m, n, b, bf16):
    C = _as_dev(_rand((m, n), 3), bf16)
    X = _rand((m, b), 4)
    y = tt.tt_pass(tt.TT_PASS_GRAMAPPLY, C, x=torch.from_numpy(X).cuda())
    Ch = _host64(C)
    bound = np.abs(Ch) @ (np.abs(Ch).T @ np.abs(X.astype(np.float64)))
    if _tc_path(n, bf16):
        # X and T = C^T X rounded to BF16; an FP32 T lying within rounding of
        # a BF16 tie may round the other way, hence the looser factor
        ref = Ch @ _bf16(Ch.T @ _bf16(X))
        assert np.max(np.abs(_host64(y) - ref)) <= 2e-4 * np.max(bound)
    else:
        ref = Ch @ (Ch.T @ X.astype(np.float64))
        assert np.max(np.abs(_host64(y) - ref)) <= 1e-5 * np.max(bound)


@pytest.mark.parametrize("m,n,b", SHAPES)
@pytest.mark.parametrize("bf16", [False, True])
def test_pass_project(tt, m, n, b, bf16):
    C = _as_dev(_rand((m, n), 5), bf16)
    X = _rand((m, b), 6)
    Ch = _host64(C)
    Xr = _bf16(X) if (_tc_path(n, bf16) and b > 32) else X.astype(np.float64)
    ref = Xr.T @ Ch
    bound = np.abs(X.astype(np.float64)).T @ np.abs(Ch)
    y = tt.tt_pass(tt.TT_PASS_PROJECT, C, x=torch.from_numpy(X).cuda())
    assert np.max(np.abs(_host64(y) - ref)) <= 1e-5 * np.max(bound)
    yb = tt.tt_pass(tt.TT_PASS_PROJECT, C, x=torch.from_numpy(X).cuda(), y_dtype=torch.bfloat16)
    assert yb.dtype == torch.bfloat16
    assert np.max(np.abs(_host64(yb) - ref)) <= 2 ** -8 * np.max(np.abs(ref)) + 1e-5 * np.max(bound)


@pytest.mark.parametrize("b", [20, 64])
@pytest.mark.parametrize("bf16_out", [False, True])
def test_pass_project_unaligned_output(tt, b, bf16_out):
    """An output that is not 16-byte aligned takes one scalar store per
    element instead of the staged 16-byte stores; both give the same bits."""
    m, n = 40, 4104
    C = _as_dev(_rand((m, n), 5), True)
    X = torch.from_numpy(_rand((m, b), 6)).cuda()
    dt = torch.bfloat16 if bf16_out else torch.float32
    y = tt.tt_pass(tt.TT_PASS_PROJECT, C, x=X, y_dtype=dt)
    big = torch.zeros(b * n + 1, dtype=dt, device="cuda")
    out = big[1:].view(b, n)
    assert out.data_ptr() % 16 != 0
    tt.tt_pass(tt.TT_PASS_PROJECT, C, x=X, out=out)
    assert torch.equal(out, y)
    assert big[0].item() == 0


@pytest.mark.parametrize("m,n", [(1, 1), (7, 31), (40, 4097), (64, 1000), (128, 333), (100, 65),
                                 (40, 4104), (128, 2048), (100, 1000), (1, 64), (17, 8200)])
@pytest.mark.parametrize("bf16", [False, True])
def test_pass_gram(tt, m, n, bf16):
    C = _as_dev(_rand((m, n), 7), bf16)
    y = tt.tt_pass(tt.TT_PASS_GRAM, C)
    Ch = _host64(C)
    ref = Ch @ Ch.T
    bound = np.abs(Ch) @ np.abs(Ch).T
    assert np.max(np.abs(_host64(y) - ref)) <= 1e-5 * np.max(bound)


def _gram_ref64(C):
    """FP64 Gram of the stored values and its |.| bound, on the device."""
    c = C.double()
    return c @ c.T, c.abs() @ c.abs().T


# 128 < m <= 2048: 128 x 256 tensor-core tiles (BF16, n % 8 == 0), SIMT
# 64 x 64 tiles otherwise; ragged in m against both tile grids and in n
# against the 64-column k-boxes and the split ranges
@pytest.mark.parametrize("m,n", [(129, 64), (200, 1000), (256, 2048), (257, 4104), (300, 777), (511, 520),
                                 (800, 1600), (800, 6400), (1024, 1032), (1500, 2000), (2048, 4096),
                                 (2048, 96), (640, 65), (1111, 8200)])
@pytest.mark.parametrize("bf16", [False, True])
def test_pass_gram_tiled(tt, m, n, bf16):
    C = _as_dev(_rand((m, n), 11), bf16)
    tt.profile_begin(event_timing=False)
    y = tt.tt_pass(tt.TT_PASS_GRAM, C)
    fams = tt.profile_end()
    ref, bound = _gram_ref64(C)
    err = (y.double() - ref).abs().max().item()
    assert err <= 1e-5 * bound.max().item()
    assert torch.equal(y, y.T)                       # both triangles from the same sums
    fam = "gram_tc_tiled" if _tc_path(n, bf16) else "gram_simt_tiled"
    assert fam in fams, fams
    assert torch.equal(tt.tt_pass(tt.TT_PASS_GRAM, C), y)   # fixed-order reduction


@pytest.mark.parametrize("m,c", [(1, 1), (17, 5), (200, 30), (800, 30), (801, 13), (1024, 64), (1537, 40),
                                 (2048, 32), (130, 63)])
def test_gram_power(tt, m, c):
    g = torch.Generator(device="cpu").manual_seed(m + c)
    A = torch.randn(m, m + 3, generator=g)
    G = (A @ A.T).float().cuda()
    ld = (c + 3) // 4 * 4 + 4                  # padded rows, 16-byte aligned
    X = torch.randn(m, ld, generator=g).cuda()[:, :c]
    W = tt.gram_power(G, X)
    ref = G.double() @ X.double()
    bound = G.double().abs() @ X.double().abs()
    assert (W.double() - ref).abs().max().item() <= 1e-5 * bound.max().item()
    assert torch.equal(tt.gram_power(G, X), W)


def test_pass_rejects_unsupported(tt):
    C = torch.zeros((2049, 10), device="cuda")
    with pytest.raises(tt.TTError):
        tt.tt_pass(tt.TT_PASS_GRAM, C)
    with pytest.raises(tt.TTError):
        tt.gram_power(torch.zeros((8, 8), device="cuda"), torch.zeros((8, 68), device="cuda")[:, :65])
    with pytest.raises(tt.TTError):        # rows not 16-byte aligned
        tt.gram_power(torch.zeros((8, 8), device="cuda"), torch.zeros((8, 11), device="cuda")[:, :10])
