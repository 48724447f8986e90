"""The allocation-free Gram-apply entry point against the workspace one.

tt_gram_apply_noalloc serves callers that cannot allocate device memory
where they call it (inside another framework's capture or memory pool, in
latency-critical loops, in plugins that do not own device memory); its
partial sums live in a fixed 16 MiB array inside the library.  This file is
named so that pytest collects it last.  It checks, through the C ABI, two
calls in a row against tt_pass(TT_PASS_GRAMAPPLY) within the tolerance the
other pass tests use (the workspace pass's BF16 roundings where it takes
the tensor cores), and that sizes beyond the array's limits are refused.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bound_and_ref(C, X):
    Ch = C.float().cpu().double().numpy()
    Xh = X.cpu().double().numpy()
    ref = Ch @ (Ch.T @ Xh)
    bound = np.abs(Ch) @ (np.abs(Ch).T @ np.abs(Xh))
    return ref, float(np.max(bound))


def test_noalloc_gram_apply_matches_workspace_entry_point():
    import paper_2308_01480_gb300 as tt
    from paper_2308_01480_gb300 import _native as N

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    L = N.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    g = torch.Generator(device="cpu").manual_seed(12)
    # two calls in a row with different shapes and dtypes; the second must
    # not see anything left in the shared array by the first
    # (256, 65536, 48): the pass would take 608 CTAs, but the array holds
    # the partials of only 4,194,304 / (256 * 48) = 341, so the cap binds
    for m, n, b, dtype in [(40, 100003, 30, torch.bfloat16), (256, 4097, 40, torch.float32),
                           (256, 65536, 48, torch.bfloat16), (7, 33, 1, torch.float32)]:
        C = torch.randn(m, n, generator=g).to(dtype).cuda()
        X = torch.randn(m, b, generator=g).cuda()
        y = torch.full((m, b), float("nan"), device="cuda")
        code = N.TT_BF16 if dtype == torch.bfloat16 else N.TT_F32
        st = L.tt_gram_apply_noalloc(ctypes.c_void_p(C.data_ptr()), code, m, n, b,
                                     ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(y.data_ptr()), stream)
        assert st == N.TT_OK, L.tt_rbki_last_error()
        y_ws = tt.tt_pass(tt.TT_PASS_GRAMAPPLY, C, x=X)
        torch.cuda.synchronize()
        ref, bound = _bound_and_ref(C, X)
        yh = y.cpu().double().numpy()
        assert np.all(np.isfinite(yh))
        # this entry point runs the FP32 SIMT pass whatever the storage
        assert np.max(np.abs(yh - ref)) <= 1e-5 * bound
        # the workspace pass takes the tensor cores for BF16 storage when n
        # is a multiple of 8 and at least 64, and rounds X and T = C^T X to
        # BF16 there (relative 2^-9 each, so at most 2^-8 of the bound)
        tc = dtype == torch.bfloat16 and n % 8 == 0 and n >= 64
        tol = 2.0 ** -8 + 1e-5 if tc else 1e-5
        assert np.max(np.abs(yh - y_ws.cpu().double().numpy())) <= tol * bound


def test_noalloc_rejects_sizes_beyond_its_limits():
    from paper_2308_01480_gb300 import _native as N

    L = N.lib()
    C = torch.zeros(300, 64, device="cuda")
    X = torch.zeros(300, 8, device="cuda")
    y = torch.zeros(300, 8, device="cuda")
    st = L.tt_gram_apply_noalloc(ctypes.c_void_p(C.data_ptr()), N.TT_F32, 300, 64, 8,
                                 ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(y.data_ptr()), None)
    assert st == N.TT_EUNSUPPORTED
    assert b"m <= 256" in L.tt_rbki_last_error()
    st = L.tt_gram_apply_noalloc(ctypes.c_void_p(C.data_ptr()), N.TT_F32, 10, 64, 49,
                                 ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(y.data_ptr()), None)
    assert st == N.TT_EUNSUPPORTED
    st = L.tt_gram_apply_noalloc(None, N.TT_F32, 10, 64, 8, ctypes.c_void_p(X.data_ptr()),
                                 ctypes.c_void_p(y.data_ptr()), None)
    assert st == N.TT_EINVAL
