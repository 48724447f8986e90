"""Host-side checks of the C ABI (no GPU needed).

The library must load and export every function include/tt_rbki.h
declares; the host-only entry points (rank clamp, workspace sizing, argument
validation) are exercised without touching the device.
"""
import ctypes
import os
import re

import pytest

import oracle
from paper_2308_01480_gb300 import _native as N
from paper_2308_01480_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(N.LIB_PATH):
        B.build()
    return N.lib()


def header_functions():
    with open(os.path.join(ROOT, "include", "tt_rbki.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^TT_API\s+[\w\s\*]*?\b(tt_\w+)\s*\(", text, flags=re.M)))


def test_header_and_binding_agree():
    assert header_functions() == N.exported_names()


def test_library_exports_every_declared_symbol(L):
    for name in header_functions():
        assert hasattr(L, name), name


def test_core_sizes_match_oracle_clamp(L):
    cases = [((16, 16, 16, 16), (4, 4, 4)), ((3, 5, 4), (10, 10)), ((2, 2, 2, 2), (9, 9, 9)),
             ((256, 256, 64, 32), (30, 30, 30)), ((40,) * 5, (20,) * 4), ((7, 1, 9), (3, 3))]
    for dims, ranks in cases:
        d = len(dims)
        ro = (ctypes.c_int64 * (d + 1))()
        ce = (ctypes.c_int64 * d)()
        assert L.tt_rbki_core_sizes(N.i64_array(dims), d, N.i64_array(ranks), ro, ce) == N.TT_OK
        rr = oracle.clamp_ranks(dims, ranks)
        assert list(ro) == rr
        assert list(ce) == [rr[k] * dims[k] * rr[k + 1] for k in range(d)]


def test_invalid_arguments_rejected_on_host(L):
    ro = (ctypes.c_int64 * 8)()
    assert L.tt_rbki_core_sizes(N.i64_array([5]), 1, N.i64_array([1]), ro, None) == N.TT_EINVAL
    assert L.tt_rbki_core_sizes(N.i64_array([5, 0, 3]), 3, N.i64_array([1, 1]), ro, None) == N.TT_EINVAL
    assert L.tt_rbki_core_sizes(N.i64_array([5, 4, 3]), 3, N.i64_array([1, 0]), ro, None) == N.TT_EINVAL
    assert b"rank" in L.tt_rbki_last_error()
    nb = ctypes.c_size_t()
    assert L.tt_rbki_workspace_size(N.i64_array([5, 4, 3]), 3, N.i64_array([2, 2]), -1, 1, None,
                                    ctypes.byref(nb)) == N.TT_EINVAL
    # block too wide for the kernels
    assert L.tt_rbki_workspace_size(N.i64_array([100, 100, 100]), 3, N.i64_array([60, 60]), 10, 1, None,
                                    ctypes.byref(nb)) == N.TT_EUNSUPPORTED
    # NULL tensor / workspace are argument errors found before any launch
    cores = N.ptr_array([1, 1, 1])
    st = L.tt_rbki_decompose(None, N.i64_array([5, 4, 3]), 3, N.i64_array([2, 2]), 1, 1,
                             ctypes.c_uint64(1), cores, None, None, 0, None, None)
    assert st == N.TT_EINVAL
    st = L.tt_rbki_decompose(ctypes.c_void_p(256), N.i64_array([5, 4, 3]), 3, N.i64_array([2, 2]), 1, 1,
                             ctypes.c_uint64(1), cores, None, ctypes.c_void_p(256), 0, None, None)
    assert st == N.TT_ENOMEM
    st = L.tt_rbki_decompose(ctypes.c_void_p(256), N.i64_array([5, 4, 3]), 3, N.i64_array([2, 2]), 1, 1,
                             ctypes.c_uint64(1), cores, None, ctypes.c_void_p(257), 1 << 30, None, None)
    assert st == N.TT_EINVAL     # misaligned workspace
    opts = N.TTOptions()
    L.tt_rbki_default_options(ctypes.byref(opts))
    opts.reserved[0] = 1
    assert L.tt_rbki_workspace_size(N.i64_array([5, 4, 3]), 3, N.i64_array([2, 2]), 1, 1, ctypes.byref(opts),
                                    ctypes.byref(nb)) == N.TT_EINVAL
    perm = (ctypes.c_int * 3)(0, 0, 1)
    assert L.tt_permute_convert(ctypes.c_void_p(256), 0, N.i64_array([2, 3, 4]), N.i64_array([12, 4, 1]),
                                perm, 3, ctypes.c_void_p(512), 0, None) == N.TT_EINVAL


def test_workspace_size_grows_with_problem(L):
    nb1, nb2 = ctypes.c_size_t(), ctypes.c_size_t()
    assert L.tt_rbki_workspace_size(N.i64_array([16] * 4), 4, N.i64_array([4] * 3), 5, 2, None,
                                    ctypes.byref(nb1)) == N.TT_OK
    assert L.tt_rbki_workspace_size(N.i64_array([32] * 5), 5, N.i64_array([10] * 4), 5, 3, None,
                                    ctypes.byref(nb2)) == N.TT_OK
    assert 0 < nb1.value < nb2.value
    # 32^5 FP32: two remainder buffers of r_1 n_1 = 10 * 32^4 floats at least
    assert nb2.value >= 2 * 10 * 32 ** 4 * 4
