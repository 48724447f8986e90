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
    opts.reserved = 1
    assert L.tt_rbki_workspace_size(N.i64_array([5, 4, 3]), 3, N.i64_array([2, 2]), 1, 1, ctypes.byref(opts),
                                    ctypes.byref(nb)) == N.TT_EINVAL
    L.tt_rbki_default_options(ctypes.byref(opts))
    assert opts.gram_power == 1
    opts.gram_power = 2
    assert L.tt_rbki_workspace_size(N.i64_array([5, 4, 3]), 3, N.i64_array([2, 2]), 1, 1, ctypes.byref(opts),
                                    ctypes.byref(nb)) == N.TT_EINVAL
    L.tt_rbki_default_options(ctypes.byref(opts))
    assert opts.paper_literal == 0
    opts.paper_literal = 2
    assert L.tt_rbki_workspace_size(N.i64_array([5, 4, 3]), 3, N.i64_array([2, 2]), 1, 1, ctypes.byref(opts),
                                    ctypes.byref(nb)) == N.TT_EINVAL
    L.tt_rbki_default_options(ctypes.byref(opts))
    assert opts.accurate_rr == 0
    opts.accurate_rr = 2
    assert L.tt_rbki_workspace_size(N.i64_array([5, 4, 3]), 3, N.i64_array([2, 2]), 1, 1, ctypes.byref(opts),
                                    ctypes.byref(nb)) == N.TT_EINVAL
    opts.accurate_rr, opts.paper_literal = 1, 1      # the two study forms exclude each other
    assert L.tt_rbki_workspace_size(N.i64_array([5, 4, 3]), 3, N.i64_array([2, 2]), 1, 1, ctypes.byref(opts),
                                    ctypes.byref(nb)) == N.TT_EINVAL
    opts.paper_literal = 0
    assert L.tt_rbki_workspace_size(N.i64_array([5, 4, 3]), 3, N.i64_array([2, 2]), 1, 1, ctypes.byref(opts),
                                    ctypes.byref(nb)) == N.TT_OK
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


def _problems(specs, keep):
    """tt_problem array for workspace sizing (fake, never dereferenced
    device pointers; sizing reads only the host arrays)."""
    arr = (N.TTProblem * len(specs))()
    for i, (dims, ranks, p, q) in enumerate(specs):
        da, ra = N.i64_array(dims), N.i64_array(ranks)
        cores = N.ptr_array([4096 * (j + 1) for j in range(len(dims))])
        keep += [da, ra, cores]
        arr[i].tensor = 1 << 20
        arr[i].dims = ctypes.cast(da, ctypes.POINTER(ctypes.c_int64))
        arr[i].ranks = ctypes.cast(ra, ctypes.POINTER(ctypes.c_int64))
        arr[i].cores_out = ctypes.cast(cores, ctypes.POINTER(ctypes.c_void_p))
        arr[i].d, arr[i].oversample, arr[i].q = len(dims), p, q
    return arr


def _single_ws(L, dims, ranks, p, q, opts):
    nb = ctypes.c_size_t()
    assert L.tt_rbki_workspace_size(N.i64_array(dims), len(dims), N.i64_array(ranks), p, q, ctypes.byref(opts),
                                    ctypes.byref(nb)) == N.TT_OK
    return nb.value


def _opts(L, streams):
    o = N.TTOptions()
    L.tt_rbki_default_options(ctypes.byref(o))
    o.storage = N.TT_BF16
    o.batch_streams = streams
    return o


SPECS = [((16, 16, 16, 16), (4, 4, 4), 5, 2), ((37, 29, 41), (5, 6), 3, 3), ((64, 8, 64, 8), (9, 12, 5), 5, 2)]


def test_batched_workspace_layout(L):
    """One 256-byte status area per problem plus one region per worker,
    sized for the largest problem the worker runs."""
    keep = []
    arr = _problems(SPECS, keep)
    singles = [_single_ws(L, d, r, p, q, _opts(L, 0)) for d, r, p, q in SPECS]
    nb = ctypes.c_size_t()
    assert L.tt_rbki_batched_workspace_size(1, arr, ctypes.byref(_opts(L, 0)), ctypes.byref(nb)) == N.TT_OK
    assert nb.value == 256 + singles[0]
    assert L.tt_rbki_batched_workspace_size(3, arr, ctypes.byref(_opts(L, 1)), ctypes.byref(nb)) == N.TT_OK
    assert nb.value == 768 + max(singles)
    assert L.tt_rbki_batched_workspace_size(3, arr, ctypes.byref(_opts(L, 3)), ctypes.byref(nb)) == N.TT_OK
    assert nb.value == 768 + sum(singles)
    assert L.tt_rbki_batched_workspace_size(3, arr, ctypes.byref(_opts(L, 2)), ctypes.byref(nb)) == N.TT_OK
    assert 768 + max(singles) <= nb.value <= 768 + sum(singles)
    assert L.tt_rbki_batched_workspace_size(0, None, ctypes.byref(_opts(L, 0)), ctypes.byref(nb)) == N.TT_OK


def test_batched_invalid_arguments(L):
    keep = []
    arr = _problems(SPECS, keep)
    nb = ctypes.c_size_t()
    assert L.tt_rbki_batched_workspace_size(-1, arr, None, ctypes.byref(nb)) == N.TT_EINVAL
    assert L.tt_rbki_batched_workspace_size(2, None, None, ctypes.byref(nb)) == N.TT_EINVAL
    assert L.tt_rbki_batched_workspace_size(3, arr, ctypes.byref(_opts(L, 65)), ctypes.byref(nb)) == N.TT_EINVAL
    arr[1].reserved = 1
    assert L.tt_rbki_batched_workspace_size(3, arr, None, ctypes.byref(nb)) == N.TT_EINVAL
    assert b"problem 1" in L.tt_rbki_last_error()
    arr[1].reserved = 0
    bad = N.i64_array([4, 0])
    keep.append(bad)
    arr[2].ranks = ctypes.cast(bad, ctypes.POINTER(ctypes.c_int64))
    arr[2].d = 3
    per = (ctypes.c_int * 3)()
    # invalid problem: rejected on the host with per-problem statuses, before any device call
    assert L.tt_rbki_decompose_batched(3, arr, ctypes.c_void_p(256), 1 << 30, None, None, per) == N.TT_EINVAL
    assert list(per) == [N.TT_OK, N.TT_OK, N.TT_EINVAL]
    arr[2].tensor = None
    arr[2].ranks = arr[0].ranks
    assert L.tt_rbki_decompose_batched(3, arr, ctypes.c_void_p(256), 1 << 30, None, None, per) == N.TT_EINVAL
    assert b"tensor is NULL" in L.tt_rbki_last_error()
    h = ctypes.c_void_p()
    assert L.tt_rbki_graph_launch(None, None) == N.TT_EINVAL
    assert L.tt_rbki_graph_destroy(None) == N.TT_OK
    assert L.tt_rbki_batched_graph_create(3, arr, ctypes.c_void_p(256), 1 << 30, None, per,
                                          ctypes.byref(h)) == N.TT_EINVAL


def test_method_option_validated(L):
    o = N.TTOptions()
    L.tt_rbki_default_options(ctypes.byref(o))
    assert o.method == N.TT_METHOD_RBKI
    nb = ctypes.c_size_t()
    dims, ranks = N.i64_array([16] * 4), N.i64_array([4] * 3)
    o.method = N.TT_METHOD_RSI
    assert L.tt_rbki_workspace_size(dims, 4, ranks, 5, 2, ctypes.byref(o), ctypes.byref(nb)) == N.TT_OK
    rsi = nb.value
    o.method = N.TT_METHOD_RBKI
    assert L.tt_rbki_workspace_size(dims, 4, ranks, 5, 2, ctypes.byref(o), ctypes.byref(nb)) == N.TT_OK
    assert rsi > 0 and nb.value > 0
    o.method = 2
    assert L.tt_rbki_workspace_size(dims, 4, ranks, 5, 2, ctypes.byref(o), ctypes.byref(nb)) == N.TT_EINVAL


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C compiler's field
    offsets, field sizes and total size."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"tt_options": N.TTOptions, "tt_mode_plan": N.TTModePlan, "tt_problem": N.TTProblem,
               "tt_kernel_stat": N.TTKernelStat}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "tt_rbki.h"', "int main(void) {"]
    for cname, cls in mirrors.items():
        lines.append(f'  printf("{cname} . %zu %zu\\n", (size_t)0, sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu %zu\\n", offsetof({cname}, {fname}), '
                         f"sizeof((({cname}*)0)->{fname}));")
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for line in filter(None, out):
        cname, fname, off, size = line.split()
        cls = mirrors[cname]
        if fname == ".":
            assert ctypes.sizeof(cls) == int(size), cname
        else:
            field = getattr(cls, fname)
            assert (field.offset, field.size) == (int(off), int(size)), (cname, fname)
        seen += 1
    assert seen == sum(len(c._fields_) + 1 for c in mirrors.values())


def test_order_limit_and_noalloc_arguments_rejected_on_host(L):
    """The order limit (d <= 64: the final kernel checks the other d - 1
    cores in one launch) and the allocation-free Gram-apply's argument and
    size checks, all taken before any CUDA call."""
    nb = ctypes.c_size_t()
    for d, want in ((64, N.TT_OK), (65, N.TT_EINVAL)):
        dims, ranks = [1] * (d - 2) + [3, 4], [1] * (d - 1)
        assert L.tt_rbki_workspace_size(N.i64_array(dims), d, N.i64_array(ranks), 1, 1, None,
                                        ctypes.byref(nb)) == want
    p = ctypes.c_void_p(256)
    cases = [((None, N.TT_F32, 10, 64, 8), N.TT_EINVAL, b"NULL"),
             ((p, 7, 10, 64, 8), N.TT_EINVAL, b"c_dtype"),
             ((p, N.TT_F32, 0, 64, 8), N.TT_EINVAL, b">= 1"),
             ((p, N.TT_BF16, 257, 64, 8), N.TT_EUNSUPPORTED, b"m <= 256"),
             ((p, N.TT_BF16, 10, 64, 49), N.TT_EUNSUPPORTED, b"b <= 48")]
    for (C, dt, m, n, b), want, msg in cases:
        assert L.tt_gram_apply_noalloc(C, dt, m, n, b, p, p, None) == want
        assert msg in L.tt_rbki_last_error()
