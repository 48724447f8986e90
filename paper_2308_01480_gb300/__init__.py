"""GB300 randomized block Krylov tensor-train approximation (TT-rBKI).

Python binding of the C ABI in include/tt_rbki.h.  Every function here only
marshals arguments: buffers are torch tensors on the current CUDA device,
work is enqueued on torch's current stream, and all arithmetic runs in the
library's CUDA kernels.  There is no CPU path.
"""
import ctypes

from . import _native as N
from ._native import (TT_BF16, TT_F32, TT_PASS_GRAM, TT_PASS_GRAMAPPLY,  # noqa: F401
                      TT_PASS_PROJECT, TT_PASS_SKETCH, TTError)

__all__ = ["decompose", "workspace_size", "core_sizes", "omega_generate", "permute_convert",
           "tt_pass", "device_status", "options", "profile_begin", "profile_end", "TTError", "TT_F32",
           "TT_BF16"]


def _torch():
    import torch
    return torch


def _dtype_code(t):
    torch = _torch()
    if t.dtype == torch.float32:
        return N.TT_F32
    if t.dtype == torch.bfloat16:
        return N.TT_BF16
    raise TypeError(f"unsupported dtype {t.dtype}")


def _stream_handle(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def options(storage=N.TT_F32, remainder=None, exhaust_gram=True):
    """tt_options with the given fields (remainder None = same as storage)."""
    o = N.TTOptions()
    N.check(N.lib().tt_rbki_default_options(ctypes.byref(o)))
    o.storage = int(storage)
    o.remainder = -1 if remainder is None else int(remainder)
    o.exhaust_gram = 1 if exhaust_gram else 0
    return o


def core_sizes(dims, ranks):
    """(clamped ranks r_0..r_d, core element counts)."""
    d = len(dims)
    ro = (ctypes.c_int64 * (d + 1))()
    ce = (ctypes.c_int64 * d)()
    N.check(N.lib().tt_rbki_core_sizes(N.i64_array(dims), d, N.i64_array(ranks), ro, ce))
    return list(ro), list(ce)


def workspace_size(dims, ranks, oversample, q, opts=None):
    nbytes = ctypes.c_size_t()
    N.check(N.lib().tt_rbki_workspace_size(N.i64_array(dims), len(dims), N.i64_array(ranks),
                                           int(oversample), int(q),
                                           ctypes.byref(opts) if opts is not None else None,
                                           ctypes.byref(nbytes)))
    return nbytes.value


def decompose(tensor, ranks, oversample, q, omega_seed=0, omegas=None, opts=None, workspace=None,
              cores=None, stream=None):
    """TT-rBKI of a dense row-major CUDA tensor.

    tensor : torch CUDA tensor (float32 or bfloat16), contiguous; its dtype
             must match opts.storage.
    omegas : optional list of d-1 float32 CUDA tensors (n_k x (r_k' + p));
             when given the explicit-Omega entry point is used.
    Returns (cores, ranks) with cores a list of float32 CUDA tensors of shape
    (r_{k-1}, I_k, r_k).  Work is enqueued on the current stream.
    """
    torch = _torch()
    if not tensor.is_cuda or not tensor.is_contiguous():
        raise ValueError("tensor must be a contiguous CUDA tensor")
    dims = list(tensor.shape)
    d = len(dims)
    if opts is None:
        opts = options(storage=_dtype_code(tensor))
    if _dtype_code(tensor) != opts.storage:
        raise ValueError("tensor dtype does not match opts.storage")
    rr, counts = core_sizes(dims, ranks)
    if cores is None:
        cores = [torch.empty((rr[k], dims[k], rr[k + 1]), dtype=torch.float32, device=tensor.device)
                 for k in range(d)]
    need = workspace_size(dims, ranks, oversample, q, opts)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=tensor.device)
    ranks_out = (ctypes.c_int64 * (d + 1))()
    core_ptrs = N.ptr_array([c.data_ptr() for c in cores])
    st = _stream_handle(stream)
    if omegas is None:
        status = N.lib().tt_rbki_decompose(
            ctypes.c_void_p(tensor.data_ptr()), N.i64_array(dims), d, N.i64_array(ranks),
            int(oversample), int(q), ctypes.c_uint64(omega_seed), core_ptrs, ranks_out,
            ctypes.c_void_p(workspace.data_ptr()), workspace.numel(), st, ctypes.byref(opts))
    else:
        for o in omegas:
            if o is not None and (not o.is_cuda or o.dtype != torch.float32 or not o.is_contiguous()):
                raise ValueError("omegas must be contiguous float32 CUDA tensors")
        om_ptrs = N.ptr_array([o.data_ptr() if o is not None else 0 for o in omegas])
        status = N.lib().tt_rbki_decompose_omega(
            ctypes.c_void_p(tensor.data_ptr()), N.i64_array(dims), d, N.i64_array(ranks),
            int(oversample), int(q), om_ptrs, core_ptrs, ranks_out,
            ctypes.c_void_p(workspace.data_ptr()), workspace.numel(), st, ctypes.byref(opts))
    N.check(status)
    decompose.last_workspace = workspace
    return cores, list(ranks_out)


def profile_begin(event_timing=True):
    """Start counting kernel launches (and timing them with CUDA events)."""
    N.check(N.lib().tt_rbki_profile_begin(1 if event_timing else 0))


def profile_end():
    """Stop accounting; returns {family: dict(launches, ms, bytes, flops)}."""
    arr = (N.TTKernelStat * 64)()
    n = ctypes.c_int()
    N.check(N.lib().tt_rbki_profile_end(arr, 64, ctypes.byref(n)))
    return {arr[i].name.decode(): dict(launches=arr[i].launches, ms=arr[i].ms, bytes=arr[i].bytes,
                                       flops=arr[i].flops) for i in range(n.value)}


def device_status(workspace, stream=None):
    """Device status word of the last decomposition that used `workspace`."""
    out = ctypes.c_int()
    N.check(N.lib().tt_rbki_device_status(ctypes.c_void_p(workspace.data_ptr()), _stream_handle(stream),
                                          ctypes.byref(out)))
    return out.value


def omega_generate(seed, mode, n, b, dtype=None, device="cuda", stream=None):
    """Omega_k (n x b) drawn on the device (Philox4x32-10 + Box-Muller)."""
    torch = _torch()
    dtype = dtype or torch.float32
    out = torch.empty((n, b), dtype=dtype, device=device)
    code = N.TT_BF16 if dtype == torch.bfloat16 else N.TT_F32
    N.check(N.lib().tt_omega_generate(ctypes.c_uint64(seed), int(mode), int(n), int(b),
                                      ctypes.c_void_p(out.data_ptr()), code, int(b), _stream_handle(stream)))
    return out


def permute_convert(src, perm=None, dst_dtype=None, stream=None):
    """Dense row-major copy of a (possibly strided) CUDA tensor with modes
    permuted (destination mode j = source mode perm[j]) and dtype converted."""
    torch = _torch()
    d = src.dim()
    perm = list(range(d)) if perm is None else [int(p) for p in perm]
    dst_dtype = dst_dtype or src.dtype
    out = torch.empty([src.shape[p] for p in perm], dtype=dst_dtype, device=src.device)
    cperm = (ctypes.c_int * d)(*perm)
    N.check(N.lib().tt_permute_convert(ctypes.c_void_p(src.data_ptr()), _dtype_code(src),
                                       N.i64_array(src.shape), N.i64_array(src.stride()), cperm, d,
                                       ctypes.c_void_p(out.data_ptr()), _dtype_code(out),
                                       _stream_handle(stream)))
    return out


def tt_pass(op, C, b=None, x=None, y_dtype=None, stream=None):
    """One streaming pass over the unfolding C (2-D CUDA tensor), see tt_pass
    in the header.  Returns the output tensor."""
    torch = _torch()
    m, n = C.shape
    if op == N.TT_PASS_GRAM:
        b = 0
        out = torch.empty((m, m), dtype=torch.float32, device=C.device)
    elif op == N.TT_PASS_PROJECT:
        b = x.shape[1]
        out = torch.empty((b, n), dtype=y_dtype or torch.float32, device=C.device)
    else:
        b = x.shape[1]
        out = torch.empty((m, b), dtype=torch.float32, device=C.device)
    nbytes = ctypes.c_size_t()
    N.check(N.lib().tt_pass_workspace_size(int(op), m, n, int(b), _dtype_code(C), ctypes.byref(nbytes)))
    ws = torch.empty(nbytes.value, dtype=torch.uint8, device=C.device)
    N.check(N.lib().tt_pass(int(op), ctypes.c_void_p(C.data_ptr()), _dtype_code(C), m, n, int(b),
                            ctypes.c_void_p(x.data_ptr() if x is not None else 0),
                            ctypes.c_void_p(out.data_ptr()), _dtype_code(out),
                            ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_handle(stream)))
    return out
