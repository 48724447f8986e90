"""GB300 randomized block Krylov tensor-train approximation (TT-rBKI).

Python binding of the C ABI in include/tt_rbki.h.  Every function here only
marshals arguments: buffers are torch tensors on the current CUDA device,
work is enqueued on torch's current stream, and all arithmetic runs in the
library's CUDA kernels.  There is no CPU path.
"""
import ctypes

from . import _native as N
from ._native import (TT_BF16, TT_F32, TT_METHOD_RBKI, TT_METHOD_RSI, TT_PASS_GRAM,  # noqa: F401
                      TT_PASS_GRAMAPPLY, TT_PASS_PROJECT, TT_PASS_SKETCH, TTError)

__all__ = ["decompose", "tt_svd", "workspace_size", "core_sizes", "omega_generate", "permute_convert",
           "tt_pass", "gram_power", "device_status", "options", "plan_modes", "profile_begin", "profile_end", "TTError", "TT_F32",
           "TT_BF16", "Problem", "batched_workspace_size", "decompose_batched", "batched_device_status",
           "BatchGraph", "tune_key", "tune_set", "tune_get", "tune_clear", "tune_entries", "tune_load"]


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


def options(storage=N.TT_F32, remainder=None, exhaust_gram=True, batch_streams=0, method=N.TT_METHOD_RBKI,
            gram_power=True, paper_literal=False, accurate_rr=False):
    """tt_options with the given fields (remainder None = same as storage;
    method TT_METHOD_RBKI (Alg. 3) or TT_METHOD_RSI (Alg. 4); q = 0 with
    either is TT-rSVD, Alg. 2; gram_power False makes every Krylov power
    stream the unfolding; paper_literal True takes the paper's steps
    literally, first-r truncation without Rayleigh-Ritz; accurate_rr True
    takes the Rayleigh-Ritz vectors from B = Q^T C without squaring it in
    FP32: compensated Gram, FP64 Cholesky, one-sided Jacobi)."""
    o = N.TTOptions()
    N.check(N.lib().tt_rbki_default_options(ctypes.byref(o)))
    o.storage = int(storage)
    o.remainder = -1 if remainder is None else int(remainder)
    o.exhaust_gram = 1 if exhaust_gram else 0
    o.batch_streams = int(batch_streams)
    o.method = int(method)
    o.gram_power = 1 if gram_power else 0
    o.paper_literal = 1 if paper_literal else 0
    o.accurate_rr = 1 if accurate_rr else 0
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


ROUTE_NAMES = {N.TT_ROUTE_KRYLOV: "krylov", N.TT_ROUTE_GRAM_ROWS: "gram_rows",
               N.TT_ROUTE_GRAM_COLS: "gram_cols", N.TT_ROUTE_GRAM_POWER: "gram_power"}


def plan_modes(dims, ranks, oversample, q, opts=None):
    """The per-mode plan tt_rbki_decompose follows for these arguments (no
    GPU needed): a list of dicts, one per mode 1..d-1, with the unfolding
    shape, clamped ranks, block width, basis columns, Krylov blocks, powers,
    the route name and whether the passes run on the tensor cores."""
    d = len(dims)
    arr = (N.TTModePlan * max(1, d - 1))()
    N.check(N.lib().tt_rbki_plan_modes(N.i64_array(dims), d, N.i64_array(ranks), int(oversample), int(q),
                                       ctypes.byref(opts) if opts is not None else None, arr, d - 1))
    out = []
    for e in arr[:d - 1]:
        out.append(dict(m=e.m, n=e.n, r_in=e.r_in, r_out=e.r_out, b=e.b, basis_cols=e.basis_cols,
                        blocks=e.blocks, powers=e.powers, route=ROUTE_NAMES[e.route],
                        tensor_cores=bool(e.tensor_cores), fused_power=bool(e.fused_power)))
    return out


def shard_plan(dims, ranks, oversample, q, world, rank, opts=None):
    """Host-side plan of rank `rank` of `world` for the sharded form (no GPU
    needed): (slab_lo, slab_w, modes), modes a list of dicts per mode with
    the unfolding's rows, whole and local columns, route and the number of
    sums over ranks (and floats summed) the mode needs."""
    d = len(dims)
    arr = (N.TTShardMode * max(1, d - 1))()
    lo, w = ctypes.c_int64(), ctypes.c_int64()
    N.check(N.lib().tt_rbki_shard_plan(N.i64_array(dims), d, N.i64_array(ranks), int(oversample), int(q),
                                       ctypes.byref(opts) if opts is not None else None, int(world), int(rank),
                                       ctypes.byref(lo), ctypes.byref(w), arr, d - 1))
    modes = [dict(m=e.m, n_global=e.n_global, n_local=e.n_local, route=ROUTE_NAMES[e.route],
                  allreduces=e.allreduces, allreduce_floats=e.allreduce_floats) for e in arr[:d - 1]]
    return lo.value, w.value, modes


def decompose_sharded(local_tensor, dims, ranks, oversample, q, world, rank, allreduce, omega_seed=0, opts=None,
                      stream=None):
    """Alg. 3 on this rank's slab A[..., lo : lo + w] of the last mode (a
    contiguous CUDA tensor).  `allreduce(buf)` receives each partial block to
    be summed over the ranks as a float32 CUDA tensor (a view into this
    call's workspace) and must sum it in place in stream order on the
    current stream (torch.distributed.all_reduce does).  Returns (cores,
    ranks): cores 1..d-1 in full, core d as this rank's slab."""
    torch = _torch()
    d = len(dims)
    if opts is None:
        opts = options(storage=_dtype_code(local_tensor))
    if not local_tensor.is_cuda or not local_tensor.is_contiguous():
        raise ValueError("local_tensor must be a contiguous CUDA tensor")
    lo, w, _ = shard_plan(dims, ranks, oversample, q, world, rank, opts)
    if list(local_tensor.shape) != list(dims[:-1]) + [w]:
        raise ValueError(f"local_tensor must have shape {list(dims[:-1]) + [w]}")
    rr, _ = core_sizes(dims, ranks)
    cores = [torch.empty((rr[k], dims[k] if k < d - 1 else w, rr[k + 1]), dtype=torch.float32,
                         device=local_tensor.device) for k in range(d)]
    nb = ctypes.c_size_t()
    N.check(N.lib().tt_rbki_sharded_workspace_size(N.i64_array(dims), d, N.i64_array(ranks), int(oversample), int(q),
                                                   ctypes.byref(opts), int(world), int(rank), ctypes.byref(nb)))
    ws = torch.empty(nb.value, dtype=torch.uint8, device=local_tensor.device)
    base = ws.data_ptr()
    errors = []

    def _cb(ptr, count, _stream, _ctx):
        try:
            off = int(ptr) - base
            view = ws[off:off + 4 * int(count)].view(torch.float32)
            allreduce(view)
            return 0
        except Exception as e:          # reported after the call
            errors.append(e)
            return 1

    cb = N.ALLREDUCE_FN(_cb)
    ranks_out = (ctypes.c_int64 * (d + 1))()
    status = N.lib().tt_rbki_decompose_sharded(
        ctypes.c_void_p(local_tensor.data_ptr()), N.i64_array(dims), d, N.i64_array(ranks), int(oversample), int(q),
        ctypes.c_uint64(omega_seed), N.ptr_array([c.data_ptr() for c in cores]), ranks_out,
        ctypes.c_void_p(base), nb.value, int(world), int(rank), cb, None, _stream_handle(stream), ctypes.byref(opts))
    if errors:
        raise errors[0]
    N.check(status)
    decompose_sharded.last_workspace = ws
    return cores, list(ranks_out)


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


def sym_eig_top(H, r, stream=None):
    """Top-r eigenpairs of the symmetric part of the k x k CUDA float32
    matrix H (the Rayleigh-Ritz eigensolver).  Returns (V (k x r), evals)."""
    torch = _torch()
    k = H.shape[0]
    if H.dtype != torch.float32 or not H.is_cuda or H.dim() != 2 or H.shape[1] != k or H.stride(1) != 1:
        raise ValueError("H must be a k x k float32 CUDA matrix with unit column stride")
    nbytes = ctypes.c_size_t()
    N.check(N.lib().tt_sym_eig_workspace_size(int(k), int(r), ctypes.byref(nbytes)))
    ws = torch.empty(nbytes.value, dtype=torch.uint8, device=H.device)
    V = torch.empty((k, r), dtype=torch.float32, device=H.device)
    ev = torch.empty((r,), dtype=torch.float32, device=H.device)
    N.check(N.lib().tt_sym_eig_top(ctypes.c_void_p(H.data_ptr()), H.stride(0), int(k), int(r),
                                   ctypes.c_void_p(V.data_ptr()), ctypes.c_void_p(ev.data_ptr()),
                                   ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_handle(stream)))
    return V, ev


def debug_fill_shared(bits=0x7FC00000, stream=None):
    """Fill every SM's shared memory with a 32-bit pattern (default: a quiet
    NaN) so that later reads of never-written shared memory show up."""
    N.check(N.lib().tt_debug_fill_shared(ctypes.c_uint32(bits), _stream_handle(stream)))


def debug_wait_timeout(workspace, stream=None):
    """Run one bounded mbarrier wait that can never complete; the status
    area at the start of `workspace` then reads TT_ETIMEOUT."""
    N.check(N.lib().tt_debug_wait_timeout(ctypes.c_void_p(workspace.data_ptr()), _stream_handle(stream)))


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


def pass_workspace_size(op, m, n, b, c_dtype):
    nbytes = ctypes.c_size_t()
    N.check(N.lib().tt_pass_workspace_size(int(op), int(m), int(n), int(b), int(c_dtype), ctypes.byref(nbytes)))
    return nbytes.value


def tt_pass(op, C, b=None, x=None, y_dtype=None, stream=None, workspace=None, out=None):
    """One streaming pass over the unfolding C (2-D CUDA tensor), see tt_pass
    in the header.  Returns the output tensor."""
    torch = _torch()
    m, n = C.shape
    if op == N.TT_PASS_GRAM:
        b = 0
        shape, dt = (m, m), torch.float32
    elif op == N.TT_PASS_PROJECT:
        b = x.shape[1]
        shape, dt = (b, n), y_dtype or torch.float32
    else:
        b = x.shape[1]
        shape, dt = (m, b), torch.float32
    if out is None:
        out = torch.empty(shape, dtype=dt, device=C.device)
    need = pass_workspace_size(op, m, n, b, _dtype_code(C))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=C.device)
    N.check(N.lib().tt_pass(int(op), ctypes.c_void_p(C.data_ptr()), _dtype_code(C), m, n, int(b),
                            ctypes.c_void_p(x.data_ptr() if x is not None else 0),
                            ctypes.c_void_p(out.data_ptr()), _dtype_code(out),
                            ctypes.c_void_p(workspace.data_ptr()), workspace.numel(), _stream_handle(stream)))
    return out


def tune_key(op, m, n, b=0):
    """The tuning-table key (op, rows, npad, nclass) of a BF16 tensor-core
    pass over an m x n unfolding with b columns (see tt_tune_set in the
    header): the same bucketing the library applies."""
    m, n, b = int(m), int(n), int(b)
    if m <= 128:
        rows = (m + 15) // 16 * 16
    else:
        rows = 256 if m <= 256 else 512 if m <= 512 else 1024 if m <= 1024 else 4096
    if op == N.TT_PASS_GRAM:
        npad = (m + 15) // 16 * 16
    elif op == N.TT_PASS_PROJECT and b <= 32:
        npad = 64
    else:
        npad = (b + 15) // 16 * 16
    return (int(op), rows, npad, 0 if n < 16384 else 1 if n < 262144 else 2)


def tune_set(key, stages, per_sm, kb=0, chunk_rows=0):
    """Sets the launch-shape entry of `key` (from tune_key)."""
    N.check(N.lib().tt_tune_set(*[int(v) for v in key], int(stages), int(per_sm), int(kb), int(chunk_rows)))


def tune_get(key):
    """The entry (stages, per_sm, kb, chunk_rows) of `key`, or None."""
    out = (ctypes.c_int * 4)()
    if N.lib().tt_tune_get(*[int(v) for v in key], out) != N.TT_OK:
        return None
    return tuple(out)


def tune_clear():
    N.check(N.lib().tt_tune_clear())


def tune_entries():
    return int(N.lib().tt_tune_entries())


def tune_load(path):
    """Replaces the table from a text file (format in the header)."""
    N.check(N.lib().tt_tune_load(str(path).encode()))


def gram_power(G, X, stream=None, out=None):
    """W = G X through a formed Gram matrix (tt_gram_power): G (m, m) and
    X (m, c) float32 CUDA tensors, X with unit column stride."""
    torch = _torch()
    m, c = X.shape
    if out is None:
        out = torch.empty((m, c), dtype=torch.float32, device=X.device)
    N.check(N.lib().tt_gram_power(ctypes.c_void_p(G.data_ptr()), int(m), ctypes.c_void_p(X.data_ptr()),
                                  int(X.stride(0)), int(c), ctypes.c_void_p(out.data_ptr()), int(out.stride(0)),
                                  _stream_handle(stream)))
    return out


class Problem:
    """One problem of a batch: a contiguous CUDA tensor (dtype = the batch's
    storage), target ranks r_1..r_{d-1}, p, q and the Omega seed.  The cores
    (float32 CUDA tensors (r_{k-1}, I_k, r_k)) are allocated here unless
    given."""

    def __init__(self, tensor, ranks, oversample, q, omega_seed, cores=None):
        torch = _torch()
        if not tensor.is_cuda or not tensor.is_contiguous():
            raise ValueError("tensor must be a contiguous CUDA tensor")
        self.tensor = tensor
        self.dims = list(tensor.shape)
        self.ranks = list(ranks)
        self.oversample, self.q, self.omega_seed = int(oversample), int(q), int(omega_seed)
        rr, _ = core_sizes(self.dims, self.ranks)
        self.rr = rr
        if cores is None:
            cores = [torch.empty((rr[k], self.dims[k], rr[k + 1]), dtype=torch.float32, device=tensor.device)
                     for k in range(len(self.dims))]
        self.cores = cores


def _problem_array(problems):
    """ctypes tt_problem array plus the host arrays it points to (kept alive
    by the caller for the duration of the C call)."""
    arr = (N.TTProblem * len(problems))()
    keep = []
    for i, pb in enumerate(problems):
        dims, ranks = N.i64_array(pb.dims), N.i64_array(pb.ranks)
        cores = N.ptr_array([c.data_ptr() for c in pb.cores])
        rout = (ctypes.c_int64 * (len(pb.dims) + 1))()
        keep += [dims, ranks, cores, rout]
        arr[i].tensor = pb.tensor.data_ptr()
        arr[i].dims = ctypes.cast(dims, ctypes.POINTER(ctypes.c_int64))
        arr[i].ranks = ctypes.cast(ranks, ctypes.POINTER(ctypes.c_int64))
        arr[i].cores_out = ctypes.cast(cores, ctypes.POINTER(ctypes.c_void_p))
        arr[i].ranks_out = ctypes.cast(rout, ctypes.POINTER(ctypes.c_int64))
        arr[i].omega_seed = pb.omega_seed
        arr[i].d, arr[i].oversample, arr[i].q, arr[i].reserved = len(pb.dims), pb.oversample, pb.q, 0
    return arr, keep


def batched_workspace_size(problems, opts):
    arr, _keep = _problem_array(problems)
    nbytes = ctypes.c_size_t()
    N.check(N.lib().tt_rbki_batched_workspace_size(len(problems), arr, ctypes.byref(opts), ctypes.byref(nbytes)))
    return nbytes.value


def _batch_ws(problems, opts, workspace):
    torch = _torch()
    need = batched_workspace_size(problems, opts)
    if workspace is None or workspace.numel() < need:
        dev = problems[0].tensor.device if problems else torch.device("cuda")
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    return workspace


def tt_svd(tensor, eps=0.0, max_ranks=None, workspace=None, stream=None):
    """TT-SVD (Alg. 1) of a dense row-major CUDA tensor (float32 or
    bfloat16) with accuracy eps and optional rank caps (tt_svd_decompose).
    Host-synchronous.  Returns (cores, ranks): float32 CUDA tensors of shape
    (r_{k-1}, I_k, r_k) with the chosen ranks, and the ranks r_0 .. r_d."""
    torch = _torch()
    if not tensor.is_cuda or not tensor.is_contiguous():
        raise ValueError("tensor must be a contiguous CUDA tensor")
    dims = list(tensor.shape)
    d = len(dims)
    storage = _dtype_code(tensor)
    caps = N.i64_array(max_ranks) if max_ranks is not None else None
    elems = (ctypes.c_int64 * d)()
    nbytes = ctypes.c_size_t()
    N.check(N.lib().tt_svd_workspace_size(N.i64_array(dims), d, caps, storage, elems, ctypes.byref(nbytes)))
    if workspace is None or workspace.numel() < nbytes.value:
        workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=tensor.device)
    bufs = [torch.empty(int(elems[k]), dtype=torch.float32, device=tensor.device) for k in range(d)]
    ranks_out = (ctypes.c_int64 * (d + 1))()
    N.check(N.lib().tt_svd_decompose(ctypes.c_void_p(tensor.data_ptr()), storage, N.i64_array(dims), d,
                                     float(eps), caps, N.ptr_array([b.data_ptr() for b in bufs]), ranks_out,
                                     ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                     _stream_handle(stream)))
    rr = [int(ranks_out[k]) for k in range(d + 1)]
    cores = [bufs[k][:rr[k] * dims[k] * rr[k + 1]].view(rr[k], dims[k], rr[k + 1]) for k in range(d)]
    return cores, rr


def decompose_batched(problems, opts, workspace=None, stream=None):
    """Enqueues every problem (tt_rbki_decompose_batched); returns the
    workspace used (read device statuses from it)."""
    workspace = _batch_ws(problems, opts, workspace)
    arr, _keep = _problem_array(problems)
    per = (ctypes.c_int * max(1, len(problems)))()
    N.check(N.lib().tt_rbki_decompose_batched(len(problems), arr, ctypes.c_void_p(workspace.data_ptr()),
                                              workspace.numel(), _stream_handle(stream), ctypes.byref(opts),
                                              per))
    return workspace


def batched_device_status(workspace, count, stream=None):
    out = (ctypes.c_int * max(1, count))()
    N.check(N.lib().tt_rbki_batched_device_status(ctypes.c_void_p(workspace.data_ptr()), int(count),
                                                  _stream_handle(stream), out))
    return list(out)[:count]


class BatchGraph:
    """The batch captured into one executable CUDA graph
    (tt_rbki_batched_graph_create); launch() replays it on a stream."""

    def __init__(self, problems, opts, workspace=None):
        self.problems = list(problems)
        self.workspace = _batch_ws(self.problems, opts, workspace)
        arr, _keep = _problem_array(self.problems)
        per = (ctypes.c_int * max(1, len(self.problems)))()
        h = ctypes.c_void_p()
        N.check(N.lib().tt_rbki_batched_graph_create(len(self.problems), arr,
                                                     ctypes.c_void_p(self.workspace.data_ptr()),
                                                     self.workspace.numel(), ctypes.byref(opts), per,
                                                     ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        N.check(N.lib().tt_rbki_graph_launch(self._h, _stream_handle(stream)))

    def device_status(self, stream=None):
        return batched_device_status(self.workspace, len(self.problems), stream)

    def close(self):
        if self._h:
            N.check(N.lib().tt_rbki_graph_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
