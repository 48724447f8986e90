"""ctypes declarations of the C ABI in include/tt_rbki.h.

Loading fails loudly when the library has not been built: there is no CPU
fallback.  Build it with ``python -m paper_2308_01480_gb300.build`` or
``__graft_entry__.build()``.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtt_rbki.so")

TT_OK, TT_EINVAL, TT_ENOMEM, TT_ECUDA, TT_EBREAKDOWN, TT_ENONFINITE, TT_EUNSUPPORTED, TT_ETIMEOUT = range(8)
TT_F32, TT_BF16 = 0, 1
TT_PASS_SKETCH, TT_PASS_GRAMAPPLY, TT_PASS_PROJECT, TT_PASS_GRAM = range(4)
TT_METHOD_RBKI, TT_METHOD_RSI = range(2)
TT_ROUTE_KRYLOV, TT_ROUTE_GRAM_ROWS, TT_ROUTE_GRAM_COLS, TT_ROUTE_GRAM_POWER = range(4)

STATUS_NAMES = {0: "TT_OK", 1: "TT_EINVAL", 2: "TT_ENOMEM", 3: "TT_ECUDA", 4: "TT_EBREAKDOWN",
                5: "TT_ENONFINITE", 6: "TT_EUNSUPPORTED", 7: "TT_ETIMEOUT"}


class TTOptions(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int32), ("remainder", ctypes.c_int32),
                ("exhaust_gram", ctypes.c_int32), ("batch_streams", ctypes.c_int32),
                ("method", ctypes.c_int32), ("gram_power", ctypes.c_int32),
                ("paper_literal", ctypes.c_int32), ("accurate_rr", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class TTModePlan(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("r_in", ctypes.c_int64), ("r_out", ctypes.c_int64),
                ("b", ctypes.c_int32), ("basis_cols", ctypes.c_int32), ("blocks", ctypes.c_int32),
                ("powers", ctypes.c_int32), ("route", ctypes.c_int32), ("tensor_cores", ctypes.c_int32),
                ("fused_power", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class TTShardMode(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n_global", ctypes.c_int64), ("n_local", ctypes.c_int64),
                ("route", ctypes.c_int32), ("allreduces", ctypes.c_int32), ("allreduce_floats", ctypes.c_int64)]


# int32 (*)(float* buf, int64 count, void* stream, void* ctx)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p)


class TTProblem(ctypes.Structure):
    _fields_ = [("tensor", ctypes.c_void_p), ("dims", ctypes.POINTER(ctypes.c_int64)),
                ("ranks", ctypes.POINTER(ctypes.c_int64)), ("cores_out", ctypes.POINTER(ctypes.c_void_p)),
                ("ranks_out", ctypes.POINTER(ctypes.c_int64)), ("omega_seed", ctypes.c_uint64),
                ("d", ctypes.c_int32), ("oversample", ctypes.c_int32), ("q", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class TTKernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


class TTError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p
_vpp = ctypes.POINTER(ctypes.c_void_p)

_SIGNATURES = {
    "tt_rbki_default_options": ([ctypes.POINTER(TTOptions)], ctypes.c_int),
    "tt_rbki_core_sizes": ([_i64p, ctypes.c_int, _i64p, _i64p, _i64p], ctypes.c_int),
    "tt_rbki_workspace_size": ([_i64p, ctypes.c_int, _i64p, ctypes.c_int, ctypes.c_int,
                                ctypes.POINTER(TTOptions), ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "tt_rbki_plan_modes": ([_i64p, ctypes.c_int, _i64p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(TTOptions),
                            ctypes.POINTER(TTModePlan), ctypes.c_int], ctypes.c_int),
    "tt_rbki_decompose": ([_vp, _i64p, ctypes.c_int, _i64p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                           _vpp, _i64p, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(TTOptions)], ctypes.c_int),
    "tt_rbki_decompose_omega": ([_vp, _i64p, ctypes.c_int, _i64p, ctypes.c_int, ctypes.c_int, _vpp,
                                 _vpp, _i64p, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(TTOptions)],
                                ctypes.c_int),
    "tt_rbki_device_status": ([_vp, _vp, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "tt_rbki_shard_plan": ([_i64p, ctypes.c_int, _i64p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(TTOptions),
                            ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                            ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(TTShardMode), ctypes.c_int], ctypes.c_int),
    "tt_rbki_sharded_workspace_size": ([_i64p, ctypes.c_int, _i64p, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(TTOptions), ctypes.c_int32, ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "tt_rbki_decompose_sharded": ([_vp, _i64p, ctypes.c_int, _i64p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                   _vpp, _i64p, _vp, ctypes.c_size_t, ctypes.c_int32, ctypes.c_int32,
                                   ALLREDUCE_FN, _vp, _vp, ctypes.POINTER(TTOptions)], ctypes.c_int),
    "tt_rbki_batched_workspace_size": ([ctypes.c_int, ctypes.POINTER(TTProblem), ctypes.POINTER(TTOptions),
                                        ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "tt_rbki_decompose_batched": ([ctypes.c_int, ctypes.POINTER(TTProblem), _vp, ctypes.c_size_t, _vp,
                                   ctypes.POINTER(TTOptions), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "tt_rbki_batched_device_status": ([_vp, ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "tt_rbki_batched_graph_create": ([ctypes.c_int, ctypes.POINTER(TTProblem), _vp, ctypes.c_size_t,
                                      ctypes.POINTER(TTOptions), ctypes.POINTER(ctypes.c_int), _vpp],
                                     ctypes.c_int),
    "tt_rbki_graph_launch": ([_vp, _vp], ctypes.c_int),
    "tt_rbki_graph_destroy": ([_vp], ctypes.c_int),
    "tt_rbki_last_error": ([], ctypes.c_char_p),
    "tt_svd_workspace_size": ([_i64p, ctypes.c_int, _i64p, ctypes.c_int, _i64p, ctypes.POINTER(ctypes.c_size_t)],
                              ctypes.c_int),
    "tt_svd_decompose": ([_vp, ctypes.c_int, _i64p, ctypes.c_int, ctypes.c_double, _i64p, _vpp, _i64p, _vp,
                          ctypes.c_size_t, _vp], ctypes.c_int),
    "tt_permute_convert": ([_vp, ctypes.c_int, _i64p, _i64p, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                            _vp, ctypes.c_int, _vp], ctypes.c_int),
    "tt_omega_generate": ([ctypes.c_uint64, ctypes.c_int, ctypes.c_int64, ctypes.c_int, _vp, ctypes.c_int,
                           ctypes.c_int64, _vp], ctypes.c_int),
    "tt_pass_workspace_size": ([ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "tt_gram_apply_noalloc": ([_vp, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, _vp, _vp,
                               _vp], ctypes.c_int),
    "tt_gram_power": ([_vp, ctypes.c_int64, _vp, ctypes.c_int64, ctypes.c_int, _vp, ctypes.c_int64, _vp],
                      ctypes.c_int),
    "tt_sym_eig_workspace_size": ([ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "tt_sym_eig_top": ([_vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, ctypes.c_size_t, _vp],
                       ctypes.c_int),
    "tt_debug_fill_shared": ([ctypes.c_uint32, _vp], ctypes.c_int),
    "tt_debug_wait_timeout": ([_vp, _vp], ctypes.c_int),
    "tt_rbki_profile_begin": ([ctypes.c_int], ctypes.c_int),
    "tt_rbki_profile_end": ([ctypes.POINTER(TTKernelStat), ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
                            ctypes.c_int),
    "tt_pass": ([ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, _vp, _vp,
                 ctypes.c_int, _vp, ctypes.c_size_t, _vp], ctypes.c_int),
    "tt_tune_set": ([ctypes.c_int] * 8, ctypes.c_int),
    "tt_tune_get": ([ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "tt_tune_clear": ([], ctypes.c_int),
    "tt_tune_entries": ([], ctypes.c_int),
    "tt_tune_load": ([ctypes.c_char_p], ctypes.c_int),
}

# The launch-shape table the offline sweep (autotune.py) wrote for this
# part; loaded with the library.
TUNE_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_table.txt")


def exported_names():
    """Names the header declares (every one must be exported by the library)."""
    return sorted(_SIGNATURES)


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"CUDA library not built: {LIB_PATH} is missing. Run "
                "`python -m paper_2308_01480_gb300.build` (there is no CPU fallback).")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        if os.path.exists(TUNE_TABLE) and L.tt_tune_load(TUNE_TABLE.encode()) != TT_OK:
            raise RuntimeError(f"invalid tuning table {TUNE_TABLE}")
        _lib = L
    return _lib


def check(status):
    if status != TT_OK:
        msg = lib().tt_rbki_last_error()
        raise TTError(status, msg.decode() if msg else "")
    return status


def i64_array(values):
    arr = (ctypes.c_int64 * len(values))(*[int(v) for v in values])
    return arr


def ptr_array(ptrs):
    return (ctypes.c_void_p * len(ptrs))(*[ctypes.c_void_p(int(p)) for p in ptrs])
