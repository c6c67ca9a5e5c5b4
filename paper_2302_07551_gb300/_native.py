"""ctypes declarations of libmc (include/mc.h).  Argument marshalling only."""
import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmc.so")
HEADER = os.path.join(HERE, "..", "include", "mc.h")

MC_OK, MC_ERR_ARG, MC_ERR_WORKSPACE, MC_ERR_CUDA = 0, 1, 2, 3
MC_ERR_SINGULAR_BLOCK, MC_ERR_NOT_FACTORED, MC_ERR_BREAKDOWN = 4, 5, 6
MC_ERR_NO_CONVERGENCE, MC_ERR_TIMEOUT = 7, 8
MC_APPLY_INVERSE, MC_APPLY_COUPLED = 0, 1
MC_F64, MC_F32, MC_BF16 = 0, 1, 2
DTYPES = {"f64": MC_F64, "f32": MC_F32, "bf16": MC_BF16}
PLANES = {"tlo": 0, "tup": 1, "tdd": 2, "lu": 3, "ninv": 4, "wlo": 5, "wup": 6}


class McDesc(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int64), ("m", ctypes.c_int32), ("stair", ctypes.c_int32),
                ("apply", ctypes.c_int32), ("dtype", ctypes.c_int32), ("paired", ctypes.c_int32),
                ("lower", ctypes.c_int32), ("upper", ctypes.c_int32)]


class McServerDesc(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("apply", ctypes.c_int32), ("stair", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("tol", ctypes.c_double),
                ("maxit", ctypes.c_int64), ("max_active", ctypes.c_int32),
                ("autotune", ctypes.c_int32)]


class McServerTuning(ctypes.Structure):
    _fields_ = [("signature", ctypes.c_uint64), ("blocks_per_sm", ctypes.c_int32),
                ("levels_per_unit", ctypes.c_int32), ("split64", ctypes.c_int32),
                ("deep", ctypes.c_int32), ("chosen", ctypes.c_int32),
                ("chunk_ms", ctypes.c_double), ("sweep_ms", ctypes.c_double),
                ("sweep_bytes", ctypes.c_double)]


class McTuning(ctypes.Structure):
    _fields_ = [("blocks_per_sm", ctypes.c_int32), ("levels_per_unit", ctypes.c_int32)]


class McResult(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int64), ("residual_l1", ctypes.c_double),
                ("step_l1", ctypes.c_double), ("contraction", ctypes.c_double),
                ("converged", ctypes.c_int32)]


_lib = None


def load():
    """Load libmc.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libmc.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, dbl, sz = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                             ctypes.c_size_t)
    pdesc = ctypes.POINTER(McDesc)
    lib.mc_workspace_bytes.argtypes = [pdesc]
    lib.mc_workspace_bytes.restype = sz
    lib.mc_create.argtypes = [pdesc, vp, vp, vp, vp, sz, vp, ctypes.POINTER(vp)]
    lib.mc_create.restype = ctypes.c_int
    lib.mc_create_banded.argtypes = [pdesc, ctypes.POINTER(vp), vp, sz, vp, ctypes.POINTER(vp)]
    lib.mc_create_banded.restype = ctypes.c_int
    lib.mc_factor.argtypes = [vp]
    lib.mc_factor.restype = ctypes.c_int
    lib.mc_sweep.argtypes = [vp, vp, vp, i64, vp]
    lib.mc_sweep.restype = ctypes.c_int
    lib.mc_profile.argtypes = [vp, vp, vp, i64, vp]
    lib.mc_profile.restype = ctypes.c_int
    lib.mc_sweep_host.argtypes = [vp, vp, vp, i64, vp]
    lib.mc_sweep_host.restype = ctypes.c_int
    lib.mc_solve.argtypes = [vp, vp, vp, dbl, dbl, i64, i32, ctypes.POINTER(McResult)]
    lib.mc_solve.restype = ctypes.c_int
    lib.mc_residual.argtypes = [vp, vp, ctypes.POINTER(dbl)]
    lib.mc_residual.restype = ctypes.c_int
    lib.mc_export.argtypes = [vp, i32, i64, i64, vp]
    lib.mc_export.restype = ctypes.c_int
    lib.mc_residual_noalloc.argtypes = [vp, vp, vp, i64, i32, vp, vp, vp]
    lib.mc_residual_noalloc.restype = ctypes.c_int
    lib.mc_wait_selftest.argtypes = [vp, i32, i64]
    lib.mc_wait_selftest.restype = ctypes.c_int
    lib.mc_server_create.argtypes = [ctypes.POINTER(McServerDesc), vp, sz, vp, ctypes.POINTER(vp)]
    lib.mc_server_create.restype = ctypes.c_int
    lib.mc_server_request_bytes.argtypes = [vp, i64, i32]
    lib.mc_server_request_bytes.restype = sz
    lib.mc_server_submit.argtypes = [vp, i64, i64, i32, vp, vp, vp]
    lib.mc_server_submit.restype = ctypes.c_int
    lib.mc_server_step.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.mc_server_step.restype = ctypes.c_int
    lib.mc_server_fetch.argtypes = [vp, ctypes.POINTER(i64), vp, i64, ctypes.POINTER(McResult),
                                    ctypes.POINTER(i32)]
    lib.mc_server_fetch.restype = ctypes.c_int
    lib.mc_server_grid.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                   ctypes.POINTER(i32)]
    lib.mc_server_grid.restype = ctypes.c_int
    lib.mc_server_trials.argtypes = [vp, ctypes.POINTER(McServerTuning), i32,
                                     ctypes.POINTER(i32)]
    lib.mc_server_trials.restype = ctypes.c_int
    lib.mc_server_destroy.argtypes = [vp]
    lib.mc_server_destroy.restype = None
    lib.mc_set_tuning.argtypes = [vp, ctypes.POINTER(McTuning)]
    lib.mc_set_tuning.restype = ctypes.c_int
    lib.mc_get_tuning.argtypes = [vp, ctypes.POINTER(McTuning)]
    lib.mc_get_tuning.restype = ctypes.c_int
    lib.mc_tune.argtypes = [vp, vp, i64, ctypes.POINTER(McTuning), ctypes.POINTER(dbl)]
    lib.mc_tune.restype = ctypes.c_int
    lib.mc_sync.argtypes = [vp]
    lib.mc_sync.restype = ctypes.c_int
    lib.mc_destroy.argtypes = [vp]
    lib.mc_destroy.restype = None
    lib.mc_status_string.argtypes = [ctypes.c_int]
    lib.mc_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def declared_functions():
    """Names of the functions include/mc.h declares."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mc_[a-z_]+)\s*\(", src)))


class McError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        msg = load().mc_status_string(status).decode()
        super().__init__(f"{where}: {msg} (status {status})")


def check(status, where=""):
    if status != MC_OK:
        raise McError(status, where)
