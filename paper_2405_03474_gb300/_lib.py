"""ctypes view of liblogdet.so (declarations mirror include/logdet.h).

The library is built in-tree by ``paper_2405_03474_gb300/build.py``.  Loading
fails loudly when it is missing: there is no CPU fallback anywhere in the
product path.
"""
import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblogdet.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "logdet.h")

c_int32 = ctypes.c_int32
c_int64 = ctypes.c_int64
c_uint64 = ctypes.c_uint64
c_double = ctypes.c_double
c_float = ctypes.c_float
c_size_t = ctypes.c_size_t
c_void_p = ctypes.c_void_p
c_char_p = ctypes.c_char_p

LD_OK = 0
LD_ERR_INVALID = -1
LD_ERR_NOT_SPD = -2
LD_ERR_NOT_CONVERGED = -3
LD_ERR_CUDA = -4
LD_ERR_WORKSPACE = -5
LD_ERR_UNSUPPORTED = -6
LD_ERR_DEVICE_TIMEOUT = -7

RBF = 0
MATERN52 = 1

FP64 = 0
FP32 = 1
BF16_TC = 2
F16_TC = 3
F16X3_TC = 4
PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16_tc": BF16_TC, "f16_tc": F16_TC, "f16x3_tc": F16X3_TC}


class LdKernel(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("reserved", c_int32), ("lengthscale", c_double),
                ("variance", c_double), ("noise", c_double)]


class LdOptions(ctypes.Structure):
    _fields_ = [("order", c_int32), ("num_probes", c_int32), ("probes_per_block", c_int32),
                ("max_iters", c_int32), ("fixed_iters", c_int32), ("precision", c_int32),
                ("residual_check", c_int32), ("dense", c_int32), ("seed", c_uint64),
                ("rel_tol", c_double), ("probe_kind", c_int32), ("probe_col0", c_int32)]


class LdResult(ctypes.Structure):
    _fields_ = [("logdet", c_double), ("logdet_P", c_double), ("trace_est", c_double),
                ("std_err", c_double), ("iters", c_int32), ("converged", c_int32),
                ("max_resid", c_double * 5), ("final_rel_resid", c_double), ("slq_logdet", c_double)]


_P = c_void_p
_SIGS = {
    "ld_status_string": (c_char_p, [c_int32]),
    "ld_last_error": (c_char_p, []),
    "ld_version": (c_int32, []),
    "ld_rk_coeffs": (c_int32, [c_int32, _P, _P, _P]),
    "ld_kz_workspace_size": (c_size_t, [c_int64, c_int32, c_int32, c_int32]),
    "ld_kz": (c_int32, [_P, c_int64, c_int32, LdKernel, _P, _P, c_int32, c_int32, _P, c_size_t, _P]),
    "ld_kz_static_capacity": (c_size_t, []),
    "ld_kz_static": (c_int32, [_P, c_int64, c_int32, LdKernel, _P, _P, c_int32, c_int32, _P]),
    "ld_kz_dl": (c_int32, [_P, c_int64, c_int32, LdKernel, _P, _P, _P, c_int32, c_int32, _P]),
    "ld_dense_bytes": (c_size_t, [c_int64, c_int32]),
    "ld_dense_materialize": (c_int32, [_P, c_int64, c_int32, LdKernel, c_int32, _P, _P]),
    "ld_dense_kz": (c_int32, [_P, c_int64, _P, _P, c_int32, c_int32, _P]),
    "ld_rademacher": (c_int32, [c_uint64, c_int64, c_int32, c_int32, _P, _P]),
    "ld_gaussian": (c_int32, [c_uint64, c_int64, c_int32, c_int32, _P, _P]),
    "precond_workspace_size": (c_size_t, [c_int64, c_int32, c_int32, c_int32]),
    "precond_build": (c_int32, [_P, c_int64, c_int32, LdKernel, c_int32, c_int32, c_uint64, c_int32,
                                _P, c_size_t, _P, _P]),
    "precond_build_scaled": (c_int32, [_P, c_int64, c_int32, LdKernel, c_int32, c_int32, c_uint64, c_double,
                                       c_int32, _P, c_size_t, _P, _P]),
    "precond_import": (c_int32, [_P, _P, c_int64, c_int32, c_int32, _P, _P]),
    "precond_export": (c_int32, [_P, _P, _P, _P, _P]),
    "precond_info": (c_int32, [_P, _P, _P, _P, _P]),
    "precond_apply": (c_int32, [_P, c_int32, _P, _P, c_int32, _P]),
    "precond_free": (None, [_P]),
    "logdet_workspace_size": (c_size_t, [c_int64, c_int32, _P, _P]),
    "logdet_estimate": (c_int32, [_P, c_int64, c_int32, LdKernel, _P, _P, _P, _P, _P, c_size_t, _P, _P]),
    "ld_combine": (c_int32, [_P, c_int32, c_double, _P]),
    "logdet_grad": (c_int32, [_P, c_int64, c_int32, LdKernel, _P, _P, _P, _P, c_size_t, _P, _P, _P]),
    "ld_launch_count": (c_int64, []),
    "ld_selftest_wait_timeout": (c_int32, [c_int64, _P]),
    "ld_profile_begin": (c_int32, []),
    "ld_profile_end": (c_int32, [_P, _P, _P, _P]),
    "ld_profile_kernel": (c_int32, [c_int32, _P, _P, _P, _P]),
    "surrogate_create": (c_int32, [c_uint64, _P, _P]),
    "surrogate_set_params": (c_int32, [_P, _P, _P]),
    "surrogate_get_params": (c_int32, [_P, _P, _P]),
    "surrogate_get_norm": (c_int32, [_P, _P, _P]),
    "surrogate_set_norm": (c_int32, [_P, _P, _P]),
    "surrogate_loss_grad": (c_int32, [_P, _P, _P, c_int32, _P, _P, _P]),
    "surrogate_train": (c_int32, [_P, _P, _P, c_int32, c_int32, c_int32, c_float, _P, _P]),
    "surrogate_infer": (c_int32, [_P, _P, c_int32, _P, _P, _P]),
    "surrogate_free": (None, [_P]),
}

_lib = None


class LogdetError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(what)


def header_functions():
    """Function names declared in include/logdet.h (parsed from the text)."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\(", text)
    skip = {"if", "while", "for", "return", "sizeof", "defined"}
    return sorted({n for n in names if n not in skip and not n.isupper()})


def load(path=LIB_PATH):
    """Load the library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("liblogdet.so not found at %s: build it with "
                           "`python -m paper_2405_03474_gb300.build`" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status, what=""):
    if status == LD_OK:
        return
    lib = load()
    msg = lib.ld_last_error().decode(errors="replace")
    name = lib.ld_status_string(status).decode()
    raise LogdetError(status, "%s: %s (%d): %s" % (what, name, status, msg))
