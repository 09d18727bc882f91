"""ctypes binding of the C ABI declared in include/sgoc.h (argument marshalling only).

Every function keeps its C name.  Device pointers are passed as integers
(e.g. torch.Tensor.data_ptr()) and streams as integers (cudaStream_t).
Loading fails loudly when the shared library has not been built: there is no
CPU fallback for any computation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsgoc.so")

SGOC_OK = 0
SGOC_ERR_INVALID_ARG = 1
SGOC_ERR_UNSUPPORTED = 2
SGOC_ERR_WORKSPACE_TOO_SMALL = 3
SGOC_ERR_CUDA = 4
SGOC_ERR_NO_CONVERGENCE = 5
SGOC_ERR_BREAKDOWN = 6
SGOC_ERR_NOT_SPD = 7
SGOC_ERR_NAN = 8
SGOC_ERR_NOT_UPLOADED = 9
STATUS_NAMES = {
    0: "SGOC_OK", 1: "SGOC_ERR_INVALID_ARG", 2: "SGOC_ERR_UNSUPPORTED", 3: "SGOC_ERR_WORKSPACE_TOO_SMALL",
    4: "SGOC_ERR_CUDA", 5: "SGOC_ERR_NO_CONVERGENCE", 6: "SGOC_ERR_BREAKDOWN", 7: "SGOC_ERR_NOT_SPD",
    8: "SGOC_ERR_NAN", 9: "SGOC_ERR_NOT_UPLOADED",
}
SGOC_FP64, SGOC_MIXED_FP32 = 0, 1
SGOC_KERNEL_KINDS = 12
SGOC_INNER_PRODUCT_WS_BYTES = 8192


class ProblemDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("M", ctypes.c_int32), ("p", ctypes.c_int32),
                ("kappa", ctypes.POINTER(ctypes.c_double)), ("beta", ctypes.c_double),
                ("gamma", ctypes.c_double), ("nt", ctypes.c_int32), ("T", ctypes.c_double),
                ("yhat", ctypes.POINTER(ctypes.c_double)), ("y0", ctypes.POINTER(ctypes.c_double)),
                ("chaos", ctypes.c_int32), ("length", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("r", ctypes.c_int32),
                ("cheb_steps", ctypes.c_int32), ("nu_pre", ctypes.c_int32), ("nu_post", ctypes.c_int32),
                ("omega", ctypes.c_double), ("precision", ctypes.c_int32), ("inner_tol", ctypes.c_double),
                ("max_outer", ctypes.c_int32), ("schur", ctypes.c_int32), ("krylov", ctypes.c_int32),
                ("restart", ctypes.c_int32), ("mass_solve", ctypes.c_int32), ("precond", ctypes.c_int32),
                ("mean_solve", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int32), ("outer_iterations", ctypes.c_int32),
                ("rel_true_residual", ctypes.c_double), ("rel_estimate", ctypes.c_double),
                ("ms_total", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_P = ctypes.c_void_p
_I32, _I64, _SZ, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_double
_PI32, _PI64, _PSZ, _PD = (ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                           ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_double))

# name -> (restype, argtypes); the exported symbol set of include/sgoc.h
SIGNATURES = {
    "sgoc_default_options": (None, [ctypes.POINTER(Options)]),
    "sgoc_problem_create": (ctypes.c_int, [ctypes.POINTER(ProblemDesc), ctypes.POINTER(Options), ctypes.POINTER(_P)]),
    "sgoc_problem_destroy": (None, [_P]),
    "sgoc_problem_sizes": (ctypes.c_int, [_P, _PI64, _PI64, _PI64, _PI64]),
    "sgoc_problem_device_bytes": (ctypes.c_int, [_P, _PSZ, _PSZ]),
    "sgoc_problem_upload": (ctypes.c_int, [_P, _P, _SZ, _P]),
    "sgoc_rhs": (ctypes.c_int, [_P, _P, _P]),
    "sgoc_solve": (ctypes.c_int, [_P, _P, _SZ, _P, _P, _P, ctypes.POINTER(Result)]),
    "sgoc_solve_batch": (ctypes.c_int, [_I32, ctypes.POINTER(_P), ctypes.POINTER(_P), _PSZ, ctypes.POINTER(_P),
                                        ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(Result)]),
    "sgoc_solve_batch_merged": (ctypes.c_int, [_I32, ctypes.POINTER(_P), ctypes.POINTER(_P), _PSZ,
                                               ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                                               ctypes.POINTER(Result)]),
    "sgoc_server_create": (ctypes.c_int, [_P, _SZ, _I32, ctypes.POINTER(_P)]),
    "sgoc_server_destroy": (None, [_P]),
    "sgoc_server_submit": (ctypes.c_int, [_P, _P, _P, ctypes.c_uint64]),
    "sgoc_server_step": (ctypes.c_int, [_P, _PI32, _PI32]),
    "sgoc_server_poll": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(Result), _I32, _PI32]),
    "sgoc_server_stats": (ctypes.c_int, [_P, _PI64, _PI64, _PI64, _PSZ]),
    "sgoc_autotune": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P, _I32, _P]),
    "sgoc_set_kernel": (ctypes.c_int, [_P, _I32, _I32, _I32]),
    "sgoc_apply_operator": (ctypes.c_int, [_P, _I32, _P, _P, _I32, _P]),
    "sgoc_apply_operator_variant": (ctypes.c_int, [_P, _I32, _I32, _P, _P, _I32, _P]),
    "sgoc_apply_kkt": (ctypes.c_int, [_P, _I32, _P, _P, _P]),
    "sgoc_apply_precond": (ctypes.c_int, [_P, _I32, _P, _P, _P, _SZ, _P]),
    "sgoc_apply_hgs": (ctypes.c_int, [_P, _I32, _P, _P, _I32, _P, _SZ, _P]),
    "sgoc_apply_vcycle": (ctypes.c_int, [_P, _I32, _P, _P, _I32, _P, _SZ, _P]),
    "sgoc_apply_chebyshev": (ctypes.c_int, [_P, _I32, _P, _P, _I32, _P, _SZ, _P]),
    "sgoc_apply_chebyshev_noalloc": (ctypes.c_int, [_P, _I32, _P, _P, _I32, _P]),
    "sgoc_inner_product": (ctypes.c_int, [_I32, _P, _P, _I64, _P, _SZ, _P, _P]),
    "sgoc_pc_indices": (ctypes.c_int, [_P, _PI32]),
    "sgoc_triple_products": (ctypes.c_int, [_P, _PI32, _PI32, _PI32, _PD, _PI64]),
    "sgoc_kernel_launches": (ctypes.c_int64, []),
    "sgoc_profile_enable": (ctypes.c_int, [_I32]),
    "sgoc_profile_query": (ctypes.c_int, [_I32, _PI64, _PD, _PD, _PD]),
    "sgoc_kernel_kind_name": (ctypes.c_char_p, [_I32]),
    "sgoc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "sgoc_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load():
    """Load libsgoc.so (built by paper_2512_23804_gb300.build); raises if missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class SgocError(RuntimeError):
    def __init__(self, status, where):
        lib = load()
        msg = lib.sgoc_last_error().decode()
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status, where):
    if status != SGOC_OK:
        raise SgocError(status, where)
    return status


def _fwd(name):
    def f(*args):
        return getattr(load(), name)(*args)
    f.__name__ = name
    return f


for _name in SIGNATURES:
    globals()[_name] = _fwd(_name)


def profile_enable(on: bool):
    check(load().sgoc_profile_enable(1 if on else 0), "sgoc_profile_enable")


def profile_report():
    """{kind name: dict(launches, ms, bytes, flops)} of the recorded launches."""
    lib = load()
    out = {}
    for k in range(SGOC_KERNEL_KINDS):
        n, ms, by, fl = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        check(lib.sgoc_profile_query(k, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by), ctypes.byref(fl)),
              "sgoc_profile_query")
        if n.value:
            out[lib.sgoc_kernel_kind_name(k).decode()] = dict(launches=n.value, ms=ms.value, bytes=by.value,
                                                             flops=fl.value)
    return out


def inner_product(a, b, stream=None):
    """sum(a * b) in float64 through sgoc_inner_product (a, b: CUDA tensors of one dtype)."""
    import torch
    ws = torch.empty(SGOC_INNER_PRODUCT_WS_BYTES // 8, dtype=torch.float64, device=a.device)
    out = torch.empty(1, dtype=torch.float64, device=a.device)
    s = stream if stream is not None else torch.cuda.current_stream()
    check(load().sgoc_inner_product(0 if a.dtype == torch.float64 else 1, ctypes.c_void_p(a.data_ptr()),
                                    ctypes.c_void_p(b.data_ptr()), a.numel(), ctypes.c_void_p(ws.data_ptr()),
                                    ws.numel() * 8, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream)),
          "sgoc_inner_product")
    return out
