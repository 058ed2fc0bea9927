"""ctypes binding of libsevennet.so (argument marshalling only).

Every computation runs in the library's CUDA kernels.  Importing this module
does not load the library; the first call does, and it raises if the library
was not built (there is no other code path).
"""

import ctypes
import os

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libsevennet.so")

OK, EINVAL, ENOMEM, ECUDA, EOVERFLOW, ETIMEDOUT, ENOMEM_ADMIT, EAGAIN = 0, -1, -2, -3, -4, -5, -6, -7
PRECISION = {"fp32": 0, "bf16": 1}


class SevenNetError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"sevennet status {status}: {message}")
        self.status = status


class ModelConfig(ctypes.Structure):
    _fields_ = [
        ("n_species", ctypes.c_int32),
        ("n_layers", ctypes.c_int32),
        ("lmax", ctypes.c_int32),
        ("mul", ctypes.c_int32 * 4),
        ("r_cut", ctypes.c_double),
        ("n_basis", ctypes.c_int32),
        ("poly_p", ctypes.c_int32),
        ("mlp_hidden", ctypes.c_int32),
        ("avg_num_neigh", ctypes.c_double),
        ("readout_hidden", ctypes.c_int32),
        ("scale", ctypes.c_double),
        ("shift", ctypes.POINTER(ctypes.c_double)),
    ]


class Request(ctypes.Structure):
    _fields_ = [
        ("n_atoms", ctypes.c_int64),
        ("species", ctypes.POINTER(ctypes.c_int32)),
        ("pos", ctypes.POINTER(ctypes.c_double)),
        ("cell", ctypes.POINTER(ctypes.c_double)),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("energy", ctypes.c_double),
        ("forces", ctypes.POINTER(ctypes.c_double)),
        ("virial", ctypes.c_double * 9),
        ("submit_s", ctypes.c_double),
        ("start_s", ctypes.c_double),
        ("done_s", ctypes.c_double),
        ("batch_id", ctypes.c_int32),
        ("batch_structs", ctypes.c_int32),
    ]


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int32)

# name -> (restype, argtypes); the C-ABI entry points of include/sevennet.h
SIGNATURES = {
    "sevennet_last_error": (ctypes.c_char_p, []),
    "sevennet_n_params": (_I64, [ctypes.POINTER(ModelConfig)]),
    "sevennet_padded_weights": (_I32, [ctypes.POINTER(ModelConfig), _D, ctypes.c_size_t, _IP, _D, ctypes.c_size_t]),
    "sevennet_create_model": (_I32, [ctypes.POINTER(ModelConfig), _D, ctypes.c_size_t, ctypes.c_int,
                                     ctypes.POINTER(_P)]),
    "sevennet_destroy_model": (None, [_P]),
    "sevennet_build_neighbors": (_I32, [_P, _I64, _D, _D, _IP, ctypes.POINTER(_P), ctypes.POINTER(_I64)]),
    "sevennet_nlist_export": (_I32, [_P, _IP, _IP, _IP]),
    "sevennet_nlist_destroy": (None, [_P]),
    "sevennet_eval_energy_forces_virial": (_I32, [_P, _I64, _IP, _D, _D, _IP, ctypes.c_int, _D, _D, _D]),
    "sevennet_eval_batch_dev": (_I32, [_P, _I32, ctypes.POINTER(_I64), _D, _IP, _P, _P, ctypes.c_int,
                                       _P, _P, _P, _P]),
    "sevennet_conv_forward_dev": (_I32, [_P, _I32, _I64, _I64, _P, _P, _P, _P, _P, ctypes.c_int, _P]),
    "sevennet_conv_backward_dev": (_I32, [_P, _I32, _I64, _I64, _P, _P, _P, _P, _P, _P, _P,
                                          ctypes.c_int, _P]),
    "sevennet_conv_forward_noalloc": (_I32, [_P, _I32, _I64, _I64, _P, _P, _P, _P, _P, ctypes.c_int, _P]),
    "sevennet_conv_dims": (_I32, [_P, _I32, _IP, _IP]),
    "sevennet_md_create": (_I32, [_P, _I64, _IP, _D, _D, _D, _D, ctypes.c_int, ctypes.POINTER(_P)]),
    "sevennet_md_step": (_I32, [_P, _I64, ctypes.c_double, _D, _D]),
    "sevennet_md_get_state": (_I32, [_P, _D, _D, _D]),
    "sevennet_eval_decomposed": (_I32, [_P, _I64, _IP, _D, _D, ctypes.c_int32, ctypes.c_int, _D, _D, _D]),
    "sevennet_md_set_skin": (_I32, [_P, ctypes.c_double]),
    "sevennet_md_set_nose_hoover": (_I32, [_P, ctypes.c_double, ctypes.c_double]),
    "sevennet_md_set_nose_hoover_ramp": (_I32, [_P, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                                ctypes.c_double]),
    "sevennet_md_get_nose_hoover": (_I32, [_P, _D, _D]),
    "sevennet_md_get_stats": (_I32, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "sevennet_md_destroy": (None, [_P]),
    "sevennet_server_create": (_I32, [_P, ctypes.c_size_t, _I32, _I32, ctypes.c_int, ctypes.POINTER(_P)]),
    "sevennet_server_submit": (_I32, [_P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "sevennet_server_poll": (_I32, [_P, ctypes.c_uint64, ctypes.POINTER(Result), ctypes.POINTER(ctypes.c_int)]),
    "sevennet_server_now": (ctypes.c_double, [_P]),
    "sevennet_server_destroy": (None, [_P]),
    "sevennet_profile": (_I32, [_P, _I32]),
    "sevennet_profile_read": (_I32, [_P, _I32, ctypes.c_char_p, _D, ctypes.POINTER(_I64), _IP]),
    "sevennet_launch_count": (_I64, []),
    "sevennet_fp32_peak": (_I32, [_I32, _I32, _I32, _D, _D]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the library (once) and declare every entry point."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: the CUDA library is not built "
                           "(run paper_2402_03789_gb300.build.build()); there is no fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status):
    if status != OK:
        msg = load().sevennet_last_error()
        raise SevenNetError(status, msg.decode() if msg else "")
    return status


def dptr(a):
    """ctypes double* of a C-contiguous float64 numpy array (or None)."""
    if a is None:
        return None
    return a.ctypes.data_as(_D)


def iptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_IP)


def as_f64(a, shape=None):
    out = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        out = out.reshape(shape)
    return out


def as_i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))
