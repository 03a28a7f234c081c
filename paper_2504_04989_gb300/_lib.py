"""ctypes view of libtsvd.so (declarations in include/tsvd.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Loading fails loudly when the library has not been built; there is
no fallback path.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtsvd.so")

TSVD_FP64, TSVD_FP32, TSVD_MIXED_TF32, TSVD_MIXED_BF16, TSVD_SPLIT_TF32 = 0, 1, 2, 3, 4
TSVD_FLAG_FP64_QR = 1
TSVD_FLAG_ALG1 = 2
TSVD_FLAG_SIMT = 4
TSVD_FLAG_QTRUNC = 8
TSVD_FLAG_DEFLATE = 16
TSVD_FLAG_GRAM_INT = 32
PRECISIONS = {"fp64": TSVD_FP64, "fp32": TSVD_FP32, "tf32": TSVD_MIXED_TF32, "bf16": TSVD_MIXED_BF16,
              "tf32x3": TSVD_SPLIT_TF32}

ERRORS = {0: "ok", -1: "invalid argument", -2: "workspace too small", -3: "CUDA failure",
          -4: "unsupported size or mode", -5: "eigen solve did not converge",
          -6: "rank-deficient Fourier slice"}


class TsvdParams(C.Structure):
    _fields_ = [("R", C.c_int), ("P", C.c_int), ("q", C.c_int), ("precision", C.c_int),
                ("seed", C.c_uint64), ("flags", C.c_int)]


class TsvdInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("m_eff", C.c_int), ("dead_columns", C.c_int), ("reserved", C.c_int)]


class TsvdRbkDesc(C.Structure):
    _fields_ = [("A", C.c_void_p), ("n1", C.c_int), ("n2", C.c_int), ("n3", C.c_int), ("params", TsvdParams),
                ("Omega", C.c_void_p), ("U", C.c_void_p), ("S", C.c_void_p), ("V", C.c_void_p),
                ("sigma_hat", C.c_void_p)]


class TsvdStageTime(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("ms", C.c_double), ("count", C.c_int)]


# name -> (restype, argtypes); mirrors include/tsvd.h
_vp, _i, _sz, _u32, _u64, _l = C.c_void_p, C.c_int, C.c_size_t, C.c_uint32, C.c_uint64, C.c_long
SIGNATURES = {
    "tsvd_rbk_workspace_size": (_i, [_i, _i, _i, C.POINTER(TsvdParams), C.POINTER(_sz)]),
    "tsvd_rbk": (_i, [_vp, _i, _i, _i, C.POINTER(TsvdParams), _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp,
                      C.POINTER(TsvdInfo)]),
    "tsvd_rbk_batched_workspace_size": (_i, [C.POINTER(TsvdRbkDesc), _i, _i, C.POINTER(_sz)]),
    "tsvd_rbk_batched": (_i, [C.POINTER(TsvdRbkDesc), _i, _i, _vp, _sz, _vp]),
    "tprod_workspace_size": (_i, [_i, _i, _i, _i, _i, C.POINTER(_sz)]),
    "tprod": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, _vp, _sz, _vp]),
    "tproj_workspace_size": (_i, [_i, _i, _i, _i, _i, C.POINTER(_sz)]),
    "tproj": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, _vp, _sz, _vp]),
    "tprod_backward_workspace_size": (_i, [_i, _i, _i, _i, _i, C.POINTER(_sz)]),
    "tprod_backward": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _i, _i, _i, _i, _vp, _sz, _vp]),
    "tproj_backward_workspace_size": (_i, [_i, _i, _i, _i, _i, C.POINTER(_sz)]),
    "tproj_backward": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _i, _i, _i, _i, _vp, _sz, _vp]),
    "ttranspose": (_i, [_vp, _vp, _i, _i, _i, _i, _vp]),
    "tsvd_masked_residual": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, C.c_long, _i, _vp]),
    "tsvd_error_workspace_size": (_i, [_i, _i, _i, _i, _i, C.POINTER(C.c_size_t)]),
    "tsvd_error": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _i, _i, _vp, _vp, C.c_size_t, _vp]),
    "tprod_noalloc": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, _vp]),
    "tsvd_rfft3": (_i, [_vp, _l, _i, _i, _vp, _vp]),
    "tsvd_irfft3": (_i, [_vp, _l, _i, _i, _vp, _vp]),
    "tsvd_rbk_fourier_workspace_size": (_i, [_i, _i, _i, _i, _i, C.POINTER(TsvdParams), C.POINTER(_sz)]),
    "tsvd_rbk_fourier": (_i, [_vp, _i, _i, _i, _i, _i, C.POINTER(TsvdParams), _vp, _vp, _vp, _vp, _vp, _sz, _vp,
                              C.POINTER(TsvdInfo)]),
    "tsvd_lowrank_workspace_size": (_i, [_i, _i, _i, _i, _i, C.POINTER(_sz)]),
    "tsvd_lowrank": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, _vp, _vp, _sz, _vp]),
    "tsvd_sigma_tubes": (_i, [_vp, _i, _i, C.c_double, _i, _vp, _vp, _sz, _vp]),
    "tsvd_fill_in": (_i, [_vp, _vp, _vp, _vp, _l, _i, _vp, _vp, _vp]),
    "tsvd_sqdiff": (_i, [_vp, _vp, _l, _i, _vp, _vp, _vp]),
    "tqr_workspace_size": (_i, [_i, _i, _i, _i, C.POINTER(_sz)]),
    "tqr": (_i, [_vp, _i, _i, _i, _i, _vp, _vp, _vp, _sz, _vp, C.POINTER(TsvdInfo)]),
    "tpinv_workspace_size": (_i, [_i, _i, _i, _i, C.POINTER(_sz)]),
    "tpinv": (_i, [_vp, _i, _i, _i, _i, _vp, _vp, _sz, _vp, C.POINTER(TsvdInfo)]),
    "tsvd_gaussian": (_i, [_u64, _u32, _u32, _l, _vp, _vp]),
    "tsvd_philox_words": (_i, [C.POINTER(_u32), _u32, _u32, _u32, _l, _vp, _vp]),
    "tsvd_profile_begin": (_i, []),
    "tsvd_profile_end": (_i, [C.POINTER(TsvdStageTime), _i, C.POINTER(_i)]),
    "tsvd_launch_count": (C.c_ulonglong, []),
    "tsvd_strerror": (C.c_char_p, [_i]),
    "tsvd_version": (_i, []),
}

_lib = None


class TsvdError(RuntimeError):
    pass


def load():
    """Load libtsvd.so (raises if it is missing: no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise TsvdError("libtsvd.so is not built (%s); run `python -c 'import __graft_entry__ as g; g.build()'`"
                            % LIB_PATH)
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(rc, what):
    if rc != 0:
        raise TsvdError("%s failed: %s (%d)" % (what, ERRORS.get(rc, "unknown"), rc))
