"""ctypes binding of ``liblbm_gb300.so`` (the C ABI declared in include/lbm.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  There is no fallback: if the library is missing or fails to load,
``load()`` raises.
"""
import ctypes
import os

from . import _build

# constants mirrored from include/lbm.h
LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSUPPORTED, LBM_ENONFINITE, LBM_ESTATE = range(7)
LBM_D3Q19 = 19
LBM_D3Q27 = 27
EQ_STANDARD, EQ_IMPROVED = 0, 1
SRT, TRT, MRT = 0, 1, 2
F64, F32, F16S, BF16S = 0, 1, 2, 3
DTYPE_F64, DTYPE_F32 = 0, 1
PATTERN_AB, PATTERN_AA = 0, 1
OPT_TRT_MAGIC, OPT_FORCE_X, OPT_FORCE_Y, OPT_FORCE_Z = 1, 2, 3, 4
OPT_WALLS_X, OPT_WALLS_Y, OPT_WALLS_Z = 5, 6, 7
OPT_RHO0_MODE, OPT_PATTERN, OPT_TAU, OPT_EQUILIBRIUM, OPT_COLLISION = 8, 9, 10, 11, 12
OPT_BLOCK_X, OPT_BLOCK_Y, OPT_CELLS_X = 13, 14, 15
OPT_MRT_OMEGA_BULK, OPT_MRT_OMEGA_4, OPT_GRAPHS = 16, 17, 18
OPT_ADJ_DEFER_SUM = 19
RED_MASS, RED_ENERGY, RED_JX, RED_JY, RED_JZ, RED_UMAX, RED_NONFINITE = range(7)
RED_COUNT = 8

_lib = None

# name -> (restype, argtypes)
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_SIGS = {
    "lbm_abi_version": (_i, []),
    "lbm_status_string": (ctypes.c_char_p, [_i]),
    "lbm_velocity_set": (_i, [ctypes.POINTER(_i), ctypes.POINTER(_d), ctypes.POINTER(_i)]),
    "lbm_velocity_set_of": (_i, [_i, ctypes.POINTER(_i), ctypes.POINTER(_d), ctypes.POINTER(_i)]),
    "lbm_create": (_i, [_i, _i, _i, _i, _i, _i, _d, _i, ctypes.POINTER(_vp)]),
    "lbm_destroy": (_i, [_vp]),
    "lbm_set_option": (_i, [_vp, _i, _d]),
    "lbm_get_option": (_i, [_vp, _i, ctypes.POINTER(_d)]),
    "lbm_required_bytes": (_i, [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(_i),
                                ctypes.POINTER(ctypes.c_size_t)]),
    "lbm_bind": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "lbm_init": (_i, [_vp, _vp, _vp, _i]),
    "lbm_step": (_i, [_vp, _i]),
    "lbm_moments": (_i, [_vp, _vp, _vp, _i]),
    "lbm_reduce": (_i, [_vp, ctypes.POINTER(_d)]),
    "lbm_enstrophy": (_i, [_vp, ctypes.POINTER(_d)]),
    "lbm_reduce_noalloc": (_i, [_vp, ctypes.POINTER(_d)]),
    "lbm_steps_done": (_i, [_vp, ctypes.POINTER(ctypes.c_longlong)]),
    "lbm_get_pdfs": (_i, [_vp, _vp]),
    "lbm_set_pdfs": (_i, [_vp, _vp]),
    "lbm_adjoint_seed": (_i, [_vp, _vp, _vp, _i, _vp]),
    "lbm_adjoint_step": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "lbm_adjoint_flush": (_i, [_vp]),
    "lbm_adjoint_init_velocity": (_i, [_vp, _vp, _vp, _i, _vp, _vp]),
    "lbm_adjoint_tau_gradient": (_i, [_vp, ctypes.POINTER(_d), ctypes.POINTER(_d)]),
    "lbm_last_error": (ctypes.c_char_p, [_vp]),
}


class LBMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d): %s" % (_status_name(status), status, msg))
        self.status = status


def _status_name(s):
    return {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ECUDA", 4: "LBM_EUNSUPPORTED",
            5: "LBM_ENONFINITE", 6: "LBM_ESTATE"}.get(s, "LBM_?")


def library_path():
    return _build.LIB


def load(build_if_missing=False):
    """Loads the compiled library (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise ImportError("liblbm_gb300.so is not built (run __graft_entry__.build() or "
                              "python -m paper_1803_04937_gb300._build); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return sorted(_SIGS)


def check(status, handle=None):
    if status != LBM_OK:
        lib = load()
        msg = lib.lbm_last_error(handle).decode() if handle else lib.lbm_status_string(status).decode()
        raise LBMError(status, msg)
    return status
