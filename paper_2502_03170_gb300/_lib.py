"""ctypes binding of libpsf.so: the C structs and the exported prototypes.

Argument marshalling only; every step of the PSF computation runs in the
library's CUDA kernels.  Loading fails loudly when the library is missing.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpsf.so")

PSF_OK = 0
PSF_ERR_ARG = -1
PSF_ERR_NOT_AXISYMMETRIC = -2
PSF_ERR_WORKSPACE = -3
PSF_ERR_PRECISION = -4
PSF_ERR_CUDA = -5
PSF_ERR_DEVICE_TIMEOUT = -6

PSF_PREC_FP32 = 0
PSF_PREC_SPLIT_FP16 = 1
PSF_PREC_SPLIT_BF16 = 2
PSF_PREC_FP32_CHIRPZ = 3
PSF_PREC_AUTO = 4
PSF_PREC_SPLIT_TF32 = 5
PSF_PREC_TF32 = 6

PSF_PROJECT_AXISYMMETRIC = 1
PSF_SCALAR = 2
PSF_FRESNEL = 4
PSF_OUTSIDE_ENVELOPE = 8

ERROR_NAMES = {
    PSF_ERR_ARG: "PSF_ERR_ARG",
    PSF_ERR_NOT_AXISYMMETRIC: "PSF_ERR_NOT_AXISYMMETRIC",
    PSF_ERR_WORKSPACE: "PSF_ERR_WORKSPACE",
    PSF_ERR_PRECISION: "PSF_ERR_PRECISION",
    PSF_ERR_CUDA: "PSF_ERR_CUDA",
    PSF_ERR_DEVICE_TIMEOUT: "PSF_ERR_DEVICE_TIMEOUT",
}


class PsfOptics(ctypes.Structure):
    _fields_ = [("NA", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("n_i", ctypes.c_double), ("n_s", ctypes.c_double),
                ("n_g", ctypes.c_double), ("n_i_design", ctypes.c_double),
                ("n_g_design", ctypes.c_double), ("t_g", ctypes.c_double),
                ("t_g_design", ctypes.c_double), ("t_i_design", ctypes.c_double),
                ("depth", ctypes.c_double), ("pol", ctypes.c_double * 4),
                ("apodize", ctypes.c_int), ("s_env", ctypes.c_double),
                ("flags", ctypes.c_int)]


class PsfGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("nz", ctypes.c_int), ("z", ctypes.POINTER(ctypes.c_double))]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_S = ctypes.c_size_t
_OPT = ctypes.POINTER(PsfOptics)
_GRID = ctypes.POINTER(PsfGrid)

# name -> (restype, argtypes); must match include/psf.h
PROTOTYPES = {
    "psf_version": (_I, []),
    "psf_last_error": (ctypes.c_char_p, []),
    "psf_workspace_status": (_I, [_P, _P]),
    "psf_fourier_workspace_size": (_S, [_OPT, _I, _GRID, _I]),
    "psf_fourier_vectorial": (_I, [_OPT, _I, _GRID, _P, _I, _P, _I, _P, _P,
                                   _P, _S, _P]),
    "psf_fourier_vectorial_noalloc": (_I, [_OPT, _I, _GRID, _P, _I, _P, _P,
                                           _P, _P]),
    "psf_fourier_backward_workspace_size": (_S, [_OPT, _I, _GRID, _I]),
    "psf_fourier_backward_workspace_size_batch": (_S, [_OPT, _I, _GRID, _I, _I]),
    "psf_fourier_vectorial_backward": (_I, [_OPT, _I, _GRID, _I, _P, _I, _P,
                                            _I, _P, _P, _P, _P, _P, _P, _S,
                                            _P]),
    "psf_kernel_timing": (_I, [_I]),
    "psf_kernel_timing_read": (_I, [_I, ctypes.POINTER(_I),
                                    ctypes.POINTER(ctypes.c_double)]),
    "psf_mlp_param_count": (_S, []),
    "psf_mlp_state_bytes": (_S, []),
    "psf_mlp_init": (_I, [_P, ctypes.c_ulonglong, _P]),
    "psf_mlp_workspace_size": (_S, [_I]),
    "psf_mlp_train_step": (_I, [_P, _P, _P, _I, ctypes.c_float, _I, _P, _P, _S,
                                _P]),
    "psf_mlp_gradients": (_I, [_P, _P, _P, _I, _P, _P, _P, _S, _P]),
    "psf_mlp_forward": (_I, [_P, _P, _I, _P, _P, _P, _S, _P]),
    "psf_mlp_get_params": (_I, [_P, _P, _P]),
    "psf_mlp_set_params": (_I, [_P, _P, _P]),
    "psf_surrogate_workspace_size": (_S, [_OPT, _I, _I, _I, _I, _I]),
    "psf_surrogate_phase": (_I, [_OPT, _P, _I, _P, _I, _P]),
    "psf_surrogate_profiles": (_I, [_P, _OPT, _P, _I, _D, _I, _I, _I, _D, _D,
                                    _I, _P, ctypes.POINTER(_I), _P, _S, _P]),
    "psf_bessel_workspace_size": (_S, [_OPT, _I, _I, _I, _I, _I, _I, _I]),
    "psf_bessel_vectorial": (_I, [_OPT, _I, _P, _P, _I, _P, _P, _P, _I, _I,
                                  _I, _I, _I, _D, _D, _I, _P, _P, _P, _S, _P]),
    "psf_bessel_backward_workspace_size": (_S, [_OPT, _I, _I, _I, _I, _I, _I,
                                                _I]),
    "psf_bessel_harmonic_order": (_I, [_P, _I, _I, _D]),
    "psf_bessel_harmonic_workspace_size": (_S, [_OPT, _I, _I, _I, _I, _I, _I, _I, _I]),
    "psf_bessel_vectorial_harmonic": (_I, [_OPT, _I, _P, _P, _I, _P, _P, _I, _I, _I,
                                           _I, _I, _D, _D, _I, _D, _I, _P, _P, _S, _P]),
    "psf_bessel_vectorial_backward": (_I, [_OPT, _I, _P, _P, _I, _P, _P, _P,
                                           _I, _I, _I, _I, _I, _D, _D, _I, _P,
                                           _P, _P, _P, _P, _P, _P, _S, _P]),
}

_lib = None


def load(path=None):
    """Load libpsf.so (built in-tree by ``build.build()``) and set prototypes."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(
            "libpsf.so not found at %s: build it with "
            "paper_2502_03170_gb300.build.build()" % p)
    lib = ctypes.CDLL(p)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


class PsfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERROR_NAMES.get(code, "?"), code, msg))
        self.code = code


def check(lib, code):
    if code != PSF_OK:
        raise PsfError(code, lib.psf_last_error().decode(errors="replace"))
    return code
