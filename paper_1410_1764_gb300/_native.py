"""ctypes declarations of libchemora.so (C ABI in include/chemora.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Loading fails loudly when the library has not been built.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libchemora.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENONFINITE, EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
WAVE, WAVE_VARC, BSSN, WAVE1 = 1, 2, 3, 4

_c_p = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)


class Params(ctypes.Structure):
    _fields_ = [("eps_diss", ctypes.c_double), ("eta", ctypes.c_double),
                ("slicing", ctypes.c_int), ("shift", ctypes.c_int), ("fd_order", ctypes.c_int)]


# name: (restype, argtypes)
SIGNATURES = {
    "chemora_grid_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_double, ctypes.POINTER(_c_p)]),
    "chemora_grid_layout": (ctypes.c_int, [_c_p, _i64p, _i64p, _i64p]),
    "chemora_system_create": (ctypes.c_int, [_c_p, ctypes.c_int, ctypes.POINTER(Params),
                                             ctypes.POINTER(_c_p)]),
    "chemora_system_set_speed": (ctypes.c_int, [_c_p, _c_p, _c_p]),
    "chemora_fill_ghosts": (ctypes.c_int, [_c_p, _c_p, _c_p]),
    "chemora_fill_ghosts_axes": (ctypes.c_int, [_c_p, _c_p, ctypes.c_int, _c_p]),
    "chemora_stage": (ctypes.c_int, [_c_p, ctypes.c_int, _c_p, _c_p, _c_p, _c_p, ctypes.c_double,
                                     ctypes.c_double, _c_p]),
    "chemora_rhs": (ctypes.c_int, [_c_p, _c_p, _c_p, _c_p]),
    "chemora_rk4_step": (ctypes.c_int, [_c_p, _c_p, ctypes.c_double, ctypes.c_int, _c_p]),
    "chemora_rk4_step_host": (ctypes.c_int, [_c_p, _c_p, ctypes.c_double, ctypes.c_int, _c_p]),
    "chemora_rk4_step_noalloc": (ctypes.c_int, [_c_p, _c_p, ctypes.c_double, ctypes.c_int, _c_p]),
    "chemora_constraints": (ctypes.c_int, [_c_p, _c_p, _c_p, _c_p]),
    "chemora_energy": (ctypes.c_int, [_c_p, _c_p, _dp, _c_p]),
    "chemora_check_finite": (ctypes.c_int, [_c_p, _c_p, _i64p, _c_p]),
    "chemora_patches_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                              ctypes.c_double, ctypes.c_int, ctypes.POINTER(Params),
                                              ctypes.POINTER(_c_p)]),
    "chemora_patches_state": (ctypes.c_int, [_c_p, ctypes.c_int, ctypes.POINTER(_c_p)]),
    "chemora_patches_inject_fault": (ctypes.c_int, [_c_p, ctypes.c_int]),
    "chemora_patches_set_time_limit": (ctypes.c_int, [_c_p, ctypes.c_double]),
    "chemora_patches_step": (ctypes.c_int, [_c_p, ctypes.c_double, ctypes.c_int, ctypes.c_int, _c_p]),
    "chemora_amr_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                          ctypes.c_double, ctypes.POINTER(_c_p)]),
    "chemora_amr_state": (ctypes.c_int, [_c_p, ctypes.c_int, ctypes.POINTER(_c_p), _i64p, _i64p, _i64p]),
    "chemora_amr_step": (ctypes.c_int, [_c_p, ctypes.c_double, ctypes.c_int, _c_p]),
    "chemora_amr_create_boxes": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                                ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                                ctypes.c_double, ctypes.POINTER(Params), ctypes.POINTER(_c_p)]),
    "chemora_system_set_chain": (ctypes.c_int, [_c_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "chemora_amr_autotune": (ctypes.c_int, [_c_p, ctypes.POINTER(ctypes.c_int), _c_p]),
    "chemora_amr_step_mode": (ctypes.c_int, [_c_p, ctypes.c_double, ctypes.c_int, ctypes.c_int, _c_p]),
    "chemora_adjoint_rk4": (ctypes.c_int, [_c_p, _c_p, _c_p, ctypes.c_double, ctypes.c_int,
                                           ctypes.c_int, _i64p, ctypes.c_int, _dp, _dp, _c_p, _c_p,
                                           _c_p]),
    "chemora_autotune": (ctypes.c_int, [_c_p, _c_p, ctypes.POINTER(ctypes.c_int), _dp, _c_p]),
    "chemora_variant_count": (ctypes.c_int, [ctypes.c_int]),
    "chemora_variant_info": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_int)]),
    "chemora_system_specialize": (ctypes.c_int, [_c_p, ctypes.c_int, ctypes.c_char_p, _dp]),
    "chemora_system_variant": (ctypes.c_int, [_c_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "chemora_profile_enable": (ctypes.c_int, [_c_p, ctypes.c_int]),
    "chemora_profile_read": (ctypes.c_int, [_c_p, _dp, _i64p, ctypes.c_int]),
    "chemora_launch_count": (ctypes.c_int64, []),
    "chemora_opcount": (ctypes.c_int, [ctypes.c_int, _i64p, _i64p]),
    "chemora_system_opcount": (ctypes.c_int, [_c_p, _i64p, _i64p]),
    "chemora_fp64_peak": (ctypes.c_int, [_dp, _c_p]),
    "chemora_last_error": (ctypes.c_char_p, []),
    "chemora_destroy": (None, [_c_p]),
}

_lib = None


class ChemoraError(RuntimeError):
    def __init__(self, code, where):
        msg = lib().chemora_last_error().decode(errors="replace")
        super().__init__("%s failed (%d): %s" % (where, code, msg))
        self.code = code


def lib():
    """The loaded libchemora.so; raises if it is missing (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libchemora.so is not built (%s); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(code, where):
    if code != OK:
        raise ChemoraError(code, where)
    return code
