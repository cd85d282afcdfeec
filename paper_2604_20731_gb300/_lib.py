"""ctypes declarations of the libadsgb C ABI (include/adsgb.h).

Marshalling only: every computation happens in the CUDA library.  Loading
fails loudly if the library has not been built or cannot be loaded; there is
no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libadsgb.so")

ADS_OK = 0
STATUS_NAMES = {0: "ok", 1: "invalid argument", 2: "out of device memory", 3: "CUDA error",
                4: "non-finite value", 5: "timeout", 6: "invalid state", 7: "unsupported",
                8: "checkpoint file error"}
ADS_F64, ADS_F32, ADS_BF16 = 0, 1, 2
ADS_PIXEL_F32, ADS_PIXEL_U8 = 0, 1
ADS_MAP_ARITHMETIC, ADS_MAP_GEOMETRIC = 0, 1
MAX_SOURCES = 8

FIELD = dict(S=0, P=1, K=2, ALPHA=3, F=4, U=5, RES=6, Z=7, GU=8, THETA=9, GRAD=10, LOSS=11,
             DT=12, MASS=13, LOSS_LOG=14)


class ads_source(C.Structure):
    _fields_ = [("center", C.c_double * 3), ("sigma", C.c_double), ("rate", C.c_double),
                ("kind", C.c_int)]


class ads_params(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int), ("phi", C.c_double), ("mu_w", C.c_double),
                ("mu_g", C.c_double), ("rho_w", C.c_double), ("rho_g", C.c_double),
                ("grav", C.c_double), ("grav_sign", C.c_double), ("kz_ratio", C.c_double),
                ("n_src", C.c_int), ("src", ads_source * MAX_SOURCES), ("ads_dtype", C.c_int)]


class crvpinn_params(C.Structure):
    _fields_ = [("width", C.c_int), ("hidden_layers", C.c_int), ("dtype", C.c_int), ("act_chunks", C.c_int)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class ads_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class hybrid_params(C.Structure):
    _fields_ = [("n_sub", C.c_int), ("dt", C.c_double), ("dt_policy", C.c_int),
                ("cfl", C.c_double), ("src_frac", C.c_double), ("adam_iters", C.c_int),
                ("lr", C.c_double)]


class hybrid_stats(C.Structure):
    _fields_ = [("dt_used", C.c_double), ("loss_last", C.c_double), ("mass_err", C.c_double),
                ("mass_total", C.c_double)]


class ads_server_config(C.Structure):
    _fields_ = [("hbm_budget", C.c_size_t), ("max_active", C.c_int), ("n_streams", C.c_int)]


class ads_request_spec(C.Structure):
    _fields_ = [("params", ads_params), ("crv", crvpinn_params), ("hp", hybrid_params),
                ("n_steps", C.c_int), ("pretrain_iters", C.c_int), ("pretrain_lr", C.c_double)]


class ads_request_result(C.Structure):
    _fields_ = [("status", C.c_int), ("steps", C.c_int), ("queue_ms", C.c_double),
                ("total_ms", C.c_double), ("p50_step_ms", C.c_double), ("p99_step_ms", C.c_double),
                ("last", hybrid_stats)]


class ads_server_stats_t(C.Structure):
    _fields_ = [("completed", C.c_int64), ("rejected", C.c_int64), ("steps", C.c_int64),
                ("pending", C.c_int64), ("active", C.c_int64), ("peak_active", C.c_int),
                ("bytes_in_use", C.c_size_t), ("peak_bytes", C.c_size_t),
                ("p50_step_ms", C.c_double), ("p99_step_ms", C.c_double)]


# every exported symbol with its signature (restype, argtypes)
_P = C.c_void_p
_D = C.POINTER(C.c_double)
SIGNATURES = {
    "ads_init": (C.c_int, [C.POINTER(ads_params), C.POINTER(crvpinn_params), _D, _D, _D, _P,
                           C.POINTER(_P)]),
    "ads_destroy": (None, [_P]),
    "ads_init_with_allocator": (C.c_int, [C.POINTER(ads_params), C.POINTER(crvpinn_params), _D, _D, _D, _P,
                                          C.POINTER(ads_allocator), C.POINTER(_P)]),
    "ads_hbm_estimate": (C.c_size_t, [C.POINTER(ads_params), C.POINTER(crvpinn_params)]),
    "ads_set_concurrency": (C.c_int, [_P, C.c_int]),
    "ads_save": (C.c_int, [_P, C.c_char_p]),
    "ads_load": (C.c_int, [_P, C.c_char_p]),
    "ads_saturation_step": (C.c_int, [_P, C.c_double, C.c_int]),
    "ads_cfl_dt": (C.c_int, [_P, C.c_double, C.c_double, C.c_double, _D]),
    "ads_galerkin_pressure": (C.c_int, [_P]),
    "ads_set_pressure_coeffs": (C.c_int, [_P, _D]),
    "ads_set_saturation": (C.c_int, [_P, _D]),
    "crvpinn_set_theta": (C.c_int, [_P, _D]),
    "crvpinn_num_params": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "crvpinn_update_coefficients": (C.c_int, [_P]),
    "crvpinn_loss_grad": (C.c_int, [_P, _D]),
    "crvpinn_vjp": (C.c_int, [_P, _D, _D]),
    "crvpinn_pretrain": (C.c_int, [_P, C.c_int, C.c_double, _D]),
    "crvpinn_pressure_update": (C.c_int, [_P, C.c_int, C.c_double, _D]),
    "ads_project_pressure": (C.c_int, [_P]),
    "hybrid_step": (C.c_int, [_P, C.POINTER(hybrid_params), C.POINTER(hybrid_stats)]),
    "hybrid_step_batch": (C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(hybrid_params),
                                    C.POINTER(hybrid_stats)]),
    "hybrid_step_batch_profile": (C.c_int, [C.POINTER(_P), C.c_int, C.c_int, _D]),
    "ads_get": (C.c_int, [_P, C.c_int, _D, C.c_size_t]),
    "ads_field_count": (C.c_int, [_P, C.c_int, C.POINTER(C.c_size_t)]),
    "ads_device_ptr": (C.c_int, [_P, C.c_int, C.POINTER(_P), C.POINTER(C.c_size_t),
                                 C.POINTER(C.c_int)]),
    "ads_sync": (C.c_int, [_P, C.c_double]),
    "ads_saturation_step_noalloc": (C.c_int, [C.POINTER(ads_params), _P, _P, _P, _P, C.c_double,
                                              _P, _P]),
    "ads_saturation_step_noalloc_status": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "ads_kernel_launches": (C.c_int, [_P, C.POINTER(C.c_ulonglong)]),
    "ads_measure_unit_rates": (C.c_int, [_D, C.c_int]),
    "ads_degree_plan_create": (C.c_int, [C.POINTER(ads_params), C.c_int, C.POINTER(_P)]),
    "ads_degree_step": (C.c_int, [_P, _P, _P, _P, _P, C.c_double, _P, _P]),
    "ads_degree_mass": (C.c_int, [_P, _P, _D, _P]),
    "ads_degree_project": (C.c_int, [_P, _P, _P, _P]),
    "ads_degree_project_vjp": (C.c_int, [_P, _P, _P, _P]),
    "ads_degree_cfl_dt": (C.c_int, [_P, _P, _P, _P, C.c_double, C.c_double, C.c_double, _D, _P]),
    "ads_degree_step_vjp": (C.c_int, [_P, _P, _P, _P, _P, C.c_double, _P, _P, _P, _D, _P]),
    "ads_degree_coeffs": (C.c_int, [_P]),
    "ads_degree_plan_destroy": (None, [_P]),
    "ads_map_from_image": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int),
                                     C.c_int, C.c_double, C.c_double, _P, _P]),
    "ads_probe_wait_expiry": (C.c_int, [_P, C.c_double, C.c_int, C.POINTER(C.c_int)]),
    "ads_profile_train": (C.c_int, [_P, C.c_int, _D]),
    "ads_profile_saturation": (C.c_int, [_P, C.c_int, _D]),
    "ads_server_create": (C.c_int, [C.POINTER(ads_server_config), C.POINTER(_P)]),
    "ads_server_submit": (C.c_int, [_P, C.POINTER(ads_request_spec), _D, _D, _D, _D,
                                    C.POINTER(C.c_int64)]),
    "ads_server_wait": (C.c_int, [_P, C.c_int64, C.c_double, _D, _D, C.POINTER(ads_request_result)]),
    "ads_server_stats": (C.c_int, [_P, C.POINTER(ads_server_stats_t)]),
    "ads_server_destroy": (None, [_P]),
    "ads_last_error": (C.c_char_p, [_P]),
    "ads_status_str": (C.c_char_p, [C.c_int]),
}

TRAIN_KERNELS = ["mlp_fwd", "residual", "gram_x", "gram_y", "gram_x_loss",
                 "adjoint_loss_finalize", "mlp_bwd", "grad_adam"]
SAT_KERNELS = ["quad_xsweep", "ysweep", "mass_finalize"]

_lib = None


def load(path: str = LIB_PATH):
    """Load libadsgb.so (raises if it is missing: build it with build.py)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libadsgb.so not found at {path}; build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class AdsError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}"
                         + (f" ({detail})" if detail else ""))
