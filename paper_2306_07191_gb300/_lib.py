"""ctypes binding of libnif.so: the C ABI declared in include/nif.h, with the
same names.  Argument marshalling only; every computation runs in the CUDA
library.  Importing this module fails loudly when the library is missing."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnif.so")

NIF_OK = 0
NIF_ERR_ARG = -1
NIF_ERR_CUDA = -2
NIF_ERR_WORKSPACE = -3
NIF_ERR_TIMEOUT = -4
NIF_ERR_NUMERIC = -5
NIF_ERR_UNSUPPORTED = -6
NIF_ERR_BOUNDS = -7

NIF_MAX_LEVELS = 24
NIF_F32, NIF_F16, NIF_BF16, NIF_E4M3 = 0, 1, 2, 3
NIF_SCHED_AUTO, NIF_SCHED_SERIAL, NIF_SCHED_PIPELINED = 0, 1, 2
NIF_ENC_MULTIRES, NIF_ENC_SPHERICAL_OUTER, NIF_ENC_SPHERICAL_INNER = 0, 1, 2
NIF_ROUND1_NEAREST, NIF_ROUND1_OUTER = 0, 1
NIF_ACT_RELU, NIF_ACT_LEAKY = 0, 1
NIF_NETS_SINGLE, NIF_NETS_CLASS, NIF_NETS_OBJECT = 0, 1, 2
NIF_QUERY_INNER = 0x80000000

P = ctypes.c_void_p
i32 = ctypes.c_int32
i64 = ctypes.c_int64
f32 = ctypes.c_float
size_t = ctypes.c_size_t


class ModelDesc(ctypes.Structure):
    _fields_ = [
        ("n_levels", i32), ("n_features", i32), ("log2_table", i32),
        ("res", i32 * NIF_MAX_LEVELS),
        ("grid_dtype", i32), ("n_objects", i32),
        ("d_obj_aabb", P), ("d_grids", P),
        ("n_hidden", i32), ("width", i32), ("act", i32), ("leaky_slope", f32),
        ("mlp_dtype", i32), ("net_mode", i32), ("n_nets", i32),
        ("d_weights", P), ("d_scales", P),
        ("tile_m", i32), ("ctas_per_sm", i32), ("schedule", i32),
        ("encoding", i32), ("res_1d", i32), ("n_features_1d", i32),
        ("n_outputs", i32), ("round1", i32),
    ]


class OptimDesc(ctypes.Structure):
    _fields_ = [
        ("lr", f32), ("beta1", f32), ("beta2", f32), ("eps", f32), ("loss_scale", f32),
        ("step", i32),
        ("d_w_master", P), ("d_w_grad", P), ("d_w_m", P), ("d_w_v", P),
        ("d_g_master", P), ("d_g_grad", P), ("d_g_m", P), ("d_g_v", P),
        ("deterministic", i32), ("d_det_ws", P), ("det_ws_bytes", size_t),
        ("half_precision", i32), ("d_loss_scale", P), ("d_scale_state", P), ("scale_window", i32),
    ]


MD = ctypes.POINTER(ModelDesc)
OD = ctypes.POINTER(OptimDesc)

# name: (restype, argtypes)
SIGNATURES = {
    "nif_last_error": (ctypes.c_char_p, []),
    "nif_version": (i32, []),
    "nif_grid_vertices": (i64, [MD]),
    "nif_weight_count": (i64, [MD]),
    "bvh_build_size": (size_t, [i64]),
    "bvh_build_workspace_size": (size_t, [i64]),
    "bvh_build": (i32, [P, i64, P, i64, P, P, size_t, P, size_t, P]),
    "bvh_build_boxes": (i32, [P, i64, P, size_t, P, size_t, P]),
    "bvh_build_boxes_ploc": (i32, [P, i64, P, size_t, P, size_t, P]),
    "bvh_build_ploc_workspace_size": (size_t, [i64]),
    "bvh_build_ploc": (i32, [P, i64, P, i64, P, P, size_t, P, size_t, P]),
    "bvh_info": (i32, [P, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i32), P]),
    "bvh_stats": (i32, [P, P, i64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                        ctypes.POINTER(ctypes.c_double), P, P]),
    "bvh_check": (i32, [P, P]),
    "bvh_cast_shadow": (i32, [P, P, i64, P, P]),
    "bvh_cast_shadow_or": (i32, [P, P, i64, P, P]),
    "nif_bits_clear": (i32, [P, i64, P]),
    "bvh_cast_closest": (i32, [P, P, i64, P, P, P]),
    "bvh_cast_pairs": (i32, [P, P, P, P, i64, P, P]),
    "bvh_cast_pairs_closest": (i32, [P, P, P, P, i64, P, P, P]),
    "nif_light_cdf": (i32, [P, i32, P, P]),
    "nif_light_samples": (i32, [P, P, P, P, P, i64, i32, P, P, i32, P, f32, f32, P, P, P]),
    "nif_shade": (i32, [P, P, i64, i32, P, P]),
    "nif_shadow_rays": (i32, [P, P, i64, i32, P, i32, f32, P, P]),
    "nif_workspace_size": (size_t, [MD, i64, i64]),
    "nif_train_workspace_size": (size_t, [MD, i64]),
    "nif_deterministic_workspace_size": (size_t, [MD, i64]),
    "nif_check": (i32, [P, ctypes.POINTER(i64), P]),
    "nif_frontend": (i32, [MD, P, P, i64, P, P, i64, P, P, P, size_t, P]),
    "nif_encode": (i32, [MD, P, P, P, i64, P, i32, P]),
    "nif_mlp_infer": (i32, [MD, P, P, i64, P, P, size_t, P]),
    "nif_tc_mma_rate": (i32, [i32, i32, i32, i32, i32, i32, P, P, size_t, P]),
    "nif_infer_queries": (i32, [MD, P, i64, P, P, P, i64, P, P, P, size_t, P]),
    "nif_infer": (i32, [MD, P, P, i64, P, P, size_t, P]),
    "nif_infer_query_counts": (i32, [MD, P, size_t, i64, P, P]),
    "nif_state_size": (size_t, [MD]),
    "nif_state_save": (i32, [MD, OD, P, size_t, P]),
    "nif_state_load": (i32, [MD, OD, P, size_t, P]),
    "nif_frontend_nearest": (i32, [MD, P, P, i64, P, P, P, i64, P, P, P, size_t, P]),
    "nif_frontend_rest": (i32, [MD, P, P, i64, P, P, P, i64, P, P, P, P, size_t, P]),
    "nif_saved_size": (size_t, [MD, i64]),
    "nif_fwd_train": (i32, [MD, P, P, P, P, i64, P, P, P]),
    "nif_loss": (i32, [P, P, i64, f32, P, P, P]),
    "nif_loss_aux": (i32, [P, P, P, i64, i32, f32, P, P, P]),
    "nif_mlp_bwd": (i32, [MD, P, P, i64, P, P, P, P, P]),
    "nif_grid_bwd": (i32, [MD, P, P, P, i64, P, P, P]),
    "nif_adam": (i32, [P, P, P, P, i64, f32, f32, f32, f32, f32, i32, P, i32, P]),
    "nif_train_step": (i32, [MD, OD, P, P, P, P, P, i64, P, P, size_t, P]),
    "nif_train_grads": (i32, [MD, OD, P, P, P, P, P, i64, P, P, size_t, P]),
    "nif_train_step_aux": (i32, [MD, OD, P, P, P, P, P, P, i64, P, P, size_t, P]),
    "nif_primary_resolve": (i32, [MD, P, i64, P, P, P, i64, P, P, P, P, P, P]),
    "nif_frontend_rest_nearer": (i32, [MD, P, P, i64, P, P, P, i64, P, P, P, P, size_t, P]),
    "nif_fill_uniform": (i32, [P, i64, ctypes.c_uint64, f32, P]),
    "nif_infer_noalloc": (i32, [MD, P, P, i64, P, P]),
    "nif_wait_selftest": (i32, [P, size_t, i64, P]),
}


class NifError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libnif error {code}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"libnif.so is not built ({LIB_PATH}); run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def last_error() -> str:
    m = lib.nif_last_error()
    return m.decode() if m else ""


def check(status: int) -> None:
    if status != NIF_OK:
        raise NifError(int(status), last_error())


def call(name: str, *args) -> None:
    check(getattr(lib, name)(*args))
