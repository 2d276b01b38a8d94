"""ctypes declarations of the C ABI in include/mcev.h.

Loads the in-tree `_build/libmcev.so` (building it with nvcc when it is
missing or older than its sources) and fails loudly if that is impossible:
there is no CPU fallback."""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

MCEV_OK = 0
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_OOM", -4: "ERR_TIMEOUT", -5: "ERR_STATE",
          -6: "ERR_NUMERIC"}

ONE_TAILED, TWO_TAILED, MEAN_ONLY, UNIFORM = 0, 1, 2, 3
SE_PAPER, SE_WELCH = 0, 1

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class SceneDesc(C.Structure):
    _fields_ = [
        ("n_vertices", C.c_int64), ("vertices", C.c_void_p),
        ("n_triangles", C.c_int64), ("triangles", C.c_void_p), ("tri_material", C.c_void_p),
        ("n_meshes", C.c_int32), ("mesh_ranges", C.c_void_p),
        ("n_instances", C.c_int32), ("inst_mesh", C.c_void_p), ("inst_material", C.c_void_p),
        ("n_keys", C.c_int32), ("key_times", C.c_void_p), ("inst_xform", C.c_void_p),
        ("cam_eye", C.c_void_p), ("cam_target", C.c_void_p), ("cam_up", C.c_void_p),
        ("fov_deg", C.c_double),
        ("n_materials", C.c_int32), ("mat_type", C.c_void_p), ("mat_albedo", C.c_void_p),
        ("mat_rough", C.c_void_p), ("mat_emit", C.c_void_p),
        ("env_w", C.c_int32), ("env_h", C.c_int32), ("env", C.c_void_p),
        ("uvs", C.c_void_p), ("mat_textured", C.c_void_p),
    ]


class Params(C.Structure):
    _fields_ = [
        ("eps", C.c_float), ("t_min", C.c_float), ("max_depth", C.c_int32), ("nee", C.c_int32),
        ("mis", C.c_int32), ("spp_min", C.c_int32), ("variant", C.c_int32), ("se_mode", C.c_int32),
        ("seed", C.c_uint64), ("wavefront", C.c_int64), ("profile", C.c_int32), ("batch_window", C.c_int32),
        ("bvh_width", C.c_int32), ("host_rounds", C.c_int32), ("device_timeout_us", C.c_int32),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("paths", C.c_int64), ("samples_used", C.c_int64), ("ref_paths", C.c_int64), ("rounds", C.c_int32),
        ("kernel_launches", C.c_int32), ("events_pos", C.c_int64), ("events_neg", C.c_int64),
        ("pixels_at_cap", C.c_int64), ("nonfinite", C.c_int64), ("gpu_ms", C.c_double),
        ("nodes_closest", C.c_int64), ("tris_closest", C.c_int64), ("nodes_shadow", C.c_int64),
        ("tris_shadow", C.c_int64), ("rays_closest", C.c_int64), ("rays_shadow", C.c_int64),
        ("kernel_count", C.c_int32 * 5), ("reserved", C.c_int32), ("kernel_ms", C.c_double * 5),
        ("h2d_bytes", C.c_int64), ("d2h_bytes", C.c_int64), ("stats_pixels", C.c_int64),
        ("boxes_closest", C.c_int64), ("boxes_shadow", C.c_int64),
    ]

    def as_dict(self):
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            d[k] = list(v) if hasattr(v, "__len__") else v
        return d


class JobDesc(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("t0", C.c_double), ("t1", C.c_double), ("events_out", C.c_void_p),
                ("spp_out", C.c_void_p), ("mean_out", C.c_void_p)]


class DetectArgs(C.Structure):
    _fields_ = [
        ("L", C.c_void_p), ("pixels", C.c_void_p), ("n_pix", C.c_int64), ("n_total", C.c_int64),
        ("spp_r", C.c_int32),
        ("reserved0", C.c_int32), ("k_base", C.c_int64),
        ("cur_n", C.c_void_p), ("cur_mean", C.c_void_p), ("cur_m2", C.c_void_p),
        ("ref_n", C.c_void_p), ("ref_mean", C.c_void_p), ("ref_m2", C.c_void_p),
        ("events", C.c_void_p), ("spp_out", C.c_void_p), ("mean_out", C.c_void_p), ("undecided", C.c_void_p),
        ("eps", C.c_float), ("C", C.c_float), ("alpha", C.c_float),
        ("spp_min", C.c_int32), ("spp_batch", C.c_int32), ("spp_max", C.c_int32),
        ("variant", C.c_int32), ("se_mode", C.c_int32),
        ("stream", C.c_void_p), ("err_msg", C.c_char_p), ("err_len", C.c_size_t),
    ]


class Quality(C.Structure):
    _fields_ = [
        ("voxels", C.c_int64), ("n_a", C.c_int64), ("n_b", C.c_int64), ("matched_a", C.c_int64),
        ("matched_b", C.c_int64), ("none_a", C.c_int64), ("none_b", C.c_int64), ("sq_diff", C.c_int64),
        ("sum_dist_a", C.c_double), ("sum_dist_b", C.c_double), ("diag", C.c_double),
        ("rmse", C.c_double), ("psnr", C.c_double), ("precision", C.c_double), ("recall", C.c_double),
        ("f1", C.c_double), ("pscd", C.c_double), ("gpu_ms", C.c_float), ("kernel_launches", C.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# every symbol include/mcev.h declares, with its ctypes signature
SIGNATURES = {
    "mcev_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int32, C.c_int32]),
    "mcev_destroy": (None, [C.c_void_p]),
    "mcev_last_error": (C.c_char_p, [C.c_void_p]),
    "mcev_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mcev_set_allocator": (C.c_int, [C.c_void_p, ALLOC_FN, FREE_FN, C.c_void_p]),
    "mcev_scene_upload": (C.c_int, [C.c_void_p, C.POINTER(SceneDesc)]),
    "mcev_build_bvh": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "mcev_set_params": (C.c_int, [C.c_void_p, C.POINTER(Params)]),
    "mcev_render_reference": (C.c_int, [C.c_void_p, C.c_double, C.c_int32]),
    "mcev_render_events": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_float, C.c_float, C.c_int32,
                                     C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Stats)]),
    "mcev_set_texture": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32]),
    "mcev_set_emission": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "mcev_render_mean": (C.c_int, [C.c_void_p, C.c_double, C.c_int32, C.c_void_p]),
    "mcev_backward": (C.c_int, [C.c_void_p, C.c_double, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mcev_event_quality": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32,
                                     C.c_int32, C.c_void_p, C.c_void_p, C.POINTER(Quality)]),
    "mcev_render_events_batch": (C.c_int, [C.c_void_p, C.POINTER(JobDesc), C.c_int32, C.c_float, C.c_float,
                                           C.c_int32, C.c_int32, C.POINTER(Stats)]),
    "mcev_trace_samples": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_int64, C.c_int64, C.c_int32,
                                     C.c_void_p, C.c_void_p]),
    "mcev_state_bytes": (C.c_size_t, [C.c_void_p]),
    "mcev_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "mcev_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "mcev_detect_batch_static": (C.c_int, [C.POINTER(DetectArgs), C.POINTER(C.c_int64)]),
}

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """The loaded libmcev.so (raises if it cannot be built or loaded)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_needed:
                _build.build()
            if not os.path.exists(_build.LIB):
                raise ImportError(f"CUDA library {_build.LIB} is missing; run __graft_entry__.build()")
            lib = C.CDLL(_build.LIB)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class McevError(RuntimeError):
    pass


def check(status: int, ctx=None, what: str = "") -> None:
    if status != MCEV_OK:
        msg = ""
        if ctx:
            raw = load().mcev_last_error(ctx)
            msg = raw.decode(errors="replace") if raw else ""
        raise McevError(f"{what}: {STATUS.get(status, status)} {msg}".strip())
