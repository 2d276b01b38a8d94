"""FP64 CPU oracle of the event renderer (arXiv 2408.07996, Alg. 1, Sec. 3).

TEST INFRASTRUCTURE ONLY: tests/, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of bench.py may import this package;
the product path never does.  It shares no code with the CUDA path: the C
sources here are a plain restatement of the paper (plus the scene, sampling
and random-number conventions written down in the design notes), compiled
with gcc into `oracle/_build/liboracle.so`.

Pinned by tests/test_oracle_*.py against published known answers, closed
forms, scipy and brute force.
"""
from __future__ import annotations

import ctypes as C
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import build as _build

ONE_TAILED, TWO_TAILED, MEAN_ONLY, UNIFORM = 0, 1, 2, 3
SE_PAPER, SE_WELCH = 0, 1

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.POINTER
        d, i32, i64, u32 = C.c_double, C.c_int32, C.c_int64, C.c_uint32
        vp = C.c_void_p
        L.orc_philox4x32_10.argtypes = [vp, vp, vp]
        L.orc_u01.argtypes = [u32]
        L.orc_u01.restype = d
        L.orc_betainc.argtypes = [d, d, d]
        L.orc_betainc.restype = d
        L.orc_t_cdf.argtypes = [d, d]
        L.orc_t_cdf.restype = d
        L.orc_t_ppf.argtypes = [d, d]
        L.orc_t_ppf.restype = d
        L.orc_scene_create.argtypes = [i64, vp, i64, vp, vp, i32, vp, i32, vp, vp, i32, vp, vp,
                                       vp, vp, vp, d, i32, vp, vp, vp, vp, i32, i32, vp]
        L.orc_scene_create.restype = vp
        L.orc_scene_free.argtypes = [vp]
        L.orc_scene_set_texture.argtypes = [vp, vp, vp, vp, i32, i32, vp]
        L.orc_scene_set_emission.argtypes = [vp, vp]
        L.orc_closest_hit.argtypes = [vp, d, vp, vp, d, d, C.c_int, P(d), P(i32), P(i32)]
        L.orc_closest_hit.restype = C.c_int
        L.orc_trace_samples.argtypes = [vp, vp, d, vp, i64, i64, i64, vp, vp]
        L.orc_trace_samples.restype = i64
        L.orc_env_sample.argtypes = [vp, d, d, vp, P(d), P(d)]
        L.orc_env_sample.restype = C.c_int
        L.orc_env_pdf.argtypes = [vp, vp]
        L.orc_env_pdf.restype = d
        L.orc_env_radiance.argtypes = [vp, vp]
        L.orc_env_radiance.restype = d
        L.orc_bsdf_eval.argtypes = [C.c_int, d, d, vp, vp, P(d)]
        L.orc_bsdf_eval.restype = d
        L.orc_bsdf_sample.argtypes = [C.c_int, d, vp, d, d, vp]
        L.orc_mean_var.argtypes = [vp, i64, P(d), P(d)]
        L.orc_detect_pixel.argtypes = [vp, vp, P(i64), P(d), P(d), P(C.c_int8), P(i32), P(d),
                                       P(d), P(d), P(d)]
        L.orc_render_events.argtypes = [vp, vp, vp, d, d, vp, i64, C.c_int, vp, vp, vp, vp, vp,
                                        vp, vp, vp, vp]
        L.orc_render_events.restype = i64
        L.orc_reference.argtypes = [vp, vp, i32, d, vp, i64, vp, vp, vp]
        L.orc_reference.restype = i64
        L.orc_camera_ray.argtypes = [vp, vp, d, d, d, vp, vp]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class Params(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("max_depth", C.c_int32),
                ("nee", C.c_int32), ("mis", C.c_int32), ("eps", C.c_double),
                ("t_min", C.c_double), ("seed", C.c_uint64)]


class Detect(C.Structure):
    _fields_ = [("C", C.c_double), ("alpha", C.c_double), ("spp_min", C.c_int32),
                ("spp_batch", C.c_int32), ("spp_max", C.c_int32), ("variant", C.c_int32),
                ("se_mode", C.c_int32)]


# ---------------------------------------------------------------- primitives

def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def u01(x: int) -> float:
    return lib().orc_u01(int(x) & 0xFFFFFFFF)


def betainc(a, b, x) -> float:
    return lib().orc_betainc(a, b, x)


def t_cdf(t, nu) -> float:
    return lib().orc_t_cdf(t, nu)


def t_ppf(p, nu) -> float:
    return lib().orc_t_ppf(p, nu)


def mean_var(y):
    y = np.ascontiguousarray(y, np.float64)
    m, v = C.c_double(), C.c_double()
    lib().orc_mean_var(_p(y), y.size, C.byref(m), C.byref(v))
    return m.value, v.value


def bsdf_eval(mtype, albedo, rough, wo, wi):
    wo = np.ascontiguousarray(wo, np.float64)
    wi = np.ascontiguousarray(wi, np.float64)
    pdf = C.c_double()
    f = lib().orc_bsdf_eval(mtype, albedo, rough, _p(wo), _p(wi), C.byref(pdf))
    return f, pdf.value


def bsdf_sample(mtype, rough, wo, u1, u2):
    wo = np.ascontiguousarray(wo, np.float64)
    wi = np.zeros(3)
    lib().orc_bsdf_sample(mtype, rough, _p(wo), u1, u2, _p(wi))
    return wi


def detect_pixel(det: Detect, y, ref):
    """Alg. 1 for one pixel on given samples; ref = (n, mean, var)."""
    y = np.ascontiguousarray(y, np.float64)
    assert y.size >= det.spp_max
    rn, rm, rv = C.c_int64(ref[0]), C.c_double(ref[1]), C.c_double(ref[2])
    ev, nu = C.c_int8(), C.c_int32()
    m, v, mt, mc = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    lib().orc_detect_pixel(C.byref(det), _p(y), C.byref(rn), C.byref(rm), C.byref(rv),
                           C.byref(ev), C.byref(nu), C.byref(m), C.byref(v), C.byref(mt),
                           C.byref(mc))
    return dict(event=ev.value, n=nu.value, mean=m.value, var=v.value, margin_t=mt.value,
                margin_c=mc.value, ref=(rn.value, rm.value, rv.value))


# ---------------------------------------------------------------- scenes

class OracleScene:
    """FP64 copy of a `scenegen.Scene` with its own per-mesh BVHs."""

    def __init__(self, sc):
        self._keep = [sc.vertices, sc.triangles, sc.tri_material, sc.mesh_ranges, sc.inst_mesh,
                      sc.inst_material, sc.key_times, sc.inst_xform, sc.cam_eye, sc.cam_target,
                      sc.cam_up, sc.mat_type, sc.mat_albedo, sc.mat_rough, sc.mat_emit, sc.env]
        env = sc.env
        self.ptr = lib().orc_scene_create(
            sc.vertices.shape[0], _p(sc.vertices), sc.triangles.shape[0], _p(sc.triangles),
            _p(sc.tri_material), sc.mesh_ranges.shape[0], _p(sc.mesh_ranges),
            sc.inst_mesh.shape[0], _p(sc.inst_mesh), _p(sc.inst_material),
            sc.key_times.shape[0], _p(sc.key_times), _p(sc.inst_xform), _p(sc.cam_eye),
            _p(sc.cam_target), _p(sc.cam_up), float(sc.fov_deg), sc.mat_type.shape[0],
            _p(sc.mat_type), _p(sc.mat_albedo), _p(sc.mat_rough), _p(sc.mat_emit),
            0 if env is None else env.shape[1], 0 if env is None else env.shape[0], _p(env))
        self._sc = sc
        if getattr(sc, "texture", None) is not None and sc.uvs is not None and sc.mat_textured is not None:
            self.set_texture(sc.texture)
        self._keep = None

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.orc_scene_free(self.ptr)
            self.ptr = None

    def closest_hit(self, time, o, d, t_min=0.0, t_max=np.inf, use_bvh=True):
        o = np.ascontiguousarray(o, np.float64)
        d = np.ascontiguousarray(d, np.float64)
        t, i, p = C.c_double(), C.c_int32(), C.c_int32()
        hit = lib().orc_closest_hit(self.ptr, time, _p(o), _p(d), t_min, t_max, int(use_bvh),
                                    C.byref(t), C.byref(i), C.byref(p))
        return bool(hit), t.value, i.value, p.value

    def set_texture(self, texture):
        """Replaces the RGB albedo texture [H, W, 3] (the scene must carry
        texture coordinates and textured-material flags)."""
        sc = self._sc
        tex = np.ascontiguousarray(texture, np.float32)
        uvs = np.ascontiguousarray(sc.uvs, np.float32)
        tris = np.ascontiguousarray(sc.triangles, np.int32)
        mtex = np.ascontiguousarray(sc.mat_textured, np.int32)
        lib().orc_scene_set_texture(self.ptr, _p(uvs), _p(tris), _p(mtex), tex.shape[1], tex.shape[0], _p(tex))

    def set_emission(self, emission):
        """Replaces the emitted radiance of the scene's emissive materials."""
        e = np.ascontiguousarray(emission, np.float32)
        assert e.shape == (len(self._sc.mat_emit),)
        lib().orc_scene_set_emission(self.ptr, _p(e))

    def camera_ray(self, p: "Params", time, fx, fy):
        o, d = np.zeros(3), np.zeros(3)
        lib().orc_camera_ray(self.ptr, C.byref(p), float(time), float(fx), float(fy), _p(o), _p(d))
        return o, d

    def env_sample(self, u1, u2):
        d = np.zeros(3)
        pdf, Le = C.c_double(), C.c_double()
        ok = lib().orc_env_sample(self.ptr, u1, u2, _p(d), C.byref(pdf), C.byref(Le))
        return bool(ok), d, pdf.value, Le.value

    def env_pdf(self, d):
        d = np.ascontiguousarray(d, np.float64)
        return lib().orc_env_pdf(self.ptr, _p(d))

    def env_radiance(self, d):
        d = np.ascontiguousarray(d, np.float64)
        return lib().orc_env_radiance(self.ptr, _p(d))


def params_of(w, **over) -> Params:
    p = Params(width=w.width, height=w.height, max_depth=w.max_depth, nee=w.nee, mis=w.mis,
               eps=w.eps, t_min=w.t_min, seed=w.seed)
    for k, v in over.items():
        setattr(p, k, v)
    return p


def detect_of(w, variant=ONE_TAILED, se_mode=SE_PAPER, **over) -> Detect:
    d = Detect(C=w.C, alpha=w.alpha, spp_min=w.spp_min, spp_batch=w.spp_batch,
               spp_max=w.spp_max, variant=variant, se_mode=se_mode)
    for k, v in over.items():
        setattr(d, k, v)
    return d


def _chunks(n, parts):
    parts = max(1, min(parts, n))
    b = np.linspace(0, n, parts + 1).astype(np.int64)
    return [(int(b[i]), int(b[i + 1])) for i in range(parts) if b[i + 1] > b[i]]


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def trace_samples(osc: OracleScene, p: Params, time, pixels, k0, count, threads=None):
    """Per-sample path radiance L and decision signature, [n_pix, count]."""
    pixels = np.ascontiguousarray(pixels, np.int32)
    n = pixels.size
    L = np.zeros((n, count), np.float64)
    sig = np.zeros((n, count), np.uint32)
    bad = [0]

    def run(a, b):
        bad[0] += lib().orc_trace_samples(osc.ptr, C.byref(p), float(time), _p(pixels[a:b]), b - a,
                                          int(k0), int(count), _p(L[a:b]), _p(sig[a:b]))

    threads = threads or default_threads()
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(lambda ab: run(*ab), _chunks(n, threads * 4)))
    return L, sig


def render_events(osc: OracleScene, p: Params, det: Detect, t0, t1, pixels, ref=None,
                  threads=None):
    """Alg. 1 frame (t0 -> t1) for the listed pixels.  `ref` is None (first
    frame: reference rendered at t0 with spp_max samples) or a dict of
    per-pixel arrays n/mean/var, updated copies of which are returned."""
    pixels = np.ascontiguousarray(pixels, np.int32)
    n = pixels.size
    make_ref = ref is None
    rn = np.zeros(n, np.int64) if make_ref else np.array(ref["n"], np.int64)
    rm = np.zeros(n) if make_ref else np.array(ref["mean"], np.float64)
    rv = np.zeros(n) if make_ref else np.array(ref["var"], np.float64)
    out = dict(events=np.zeros(n, np.int8), n=np.zeros(n, np.int32), mean=np.zeros(n),
               var=np.zeros(n), margin_t=np.zeros(n), margin_c=np.zeros(n))
    def run(a, b):
        lib().orc_render_events(osc.ptr, C.byref(p), C.byref(det), float(t0), float(t1),
                                _p(pixels[a:b]), b - a, int(make_ref), _p(rn[a:b]), _p(rm[a:b]),
                                _p(rv[a:b]), _p(out["events"][a:b]), _p(out["n"][a:b]),
                                _p(out["mean"][a:b]), _p(out["var"][a:b]),
                                _p(out["margin_t"][a:b]), _p(out["margin_c"][a:b]))

    threads = threads or default_threads()
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(lambda ab: run(*ab), _chunks(n, threads * 4)))
    out["ref"] = dict(n=rn, mean=rm, var=rv)
    return out


def reference(osc: OracleScene, p: Params, spp: int, time, pixels, threads=None):
    """First frame of Alg. 1: count, mean and unbiased variance of `spp`
    log-luminance samples per pixel at `time`."""
    pixels = np.ascontiguousarray(pixels, np.int32)
    n = pixels.size
    rn = np.zeros(n, np.int64)
    rm = np.zeros(n)
    rv = np.zeros(n)

    def run(a, b):
        lib().orc_reference(osc.ptr, C.byref(p), int(spp), float(time), _p(pixels[a:b]), b - a,
                            _p(rn[a:b]), _p(rm[a:b]), _p(rv[a:b]))

    threads = threads or default_threads()
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(lambda ab: run(*ab), _chunks(n, threads * 4)))
    return dict(n=rn, mean=rm, var=rv)
