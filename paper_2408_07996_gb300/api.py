"""Python face of the C ABI: argument marshalling only.

PyTorch supplies device memory (through its caching allocator, installed as
the library's allocator) and the CUDA stream; every step of the method runs
in the library's kernels."""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, replace

import numpy as np
import torch

from . import _lib as L


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _tptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


@dataclass
class RenderSettings:
    eps: float = 1e-3
    t_min: float = 1e-4
    max_depth: int = 4
    nee: int = 1
    mis: int = 1
    spp_min: int = 16
    variant: int = L.ONE_TAILED
    se_mode: int = L.SE_PAPER
    seed: int = 20240815
    wavefront: int = 0
    profile: int = 0
    batch_window: int = 0
    bvh_width: int = 0
    host_rounds: int = 0
    device_timeout_us: int = 0


class Renderer:
    """One rendering context (scene, BVH, per-pixel reference state) on one GPU.

    Mirrors include/mcev.h: `upload`, `build_bvh`, `set_params`,
    `render_reference`, `render_events`, `trace_samples`, `get_state`,
    `set_state`."""

    def __init__(self, width: int, height: int, device: int = 0, use_torch_allocator: bool = True):
        if not torch.cuda.is_available():
            raise RuntimeError("mcev needs a CUDA device; there is no CPU path")
        self.lib = L.load()
        self.width, self.height = int(width), int(height)
        self.device = torch.device("cuda", device)
        h = C.c_void_p()
        L.check(self.lib.mcev_create(C.byref(h), device, self.width, self.height), None, "mcev_create")
        self.ctx = h
        self._keep = []
        if use_torch_allocator:
            dev = device

            def _alloc(nbytes, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev,
                                                              torch.cuda.current_stream(dev).cuda_stream)
                except Exception:  # reported to the library as NULL -> MCEV_ERR_OOM
                    return None

            def _free(ptr, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc_cb = L.ALLOC_FN(_alloc)
            self._free_cb = L.FREE_FN(_free)
            L.check(self.lib.mcev_set_allocator(self.ctx, self._alloc_cb, self._free_cb, None), self.ctx,
                    "mcev_set_allocator")
        self.set_stream(torch.cuda.current_stream(self.device))
        self.settings = RenderSettings()

    # ------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "ctx", None):
            torch.cuda.synchronize(self.device)
            self.lib.mcev_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------ setup
    def set_stream(self, stream: torch.cuda.Stream):
        self.stream = stream
        L.check(self.lib.mcev_set_stream(self.ctx, C.c_void_p(stream.cuda_stream)), self.ctx, "mcev_set_stream")

    def upload(self, scene) -> None:
        """Copies a `scenegen.Scene`-shaped object (host arrays) to the device."""
        arrs = dict(
            vertices=np.ascontiguousarray(scene.vertices, np.float32),
            triangles=np.ascontiguousarray(scene.triangles, np.int32),
            tri_material=np.ascontiguousarray(scene.tri_material, np.int32),
            mesh_ranges=np.ascontiguousarray(scene.mesh_ranges, np.int32),
            inst_mesh=np.ascontiguousarray(scene.inst_mesh, np.int32),
            inst_material=np.ascontiguousarray(scene.inst_material, np.int32),
            key_times=np.ascontiguousarray(scene.key_times, np.float64),
            inst_xform=np.ascontiguousarray(scene.inst_xform, np.float64),
            cam_eye=np.ascontiguousarray(scene.cam_eye, np.float64),
            cam_target=np.ascontiguousarray(scene.cam_target, np.float64),
            cam_up=np.ascontiguousarray(scene.cam_up, np.float64),
            mat_type=np.ascontiguousarray(scene.mat_type, np.int32),
            mat_albedo=np.ascontiguousarray(scene.mat_albedo, np.float32),
            mat_rough=np.ascontiguousarray(scene.mat_rough, np.float32),
            mat_emit=np.ascontiguousarray(scene.mat_emit, np.float32),
        )
        env = None if scene.env is None else np.ascontiguousarray(scene.env, np.float32)
        uvs = getattr(scene, "uvs", None)
        uvs = None if uvs is None else np.ascontiguousarray(uvs, np.float32)
        mtex = getattr(scene, "mat_textured", None)
        mtex = None if mtex is None else np.ascontiguousarray(mtex, np.int32)
        d = L.SceneDesc(
            n_vertices=arrs["vertices"].shape[0], vertices=_ptr(arrs["vertices"]),
            n_triangles=arrs["triangles"].shape[0], triangles=_ptr(arrs["triangles"]),
            tri_material=_ptr(arrs["tri_material"]),
            n_meshes=arrs["mesh_ranges"].shape[0], mesh_ranges=_ptr(arrs["mesh_ranges"]),
            n_instances=arrs["inst_mesh"].shape[0], inst_mesh=_ptr(arrs["inst_mesh"]),
            inst_material=_ptr(arrs["inst_material"]),
            n_keys=arrs["key_times"].shape[0], key_times=_ptr(arrs["key_times"]),
            inst_xform=_ptr(arrs["inst_xform"]), cam_eye=_ptr(arrs["cam_eye"]),
            cam_target=_ptr(arrs["cam_target"]), cam_up=_ptr(arrs["cam_up"]), fov_deg=float(scene.fov_deg),
            n_materials=arrs["mat_type"].shape[0], mat_type=_ptr(arrs["mat_type"]),
            mat_albedo=_ptr(arrs["mat_albedo"]), mat_rough=_ptr(arrs["mat_rough"]),
            mat_emit=_ptr(arrs["mat_emit"]),
            env_w=0 if env is None else env.shape[1], env_h=0 if env is None else env.shape[0], env=_ptr(env),
            uvs=_ptr(uvs), mat_textured=_ptr(mtex))
        L.check(self.lib.mcev_scene_upload(self.ctx, C.byref(d)), self.ctx, "mcev_scene_upload")
        tex = getattr(scene, "texture", None)
        if tex is not None:
            self.set_texture(torch.from_numpy(np.ascontiguousarray(tex, np.float32)).to(self.device))

    def build_bvh(self, sah_bins: int = 32, max_leaf: int = 4) -> None:
        L.check(self.lib.mcev_build_bvh(self.ctx, sah_bins, max_leaf), self.ctx, "mcev_build_bvh")

    def set_params(self, **kw) -> RenderSettings:
        """Updates the named settings; on an error the previous settings stay."""
        for k in kw:
            if not hasattr(self.settings, k):
                raise KeyError(k)
        s = replace(self.settings, **kw)
        p = L.Params(eps=s.eps, t_min=s.t_min, max_depth=s.max_depth, nee=s.nee, mis=s.mis,
                     spp_min=s.spp_min, variant=s.variant, se_mode=s.se_mode, seed=s.seed,
                     wavefront=s.wavefront, profile=s.profile, batch_window=s.batch_window, bvh_width=s.bvh_width,
                     host_rounds=s.host_rounds, device_timeout_us=s.device_timeout_us)
        L.check(self.lib.mcev_set_params(self.ctx, C.byref(p)), self.ctx, "mcev_set_params")
        self.settings = s
        return s

    def configure(self, w) -> None:
        """Settings of a `scenegen.Workload`."""
        self.set_params(eps=w.eps, t_min=w.t_min, max_depth=w.max_depth, nee=w.nee, mis=w.mis,
                        spp_min=w.spp_min, seed=w.seed)

    # ------------------------------------------------------------ rendering
    def render_reference(self, t0: float, spp: int) -> None:
        L.check(self.lib.mcev_render_reference(self.ctx, float(t0), int(spp)), self.ctx, "mcev_render_reference")

    def render_events(self, t0: float, t1: float, C_: float, alpha: float, spp_batch: int, spp_max: int,
                      out: dict | None = None, stats: bool = True) -> dict:
        """One Alg. 1 frame; returns events (int8 [H,W]), spp (int32), mean (float32)."""
        H, W = self.height, self.width
        if out is None:
            out = dict(events=torch.empty((H, W), dtype=torch.int8, device=self.device),
                       spp=torch.empty((H, W), dtype=torch.int32, device=self.device),
                       mean=torch.empty((H, W), dtype=torch.float32, device=self.device))
        st = L.Stats()
        L.check(self.lib.mcev_render_events(self.ctx, float(t0), float(t1), float(C_), float(alpha), int(spp_batch),
                                            int(spp_max), _tptr(out["events"]), _tptr(out.get("spp")),
                                            _tptr(out.get("mean")), C.byref(st) if stats else None),
                self.ctx, "mcev_render_events")
        if stats:
            out["stats"] = st.as_dict()
        return out

    def trace_samples(self, t: float, pixels: torch.Tensor, k0: int, count: int, want_sig: bool = True):
        """tracePaths: per-sample radiance [n, count] (and decision signatures)."""
        pixels = pixels.to(device=self.device, dtype=torch.int32).contiguous()
        n = pixels.numel()
        Lo = torch.empty((n, count), dtype=torch.float32, device=self.device)
        sig = torch.empty((n, count), dtype=torch.int32, device=self.device) if want_sig else None
        L.check(self.lib.mcev_trace_samples(self.ctx, float(t), _tptr(pixels), n, int(k0), int(count), _tptr(Lo),
                                            _tptr(sig)), self.ctx, "mcev_trace_samples")
        return Lo, sig

    # ------------------------------------------------------------ differentiable rendering
    def set_texture(self, texture: torch.Tensor | None) -> None:
        """RGB albedo texture [H, W, 3] on the device (kept by reference)."""
        if texture is None:
            L.check(self.lib.mcev_set_texture(self.ctx, None, 0, 0), self.ctx, "mcev_set_texture")
            self._texture = None
            return
        if not (texture.is_cuda and texture.dtype == torch.float32 and texture.is_contiguous() and
                texture.dim() == 3 and texture.shape[2] == 3):
            raise ValueError("texture must be a contiguous float32 CUDA tensor [H, W, 3]")
        self._texture = texture
        L.check(self.lib.mcev_set_texture(self.ctx, _tptr(texture), texture.shape[1], texture.shape[0]), self.ctx,
                "mcev_set_texture")

    def set_emission(self, emission: torch.Tensor | None) -> None:
        """Emitted radiance per material on the device (kept by reference);
        it replaces the table's value for the scene's emissive materials."""
        if emission is not None and not (emission.is_cuda and emission.dtype == torch.float32 and
                                         emission.is_contiguous()):
            raise ValueError("emission must be a contiguous float32 CUDA tensor")
        self._emission = emission
        n = 0 if emission is None else emission.numel()
        L.check(self.lib.mcev_set_emission(self.ctx, _tptr(emission), n), self.ctx, "mcev_set_emission")

    def render_mean(self, t: float, spp: int) -> torch.Tensor:
        """Per-pixel mean of ln(L + eps) over samples 0..spp-1 at time t."""
        out = torch.empty((self.height, self.width), dtype=torch.float32, device=self.device)
        L.check(self.lib.mcev_render_mean(self.ctx, float(t), int(spp), _tptr(out)), self.ctx, "mcev_render_mean")
        return out

    def backward(self, t: float, spp: int, grad_mean: torch.Tensor, grad_texture: torch.Tensor | None,
                 grad_emission: torch.Tensor | None) -> None:
        """Path-replay adjoint of render_mean(t, spp): adds d loss / d texel RGB
        to grad_texture and d loss / d emitted radiance to grad_emission, given
        grad_mean = d loss / d mean [H, W]."""
        g = grad_mean.to(device=self.device, dtype=torch.float32).contiguous()
        L.check(self.lib.mcev_backward(self.ctx, float(t), int(spp), _tptr(g), _tptr(grad_texture),
                                       _tptr(grad_emission)), self.ctx, "mcev_backward")

    def state_bytes(self) -> int:
        return int(self.lib.mcev_state_bytes(self.ctx))

    def get_state(self) -> torch.Tensor:
        buf = torch.empty(self.state_bytes(), dtype=torch.uint8, device=self.device)
        L.check(self.lib.mcev_get_state(self.ctx, _tptr(buf), buf.numel()), self.ctx, "mcev_get_state")
        return buf

    def set_state(self, buf: torch.Tensor) -> None:
        buf = buf.to(self.device).contiguous()
        L.check(self.lib.mcev_set_state(self.ctx, _tptr(buf), buf.numel()), self.ctx, "mcev_set_state")

    def reference_arrays(self):
        """Reference state as (n, mean, M2) tensors [H, W] (views of a state copy)."""
        b = self.get_state()
        n = self.width * self.height
        body = b[16:]
        cnt = body[: 4 * n].view(torch.int32).view(self.height, self.width)
        mean = body[4 * n: 8 * n].view(torch.float32).view(self.height, self.width)
        m2 = body[8 * n: 12 * n].view(torch.float32).view(self.height, self.width)
        return cnt, mean, m2


def render_events_batch(runner: Renderer, jobs, C_: float, alpha: float, spp_batch: int, spp_max: int,
                        stats: bool = True):
    """Batched Alg. 1 frames (include/mcev.h, mcev_render_events_batch).

    jobs: list of (renderer, t0, t1); returns one dict of events / spp / mean
    tensors per job, plus the runner's counters under "stats"."""
    outs, descs = [], (L.JobDesc * len(jobs))()
    for i, (r, t0, t1) in enumerate(jobs):
        o = dict(events=torch.empty((r.height, r.width), dtype=torch.int8, device=r.device),
                 spp=torch.empty((r.height, r.width), dtype=torch.int32, device=r.device),
                 mean=torch.empty((r.height, r.width), dtype=torch.float32, device=r.device))
        descs[i] = L.JobDesc(ctx=r.ctx, t0=float(t0), t1=float(t1), events_out=_tptr(o["events"]),
                             spp_out=_tptr(o["spp"]), mean_out=_tptr(o["mean"]))
        outs.append(o)
    st = L.Stats()
    L.check(runner.lib.mcev_render_events_batch(runner.ctx, descs, len(jobs), float(C_), float(alpha),
                                                int(spp_batch), int(spp_max), C.byref(st) if stats else None),
            runner.ctx, "mcev_render_events_batch")
    return outs, (st.as_dict() if stats else None)


def event_quality(a: torch.Tensor, b: torch.Tensor, tau2: int = 3, want_d2: bool = False,
                  runner: "Renderer | None" = None) -> dict:
    """RMSE, PSNR, polarity-aware F1 and chamfer distance of event video
    `a` against `b` (int8 [T, H, W] or [H, W] of {-1, 0, 1} on the device),
    computed by mcev_event_quality.  `runner`: a context to run on (its
    stream and allocator); by default one cached per device.  With
    `want_d2`, also the per-voxel squared distances d2_a, d2_b."""
    if not (a.shape == b.shape and a.dim() in (2, 3) and a.dtype == torch.int8 and b.dtype == torch.int8 and
            a.is_cuda and b.is_cuda):
        raise ValueError("a and b must be int8 CUDA tensors of one shape, [T, H, W] or [H, W]")
    shp = (1,) * (3 - a.dim()) + tuple(a.shape)
    T, H, W = shp
    if runner is None:
        runner = _quality_ctx(a.device)
    a = a.contiguous()
    b = b.contiguous()
    d2a = torch.empty(shp, dtype=torch.int32, device=a.device) if want_d2 else None
    d2b = torch.empty(shp, dtype=torch.int32, device=a.device) if want_d2 else None
    q = L.Quality()
    L.check(runner.lib.mcev_event_quality(runner.ctx, _tptr(a), _tptr(b), W, H, T, int(tau2), _tptr(d2a), _tptr(d2b),
                                          C.byref(q)), runner.ctx, "mcev_event_quality")
    out = q.as_dict()
    if want_d2:
        out["d2_a"], out["d2_b"] = d2a, d2b
    return out


_QCTX: dict = {}


def _quality_ctx(device: torch.device) -> "Renderer":
    idx = device.index if device.index is not None else torch.cuda.current_device()
    r = _QCTX.get(idx)
    if r is None:
        r = _QCTX[idx] = Renderer(1, 1, idx)
    r.set_stream(torch.cuda.current_stream(r.device))
    return r


class EventFrames(torch.autograd.Function):
    """(texture, emission) -> per-pixel mean ln(L + eps) at t0 and t1.

    The backward pass is the library's path-replay adjoint (mcev_backward):
    gradients with respect to the RGB albedo texture of textured Lambertian
    materials and to every material's emitted radiance."""

    @staticmethod
    def forward(ctx, texture, emission, renderer, t0, t1, spp):
        renderer.set_texture(texture)
        renderer.set_emission(emission)
        m0 = renderer.render_mean(t0, spp)
        m1 = renderer.render_mean(t1, spp)
        ctx.save_for_backward(texture, emission)
        ctx.renderer, ctx.frame = renderer, (t0, t1, spp)
        return m0, m1

    @staticmethod
    def backward(ctx, g0, g1):
        texture, emission = ctx.saved_tensors
        r = ctx.renderer
        t0, t1, spp = ctx.frame
        gt = torch.zeros_like(texture)
        ge = torch.zeros_like(emission)
        r.set_texture(texture)
        r.set_emission(emission)
        if g0 is not None:
            r.backward(t0, spp, g0, gt, ge)
        if g1 is not None:
            r.backward(t1, spp, g1, gt, ge)
        return gt, ge, None, None, None, None


def event_loss(m0: torch.Tensor, m1: torch.Tensor, target_events: torch.Tensor, C_: float,
               tau: float = 0.05) -> torch.Tensor:
    """Smooth event loss: where the target has an event of polarity p, a
    softplus push of p * (m1 - m0) above C; elsewhere a softplus push of
    |m1 - m0| below C (temperature tau)."""
    d = m1 - m0
    p = target_events.to(d.dtype)
    on = target_events != 0
    on_term = torch.nn.functional.softplus((C_ - p * d) / tau)
    off_term = torch.nn.functional.softplus((d.abs() - C_) / tau)
    return torch.where(on, on_term, off_term).sum()
