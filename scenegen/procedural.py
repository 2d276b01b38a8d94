"""Procedural scenes shaped like the paper's workloads (Sec. 4: indoor boxes,
object motion, camera fly-throughs), plus the closed-form test scenes.

A scene is plain arrays (see `Scene`).  Conventions every consumer relies on:

* vertices are float32 object-space positions; triangles index them;
* a mesh is a contiguous range of triangles; an instance places one mesh in
  the world with a 3x4 row-major object->world affine matrix per keyframe;
* `inst_material[i] >= 0` overrides the per-triangle material of instance i;
* materials: type 0 = Lambertian, 1 = GGX microfacet reflector; `albedo` is
  the diffuse albedo or the GGX normal-incidence reflectance, `rough` the
  GGX alpha, `emit` a one-sided radiance emitted on the side the triangle's
  winding normal (v1-v0) x (v2-v0) points to;
* the environment map is float32 [H, W] scalar radiance, latitude-longitude,
  row 0 at the +y pole, column 0 at azimuth 0 measured from +x towards +z;
* camera keyframes are (eye, target, up); `fov_deg` spans the shorter image
  axis.  Keyframe times are strictly increasing.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

DIFFUSE = 0
GGX = 1


@dataclass
class Scene:
    vertices: np.ndarray          # float32 [Nv, 3]
    triangles: np.ndarray         # int32   [Nt, 3]
    tri_material: np.ndarray      # int32   [Nt]
    mesh_ranges: np.ndarray       # int32   [Nm, 2]  (first triangle, count)
    inst_mesh: np.ndarray         # int32   [Ni]
    inst_material: np.ndarray     # int32   [Ni]
    key_times: np.ndarray         # float64 [K]
    inst_xform: np.ndarray        # float64 [K, Ni, 12]
    cam_eye: np.ndarray           # float64 [K, 3]
    cam_target: np.ndarray        # float64 [K, 3]
    cam_up: np.ndarray            # float64 [K, 3]
    fov_deg: float
    mat_type: np.ndarray          # int32   [Nm]
    mat_albedo: np.ndarray        # float32 [Nm]
    mat_rough: np.ndarray         # float32 [Nm]
    mat_emit: np.ndarray          # float32 [Nm]
    env: np.ndarray | None = None  # float32 [H, W]
    uvs: np.ndarray | None = None          # float32 [Nv, 2] texture coordinates, optional
    mat_textured: np.ndarray | None = None  # int32 [Nm]: 1 = Lambertian albedo from the texture
    texture: np.ndarray | None = None      # float32 [Ht, Wt, 3] RGB albedo texture, optional

    def __post_init__(self):
        self.vertices = np.ascontiguousarray(self.vertices, np.float32).reshape(-1, 3)
        self.triangles = np.ascontiguousarray(self.triangles, np.int32).reshape(-1, 3)
        self.tri_material = np.ascontiguousarray(self.tri_material, np.int32).reshape(-1)
        self.mesh_ranges = np.ascontiguousarray(self.mesh_ranges, np.int32).reshape(-1, 2)
        self.inst_mesh = np.ascontiguousarray(self.inst_mesh, np.int32).reshape(-1)
        self.inst_material = np.ascontiguousarray(self.inst_material, np.int32).reshape(-1)
        self.key_times = np.ascontiguousarray(self.key_times, np.float64).reshape(-1)
        k, ni = len(self.key_times), len(self.inst_mesh)
        self.inst_xform = np.ascontiguousarray(self.inst_xform, np.float64).reshape(k, ni, 12)
        for name in ("cam_eye", "cam_target", "cam_up"):
            setattr(self, name, np.ascontiguousarray(getattr(self, name), np.float64).reshape(k, 3))
        self.mat_type = np.ascontiguousarray(self.mat_type, np.int32).reshape(-1)
        for name in ("mat_albedo", "mat_rough", "mat_emit"):
            setattr(self, name, np.ascontiguousarray(getattr(self, name), np.float32).reshape(-1))
        if self.env is not None:
            self.env = np.ascontiguousarray(self.env, np.float32)
            assert self.env.ndim == 2
        if self.uvs is not None:
            self.uvs = np.ascontiguousarray(self.uvs, np.float32).reshape(-1, 2)
        if self.mat_textured is not None:
            self.mat_textured = np.ascontiguousarray(self.mat_textured, np.int32).reshape(-1)
        if self.texture is not None:
            self.texture = np.ascontiguousarray(self.texture, np.float32)
            assert self.texture.ndim == 3 and self.texture.shape[2] == 3

    @property
    def n_triangles(self) -> int:
        return int(self.triangles.shape[0])


@dataclass
class Workload:
    """A scene plus the render settings of one benchmark or test case."""
    name: str
    scene: Scene
    width: int
    height: int
    times: list            # frame times; frame pairs are (times[k], times[k+1])
    spp_min: int
    spp_batch: int
    spp_max: int
    C: float
    alpha: float
    max_depth: int
    eps: float = 1e-3
    seed: int = 20240815
    t_min: float = 1e-4
    nee: int = 1
    mis: int = 1
    extra: dict = field(default_factory=dict)


# --------------------------------------------------------------------------
# small helpers (geometry generation only)
# --------------------------------------------------------------------------

IDENTITY = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float64)


def _affine(scale=1.0, rot_y=0.0, translate=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Row-major 3x4 matrix T(translate) * R_y(rot_y) * S(scale)."""
    c, s = math.cos(rot_y), math.sin(rot_y)
    sx = sy = sz = scale
    m = np.array([
        [c * sx, 0.0, s * sz, translate[0]],
        [0.0, sy, 0.0, translate[1]],
        [-s * sx, 0.0, c * sz, translate[2]],
    ], np.float64)
    return m.reshape(12)


def _quad(p0, p1, p2, p3):
    """Two triangles (p0,p1,p2), (p0,p2,p3); winding normal (p1-p0)x(p2-p0)."""
    v = np.array([p0, p1, p2, p3], np.float32)
    t = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    return v, t


class _MeshBuilder:
    def __init__(self):
        self.v, self.t, self.m = [], [], []
        self.nv = 0

    def add(self, verts, tris, material):
        verts = np.asarray(verts, np.float32)
        tris = np.asarray(tris, np.int32) + self.nv
        self.v.append(verts)
        self.t.append(tris)
        mat = np.broadcast_to(np.asarray(material, np.int32), (tris.shape[0],))
        self.m.append(np.array(mat, np.int32))
        self.nv += verts.shape[0]

    def arrays(self):
        if not self.t:
            return (np.zeros((0, 3), np.float32), np.zeros((0, 3), np.int32),
                    np.zeros((0,), np.int32))
        return np.concatenate(self.v), np.concatenate(self.t), np.concatenate(self.m)


def _box_faces(lo, hi, rot_y=0.0, pivot=None, bottom=False):
    """Axis-aligned box [lo, hi] rotated about the vertical axis through
    `pivot`; returns a list of quads (4 corners each)."""
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    quads = [
        [(x0, y1, z0), (x0, y1, z1), (x1, y1, z1), (x1, y1, z0)],  # top
        [(x0, y0, z1), (x1, y0, z1), (x1, y1, z1), (x0, y1, z1)],  # +z
        [(x1, y0, z0), (x0, y0, z0), (x0, y1, z0), (x1, y1, z0)],  # -z
        [(x1, y0, z1), (x1, y0, z0), (x1, y1, z0), (x1, y1, z1)],  # +x
        [(x0, y0, z0), (x0, y0, z1), (x0, y1, z1), (x0, y1, z0)],  # -x
    ]
    if bottom:
        quads.append([(x0, y0, z0), (x1, y0, z0), (x1, y0, z1), (x0, y0, z1)])
    if pivot is None:
        pivot = 0.5 * (lo + hi)
    c, s = math.cos(rot_y), math.sin(rot_y)
    out = []
    for q in quads:
        rq = []
        for p in q:
            dx, dz = p[0] - pivot[0], p[2] - pivot[2]
            rq.append((pivot[0] + c * dx + s * dz, p[1], pivot[2] - s * dx + c * dz))
        out.append(rq)
    return out


def _icosphere(level: int):
    """Unit icosphere by repeated 4-way subdivision; outward winding."""
    p = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [(-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0),
             (0, -1, p), (0, 1, p), (0, -1, -p), (0, 1, -p),
             (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1)]
    verts = [np.array(v, np.float64) / np.linalg.norm(v) for v in verts]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return np.array(verts, np.float64), np.array(faces, np.int32)


def _static_keys(times, n_inst, xforms, eye, target, up):
    k = len(times)
    xf = np.broadcast_to(np.asarray(xforms, np.float64).reshape(1, n_inst, 12), (k, n_inst, 12)).copy()
    e = np.broadcast_to(np.asarray(eye, np.float64), (k, 3)).copy()
    t = np.broadcast_to(np.asarray(target, np.float64), (k, 3)).copy()
    u = np.broadcast_to(np.asarray(up, np.float64), (k, 3)).copy()
    return xf, e, t, u


# --------------------------------------------------------------------------
# environment texture
# --------------------------------------------------------------------------

def sky_texture(width=512, height=256, sun_elev_deg=35.0, sun_azim_deg=120.0,
                sun_radius_deg=1.5, sun_radiance=1.0e3, lo=1.0e-2, hi=1.0e3):
    """Procedural HDR sky baked at texel centres: zenith-to-horizon gradient,
    sun disk with a glow, dim ground below the horizon; clamped to [lo, hi]."""
    i = (np.arange(height) + 0.5) / height * math.pi           # polar angle from +y
    j = (np.arange(width) + 0.5) / width * 2.0 * math.pi       # azimuth from +x to +z
    th, ph = np.meshgrid(i, j, indexing="ij")
    d = np.stack([np.sin(th) * np.cos(ph), np.cos(th), np.sin(th) * np.sin(ph)], -1)
    el, az = math.radians(sun_elev_deg), math.radians(sun_azim_deg)
    sun = np.array([math.cos(el) * math.cos(az), math.sin(el), math.cos(el) * math.sin(az)])
    cosang = np.clip(d @ sun, -1.0, 1.0)
    ang = np.arccos(cosang)
    up = d[..., 1]
    sky = np.where(up > 0.0, 0.8 + 2.2 * (1.0 - up) ** 3, 0.05 + 0.0 * up)
    glow = 60.0 * np.exp(-ang / 0.08) * (up > -0.05)
    disk = np.where(ang < math.radians(sun_radius_deg), sun_radiance, 0.0)
    env = np.clip(sky + glow + disk, lo, hi)
    return env.astype(np.float32)


# --------------------------------------------------------------------------
# configuration 1: Cornell-like box, 32 triangles
# --------------------------------------------------------------------------

def cornell_box(seed: int = 20240815, shift: float = 0.02) -> Scene:
    """Unit room [0,1]^3: floor, ceiling, back, left and right walls (10 tris),
    a short and a tall box without bottoms (20 tris) and a one-sided ceiling
    light quad of radiance 10 (2 tris) = 32 triangles.  The front (z=1) is
    open; the camera looks in through it and shifts by `shift` along +x
    between the two keyframes t=0 and t=1."""
    rng = np.random.default_rng(seed)
    mb = _MeshBuilder()
    albedo = []

    def new_mat():
        albedo.append(float(rng.uniform(0.3, 0.8)))
        return len(albedo) - 1

    walls = [
        [(0, 0, 0), (1, 0, 0), (1, 0, 1), (0, 0, 1)],    # floor
        [(0, 1, 0), (0, 1, 1), (1, 1, 1), (1, 1, 0)],    # ceiling
        [(0, 0, 0), (0, 1, 0), (1, 1, 0), (1, 0, 0)],    # back
        [(0, 0, 0), (0, 0, 1), (0, 1, 1), (0, 1, 0)],    # left
        [(1, 0, 0), (1, 1, 0), (1, 1, 1), (1, 0, 1)],    # right
    ]
    for q in walls:
        v, t = _quad(*q)
        mb.add(v, t, new_mat())
    for lo, hi, rot in [((0.13, 0.0, 0.47), (0.43, 0.30, 0.77), -0.30),
                        ((0.55, 0.0, 0.15), (0.85, 0.60, 0.45), 0.28)]:
        for q in _box_faces(lo, hi, rot_y=rot):
            v, t = _quad(*q)
            mb.add(v, t, new_mat())
    n_diffuse = len(albedo)
    # light quad just below the ceiling, winding normal pointing down (-y)
    y = 0.999
    v, t = _quad((0.35, y, 0.35), (0.65, y, 0.35), (0.65, y, 0.65), (0.35, y, 0.65))
    mb.add(v, t, n_diffuse)
    verts, tris, tmat = mb.arrays()
    assert tris.shape[0] == 32
    nm = n_diffuse + 1
    mat_type = np.zeros(nm, np.int32)
    mat_albedo = np.array(albedo + [0.0], np.float32)
    mat_rough = np.zeros(nm, np.float32)
    mat_emit = np.zeros(nm, np.float32)
    mat_emit[-1] = 10.0
    times = np.array([0.0, 1.0])
    xf, _, _, up = _static_keys(times, 1, IDENTITY, (0, 0, 0), (0, 0, 0), (0, 1, 0))
    eye = np.array([[0.5, 0.5, 2.3], [0.5 + shift, 0.5, 2.3]])
    target = np.array([[0.5, 0.5, 0.0], [0.5 + shift, 0.5, 0.0]])
    return Scene(verts, tris, tmat, [[0, tris.shape[0]]], [0], [-1], times, xf,
                 eye, target, up, 40.0, mat_type, mat_albedo, mat_rough, mat_emit, None)


# --------------------------------------------------------------------------
# configuration 2: 64 displaced icospheres on a ground plane, one spinning
# --------------------------------------------------------------------------

def icosphere_field(seed: int = 20240816, n_spheres: int = 64, level: int = 4,
                    n_frames: int = 33, dt: float = 1.0e-3, spin_hz: float = 1.0,
                    env_w: int = 512, env_h: int = 256, n_spin: int = 1) -> Scene:
    """64 icospheres (subdivision `level`, 20*4^level triangles each) with a
    radial vertex displacement ~U(0, 0.05), seed-placed on a 2-triangle
    ground plane.  All surfaces Lambertian with albedo ~U(0.2, 0.9).  Spheres
    s < n_spin spin about their vertical axes, sphere s at spin_hz * (1 + s/4)
    turns per second (default: sphere 0 alone); keyframes at k*dt for
    k < n_frames.  Lit by the procedural sky."""
    rng = np.random.default_rng(seed)
    base_v, base_f = _icosphere(level)
    mb = _MeshBuilder()
    ranges = []
    positions = []
    radii = []
    tries = 0
    while len(positions) < n_spheres:
        tries += 1
        r = float(rng.uniform(0.35, 0.7))
        p = rng.uniform(-6.0, 6.0, size=2)
        if all(np.hypot(*(p - q)) > r + rq + 0.05 for q, rq in zip(positions, radii)) or tries > 20000:
            positions.append(p)
            radii.append(r)
    albedo = []
    for s in range(n_spheres):
        disp = rng.uniform(0.0, 0.05, size=base_v.shape[0])
        v = base_v * (radii[s] + disp)[:, None]
        first = sum(c for _, c in ranges)
        mb.add(v.astype(np.float32), base_f, s)
        ranges.append((first, base_f.shape[0]))
        albedo.append(float(rng.uniform(0.2, 0.9)))
    first = sum(c for _, c in ranges)
    g = 40.0
    v, t = _quad((-g, 0, -g), (-g, 0, g), (g, 0, g), (g, 0, -g))
    mb.add(v, t, n_spheres)
    ranges.append((first, 2))
    albedo.append(float(rng.uniform(0.2, 0.9)))
    verts, tris, tmat = mb.arrays()
    ni = n_spheres + 1
    times = np.arange(n_frames, dtype=np.float64) * dt
    xf = np.zeros((n_frames, ni, 12))
    for k, tk in enumerate(times):
        for s in range(n_spheres):
            rot = 2.0 * math.pi * spin_hz * (1.0 + s / 4.0) * tk if s < n_spin else 0.0
            xf[k, s] = _affine(1.0, rot, (positions[s][0], radii[s], positions[s][1]))
        xf[k, n_spheres] = IDENTITY
    eye = np.broadcast_to([0.0, 7.5, 11.0], (n_frames, 3))
    target = np.broadcast_to([0.0, 0.0, 0.5], (n_frames, 3))
    up = np.broadcast_to([0.0, 1.0, 0.0], (n_frames, 3))
    nm = n_spheres + 1
    return Scene(verts, tris, tmat, ranges, np.arange(ni), -np.ones(ni), times, xf,
                 eye, target, up, 55.0, np.zeros(nm), albedo, np.zeros(nm), np.zeros(nm),
                 sky_texture(env_w, env_h))


# --------------------------------------------------------------------------
# configuration 3: 1024^2 heightfield terrain + 200 instanced boxes, HDR sky
# --------------------------------------------------------------------------

def _fractal_height(n: int, rng, beta: float = 2.2, amplitude: float = 6.0) -> np.ndarray:
    kx = np.fft.fftfreq(n)[:, None]
    kz = np.fft.rfftfreq(n)[None, :]
    k = np.sqrt(kx * kx + kz * kz)
    k[0, 0] = 1.0
    spec = (rng.normal(size=k.shape) + 1j * rng.normal(size=k.shape)) * k ** (-beta)
    spec[0, 0] = 0.0
    h = np.fft.irfft2(spec, s=(n, n))
    h = h / np.max(np.abs(h)) * amplitude
    return h


def terrain_with_boxes(seed: int = 20240817, grid: int = 1024, extent: float = 100.0,
                       n_boxes: int = 200, n_frames: int = 100, dt: float = 0.01,
                       patches: int = 16, env_w: int = 512, env_h: int = 256) -> Scene:
    """Heightfield terrain of `grid`^2 vertices ((grid-1)^2*2 triangles) over
    [-extent/2, extent/2]^2 plus `n_boxes` instances of one closed 12-triangle
    box.  Materials: a 50/50 mix of Lambertian (albedo U(0.2,0.8)) and GGX
    (reflectance U(0.2,0.8), alpha U(0.1,0.6)), per terrain patch and per box.
    The camera moves on a straight line across a quarter of the terrain's
    extent over `n_frames` keyframes spaced `dt` apart.  HDR sky 512x256."""
    rng = np.random.default_rng(seed)
    h = _fractal_height(grid, rng)
    xs = np.linspace(-extent / 2, extent / 2, grid)
    X, Z = np.meshgrid(xs, xs, indexing="ij")
    verts = np.stack([X, h, Z], -1).reshape(-1, 3).astype(np.float32)
    i, j = np.meshgrid(np.arange(grid - 1), np.arange(grid - 1), indexing="ij")
    v00 = (i * grid + j).reshape(-1)
    v01 = v00 + 1
    v10 = v00 + grid
    v11 = v10 + 1
    tris = np.empty((2 * v00.size, 3), np.int32)
    tris[0::2] = np.stack([v00, v01, v11], -1)
    tris[1::2] = np.stack([v00, v11, v10], -1)
    # materials: patches x patches terrain patches, then one per box
    n_mat = patches * patches + n_boxes
    mtype = (rng.uniform(size=n_mat) < 0.5).astype(np.int32)
    malb = rng.uniform(0.2, 0.8, size=n_mat)
    mrough = np.where(mtype == GGX, rng.uniform(0.1, 0.6, size=n_mat), 0.0)
    pi = (i * patches // (grid - 1)).reshape(-1)
    pj = (j * patches // (grid - 1)).reshape(-1)
    cell_mat = (pi * patches + pj).astype(np.int32)
    tmat = np.repeat(cell_mat, 2)
    # closed box mesh [-0.5,0.5] x [0,1] x [-0.5,0.5]
    bv, bt = [], []
    for q in _box_faces((-0.5, 0.0, -0.5), (0.5, 1.0, 0.5), bottom=True):
        v, t = _quad(*q)
        bt.append(t + 4 * len(bv))
        bv.append(v)
    bv = np.concatenate(bv).astype(np.float32)
    bt = np.concatenate(bt).astype(np.int32) + verts.shape[0]
    all_v = np.concatenate([verts, bv])
    all_t = np.concatenate([tris, bt])
    all_m = np.concatenate([tmat, np.zeros(12, np.int32)])
    ranges = [(0, tris.shape[0]), (tris.shape[0], 12)]
    ni = 1 + n_boxes
    inst_mesh = np.array([0] + [1] * n_boxes, np.int32)
    inst_mat = np.array([-1] + [patches * patches + b for b in range(n_boxes)], np.int32)
    xf0 = np.zeros((ni, 12))
    xf0[0] = IDENTITY
    for b in range(n_boxes):
        gx, gz = rng.integers(0, grid, size=2)
        s = float(rng.uniform(0.6, 2.5))
        xf0[1 + b] = _affine(s, float(rng.uniform(0, 2 * math.pi)),
                             (xs[gx], h[gx, gz] - 0.15 * s, xs[gz]))
    times = np.arange(n_frames, dtype=np.float64) * dt
    xf = np.broadcast_to(xf0, (n_frames, ni, 12)).copy()
    travel = 0.25 * extent
    frac = np.arange(n_frames) / max(n_frames - 1, 1)
    eye = np.stack([-travel / 2 + travel * frac, np.full(n_frames, 32.0),
                    np.full(n_frames, 38.0)], -1)
    target = eye + np.array([0.0, -22.0, -42.0])
    up = np.broadcast_to([0.0, 1.0, 0.0], (n_frames, 3))
    return Scene(all_v, all_t, all_m, ranges, inst_mesh, inst_mat, times, xf,
                 eye, target, up, 50.0, mtype, malb, mrough, np.zeros(n_mat),
                 sky_texture(env_w, env_h))


# --------------------------------------------------------------------------
# closed-form test scenes
# --------------------------------------------------------------------------

def furnace_sphere(albedo: float = 0.5, emit: float = 1.0, level: int = 2,
                   radius: float = 1.0) -> Scene:
    """Closed icosphere, winding flipped so every triangle emits inwards; the
    camera sits at the centre.  With BSDF sampling only, every path's
    radiance is emit * sum_{k=0..D} albedo^k."""
    v, f = _icosphere(level)
    f = f[:, [0, 2, 1]]
    times = np.array([0.0, 1.0])
    xf, eye, target, up = _static_keys(times, 1, IDENTITY, (0, 0, 0), (0, 0, -1), (0, 1, 0))
    return Scene((v * radius).astype(np.float32), f, np.zeros(f.shape[0]), [[0, f.shape[0]]],
                 [0], [-1], times, xf, eye, target, up, 60.0,
                 [DIFFUSE], [albedo], [0.0], [emit], None)


def plane_under_env(albedo: float = 0.5, env_value: float = 2.0, half: float = 50.0,
                    height: float = 1.0) -> Scene:
    """Lambertian plane y=0 under a constant environment, camera looking
    straight down from `height`.  With BSDF sampling only, each path's
    radiance is albedo * env_value exactly."""
    v, t = _quad((-half, 0, -half), (-half, 0, half), (half, 0, half), (half, 0, -half))
    times = np.array([0.0, 1.0])
    xf, eye, target, up = _static_keys(times, 1, IDENTITY, (0, height, 0), (0, 0, 0), (0, 0, -1))
    env = np.full((8, 16), env_value, np.float32)
    return Scene(v, t, [0, 0], [[0, 2]], [0], [-1], times, xf, eye, target, up, 40.0,
                 [DIFFUSE], [albedo], [0.0], [0.0], env)


def textured_plane(texture: np.ndarray, repeat: float = 3.0, env_value: float = 2.0, half: float = 0.5,
                   height: float = 1.0) -> Scene:
    """plane_under_env with texture coordinates (u, v) = repeat * ((x, z) +
    half) / (2 half) and a textured Lambertian material: with BSDF sampling
    only, each path's radiance is env_value times the Rec. 709 luminance of
    the nearest texel at the wrapped coordinates of its first hit."""
    sc = plane_under_env(0.5, env_value, half, height)
    uv = repeat * (sc.vertices[:, [0, 2]].astype(np.float64) + half) / (2.0 * half)
    return replace(sc, uvs=uv.astype(np.float32), mat_textured=np.array([1], np.int32),
                   texture=np.ascontiguousarray(texture, np.float32))


def empty_env(env_value: float = 3.0) -> Scene:
    """No geometry at all, constant environment: every path's radiance is
    env_value (the degenerate zero-triangle scene)."""
    times = np.array([0.0, 1.0])
    xf, eye, target, up = _static_keys(times, 0, np.zeros((0, 12)), (0, 0, 0), (0, 0, -1), (0, 1, 0))
    return Scene(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0), np.zeros((0, 2)),
                 np.zeros(0), np.zeros(0), times, xf.reshape(2, 0, 12), eye, target, up, 45.0,
                 [DIFFUSE], [0.5], [0.0], [0.0], np.full((4, 8), env_value, np.float32))


def static_variant(scene: Scene) -> Scene:
    """Same scene with every keyframe equal to the first: nothing moves."""
    k = len(scene.key_times)
    return replace(
        scene,
        inst_xform=np.broadcast_to(scene.inst_xform[:1], scene.inst_xform.shape).copy(),
        cam_eye=np.broadcast_to(scene.cam_eye[:1], (k, 3)).copy(),
        cam_target=np.broadcast_to(scene.cam_target[:1], (k, 3)).copy(),
        cam_up=np.broadcast_to(scene.cam_up[:1], (k, 3)).copy(),
    )


# --------------------------------------------------------------------------
# named workloads (paper-shaped synthetic stand-ins for its scenes)
# --------------------------------------------------------------------------

def _bbox_diag(scene: Scene) -> float:
    if scene.n_triangles == 0:
        return 1.0
    lo = np.full(3, np.inf)
    hi = np.full(3, -np.inf)
    for i, m in enumerate(scene.inst_mesh):
        first, cnt = scene.mesh_ranges[m]
        idx = np.unique(scene.triangles[first:first + cnt].reshape(-1))
        p = scene.vertices[idx].astype(np.float64)
        M = scene.inst_xform[0, i].reshape(3, 4)
        w = p @ M[:, :3].T + M[:, 3]
        lo = np.minimum(lo, w.min(0))
        hi = np.maximum(hi, w.max(0))
    return float(np.linalg.norm(hi - lo))


def workload(name: str, **over) -> Workload:
    """Named workloads.  `cornell64` (64x64, 32 tris), `spheres512` (512x512,
    64 displaced icospheres), `terrain720p` (1280x720, ~2.1M tris)."""
    if name == "cornell64":
        sc = cornell_box(20240815)
        w = Workload(name, sc, 64, 64, [0.0, 1.0], spp_min=16, spp_batch=16, spp_max=256,
                     C=0.2, alpha=0.05, max_depth=4, seed=20240815)
    elif name == "spheres512":
        sc = icosphere_field(20240816)
        w = Workload(name, sc, 512, 512, list(sc.key_times), spp_min=256, spp_batch=32,
                     spp_max=4096, C=0.25, alpha=0.01, max_depth=4, seed=20240816)
    elif name == "diff256":
        sc = textured_room(20240819)
        w = Workload(name, sc, 256, 256, [0.0, 1.0], spp_min=64, spp_batch=64, spp_max=64,
                     C=0.2, alpha=0.05, max_depth=3, seed=20240819)
    elif name == "terrain720p":
        sc = terrain_with_boxes(20240817)
        w = Workload(name, sc, 1280, 720, list(sc.key_times), spp_min=512, spp_batch=64,
                     spp_max=8192, C=0.2, alpha=0.05, max_depth=6, seed=20240817)
    else:
        raise KeyError(name)
    w.t_min = 1e-4 * _bbox_diag(w.scene)
    for k, v in over.items():
        setattr(w, k, v)
    return w


def albedo_texture(size: int = 512, seed: int = 0, lo: float = 0.2, hi: float = 0.8) -> np.ndarray:
    """RGB albedo texture [size, size, 3]: smooth random blobs in [lo, hi]."""
    rng = np.random.default_rng(seed)
    k = np.fft.fftfreq(size)[:, None] ** 2 + np.fft.fftfreq(size)[None, :] ** 2
    out = np.empty((size, size, 3))
    for c in range(3):
        spec = (rng.normal(size=(size, size)) + 1j * rng.normal(size=(size, size))) * np.exp(-k * 400.0)
        f = np.real(np.fft.ifft2(spec))
        f = (f - f.min()) / (f.max() - f.min() + 1e-12)
        out[..., c] = lo + (hi - lo) * f
    return out.astype(np.float32)


def textured_room(seed: int = 20240819, grid: int = 158, tex_size: int = 512, shift: float = 0.05,
                  texture: np.ndarray | None = None) -> Scene:
    """Differentiation scene (256x256 frames, 64 spp): a (grid-1)^2*2-triangle floor (about
    50k triangles at grid 158) carrying an RGB albedo texture, a few
    untextured boxes, and 4 one-sided emissive quads (one material each)
    above it.  Camera looks down at the floor and shifts by `shift` along x
    between t = 0 and t = 1."""
    rng = np.random.default_rng(seed)
    mb = _MeshBuilder()
    xs = np.linspace(-2.0, 2.0, grid)
    X, Z = np.meshgrid(xs, xs, indexing="ij")
    verts = np.stack([X, np.zeros_like(X), Z], -1).reshape(-1, 3)
    i, j = np.meshgrid(np.arange(grid - 1), np.arange(grid - 1), indexing="ij")
    v00 = (i * grid + j).reshape(-1)
    tris = np.concatenate([np.stack([v00, v00 + 1, v00 + grid + 1], -1),
                           np.stack([v00, v00 + grid + 1, v00 + grid], -1)])
    uv_floor = np.stack([(X + 2.0) / 4.0, (Z + 2.0) / 4.0], -1).reshape(-1, 2)
    mb.add(verts, tris, 0)
    uvs = [uv_floor]
    n_box = 3
    for b in range(n_box):
        c = rng.uniform(-1.2, 1.2, size=2)
        h = float(rng.uniform(0.2, 0.6))
        for q in _box_faces((c[0] - 0.25, 0.0, c[1] - 0.25), (c[0] + 0.25, h, c[1] + 0.25), rot_y=float(rng.uniform(0, 3))):
            v, t = _quad(*q)
            mb.add(v, t, 1 + b)
            uvs.append(np.zeros((4, 2)))
    n_lights = 4
    for l in range(n_lights):
        cx, cz = [(-1.0, -1.0), (1.0, -1.0), (-1.0, 1.0), (1.0, 1.0)][l]
        y = 2.0
        v, t = _quad((cx - 0.3, y, cz - 0.3), (cx + 0.3, y, cz - 0.3), (cx + 0.3, y, cz + 0.3), (cx - 0.3, y, cz + 0.3))
        mb.add(v, t, 1 + n_box + l)
        uvs.append(np.zeros((4, 2)))
    verts, tris, tmat = mb.arrays()
    nm = 1 + n_box + n_lights
    mat_type = np.zeros(nm, np.int32)
    mat_albedo = np.array([0.5] + [float(rng.uniform(0.3, 0.8)) for _ in range(n_box)] + [0.0] * n_lights)
    mat_emit = np.array([0.0] * (1 + n_box) + [float(rng.uniform(4.0, 8.0)) for _ in range(n_lights)])
    textured = np.zeros(nm, np.int32)
    textured[0] = 1
    times = np.array([0.0, 1.0])
    xf, _, _, up = _static_keys(times, 1, IDENTITY, (0, 0, 0), (0, 0, 0), (0, 0, -1))
    eye = np.array([[0.0, 3.2, 0.0], [shift, 3.2, 0.0]])
    target = np.array([[0.0, 0.0, 0.0], [shift, 0.0, 0.0]])
    up = np.array([[0.0, 0.0, -1.0], [0.0, 0.0, -1.0]])
    tex = albedo_texture(tex_size, seed) if texture is None else texture
    return Scene(verts, tris, tmat, [[0, tris.shape[0]]], [0], [-1], times, xf, eye, target, up, 70.0,
                 mat_type, mat_albedo, np.zeros(nm), mat_emit, None,
                 uvs=np.concatenate(uvs).astype(np.float32), mat_textured=textured, texture=tex)


WORKLOADS = ("cornell64", "spheres512", "terrain720p")

BATCH_RESOLUTIONS = ((128, 128), (320, 240), (346, 260), (640, 480))


def batch_workloads(n_jobs: int = 64, seed: int = 20240818) -> list:
    """Independent frame-pair jobs for batched rendering: image
    sizes drawn uniformly from BATCH_RESOLUTIONS, scenes of 5k-100k
    triangles (displaced icosphere fields of 1-19 level-4 spheres, or 4-78
    level-3 spheres, each with one spinning sphere and a moving camera),
    schedule spp 16 -> +16 -> 4096, C = 0.2, alpha = 0.05."""
    rng = np.random.default_rng(seed)
    jobs = []
    for j in range(n_jobs):
        W, H = BATCH_RESOLUTIONS[int(rng.integers(len(BATCH_RESOLUTIONS)))]
        target = int(rng.uniform(5_000, 100_000))
        level = int(rng.integers(3, 5))
        per = 20 * 4 ** level
        n_sph = int(max(1, min(target // per, 19 if level == 4 else 78)))
        sc = icosphere_field(seed + 1000 + j, n_spheres=n_sph, level=level, n_frames=9, dt=2.0e-3,
                             env_w=128, env_h=64)
        k = len(sc.key_times)
        shift = np.linspace(0.0, 0.08, k)[:, None] * np.array([1.0, 0.0, 0.0])
        sc.cam_eye = sc.cam_eye + shift
        sc.cam_target = sc.cam_target + shift
        w = Workload(f"batch{j}", sc, W, H, list(sc.key_times), spp_min=16, spp_batch=16, spp_max=4096,
                     C=0.2, alpha=0.05, max_depth=4, seed=seed + j)
        w.t_min = 1e-4 * _bbox_diag(sc)
        jobs.append(w)
    return jobs


def event_video_pair(width: int, height: int, frames: int, seed: int = 20240820, move: float = 0.05,
                     drop: float = 0.03, flip: float = 0.01, noise: float = 2e-4):
    """Two int8 event videos [frames, height, width] of {-1, 0, +1} for the
    quality metrics: `a` holds the events of a drifting sinusoidal grating
    seen by an ideal log sensor (a pixel fires when its level index
    floor(4 * I) changes between frames, polarity = sign of the change),
    `b` is `a` with each event moved by one lattice step (probability
    `move`), dropped (`drop`) or flipped (`flip`), plus spurious events at
    rate `noise` per voxel."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:height, 0:width].astype(np.float64)
    kx, ky = rng.uniform(0.02, 0.08, 2)
    vx, vy = rng.uniform(0.3, 1.5, 2)
    levels = []
    for t in range(frames + 1):
        I = 0.5 + 0.25 * np.sin(kx * (x - vx * t)) + 0.25 * np.sin(ky * (y - vy * t) + 0.3 * np.sin(0.05 * x))
        levels.append(np.floor(4.0 * I))
    lv = np.stack(levels)
    a = np.sign(lv[1:] - lv[:-1]).astype(np.int8)
    b = np.zeros_like(a)
    t, r, c = np.nonzero(a)
    pol = a[t, r, c]
    u = rng.random(t.size)
    keep = u >= drop
    moved = (u >= drop) & (u < drop + move)
    axis = rng.integers(0, 3, t.size)
    step = rng.choice(np.array([-1, 1]), t.size)
    t2, r2, c2 = t.copy(), r.copy(), c.copy()
    t2[moved & (axis == 0)] += step[moved & (axis == 0)]
    r2[moved & (axis == 1)] += step[moved & (axis == 1)]
    c2[moved & (axis == 2)] += step[moved & (axis == 2)]
    ok = keep & (t2 >= 0) & (t2 < frames) & (r2 >= 0) & (r2 < height) & (c2 >= 0) & (c2 < width)
    fl = rng.random(t.size) < flip
    b[t2[ok], r2[ok], c2[ok]] = np.where(fl[ok], -pol[ok], pol[ok])
    spur = rng.random(a.shape) < noise
    b[spur] = rng.choice(np.array([-1, 1], np.int8), int(spur.sum()))
    return a, b
