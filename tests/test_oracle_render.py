"""Pins of the oracle's path tracer (tracePaths of Alg. 1, Sec. 3.1) against
closed forms, brute force and sampling identities that do not reuse the
oracle's own formulas."""
import math

import numpy as np
import pytest

import oracle as O
import scenegen as sg


def params(w=8, h=8, depth=4, nee=1, mis=1, eps=1e-3, t_min=1e-4, seed=7):
    return O.Params(width=w, height=h, max_depth=depth, nee=nee, mis=mis, eps=eps,
                    t_min=t_min, seed=seed)


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("albedo,emit,depth", [(0.5, 1.0, 4), (0.8, 2.0, 6), (0.3, 0.7, 1), (0.9, 1.0, 0)])
def test_white_furnace_exact(albedo, emit, depth):
    # closed emitting sphere, camera inside, BSDF sampling only: every path
    # collects emit at each of its depth+1 vertices, scaled by albedo^k
    osc = O.OracleScene(sg.furnace_sphere(albedo, emit))
    L, _ = O.trace_samples(osc, params(depth=depth, nee=0, mis=0), 0.0, np.arange(64), 0, 8)
    a, e = float(np.float32(albedo)), float(np.float32(emit))   # scene values are FP32
    expect = e * sum(a ** k for k in range(depth + 1))
    np.testing.assert_allclose(L, expect, rtol=1e-12)


@pytest.mark.parametrize("mis", [0, 1])
def test_white_furnace_nee_unbiased(mis):
    # NEE over all emissive triangles (area-light pdf) and, with mis=1, the
    # power heuristic: unbiased estimates of the same closed form
    osc = O.OracleScene(sg.furnace_sphere(0.5, 1.0))
    L, _ = O.trace_samples(osc, params(depth=4, mis=mis), 0.0, np.arange(64), 0, 256)
    expect = sum(0.5 ** k for k in range(5))
    se = L.std() / math.sqrt(L.size)
    assert abs(L.mean() - expect) < 5 * se + 1e-12


def test_plane_under_constant_env_exact():
    osc = O.OracleScene(sg.plane_under_env(0.5, 2.0))
    L, _ = O.trace_samples(osc, params(depth=3, nee=0, mis=0), 0.0, np.arange(64), 0, 16)
    np.testing.assert_allclose(L, 1.0, rtol=1e-12)


@pytest.mark.parametrize("mis", [0, 1])
def test_plane_under_constant_env_nee_unbiased(mis):
    osc = O.OracleScene(sg.plane_under_env(0.5, 2.0))
    L, _ = O.trace_samples(osc, params(depth=3, mis=mis), 0.0, np.arange(64), 0, 1024)
    se = L.std() / math.sqrt(L.size)
    assert abs(L.mean() - 1.0) < 5 * se


def test_empty_scene_sees_environment():
    osc = O.OracleScene(sg.empty_env(3.0))
    L, sig = O.trace_samples(osc, params(), 0.0, np.arange(64), 0, 4)
    np.testing.assert_array_equal(L, 3.0)


def test_log_luminance_of_deterministic_paths():
    # var = 0 and mean ln(L + eps) = ln(closed form + eps) exactly
    osc = O.OracleScene(sg.furnace_sphere(0.5, 1.0))
    p = params(depth=4, nee=0, mis=0)
    w = sg.Workload("furnace", sg.furnace_sphere(0.5, 1.0), 8, 8, [0.0, 1.0], spp_min=16,
                    spp_batch=16, spp_max=64, C=0.2, alpha=0.05, max_depth=4)
    ref = O.reference(osc, p, 64, 0.0, np.arange(64))
    np.testing.assert_allclose(ref["mean"], math.log(1.9375 + 1e-3), rtol=1e-14)
    assert (ref["var"] < 1e-25).all()      # zero up to the rounding of the mean
    out = O.render_events(osc, p, O.detect_of(w), 0.0, 1.0, np.arange(64), ref=ref)
    # zero variance, zero gap: stop at the first test, no event
    assert (out["n"] == 16).all() and (out["events"] == 0).all()


# ---------------------------------------------------------------- camera

def test_camera_center_and_field_of_view():
    sc = sg.cornell_box()
    osc = O.OracleScene(sc)
    for (w, h) in [(64, 64), (128, 64), (40, 80)]:
        p = params(w=w, h=h)
        o, d = osc.camera_ray(p, 0.0, w / 2, h / 2)
        np.testing.assert_allclose(o, sc.cam_eye[0])
        fwd = sc.cam_target[0] - sc.cam_eye[0]
        np.testing.assert_allclose(d, fwd / np.linalg.norm(fwd), atol=1e-15)
        half = math.radians(sc.fov_deg) / 2
        if w <= h:
            _, d1 = osc.camera_ray(p, 0.0, 0.0, h / 2)
        else:
            _, d1 = osc.camera_ray(p, 0.0, w / 2, 0.0)
        assert math.acos(np.dot(d1, d)) == pytest.approx(half, rel=1e-12)
        # pixel (0, 0) is top-left: left of and above the view axis
        _, d2 = osc.camera_ray(p, 0.0, 0.0, 0.0)
        assert d2[0] < 0 and d2[1] > d[1]


def test_keyframes_interpolate_linearly():
    sc = sg.cornell_box(shift=0.02)
    osc = O.OracleScene(sc)
    p = params()
    for t, dx in [(0.0, 0.0), (0.25, 0.005), (1.0, 0.02), (2.0, 0.02), (-1.0, 0.0)]:
        o, _ = osc.camera_ray(p, t, 4, 4)
        assert o[0] == pytest.approx(0.5 + dx, abs=1e-15)


# ---------------------------------------------------------------- geometry

def _random_rays(rng, n, lo, hi):
    o = rng.uniform(lo, hi, size=(n, 3))
    d = rng.normal(size=(n, 3))
    return o, d / np.linalg.norm(d, axis=1, keepdims=True)


def test_bvh_matches_brute_force_cornell():
    osc = O.OracleScene(sg.cornell_box())
    rng = np.random.default_rng(20)
    o, d = _random_rays(rng, 3000, 0.02, 0.98)
    for i in range(len(o)):
        a = osc.closest_hit(0.0, o[i], d[i], 1e-4, np.inf, True)
        b = osc.closest_hit(0.0, o[i], d[i], 1e-4, np.inf, False)
        assert a == b


def test_bvh_matches_brute_force_instanced_spheres():
    sc = sg.icosphere_field(n_spheres=12, level=3, n_frames=3)
    osc = O.OracleScene(sc)
    rng = np.random.default_rng(21)
    hits = 0
    for i in range(300):
        o = np.array([rng.uniform(-7, 7), rng.uniform(2, 4), rng.uniform(-7, 7)])
        d = np.array([rng.uniform(-0.3, 0.3), -1.0, rng.uniform(-0.3, 0.3)])
        d /= np.linalg.norm(d)
        t = [0.0, 0.001, 0.0015][i % 3]
        a = osc.closest_hit(t, o, d, 1e-4, np.inf, True)
        b = osc.closest_hit(t, o, d, 1e-4, np.inf, False)
        assert a == b
        hits += a[0] and a[2] < 12
    assert hits > 10


def test_bvh_matches_brute_force_many_moving_instances():
    # eight of twelve spheres spin (the moving-instance parity scene's kind),
    # at times between and on keyframes, so the oracle's per-frame instance
    # transforms are exercised for several instances at once
    sc = sg.icosphere_field(11, n_spheres=12, level=3, n_frames=4, dt=0.05, env_w=64, env_h=32, n_spin=8)
    moving = [s for s in range(12) if not np.allclose(sc.inst_xform[0, s], sc.inst_xform[-1, s])]
    assert moving == list(range(8))
    osc = O.OracleScene(sc)
    rng = np.random.default_rng(22)
    hits = set()
    for i in range(400):
        o = np.array([rng.uniform(-7, 7), rng.uniform(2, 4), rng.uniform(-7, 7)])
        d = np.array([rng.uniform(-0.3, 0.3), -1.0, rng.uniform(-0.3, 0.3)])
        d /= np.linalg.norm(d)
        t = [0.0, 0.05, 0.075, 0.1][i % 4]
        a = osc.closest_hit(t, o, d, 1e-4, np.inf, True)
        b = osc.closest_hit(t, o, d, 1e-4, np.inf, False)
        assert a == b
        if a[0] and a[2] < 8:
            hits.add(a[2])
    assert len(hits) >= 3


def test_watertight_shared_edge():
    # rays aimed at points of the shared diagonal of a split quad never leak
    osc = O.OracleScene(sg.plane_under_env(0.5, 1.0, half=1.0))
    rng = np.random.default_rng(22)
    for _ in range(2000):
        s = rng.uniform(-1, 1)
        target = np.array([s, 0.0, s])         # the diagonal (-1,0,-1)-(1,0,1)
        o = target + rng.normal(size=3) * np.array([1, 0, 1]) + np.array([0, rng.uniform(0.1, 3), 0])
        d = target - o
        hit, t, inst, prim = osc.closest_hit(0.0, o, d / np.linalg.norm(d), 0.0, np.inf, False)
        assert hit and prim in (0, 1)


def test_instance_transform_moves_geometry():
    # sphere 0 spins; a ray through its centre hits it at every key time and
    # the hit triangle changes as it turns
    sc = sg.icosphere_field(n_spheres=2, level=3, n_frames=3, dt=0.05)
    osc = O.OracleScene(sc)
    c = sc.inst_xform[0, 0].reshape(3, 4)[:, 3]
    o = c + np.array([0.0, 0.0, 5.0])
    prims = []
    for t in sc.key_times:
        hit, dist, inst, prim = osc.closest_hit(t, o, np.array([0.0, 0.0, -1.0]), 1e-4, np.inf, True)
        assert hit and inst == 0
        prims.append(prim)
    assert len(set(prims)) > 1


# ---------------------------------------------------------------- samplers

def test_env_sampler_integrates_environment():
    rng = np.random.default_rng(23)
    env = rng.uniform(0.01, 10.0, size=(8, 16)).astype(np.float32)
    env[3, 5] = 500.0
    sc = sg.empty_env(1.0)
    sc.env = env
    osc = O.OracleScene(sc)
    H, W = env.shape
    th = np.linspace(0, math.pi, H + 1)
    exact = sum(float(env[i, j]) * (2 * math.pi / W) * (math.cos(th[i]) - math.cos(th[i + 1]))
                for i in range(H) for j in range(W))
    n = 20000
    acc = []
    for k in range(n):
        u1, u2 = (k + 0.5) / n, rng.uniform()
        ok, d, pdf, Le = osc.env_sample(u1, u2)
        assert ok and pdf > 0
        assert abs(np.linalg.norm(d) - 1) < 1e-12
        acc.append(Le / pdf)
        if k % 50 == 0:
            assert osc.env_radiance(d) == Le
            assert osc.env_pdf(d) == pytest.approx(pdf, rel=1e-9)
    est = np.mean(acc)
    assert est == pytest.approx(exact, rel=5 * np.std(acc) / math.sqrt(n) / exact + 1e-9)


def test_env_pdf_normalised():
    rng = np.random.default_rng(24)
    env = rng.uniform(0.1, 5.0, size=(6, 12)).astype(np.float32)
    sc = sg.empty_env(1.0)
    sc.env = env
    osc = O.OracleScene(sc)
    nt, nphi = 300, 240
    tot = 0.0
    for i in range(nt):
        th = (i + 0.5) / nt * math.pi
        for j in range(nphi):
            ph = (j + 0.5) / nphi * 2 * math.pi
            d = np.array([math.sin(th) * math.cos(ph), math.cos(th), math.sin(th) * math.sin(ph)])
            tot += osc.env_pdf(d) * math.sin(th) * (math.pi / nt) * (2 * math.pi / nphi)
    assert tot == pytest.approx(1.0, rel=1e-9)


def _sph(ct, ph):
    st_ = math.sqrt(max(0.0, 1 - ct * ct))
    return np.array([st_ * math.cos(ph), st_ * math.sin(ph), ct])


def test_lambertian_sampler_is_cosine_weighted():
    rng = np.random.default_rng(25)
    wo = _sph(0.6, 0.3)
    n, inside = 20000, 0
    for _ in range(n):
        wi = O.bsdf_sample(0, 0.0, wo, rng.uniform(), rng.uniform())
        f, pdf = O.bsdf_eval(0, 0.7, 0.0, wo, wi)
        assert pdf == pytest.approx(wi[2] / math.pi)
        assert f * wi[2] / pdf == pytest.approx(0.7)
        inside += wi[2] > math.cos(math.radians(30))
    # cosine-weighted: P(theta < 30 deg) = sin^2(30 deg) = 1/4
    assert abs(inside / n - 0.25) < 4 * math.sqrt(0.25 * 0.75 / n)


@pytest.mark.parametrize("alpha", [0.1, 0.3, 0.6])
def test_ggx_normal_incidence_visible_fraction(alpha):
    # at normal incidence pdf(wi) = D(h)/4 and the reflected directions above
    # the horizon are the half vectors within 45 degrees, whose D-mass is
    # alpha^2 int_{1/2}^{1} du / (u (alpha^2-1) + 1)^2 = 1 / (1 + alpha^2)
    wo = np.array([0.0, 0.0, 1.0])
    nt, nphi = 4000, 8
    tot = 0.0
    for i in range(nt):
        ct = (i + 0.5) / nt
        for j in range(nphi):
            ph = (j + 0.5) / nphi * 2 * math.pi
            f, pdf = O.bsdf_eval(1, 1.0, alpha, wo, _sph(ct, ph))
            tot += pdf * (1.0 / nt) * (2 * math.pi / nphi)
    assert tot == pytest.approx(1.0 / (1.0 + alpha * alpha), rel=2e-3)


@pytest.mark.parametrize("alpha,ct", [(0.3, 0.9), (0.6, 0.4), (0.45, 0.15)])
def test_ggx_sampler_matches_pdf_chi2(alpha, ct):
    # histogram of visible-normal samples vs the pdf integrated over bins
    rng = np.random.default_rng(int(alpha * 100 + ct * 10))
    wo = _sph(ct, 0.7)
    nb_t, nb_p, sub = 10, 12, 6
    expected = np.zeros((nb_t, nb_p))
    for a in range(nb_t):
        for b in range(nb_p):
            acc = 0.0
            for s in range(sub):
                for r in range(sub):
                    c = (a + (s + 0.5) / sub) / nb_t
                    ph = (b + (r + 0.5) / sub) / nb_p * 2 * math.pi
                    acc += O.bsdf_eval(1, 1.0, alpha, wo, _sph(c, ph))[1]
            expected[a, b] = acc / sub / sub * (1.0 / nb_t) * (2 * math.pi / nb_p)
    n = 40000
    counts = np.zeros((nb_t, nb_p))
    for _ in range(n):
        wi = O.bsdf_sample(1, alpha, wo, rng.uniform(), rng.uniform())
        if wi[2] <= 0:
            continue
        a = min(int(wi[2] * nb_t), nb_t - 1)
        ph = math.atan2(wi[1], wi[0]) % (2 * math.pi)
        b = min(int(ph / (2 * math.pi) * nb_p), nb_p - 1)
        counts[a, b] += 1
    exp_n = expected * n
    mask = exp_n > 5
    chi2 = float(np.sum((counts[mask] - exp_n[mask]) ** 2 / exp_n[mask]))
    dof = int(mask.sum())
    assert chi2 < dof + 6 * math.sqrt(2 * dof)
    assert abs(counts.sum() - exp_n.sum()) < 6 * math.sqrt(n) + 0.01 * n


@pytest.mark.parametrize("alpha", [0.1, 0.35, 0.6])
def test_ggx_reciprocity_and_energy(alpha):
    rng = np.random.default_rng(26)
    for _ in range(200):
        wo = _sph(rng.uniform(0.05, 1), rng.uniform(0, 6.28))
        wi = _sph(rng.uniform(0.05, 1), rng.uniform(0, 6.28))
        f1, _ = O.bsdf_eval(1, 0.4, alpha, wo, wi)
        f2, _ = O.bsdf_eval(1, 0.4, alpha, wi, wo)
        assert f1 == pytest.approx(f2, rel=1e-12)
    # directional albedo with F0 = 1 never exceeds 1, even at grazing angles
    for ct in [1.0, 0.5, 0.1, 0.03]:
        wo = _sph(ct, 0.0)
        est = []
        for _ in range(4000):
            wi = O.bsdf_sample(1, alpha, wo, rng.uniform(), rng.uniform())
            f, pdf = O.bsdf_eval(1, 1.0, alpha, wo, wi)
            est.append(f * wi[2] / pdf if pdf > 0 else 0.0)
        assert np.mean(est) <= 1.0 + 1e-9
        assert max(est) <= 1.0 + 1e-9
    # single scattering loses little energy at normal incidence for small alpha
    if alpha == 0.1:
        assert np.mean(est) < 1.0


def test_schlick_fresnel_at_normal_incidence():
    # F(1) = F0: with alpha small, the normal-incidence albedo tends to F0
    wo = np.array([0.0, 0.0, 1.0])
    rng = np.random.default_rng(27)
    est = []
    for _ in range(4000):
        wi = O.bsdf_sample(1, 0.05, wo, rng.uniform(), rng.uniform())
        f, pdf = O.bsdf_eval(1, 0.3, 0.05, wo, wi)
        est.append(f * wi[2] / pdf if pdf > 0 else 0.0)
    assert np.mean(est) == pytest.approx(0.3, rel=0.01)


# ---------------------------------------------------------------- Alg. 1 on scenes

def test_static_scene_false_events_below_alpha():
    # Nothing moves and t0, t1 draw independent streams: the true gap is 0.
    # With the paper's schedule (Sec. 3.3: first test at 256, +64, cap 4096)
    # the standard error at the cap is far below C, so false events stay
    # under alpha and most pixels stop long before the cap.
    w = sg.workload("cornell64")
    sc = sg.static_variant(w.scene)
    osc = O.OracleScene(sc)
    rng = np.random.default_rng(29)
    pix = np.sort(rng.choice(w.width * w.height, size=256, replace=False)).astype(np.int32)
    d = O.detect_of(w, spp_min=256, spp_batch=64, spp_max=4096)
    out = O.render_events(osc, O.params_of(w), d, 0.0, 1.0, pix)
    assert np.mean(out["events"] != 0) <= w.alpha
    assert np.median(out["n"]) < 0.25 * 4096


def test_cornell_frame_invariants_and_prefix():
    w = sg.workload("cornell64")
    osc = O.OracleScene(w.scene)
    p, d = O.params_of(w), O.detect_of(w)
    rng = np.random.default_rng(28)
    pix = np.sort(rng.choice(w.width * w.height, size=300, replace=False)).astype(np.int32)
    out = O.render_events(osc, p, d, 0.0, 1.0, pix)
    ev, n = out["events"], out["n"]
    assert ((n - w.spp_min) % w.spp_batch == 0).all() | (n == w.spp_max).all()
    assert (ev[n < w.spp_max] == 0).all()
    assert (ev != 0).any() and (n < w.spp_max).any()
    # the adaptive samples are the first n of the uniform pixel's samples
    ref = O.reference(osc, p, w.spp_max, 0.0, pix)
    L, _ = O.trace_samples(osc, p, 1.0, pix[:20], 0, w.spp_max)
    for i in range(20):
        y = np.log(L[i, :n[i]] + w.eps)
        assert out["mean"][i] == pytest.approx(float(np.mean(y)), rel=1e-12, abs=1e-12)
    # reference of the first frame = plain statistics of spp_max samples at t0
    L0, _ = O.trace_samples(osc, p, 0.0, pix[:5], 0, w.spp_max)
    for i in range(5):
        y = np.log(L0[i] + w.eps)
        assert ref["mean"][i] == pytest.approx(float(np.mean(y)), rel=1e-12, abs=1e-12)
        assert ref["var"][i] == pytest.approx(float(np.var(y, ddof=1)), rel=1e-10)
    # uniform variant runs every pixel to the cap
    u = O.render_events(osc, p, O.detect_of(w, variant=O.UNIFORM), 0.0, 1.0, pix[:30])
    assert (u["n"] == w.spp_max).all()


def test_streams_independent_across_times_and_pixels():
    w = sg.workload("cornell64")
    osc = O.OracleScene(w.scene)
    p = O.params_of(w)
    La, _ = O.trace_samples(osc, p, 0.0, [100, 101], 0, 64)
    Lb, _ = O.trace_samples(osc, p, 0.5, [100, 101], 0, 64)
    assert not np.allclose(La, Lb)
    assert not np.allclose(La[0], La[1])
    Lc, _ = O.trace_samples(osc, p, 0.0, [100, 101], 0, 64)
    np.testing.assert_array_equal(La, Lc)
