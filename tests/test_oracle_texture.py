"""Oracle texturing and the gradient references built on it.

Pins: on a textured plane under a constant environment with BSDF sampling
only, every path's radiance is the environment value times the Rec. 709
luminance of the nearest texel at the wrapped, barycentrically interpolated
coordinates of its first hit (checked on pixels whose whole footprint lies
in one texel, with a non-square texture and distinct RGB so that a
transposed lookup, a wrong weight or an off-by-one cell shows); a constant
texture renders like the untextured material of the same luminance; the
finite-difference gradient matches the closed-form derivative on the plane;
the emission derivative obeys degree-1 homogeneity."""
import numpy as np
import pytest

import oracle as O
import scenegen as sg
from diffref import Y709, emission_fd, oracle_means, single_texel_pixels, texel_fd

REPEAT, HALF, LE = 3.0, 0.5, 2.0


def plane_case(seed=3, tw=5, th=3):
    tex = np.random.default_rng(seed).uniform(0.1, 0.9, size=(th, tw, 3)).astype(np.float32)
    sc = sg.textured_plane(tex, REPEAT, LE, HALF)
    p = O.Params(width=48, height=32, max_depth=3, nee=0, mis=0, eps=1e-3, t_min=1e-5, seed=11)
    return sc, tex, p


def test_textured_plane_radiance_is_texel_luminance():
    sc, tex, p = plane_case()
    osc = O.OracleScene(sc)
    cells = single_texel_pixels(osc, p, p.width, p.height, REPEAT, HALF, tex.shape[1], tex.shape[0])
    assert len(cells) > 0.3 * p.width * p.height
    assert len(set(cells.values())) >= 10          # most texels of the 5x3 texture are seen
    pix = np.array(sorted(cells), np.int32)
    L, _ = O.trace_samples(osc, p, 0.0, pix, 0, 8)
    want = np.array([LE * float(Y709 @ tex[cells[q]].astype(np.float64)) for q in pix])
    np.testing.assert_allclose(L, np.repeat(want[:, None], 8, 1), rtol=1e-12)


def test_constant_texture_matches_untextured_material():
    w = sg.workload("diff256")
    rgb = np.array([0.3, 0.6, 0.45], np.float32)
    tex = np.broadcast_to(rgb, (4, 4, 3)).copy()
    sc_t = sg.textured_room(20240819, grid=16, texture=tex)
    y = np.float32(float(Y709 @ rgb.astype(np.float64)))
    alb = sc_t.mat_albedo.copy()
    alb[0] = y
    sc_u = sg.Scene(**{**sc_t.__dict__, "mat_albedo": alb, "mat_textured": np.zeros_like(sc_t.mat_textured)})
    p = O.params_of(w, width=48, height=48)
    pix = np.arange(0, 48 * 48, 5)
    Lt, st = O.trace_samples(O.OracleScene(sc_t), p, 0.0, pix, 0, 16)
    Lu, su = O.trace_samples(O.OracleScene(sc_u), p, 0.0, pix, 0, 16)
    assert Lt.max() > 0
    np.testing.assert_allclose(Lt, Lu, rtol=1e-6, atol=1e-12)   # albedo rounds to float32 once
    assert (st != su).mean() > 0.5                               # the texel joins the signature


def test_plane_texel_gradient_closed_form():
    sc, tex, p = plane_case()
    osc = O.OracleScene(sc)
    cells = single_texel_pixels(osc, p, p.width, p.height, REPEAT, HALF, tex.shape[1], tex.shape[0])
    pix = np.array(sorted(cells), np.int32)
    texels = sorted(set(cells.values()))[:6]
    fd = texel_fd(osc, tex, lambda: oracle_means(osc, p, 0.0, pix, 4, p.eps).sum(), texels, 1e-3)
    for (iy, ix), g in zip(texels, fd):
        n = sum(1 for q in pix if cells[q] == (iy, ix))
        y = float(Y709 @ tex[iy, ix].astype(np.float64))
        # the analytic derivative, up to the central difference's O(h^2) term ...
        assert g == pytest.approx(n * LE / (y * LE + p.eps), rel=1e-4)
        # ... and exactly the central difference of the closed form
        yp, ym = [float(Y709 @ (tex[iy, ix].astype(np.float64) + s * 1e-3).astype(np.float32).astype(np.float64))
                  for s in (1, -1)]
        want = n * (np.log(yp * LE + p.eps) - np.log(ym * LE + p.eps)) / (yp - ym)
        assert g == pytest.approx(want, rel=1e-9)


def test_emission_gradient_homogeneity():
    """Without an environment every path's radiance is linear in the
    emitters' radiance, so sum_m e_m dL/de_m = L for each sample."""
    sc = sg.textured_room(20240819, grid=16)
    w = sg.workload("diff256")
    p = O.params_of(w, width=32, height=32)
    osc = O.OracleScene(sc)
    pix = np.arange(0, 32 * 32, 3)
    L, _ = O.trace_samples(osc, p, 0.0, pix, 0, 8)
    emitters = [m for m in range(len(sc.mat_emit)) if sc.mat_emit[m] > 0]
    fd = emission_fd(osc, sc.mat_emit, lambda: oracle_means(osc, p, 0.0, pix, 8, p.eps).sum(), emitters, 1e-3)
    lhs = float(np.dot(np.asarray(sc.mat_emit, np.float64)[emitters], fd))
    rhs = float((L / (L + p.eps)).mean(axis=1).sum())
    assert lhs == pytest.approx(rhs, rel=1e-6)
    assert np.all(fd > 0)
