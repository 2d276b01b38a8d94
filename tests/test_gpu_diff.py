"""Differentiable event rendering on the GPU: the path-replay adjoint
(mcev_backward) against closed forms, against central finite differences
of the GPU forward pass, and against finite differences of the FP64 oracle
on pixels whose every sample made the same discrete decisions on both
sides.  Texture gradients are compared per texel in luminance units
(the kernel spreads dL/dY over the channels by the Rec. 709 weights)."""
import numpy as np
import pytest
import torch

import oracle as O
import scenegen as sg
from diffref import Y709, emission_fd, oracle_means, single_texel_pixels, texel_fd
from parity import per_sample, renderer_for, summary

pytestmark = pytest.mark.gpu

REPEAT, HALF, LE = 3.0, 0.5, 2.0
SPP = 64
H_FD = 1e-3
Y32 = torch.tensor(Y709, dtype=torch.float32)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


# ---------------------------------------------------------------- closed forms

def test_textured_plane_forward_and_adjoint_closed_form():
    tex = np.random.default_rng(3).uniform(0.1, 0.9, size=(3, 5, 3)).astype(np.float32)
    sc = sg.textured_plane(tex, REPEAT, LE, HALF)
    w = sg.Workload("tplane", sc, 48, 32, [0.0, 1.0], spp_min=16, spp_batch=16, spp_max=64, C=0.2,
                    alpha=0.05, max_depth=3, nee=0, mis=0)
    r = renderer_for(w)
    osc = O.OracleScene(sc)
    cells = single_texel_pixels(osc, O.params_of(w), 48, 32, REPEAT, HALF, 5, 3)
    pix = np.array(sorted(cells), np.int32)
    L, _ = r.trace_samples(0.0, torch.from_numpy(pix), 0, 16)
    want = np.array([LE * float(Y709 @ tex[cells[q]].astype(np.float64)) for q in pix])
    np.testing.assert_allclose(L.cpu().numpy(), np.repeat(want[:, None], 16, 1), rtol=2e-6)
    # d/dtexel of sum over those pixels of mean ln(L + eps)
    g = torch.zeros(32 * 48, device="cuda")
    g[torch.from_numpy(pix).long().cuda()] = 1.0
    gt = torch.zeros(3, 5, 3, device="cuda")
    r.backward(0.0, 16, g.view(32, 48), gt, None)
    expect = np.zeros((3, 5, 3))
    for q in pix:
        iy, ix = cells[q]
        y = float(Y709 @ tex[iy, ix].astype(np.float64))
        expect[iy, ix] += LE / (y * LE + w.eps) * Y709
    np.testing.assert_allclose(gt.cpu().numpy(), expect, rtol=1e-4, atol=1e-4)
    r.close()


def test_furnace_emission_gradient_closed_form():
    sc = sg.furnace_sphere(0.5, 1.0)
    w = sg.Workload("furnace", sc, 16, 16, [0.0, 1.0], spp_min=16, spp_batch=16, spp_max=64, C=0.2,
                    alpha=0.05, max_depth=4, nee=0, mis=0)
    r = renderer_for(w)
    e = _dev(sc.mat_emit)
    r.set_emission(e)
    g = torch.randn(16, 16, generator=torch.Generator().manual_seed(5)).cuda()
    ge = torch.zeros(1, device="cuda")
    r.backward(0.0, 32, g, None, ge)
    S = 1.9375                                   # sum_{k=0..4} 0.5^k
    want = float(g.double().sum()) * S / (S + w.eps)
    assert float(ge[0]) == pytest.approx(want, rel=1e-4, abs=1e-4)
    r.close()


# ---------------------------------------------------------------- textured room, 256x256, 64 spp

@pytest.fixture(scope="module")
def room():
    w = sg.workload("diff256")
    osc = O.OracleScene(w.scene)
    r = renderer_for(w)
    tex = _dev(w.scene.texture)
    emit = _dev(w.scene.mat_emit)
    r.set_texture(tex)
    r.set_emission(emit)
    yield w, osc, r, tex, emit
    r.close()


@pytest.mark.parametrize("t", [0.0, 1.0])
def test_room_per_sample_parity(room, t):
    w, osc, r, _, _ = room
    rng = np.random.default_rng(50 + int(t))
    pix = np.sort(rng.choice(w.width * w.height, size=1500, replace=False))
    ps = per_sample(r, osc, O.params_of(w), t, pix, 0, 24, w.eps)
    s = summary(ps)
    print("room per-sample", t, s)
    assert s["mismatch"] <= 2e-3
    assert s["p999_dy"] < 1e-4 and s["max_dy"] < 1e-3
    full = ps["match"].all(axis=1)
    assert np.abs(ps["yg"].mean(1) - ps["yo"].mean(1))[full].max() < 1e-4


def test_render_mean_matches_samples(room):
    w, _, r, _, _ = room
    m = r.render_mean(0.0, SPP).double().cpu().numpy().reshape(-1)
    L, _ = r.trace_samples(0.0, torch.arange(w.width * w.height, dtype=torch.int32), 0, SPP, want_sig=False)
    y = np.log(L.double().cpu().numpy() + w.eps).mean(1)
    assert np.abs(m - y).max() < 4e-6


def _grads(r, t, g, tex_shape, n_mat):
    gt = torch.zeros(tex_shape, device="cuda")
    ge = torch.zeros(n_mat, device="cuda")
    r.backward(t, SPP, g, gt, ge)
    torch.cuda.synchronize()
    return gt, ge


def _lin_loss(r, t, g):
    return float((r.render_mean(t, SPP).double() * g.double()).sum())


def _texels(G, n_top, n_rand, seed):
    flat = G.abs().reshape(-1)
    order = torch.argsort(flat, descending=True).cpu().numpy()
    top = order[:n_top]
    rest = order[n_top:][(flat.cpu().numpy()[order[n_top:]] > 1e-3 * float(flat.max()))]
    rnd = np.random.default_rng(seed).choice(rest, size=min(n_rand, rest.size), replace=False)
    W = G.shape[1]
    return [(int(i) // W, int(i) % W) for i in np.concatenate([top, rnd])]


def test_room_adjoint_vs_gpu_finite_differences(room):
    """32 texels and the 4 emitters, central differences with h = 1e-3 of
    sum_p g_p mean_p(t) for a fixed random g."""
    w, _, r, tex, emit = room
    g = torch.randn(w.height, w.width, generator=torch.Generator().manual_seed(9)).cuda()
    gt, ge = _grads(r, 0.0, g, tex.shape, emit.numel())
    # channel split is the Rec. 709 weights
    ratio = gt / Y32.cuda()
    nz = gt.abs().sum(-1) > 0
    assert nz.sum() > 1000
    np.testing.assert_allclose(ratio[nz][:, 0].cpu().numpy(), ratio[nz][:, 1].cpu().numpy(), rtol=1e-5, atol=1e-6)
    G = gt[..., 1] / float(Y709[1])
    texels = _texels(G, 16, 16, 1)
    fd = []
    for iy, ix in texels:
        keep = tex[iy, ix].clone()
        vals, lum = [], []
        for s in (1.0, -1.0):
            tex[iy, ix] = keep + s * H_FD
            lum.append(float((tex[iy, ix].double().cpu() * torch.tensor(Y709)).sum()))
            vals.append(_lin_loss(r, 0.0, g))
        tex[iy, ix] = keep
        fd.append((vals[0] - vals[1]) / (lum[0] - lum[1]))
    adj = np.array([float(G[iy, ix]) for iy, ix in texels])
    fd = np.array(fd)
    print("texel adjoint vs fd", np.c_[adj, fd][:8])
    big = np.abs(adj).max()
    assert np.all(np.abs(fd - adj) <= 1e-2 * np.abs(adj) + 1e-3 * big)
    emitters = [m for m in range(emit.numel()) if float(w.scene.mat_emit[m]) > 0]
    for m in emitters:
        keep = float(emit[m])
        vals = []
        for s in (1.0, -1.0):
            emit[m] = keep + s * 1e-2
            vals.append(_lin_loss(r, 0.0, g))
        step = float(torch.tensor([keep + 1e-2], dtype=torch.float32)) - float(torch.tensor([keep - 1e-2],
                                                                                              dtype=torch.float32))
        emit[m] = keep
        efd = (vals[0] - vals[1]) / step
        print("emitter", m, float(ge[m]), efd)
        assert float(ge[m]) == pytest.approx(efd, rel=1e-3, abs=1e-3 * float(ge.abs().max()))
    non = [m for m in range(emit.numel()) if m not in emitters]
    assert torch.all(ge[non] == 0)


def test_room_emission_homogeneity_full_frame(room):
    """No environment: every sample's radiance is linear in the emitters,
    so sum_m e_m dF/de_m = sum_p g_p mean_k L/(L + eps) for F = sum_p g_p mean_p."""
    w, _, r, tex, emit = room
    g = torch.randn(w.height, w.width, generator=torch.Generator().manual_seed(13)).cuda()
    _, ge = _grads(r, 1.0, g, tex.shape, emit.numel())
    lhs = float((ge.double() * emit.double()).sum())
    L, _ = r.trace_samples(1.0, torch.arange(w.width * w.height, dtype=torch.int32), 0, SPP, want_sig=False)
    L = L.double()
    rhs = float(((L / (L + w.eps)).mean(1) * g.reshape(-1).double()).sum())
    scale = float(((L / (L + w.eps)).mean(1) * g.reshape(-1).double()).abs().sum())
    assert abs(lhs - rhs) < 1e-4 * scale


def test_room_adjoint_vs_fp64_oracle(room):
    """FP64 CPU reference gradient: central differences of the oracle's
    means over a 20x20 window, restricted to pixels whose 64 samples made
    the same decisions on both sides."""
    w, osc, r, tex, emit = room
    p = O.params_of(w)
    ys, xs = np.mgrid[118:138, 118:138]
    win = (ys * w.width + xs).reshape(-1).astype(np.int32)
    ps = per_sample(r, osc, p, 0.0, win, 0, SPP, w.eps)
    keep = ps["match"].all(axis=1)
    assert keep.mean() > 0.9
    gw = np.random.default_rng(17).normal(size=win.size) * keep
    g = torch.zeros(w.height * w.width, dtype=torch.float32)
    g[torch.from_numpy(win).long()] = torch.from_numpy(gw.astype(np.float32))
    gt, ge = _grads(r, 0.0, g.view(w.height, w.width).cuda(), tex.shape, emit.numel())
    G = gt[..., 1] / float(Y709[1])
    texels = _texels(G, 16, 0, 0)
    gw32 = gw.astype(np.float32).astype(np.float64)
    loss = lambda: float((gw32 * oracle_means(osc, p, 0.0, win, SPP, w.eps)).sum())  # noqa: E731
    fd = texel_fd(osc, w.scene.texture, loss, texels, H_FD)
    adj = np.array([float(G[iy, ix]) for iy, ix in texels])
    print("texel adjoint vs fp64 fd", np.c_[adj, fd][:8])
    assert np.all(np.abs(fd - adj) <= 2e-3 * np.abs(adj) + 1e-4 * np.abs(adj).max())
    emitters = [m for m in range(emit.numel()) if float(w.scene.mat_emit[m]) > 0]
    efd = emission_fd(osc, w.scene.mat_emit, loss, emitters, 1e-3)
    eadj = ge.double().cpu().numpy()[emitters]
    print("emission adjoint vs fp64 fd", eadj, efd)
    np.testing.assert_allclose(eadj, efd, rtol=2e-3, atol=1e-4 * np.abs(efd).max())


def test_autograd_event_loss(room):
    """EventFrames + event_loss: the texture and emission gradients equal
    the adjoint of dloss/dmean at both times, and a few central
    differences of the whole loss agree."""
    from paper_2408_07996_gb300.api import EventFrames, event_loss
    w, _, r, tex, emit = room
    # target events from a different texture
    other = _dev(sg.albedo_texture(w.scene.texture.shape[0], 77))
    r.set_texture(other)
    d = r.render_mean(1.0, SPP) - r.render_mean(0.0, SPP)
    target = (torch.sign(d) * (d.abs() > w.C)).to(torch.int8)
    T = tex.clone().requires_grad_(True)
    E = emit.clone().requires_grad_(True)
    m0, m1 = EventFrames.apply(T, E, r, 0.0, 1.0, SPP)
    loss = event_loss(m0.double(), m1.double(), target, w.C)
    loss.backward()
    # manual chain
    mm0 = m0.detach().double().requires_grad_(True)
    mm1 = m1.detach().double().requires_grad_(True)
    g0, g1 = torch.autograd.grad(event_loss(mm0, mm1, target, w.C), (mm0, mm1))
    gt = torch.zeros_like(tex)
    ge = torch.zeros_like(emit)
    r.set_texture(tex)
    r.backward(0.0, SPP, g0.float(), gt, ge)
    r.backward(1.0, SPP, g1.float(), gt, ge)
    torch.testing.assert_close(T.grad, gt, rtol=1e-4, atol=1e-4 * float(gt.abs().max()))
    torch.testing.assert_close(E.grad, ge, rtol=1e-4, atol=1e-4 * float(ge.abs().max()))
    # whole-loss central differences on the 6 texels of largest gradient
    G = T.grad[..., 1] / float(Y709[1])
    for iy, ix in _texels(G, 6, 0, 0):
        keep = tex[iy, ix].clone()
        vals, lum = [], []
        for s in (1.0, -1.0):
            tex[iy, ix] = keep + s * 1e-2
            lum.append(float((tex[iy, ix].double().cpu() * torch.tensor(Y709)).sum()))
            vals.append(float(event_loss(r.render_mean(0.0, SPP).double(), r.render_mean(1.0, SPP).double(),
                                         target, w.C)))
        tex[iy, ix] = keep
        fdv = (vals[0] - vals[1]) / (lum[0] - lum[1])
        assert float(G[iy, ix]) == pytest.approx(fdv, rel=5e-2, abs=1e-3 * float(G.abs().max()))
    r.set_emission(emit)


def test_texture_descent_reduces_loss(room):
    """Five Adam steps from a flat texture towards a target rendering."""
    from paper_2408_07996_gb300.api import EventFrames
    w, _, r, tex, emit = room
    with torch.no_grad():
        m0_t, m1_t = r.render_mean(0.0, SPP).clone(), r.render_mean(1.0, SPP).clone()
    T = torch.full_like(tex, 0.5).requires_grad_(True)
    opt = torch.optim.Adam([T], lr=0.05)
    losses = []
    for _ in range(6):
        opt.zero_grad()
        m0, m1 = EventFrames.apply(T, emit, r, 0.0, 1.0, SPP)
        loss = ((m0 - m0_t) ** 2).sum() + ((m1 - m1_t) ** 2).sum()
        loss.backward()
        opt.step()
        with torch.no_grad():
            T.clamp_(0.0, 1.0)
        losses.append(float(loss))
    r.set_texture(tex)
    print("descent", losses)
    assert losses[-1] < 0.7 * losses[0]


def test_diff_argument_errors(room):
    from paper_2408_07996_gb300._lib import McevError
    w, _, r, tex, emit = room
    with pytest.raises(McevError):
        r.render_mean(0.0, 0)
    with pytest.raises(McevError):
        r.backward(0.0, 0, torch.zeros(w.height, w.width, device="cuda"), None, None)
    with pytest.raises(McevError):
        r.set_emission(emit[:-1].contiguous())
    r.set_emission(emit)
