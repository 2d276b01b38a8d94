"""Helpers that compare the CUDA path with the oracle on identical sample
streams (used by the -m gpu tests)."""
import numpy as np
import torch

import oracle as O


def renderer_for(w, width=None, height=None, **params):
    from paper_2408_07996_gb300.api import Renderer
    r = Renderer(width or w.width, height or w.height, 0)
    r.upload(w.scene)
    r.configure(w)
    if params:
        r.set_params(**params)
    return r


def per_sample(r, osc, p, t, pixels, k0, count, eps):
    """GPU and oracle per-sample log luminance with decision signatures."""
    pix = np.ascontiguousarray(pixels, np.int32)
    Lg, sg = r.trace_samples(t, torch.from_numpy(pix), k0, count)
    Lg = Lg.cpu().numpy().astype(np.float64)
    sg = sg.cpu().numpy().view(np.uint32)
    Lo, so = O.trace_samples(osc, p, t, pix, k0, count)
    return dict(yg=np.log(Lg + eps), yo=np.log(Lo + eps), Lg=Lg, Lo=Lo, match=(sg == so))


def summary(ps):
    m = ps["match"]
    d = np.abs(ps["yg"] - ps["yo"])
    return dict(mismatch=float(1 - m.mean()), max_dy=float(d[m].max()) if m.any() else 0.0,
                p999_dy=float(np.quantile(d[m], 0.999)) if m.any() else 0.0)


# Bands around the two floating-point decisions of Alg. 1 (see the module
# docstrings of the parity tests): |t - t_crit| and | |gap| - C |.
T_BAND = 1e-3
C_BAND = 1e-5


def topology_ok(r, osc, p, t, pix, counts, eps):
    """Per pixel: True when every sample k < counts[i] made the same discrete
    decisions (hit ids, visibility, texel, flags) on both sides."""
    counts = np.asarray(counts, np.int64)
    kmax = int(counts.max()) if counts.size else 0
    if kmax == 0:
        return np.ones(len(pix), bool)
    m = per_sample(r, osc, p, t, pix, 0, kmax, eps)["match"]
    used = np.arange(kmax)[None, :] < counts[:, None]
    return np.where(used, m, True).all(1)


def in_band(o):
    """Pixels whose oracle decision lay within a band of a threshold."""
    return (o["margin_t"] < T_BAND) | (o["margin_c"] < C_BAND)


def frame_mismatches(ev, n, mean, o, keep, mean_tol):
    """Element-wise comparison of one Alg. 1 frame with the oracle's on the
    kept pixels: counts of differing events and sample counts, and the worst
    mean difference at equal sample counts."""
    bad_ev = keep & (ev != o["events"])
    bad_n = keep & (n != o["n"])
    same_n = keep & (n == o["n"])
    dmean = np.abs(mean - o["mean"])[same_n]
    return dict(bad_ev=int(bad_ev.sum()), bad_n=int(bad_n.sum()),
                max_dmean=float(dmean.max()) if dmean.size else 0.0, kept=int(keep.sum()),
                mean_ok=bool(dmean.size == 0 or dmean.max() < mean_tol))


def worst_sample(ps, pix, k0):
    """Pixel, sample index, both radiances and |dy| of the matched sample
    with the largest log difference."""
    m = ps["match"]
    d = np.where(m, np.abs(ps["yg"] - ps["yo"]), -1.0)
    i, k = np.unravel_index(int(np.argmax(d)), d.shape)
    return dict(pixel=int(pix[i]), sample=int(k0 + k), Lg=float(ps["Lg"][i, k]), Lo=float(ps["Lo"][i, k]),
                dy=float(d[i, k]))
