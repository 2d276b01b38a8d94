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
