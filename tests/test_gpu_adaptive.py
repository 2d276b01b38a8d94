"""The adaptive detector against the uniform-sampling baseline on the GPU,
and the properties the paper states about it (Sec. 3.3, Sec. 4): event maps
within 0.5 % of pixels of the uniform-spp maps from the same reference, and
fewer samples where fewer events happen (the speed-up falls as event density
rises)."""
import numpy as np
import pytest

import scenegen as sg
from parity import renderer_for

pytestmark = pytest.mark.gpu


def _frame(r, w, k, variant):
    r.set_params(variant=variant)
    return r.render_events(w.times[k], w.times[k + 1], w.C, w.alpha, w.spp_batch, w.spp_max)


@pytest.mark.slow
def test_adaptive_event_map_matches_uniform():
    from paper_2408_07996_gb300 import ONE_TAILED, UNIFORM
    w = sg.workload("spheres512")
    r = renderer_for(w)
    r.render_reference(w.times[4], w.spp_max)
    state = r.get_state().clone()
    ad = _frame(r, w, 4, ONE_TAILED)
    ev_ad = ad["events"].cpu().numpy()
    r.set_state(state)
    un = _frame(r, w, 4, UNIFORM)
    ev_un = un["events"].cpu().numpy()
    err = float(np.mean(ev_ad != ev_un))
    n_ad = ad["spp"].cpu().numpy()
    print("adaptive vs uniform: event error %.4f%%, mean spp %.0f of %d, paths %.3g vs %.3g" % (
        100 * err, n_ad.mean(), w.spp_max, ad["stats"]["samples_used"], un["stats"]["samples_used"]))
    assert err <= 0.005
    assert (un["spp"].cpu().numpy() == w.spp_max).all()
    assert ad["stats"]["samples_used"] < 0.5 * un["stats"]["samples_used"]
    r.close()


def test_fewer_samples_where_fewer_events():
    from paper_2408_07996_gb300 import ONE_TAILED
    w = sg.workload("cornell64")
    moving = renderer_for(w)
    out_m = _frame(moving, w, 0, ONE_TAILED)
    ws = sg.workload("cornell64")
    ws.scene = sg.static_variant(ws.scene)
    still = renderer_for(ws)
    out_s = _frame(still, ws, 0, ONE_TAILED)
    ev_m = int((out_m["events"] != 0).sum())
    ev_s = int((out_s["events"] != 0).sum())
    n_m = float(out_m["spp"].float().mean())
    n_s = float(out_s["spp"].float().mean())
    print("moving: %d events, mean spp %.1f; static: %d events, mean spp %.1f" % (ev_m, n_m, ev_s, n_s))
    assert ev_s < ev_m
    assert n_s < n_m
    moving.close()
    still.close()
