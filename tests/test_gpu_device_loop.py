"""The device-resident round loop (one CUDA graph per call: trace a chunk,
merge and test, size the next chunk or round on the device) against the
host-driven rounds (the undecided count read back after every round): the
same samples and decisions, so identical outputs and counters, for single
frames with a carried reference, batched jobs and the mean pass; and its
bound: a loop that runs past device_timeout_us stops with MCEV_ERR_TIMEOUT
and leaves a usable context."""
import numpy as np
import pytest
import torch

import scenegen as sg
from paper_2408_07996_gb300 import McevError
from paper_2408_07996_gb300.api import Renderer, render_events_batch
from parity import renderer_for

pytestmark = pytest.mark.gpu

KEYS = ("events", "spp", "mean")


def _small_spheres():
    sc = sg.icosphere_field(7, n_spheres=6, level=3, n_frames=4, dt=5e-3, env_w=64, env_h=32, n_spin=3)
    return sg.Workload("spheres_small", sc, 96, 64, [0.0, 1.0, 2.0, 3.0], spp_min=16, spp_batch=16, spp_max=512,
                       C=0.2, alpha=0.05, max_depth=4, seed=7, t_min=2e-4)


@pytest.mark.parametrize("name", ["cornell64", "spheres_small"])
def test_device_loop_equals_host_rounds(name):
    w = sg.workload(name) if name == "cornell64" else _small_spheres()
    outs = {}
    for host in (0, 1):
        # a small wavefront: rounds of several chunks with a ragged last one
        r = renderer_for(w, host_rounds=host, wavefront=20000)
        res = []
        for t0, t1 in ((0.0, 1.0), (1.0, 2.0)):      # the reference carried into the second frame
            o = r.render_events(t0, t1, w.C, w.alpha, w.spp_batch, w.spp_max)
            res.append(({k_: o[k_].clone() for k_ in KEYS}, o["stats"]))
        outs[host] = res
        r.close()
    for (a, sa), (b, sb) in zip(outs[0], outs[1]):
        for k_ in KEYS:
            assert torch.equal(a[k_], b[k_]), k_
        for c in ("paths", "samples_used", "ref_paths", "rounds", "events_pos", "events_neg", "pixels_at_cap",
                  "nodes_closest", "tris_closest", "rays_closest", "rays_shadow", "stats_pixels"):
            assert sa[c] == sb[c], c
        assert sa["rounds"] > 2


def test_device_loop_batched_and_mean():
    c = sg.workload("cornell64")
    ws = [c, _small_spheres()]
    res = {}
    for host in (0, 1):
        rs = [renderer_for(w, host_rounds=host) for w in ws]
        runner = Renderer(8, 8)
        runner.set_params(host_rounds=host, wavefront=50000)
        outs, st = render_events_batch(runner, [(r, 0.0, 1.0) for r in rs], 0.2, 0.05, 16, 256)
        means = [r.render_mean(0.5, 24).clone() for r in rs]
        res[host] = ([{k: o[k].clone() for k in KEYS} for o in outs], st, means)
        for r in rs:
            r.close()
        runner.close()
    for a, b in zip(res[0][0], res[1][0]):
        for k in KEYS:
            assert torch.equal(a[k], b[k])
    assert res[0][1]["paths"] == res[1][1]["paths"] and res[0][1]["rounds"] == res[1][1]["rounds"]
    for a, b in zip(res[0][2], res[1][2]):
        assert torch.equal(a, b)


def test_device_loop_timeout_is_reported_and_recoverable():
    w = sg.workload("cornell64")
    r = renderer_for(w)
    r.render_events(0.0, 1.0, w.C, w.alpha, w.spp_batch, w.spp_max)
    # a 1-us bound: the loop stops after its first chunk
    r.set_params(device_timeout_us=1)
    with pytest.raises(McevError, match="TIMEOUT"):
        r.render_events(1.0, 2.0, w.C, w.alpha, w.spp_batch, w.spp_max)
    # the context stays usable; the interrupted frame invalidated the
    # reference, so the next call renders it again and matches a fresh context
    r.set_params(device_timeout_us=0)
    o = r.render_events(1.0, 2.0, w.C, w.alpha, w.spp_batch, w.spp_max)
    assert o["stats"]["ref_paths"] == w.width * w.height * w.spp_max
    r2 = renderer_for(w)
    e = r2.render_events(1.0, 2.0, w.C, w.alpha, w.spp_batch, w.spp_max)
    for k in KEYS:
        assert torch.equal(o[k], e[k])
    r.close()
    r2.close()
