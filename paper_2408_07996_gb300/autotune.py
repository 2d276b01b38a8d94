"""Autotuner for batched event rendering.

Picks the wavefront width (paths per chunk, hence queue chunk size in pixels
= width / samples per pixel), the speculative batch window, the BVH node
layout (two-wide or compressed 8-wide) and the BVH leaf size by timing one
batched frame per candidate from the same reference states.  None of these
settings changes what is rendered (the samples and the decisions are the
same; the two node layouts find the same closest hits up to rare FP32
box-culling decisions next to a ray's origin), only how fast: the tuner only
reads `mcev_stats.gpu_ms`."""
from __future__ import annotations

import itertools

from .api import Renderer, render_events_batch

WAVEFRONTS = (1 << 22, 1 << 23, 1 << 24, 1 << 25)
WINDOWS = (4, 16)
LEAF_SIZES = (2, 4)
BVH_WIDTHS = (2, 8)


def tune_batch(runner: Renderer, renderers: list, pair: tuple, schedule: dict, wavefronts=WAVEFRONTS,
               windows=WINDOWS, leaf_sizes=LEAF_SIZES, sah_bins: int = 32, bvh_widths=BVH_WIDTHS) -> dict:
    """Times one batched frame `pair` = (t0, t1) for every candidate and
    leaves the fastest configuration applied (the leaf size only on the
    renderers passed in).  Tune where the references at t0 already exist,
    or every trial also renders them.  `schedule` holds C, alpha,
    spp_batch, spp_max.  The renderers' reference states are restored after
    every trial, so tuning does not advance the frame sequence."""
    states = [r.get_state().clone() for r in renderers]
    trials = []
    current = None

    def build(width, leaf):
        for r in renderers:
            r.set_params(bvh_width=width)
            r.build_bvh(sah_bins, leaf)

    for width, leaf, wf, win in itertools.product(bvh_widths, leaf_sizes, wavefronts, windows):
        if (width, leaf) != current:
            build(width, leaf)
            current = (width, leaf)
        runner.set_params(wavefront=wf, batch_window=win)
        for r, s in zip(renderers, states):
            r.set_state(s)
        _, st = render_events_batch(runner, [(r, pair[0], pair[1]) for r in renderers], schedule["C"],
                                    schedule["alpha"], schedule["spp_batch"], schedule["spp_max"])
        trials.append({"bvh_width": width, "max_leaf": leaf, "wavefront": wf, "batch_window": win,
                       "gpu_ms": st["gpu_ms"]})
    best = min(trials, key=lambda t: t["gpu_ms"])
    if (best["bvh_width"], best["max_leaf"]) != current:
        build(best["bvh_width"], best["max_leaf"])
    runner.set_params(wavefront=best["wavefront"], batch_window=best["batch_window"])
    for r, s in zip(renderers, states):
        r.set_state(s)
    return {"best": best, "trials": trials}


def tune_renderer(r: Renderer, pair: tuple, schedule: dict, bvh_widths=BVH_WIDTHS, leaf_sizes=LEAF_SIZES,
                  sah_bins: int = 32) -> dict:
    """The same search for one context: times the frame `pair` = (t0, t1)
    for every BVH node layout and leaf size from the same reference state
    and leaves the fastest applied (the reference state is restored, so
    tuning does not advance the frame sequence).  `schedule` holds C, alpha,
    spp_batch, spp_max."""
    state = r.get_state().clone()
    trials = []
    for width, leaf in itertools.product(bvh_widths, leaf_sizes):
        r.set_params(bvh_width=width)
        r.build_bvh(sah_bins, leaf)
        r.set_state(state)
        st = r.render_events(pair[0], pair[1], schedule["C"], schedule["alpha"], schedule["spp_batch"],
                             schedule["spp_max"])["stats"]
        trials.append({"bvh_width": width, "max_leaf": leaf, "gpu_ms": st["gpu_ms"]})
    best = min(trials, key=lambda t: t["gpu_ms"])
    r.set_params(bvh_width=best["bvh_width"])
    r.build_bvh(sah_bins, best["max_leaf"])
    r.set_state(state)
    return {"best": best, "trials": trials}
