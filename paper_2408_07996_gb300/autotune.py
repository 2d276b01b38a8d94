"""Autotuner for batched event rendering.

Picks the wavefront width (paths per chunk, hence queue chunk size in pixels
= width / samples per pixel), the speculative batch window and the BVH leaf
size by timing one batched frame per candidate from the same reference
states.  None of these settings changes what is rendered (the samples, the
closest hits and the decisions are the same), only how fast: the tuner only
reads `mcev_stats.gpu_ms`."""
from __future__ import annotations

import itertools

from .api import Renderer, render_events_batch

WAVEFRONTS = (1 << 22, 1 << 23, 1 << 24, 1 << 25)
WINDOWS = (4, 16)
LEAF_SIZES = (2, 4)


def tune_batch(runner: Renderer, renderers: list, pair: tuple, schedule: dict, wavefronts=WAVEFRONTS,
               windows=WINDOWS, leaf_sizes=LEAF_SIZES, sah_bins: int = 32) -> dict:
    """Times one batched frame `pair` = (t0, t1) for every candidate and
    leaves the fastest configuration applied (the leaf size only on the
    renderers passed in).  Tune where the references at t0 already exist,
    or every trial also renders them.  `schedule` holds C, alpha,
    spp_batch, spp_max.  The renderers' reference states are restored after
    every trial, so tuning does not advance the frame sequence."""
    states = [r.get_state().clone() for r in renderers]
    trials = []
    current_leaf = None
    for leaf, wf, win in itertools.product(leaf_sizes, wavefronts, windows):
        if leaf != current_leaf:
            for r in renderers:
                r.build_bvh(sah_bins, leaf)
            current_leaf = leaf
        runner.set_params(wavefront=wf, batch_window=win)
        for r, s in zip(renderers, states):
            r.set_state(s)
        _, st = render_events_batch(runner, [(r, pair[0], pair[1]) for r in renderers], schedule["C"],
                                    schedule["alpha"], schedule["spp_batch"], schedule["spp_max"])
        trials.append({"max_leaf": leaf, "wavefront": wf, "batch_window": win, "gpu_ms": st["gpu_ms"]})
    best = min(trials, key=lambda t: t["gpu_ms"])
    if best["max_leaf"] != current_leaf:
        for r in renderers:
            r.build_bvh(sah_bins, best["max_leaf"])
    runner.set_params(wavefront=best["wavefront"], batch_window=best["batch_window"])
    for r, s in zip(renderers, states):
        r.set_state(s)
    return {"best": best, "trials": trials}
