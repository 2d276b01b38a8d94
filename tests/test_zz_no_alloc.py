"""mcev_detect_batch_static, the allocation-free detector step, against
mcev_render_events.

The step exists for callers that cannot have device memory allocated on
their behalf (a renderer inside a host application that owns the GPU's
memory, or a real-time loop that cannot afford the device-wide
synchronisation of cudaMalloc/cudaFree).  Such a caller brings its own path
samples and per-pixel state buffers; the step keeps its scratch in a fixed
array inside the library.  This test is that caller: it takes the samples
from mcev_trace_samples and its buffers from torch, runs the step batch
after batch for two frames in a row, and must end with the same event,
sample-count and mean maps as mcev_render_events."""
import ctypes as C

import pytest
import torch

import scenegen as sg
from paper_2408_07996_gb300 import _lib as L
from parity import renderer_for

pytestmark = pytest.mark.gpu

MEAN_TOL = 1e-4   # the per-pixel mean tolerance of the parity tests


def _step(args: L.DetectArgs):
    n = C.c_int64(-1)
    msg = C.create_string_buffer(512)
    args.err_msg = C.cast(msg, C.c_char_p)
    args.err_len = len(msg)
    status = L.load().mcev_detect_batch_static(C.byref(args), C.byref(n))
    return status, n.value, msg.value.decode()


def _p(t):
    return C.c_void_p(t.data_ptr())


def test_static_step_reproduces_render_events_two_frames():
    w = sg.workload("cornell64")
    frames = [(0.0, 1.0), (1.0, 2.0)]
    H, W = w.height, w.width
    n_all = H * W

    ra = renderer_for(w)
    expect = []
    for t0, t1 in frames:
        o = ra.render_events(t0, t1, w.C, w.alpha, w.spp_batch, w.spp_max)
        expect.append({k: o[k].reshape(-1).clone() for k in ("events", "spp", "mean")})
    ra.close()

    rb = renderer_for(w)
    rb.render_reference(frames[0][0], w.spp_max)
    cnt, mean, m2 = rb.reference_arrays()
    dev = rb.device
    ref = [cnt.reshape(-1).clone(), mean.reshape(-1).clone(), m2.reshape(-1).clone()]
    cur = [torch.zeros(n_all, dtype=torch.int32, device=dev), torch.zeros(n_all, device=dev),
           torch.zeros(n_all, device=dev)]
    stream = torch.cuda.current_stream(dev).cuda_stream
    calls = 0
    for (t0, t1), exp in zip(frames, expect):
        ev = torch.full((n_all,), 7, dtype=torch.int8, device=dev)
        spp = torch.zeros(n_all, dtype=torch.int32, device=dev)
        mo = torch.zeros(n_all, device=dev)
        queue = torch.arange(n_all, dtype=torch.int32, device=dev)
        k = 0
        while queue.numel() > 0:
            spp_r = w.spp_min if k == 0 else min(w.spp_batch, w.spp_max - k)
            samples, _ = rb.trace_samples(t1, queue, k, spp_r, want_sig=False)
            undecided = torch.empty_like(queue)
            args = L.DetectArgs(L=_p(samples), pixels=_p(queue), n_pix=queue.numel(), n_total=n_all,
                                spp_r=spp_r, reserved0=0, k_base=k,
                                cur_n=_p(cur[0]), cur_mean=_p(cur[1]), cur_m2=_p(cur[2]),
                                ref_n=_p(ref[0]), ref_mean=_p(ref[1]), ref_m2=_p(ref[2]),
                                events=_p(ev), spp_out=_p(spp), mean_out=_p(mo), undecided=_p(undecided),
                                eps=w.eps, C=w.C, alpha=w.alpha, spp_min=w.spp_min, spp_batch=w.spp_batch,
                                spp_max=w.spp_max, variant=L.ONE_TAILED, se_mode=L.SE_PAPER,
                                stream=C.c_void_p(stream))
            status, n_und, msg = _step(args)
            assert status == 0, msg
            assert 0 <= n_und <= queue.numel()
            calls += 1
            queue = undecided[:n_und].clone()
            k += spp_r
        assert not (ev == 7).any(), "every pixel is decided exactly once per frame"
        assert torch.equal(ev, exp["events"])
        assert torch.equal(spp, exp["spp"])
        assert (mo - exp["mean"]).abs().max().item() <= MEAN_TOL
    assert calls > 2
    rb.close()


def test_static_step_rejects_schedules_beyond_its_scratch():
    dummy = torch.zeros(16, dtype=torch.int32, device="cuda")
    f = torch.zeros(16, device="cuda")
    args = L.DetectArgs(L=_p(f), pixels=_p(dummy), n_pix=16, n_total=16, spp_r=2, reserved0=0, k_base=0,
                        cur_n=_p(dummy), cur_mean=_p(f), cur_m2=_p(f), ref_n=_p(dummy), ref_mean=_p(f),
                        ref_m2=_p(f), events=_p(dummy), spp_out=None, mean_out=None, undecided=_p(dummy),
                        eps=1e-3, C=0.2, alpha=0.05, spp_min=2, spp_batch=1, spp_max=5000,
                        variant=L.ONE_TAILED, se_mode=L.SE_PAPER, stream=None)
    status, _, msg = _step(args)
    assert status == -1 and "4096" in msg
