"""mcev_detect_batch_static, the allocation-free detector step, against
mcev_render_events.

The step exists for callers that cannot have device memory allocated on
their behalf (a renderer inside a host application that owns the GPU's
memory, or a real-time loop that cannot afford the device-wide
synchronisation of cudaMalloc/cudaFree).  Such a caller brings its own path
samples and per-pixel state buffers; the step keeps its scratch in a fixed
array inside the library.  This test is that caller: it takes the samples
from mcev_trace_samples and its buffers from torch, runs the step window
after window for two frames in a row, and must end with the same event,
sample-count and mean maps as mcev_render_events.  Around every step call
after the first it also checks that no device memory was allocated."""
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


def _mem():
    """Device memory as this process and the driver see it."""
    torch.cuda.synchronize()
    st = torch.cuda.memory_stats()
    return (torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated(), st.get("allocation.all.allocated", 0),
            st.get("segment.all.allocated", 0))


def _args(w, variant, samples, queue, n_all, spp_r, k, cur, ref, ev, spp, mo, undecided, stream):
    return L.DetectArgs(L=_p(samples), pixels=_p(queue), n_pix=queue.numel(), n_total=n_all,
                        spp_r=spp_r, reserved0=0, k_base=k,
                        cur_n=_p(cur[0]), cur_mean=_p(cur[1]), cur_m2=_p(cur[2]),
                        ref_n=_p(ref[0]), ref_mean=_p(ref[1]), ref_m2=_p(ref[2]),
                        events=_p(ev), spp_out=_p(spp), mean_out=_p(mo), undecided=_p(undecided),
                        eps=w.eps, C=w.C, alpha=w.alpha, spp_min=w.spp_min, spp_batch=w.spp_batch,
                        spp_max=w.spp_max, variant=variant, se_mode=L.SE_PAPER, stream=C.c_void_p(stream))


@pytest.mark.parametrize("variant,window", [(L.ONE_TAILED, 1), (L.ONE_TAILED, 2), (L.TWO_TAILED, 3)])
def test_static_step_reproduces_render_events_two_frames(variant, window):
    """`window` batches of spp_batch per call after the first batch; every
    schedule point inside a window is still tested."""
    w = sg.workload("cornell64")
    frames = [(0.0, 1.0), (1.0, 2.0)]
    H, W = w.height, w.width
    n_all = H * W

    ra = renderer_for(w, variant=variant)
    expect = []
    for t0, t1 in frames:
        o = ra.render_events(t0, t1, w.C, w.alpha, w.spp_batch, w.spp_max)
        expect.append({k: o[k].reshape(-1).clone() for k in ("events", "spp", "mean")})
    ra.close()

    rb = renderer_for(w, variant=variant)
    rb.render_reference(frames[0][0], w.spp_max)
    cnt, mean, m2 = rb.reference_arrays()
    dev = rb.device
    ref = [cnt.reshape(-1).clone(), mean.reshape(-1).clone(), m2.reshape(-1).clone()]
    cur = [torch.zeros(n_all, dtype=torch.int32, device=dev), torch.zeros(n_all, device=dev),
           torch.zeros(n_all, device=dev)]
    stream = torch.cuda.current_stream(dev).cuda_stream
    calls = 0
    mem_checked = 0
    for (t0, t1), exp in zip(frames, expect):
        ev = torch.full((n_all,), 7, dtype=torch.int8, device=dev)
        spp = torch.zeros(n_all, dtype=torch.int32, device=dev)
        mo = torch.zeros(n_all, device=dev)
        queue = torch.arange(n_all, dtype=torch.int32, device=dev)
        k = 0
        while queue.numel() > 0:
            spp_r = w.spp_min if k == 0 else min(window * w.spp_batch, w.spp_max - k)
            samples, _ = rb.trace_samples(t1, queue, k, spp_r, want_sig=False)
            undecided = torch.empty_like(queue)
            args = _args(w, variant, samples, queue, n_all, spp_r, k, cur, ref, ev, spp, mo, undecided, stream)
            before = _mem() if calls > 0 else None
            status, n_und, msg = _step(args)
            if before is not None:
                assert _mem() == before, "the allocation-free step changed device memory"
                mem_checked += 1
            assert status == 0, msg
            assert 0 <= n_und <= queue.numel()
            calls += 1
            queue = undecided[:n_und].clone()
            k += spp_r
        assert not (ev == 7).any(), "every pixel is decided exactly once per frame"
        assert torch.equal(ev, exp["events"])
        assert torch.equal(spp, exp["spp"])
        assert (mo - exp["mean"]).abs().max().item() <= MEAN_TOL
    assert calls > 2 and mem_checked == calls - 1
    rb.close()


def _first_batch_fixture():
    """Buffers of a 64x64 Cornell frame after its reference, ready for the
    first window of the t1 frame."""
    w = sg.workload("cornell64")
    n_all = w.width * w.height
    r = renderer_for(w)
    r.render_reference(0.0, w.spp_max)
    cnt, mean, m2 = r.reference_arrays()
    dev = r.device
    ref = [cnt.reshape(-1).clone(), mean.reshape(-1).clone(), m2.reshape(-1).clone()]
    cur = [torch.zeros(n_all, dtype=torch.int32, device=dev), torch.zeros(n_all, device=dev),
           torch.zeros(n_all, device=dev)]
    outs = (torch.full((n_all,), 7, dtype=torch.int8, device=dev), torch.zeros(n_all, dtype=torch.int32, device=dev),
            torch.zeros(n_all, device=dev))
    return w, r, n_all, ref, cur, outs, torch.cuda.current_stream(dev).cuda_stream


def test_static_step_rejects_off_schedule_windows():
    w, r, n_all, ref, cur, (ev, spp, mo), stream = _first_batch_fixture()
    queue = torch.arange(n_all, dtype=torch.int32, device=r.device)
    samples, _ = r.trace_samples(1.0, queue, 0, w.spp_min, want_sig=False)
    und = torch.empty_like(queue)
    status, n_und, msg = _step(_args(w, L.ONE_TAILED, samples, queue, n_all, w.spp_min, 0, cur, ref, ev, spp, mo,
                                     und, stream))
    assert status == 0, msg
    q = und[:n_und].clone()
    assert q.numel() > 0
    more, _ = r.trace_samples(1.0, q, w.spp_min, 2 * w.spp_batch + 1, want_sig=False)
    und2 = torch.empty_like(q)
    bad = [
        (w.spp_min + 1, w.spp_batch),          # k_base between two test points
        (w.spp_min - 2, w.spp_batch),          # k_base below spp_min
        (w.spp_min, w.spp_batch + 1),          # a partial batch that does not end at spp_max
        (w.spp_min, 2 * w.spp_batch + 1),
    ]
    snap = [t.clone() for t in cur + [ev, spp, mo]]
    for k_base, spp_r in bad:
        status, _, msg = _step(_args(w, L.ONE_TAILED, more, q, n_all, spp_r, k_base, cur, ref, ev, spp, mo, und2,
                                     stream))
        assert status == -1 and "schedule" in msg, (k_base, spp_r, msg)
    # a refused call touches nothing
    for a, b in zip(snap, cur + [ev, spp, mo]):
        assert torch.equal(a, b)
    r.close()


def test_static_step_skips_out_of_range_pixel_ids():
    """An id outside [0, n_total) is skipped by the kernel's own range check
    (nothing is read or written for it) and the call reports MCEV_ERR_ARG;
    every other listed pixel is processed as without the bad id."""
    w, r, n_all, ref, cur, (ev, spp, mo), stream = _first_batch_fixture()
    dev = r.device
    queue = torch.arange(n_all, dtype=torch.int32, device=dev)
    samples, _ = r.trace_samples(1.0, queue, 0, w.spp_min, want_sig=False)
    und = torch.empty_like(queue)
    good = [t.clone() for t in cur], [t.clone() for t in ref], [t.clone() for t in (ev, spp, mo)]
    status, n_good, msg = _step(_args(w, L.ONE_TAILED, samples, queue, n_all, w.spp_min, 0, good[0], good[1],
                                      *good[2], und, stream))
    assert status == 0, msg
    und_good = und[:n_good].clone()
    # the same call with pixel 5's id replaced by n_total (its samples stay in place)
    q_bad = queue.clone()
    q_bad[5] = n_all
    und_b = torch.empty_like(queue)
    status, n_bad, msg = _step(_args(w, L.ONE_TAILED, samples, q_bad, n_all, w.spp_min, 0, cur, ref, ev, spp, mo,
                                     und_b, stream))
    assert status == -1 and "outside" in msg
    keep = torch.ones(n_all, dtype=torch.bool, device=dev)
    keep[5] = False
    for a, b in zip(good[0] + good[1] + good[2], cur + ref + [ev, spp, mo]):
        assert torch.equal(a[keep], b[keep])
    assert cur[0][5].item() == 0 and ev[5].item() == 7
    expect_und = und_good[und_good != 5]
    assert n_bad == expect_und.numel()
    assert torch.equal(torch.sort(und_b[:n_bad]).values, torch.sort(expect_und).values)
    r.close()


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
