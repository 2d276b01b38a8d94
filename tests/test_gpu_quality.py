"""Event-video quality metrics on the GPU (mcev_event_quality) against the
FP64 oracle (oracle/quality.py): integer counts and every per-event squared
distance bit-exact, distance sums and the derived metrics to 1e-12
relative.  Shapes span ragged rows (W not a multiple of 32), single rows,
single frames, a single voxel, empty and one-polarity videos; the
1280x720x100 case is checked on sampled events against an exact
nearest-neighbour search."""
import math

import numpy as np
import pytest
import torch

import scenegen as sg
from oracle import quality as Q

pytestmark = pytest.mark.gpu

EXACT = ("voxels", "n_a", "n_b", "matched_a", "matched_b", "sq_diff")
CLOSE = ("sum_dist_a", "sum_dist_b", "diag", "rmse", "psnr", "precision", "recall", "f1", "pscd")


def _gpu(a, b, tau2=3, want_d2=True):
    from paper_2408_07996_gb300.api import event_quality
    return event_quality(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), tau2, want_d2)


def _d2_at_points(d2_vol, v):
    """GPU per-voxel distances at the oracle's point order (-2 -> -1)."""
    idx = np.argwhere(v != 0)
    d = d2_vol.cpu().numpy()[idx[:, 0], idx[:, 1], idx[:, 2]].astype(np.int64)
    return np.where(d == -2, -1, d)


def _compare(a, b, tau2=3):
    g = _gpu(a, b, tau2)
    o = Q.quality(a, b, tau2)
    for k in EXACT:
        assert g[k] == o[k], k
    for k in CLOSE:
        if math.isinf(o[k]):
            assert math.isinf(g[k]) and g[k] > 0, k
        else:
            assert g[k] == pytest.approx(o[k], rel=1e-12, abs=1e-300), k
    np.testing.assert_array_equal(_d2_at_points(g["d2_a"], a), o["d2_a"])
    np.testing.assert_array_equal(_d2_at_points(g["d2_b"], b), o["d2_b"])
    # voxels without an event are -1
    assert np.all(g["d2_a"].cpu().numpy()[a == 0] == -1)
    return g, o


@pytest.mark.parametrize("shape,seed", [((10, 64, 96), 1), ((7, 33, 70), 2), ((1, 45, 61), 3), ((5, 1, 200), 4),
                                        ((12, 40, 1), 5), ((3, 130, 257), 6),
                                        # long columns and many frames
                                        ((2, 300, 40), 7), ((260, 8, 12), 8)])
def test_quality_parity(shape, seed):
    T, H, W = shape
    a, b = sg.event_video_pair(W, H, T, seed=seed, move=0.1, noise=1e-3)
    g, o = _compare(a, b)
    print(shape, {k: g[k] for k in ("n_a", "matched_a", "f1", "pscd", "rmse")})
    _compare(b, a, tau2=1)
    _compare(a, b, tau2=0)


def test_quality_degenerate_cases():
    z = np.zeros((4, 9, 11), np.int8)
    a, _ = sg.event_video_pair(11, 9, 4, seed=8)
    pos = np.where(a > 0, a, 0).astype(np.int8)
    for x, y in [(z, z), (z, a), (a, z), (pos, a), (a, -a), (a, a)]:
        _compare(x, y)
    one = np.ones((1, 1, 1), np.int8)
    g, _ = _compare(one, -one)
    assert g["diag"] == 0.0 and g["pscd"] == 0.0


def test_quality_rejects_bad_values_and_extents():
    from paper_2408_07996_gb300._lib import McevError
    from paper_2408_07996_gb300.api import event_quality
    a = torch.zeros(2, 3, 4, dtype=torch.int8, device="cuda")
    b = a.clone()
    b[1, 2, 3] = 2
    with pytest.raises(McevError, match="ARG"):
        event_quality(a, b)
    with pytest.raises(McevError, match="ARG"):
        event_quality(a, a, tau2=-1)
    big = torch.zeros(1, 1, 16385, dtype=torch.int8, device="cuda")
    with pytest.raises(McevError, match="ARG"):
        event_quality(big, big)
    assert event_quality(a, a)["f1"] == 1.0


def test_quality_unaligned_inputs():
    a, b = sg.event_video_pair(37, 21, 5, seed=9)
    ta = torch.zeros(a.size + 3, dtype=torch.int8, device="cuda")
    tb = torch.zeros(b.size + 5, dtype=torch.int8, device="cuda")
    ta[3:] = torch.from_numpy(a.reshape(-1)).cuda()
    tb[5:] = torch.from_numpy(b.reshape(-1)).cuda()
    from paper_2408_07996_gb300.api import event_quality
    g = event_quality(ta[3:].view(a.shape), tb[5:].view(b.shape))
    o = Q.quality(a, b)
    for k in EXACT:
        assert g[k] == o[k]
    assert g["pscd"] == pytest.approx(o["pscd"], rel=1e-12)


@pytest.mark.slow
def test_quality_full_size_sampled():
    """1280x720, 100 frames (92M voxels, the terrain benchmark's frame size
    over its 100 keyframes): totals exact; 3000 sampled events per video
    against an exact nearest-neighbour search."""
    spatial = pytest.importorskip("scipy.spatial")
    T, H, W = 100, 720, 1280
    a, b = sg.event_video_pair(W, H, T, seed=11)
    g = _gpu(a, b)
    assert g["n_a"] == int(np.count_nonzero(a)) and g["n_b"] == int(np.count_nonzero(b))
    assert g["sq_diff"] == int(np.sum((a.astype(np.int64) - b.astype(np.int64)) ** 2))
    rng = np.random.default_rng(12)
    for src, dst, d2 in ((a, b, g["d2_a"]), (b, a, g["d2_b"])):
        ps, qs = Q.signed_points(src)
        pd, qd = Q.signed_points(dst)
        pick = rng.choice(ps.shape[0], size=3000, replace=False)
        want = np.full(pick.size, -1, np.int64)
        for pol in (-1, 1):
            sel = qs[pick] == pol
            if not np.any(qd == pol) or not np.any(sel):
                continue
            tree = spatial.cKDTree(pd[qd == pol].astype(np.float64))
            dist, _ = tree.query(ps[pick][sel].astype(np.float64), k=1)
            want[sel] = np.rint(dist ** 2).astype(np.int64)
        x, y, t = ps[pick, 0], ps[pick, 1], ps[pick, 2]
        got = d2[torch.from_numpy(t).cuda(), torch.from_numpy(y).cuda(), torch.from_numpy(x).cuda()]
        got = got.cpu().numpy().astype(np.int64)
        np.testing.assert_array_equal(np.where(got == -2, -1, got), want)
    print("full size", {k: g[k] for k in ("n_a", "f1", "pscd", "rmse", "gpu_ms")})
