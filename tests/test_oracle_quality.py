"""Pins of the quality-metric oracle (Sec. 4.2 metrics, readings in
oracle/quality.py): closed forms of the frame error, a hand-computed point
cloud, scipy's exact Euclidean distance transform (the nearest same-polarity
event of B at each event of A), and the invariants of the definitions."""
import math

import numpy as np
import pytest

import scenegen as sg
from oracle import quality as Q


def test_frame_error_closed_forms():
    z = np.zeros((2, 3, 4), np.int8)
    p = np.ones_like(z)
    assert Q.frame_error(z, z)[1:] == (0.0, 0.0, math.inf)
    sq, mse, rmse, psnr = Q.frame_error(p, -p)
    assert (sq, mse, rmse, psnr) == (4 * 24, 1.0, 1.0, 0.0)
    sq, mse, rmse, psnr = Q.frame_error(z, p)
    assert (sq, rmse) == (24, 0.5) and psnr == pytest.approx(20 * math.log10(2), rel=1e-15)
    one = z.copy()
    one[1, 2, 3] = -1
    assert Q.frame_error(one, z)[2] == pytest.approx(math.sqrt(0.25 / 24), rel=1e-15)
    assert Q.frame_error(one, -one)[2] == pytest.approx(math.sqrt(1.0 / 24), rel=1e-15)


def test_hand_computed_clouds():
    # video [T=2][H=3][W=4]; points written as (x, y, t, polarity)
    a = np.zeros((2, 3, 4), np.int8)
    b = np.zeros_like(a)
    a[0, 0, 0] = 1          # (0,0,0,+): nearest B+ is (1,1,1): d^2 = 3  -> matched at tau2 = 3
    a[1, 2, 3] = 1          # (3,2,1,+): nearest B+ is (1,1,1): d^2 = 4+1 = 5, or (3,0,0): 4+1 = 5
    a[0, 2, 0] = -1         # (0,2,0,-): B has no negative point -> d = D
    b[1, 1, 1] = 1
    b[0, 0, 3] = 1          # (3,0,0,+): nearest A+ is (0,0,0): 9, or (3,2,1): 4+1 = 5
    r = Q.quality(a, b, tau2=3)
    D = math.sqrt(9 + 4 + 1)
    assert r["diag"] == D
    # signed_points order is t, then row, then column: (0,0,0) (0,2,0) (3,2,1) for a
    assert list(r["d2_a"]) == [3, -1, 5]
    assert list(r["d2_b"]) == [5, 3]          # (3,0,0) then (1,1,1)
    assert (r["n_a"], r["n_b"], r["matched_a"], r["matched_b"]) == (3, 2, 1, 1)
    assert r["precision"] == pytest.approx(1 / 3) and r["recall"] == pytest.approx(1 / 2)
    assert r["f1"] == pytest.approx(2 * (1 / 3) * (1 / 2) / (1 / 3 + 1 / 2))
    sda = math.sqrt(3) + D + math.sqrt(5)
    sdb = math.sqrt(5) + math.sqrt(3)
    assert r["sum_dist_a"] == pytest.approx(sda, rel=1e-15)
    assert r["pscd"] == pytest.approx((sda / 3 + sdb / 2) / (2 * D), rel=1e-15)
    assert Q.quality(a, b, tau2=4)["matched_a"] == 1
    assert Q.quality(a, b, tau2=5)["matched_a"] == 2


@pytest.mark.parametrize("shape,seed", [((7, 40, 56), 1), ((3, 17, 90), 2)])
def test_nearest_distances_match_scipy_edt(shape, seed):
    ndimage = pytest.importorskip("scipy.ndimage")
    a, b = sg.event_video_pair(shape[2], shape[1], shape[0], seed=seed, move=0.2, noise=1e-3)
    r = Q.quality(a, b)
    pa, qa = Q.signed_points(a)
    want = np.full(pa.shape[0], -1, np.int64)
    for pol in (-1, 1):
        if not np.any(b == pol):
            continue
        edt = ndimage.distance_transform_edt(b != pol)     # distance to the nearest b == pol voxel
        sel = qa == pol
        x, y, t = pa[sel, 0], pa[sel, 1], pa[sel, 2]
        want[sel] = np.rint(edt[t, y, x] ** 2).astype(np.int64)
    np.testing.assert_array_equal(r["d2_a"], want)


def test_invariants():
    a, b = sg.event_video_pair(48, 32, 6, seed=4)
    r = Q.quality(a, b)
    s = Q.quality(b, a)
    assert (s["precision"], s["recall"]) == (r["recall"], r["precision"])
    assert s["f1"] == pytest.approx(r["f1"], rel=1e-15) and s["pscd"] == pytest.approx(r["pscd"], rel=1e-15)
    f = Q.quality(-a, -b)
    for k in ("matched_a", "matched_b", "sq_diff", "f1", "pscd", "rmse"):
        assert f[k] == r[k]
    same = Q.quality(a, a)
    assert (same["f1"], same["pscd"], same["rmse"], same["sum_dist_a"]) == (1.0, 0.0, 0.0, 0.0)
    # a video one frame late: every event that stays in range is one lattice step away
    late = np.zeros_like(a)
    late[1:] = a[:-1]
    d = Q.quality(a, late)
    assert set(np.unique(d["d2_b"])) <= {0, 1}
    z = np.zeros_like(a)
    e = Q.quality(z, z)
    assert (e["precision"], e["recall"], e["f1"], e["pscd"]) == (1.0, 1.0, 1.0, 0.0)
    h = Q.quality(z, a)
    assert (h["precision"], h["recall"], h["f1"]) == (1.0, 0.0, 0.0)
    assert h["pscd"] == pytest.approx(0.5, rel=1e-15)
