"""Quality metrics of event videos (Sec. 4.2), plain FP64 definitions.

TEST INFRASTRUCTURE ONLY (same rule as the rest of `oracle/`).

The paper scores an event video against the baseline's with four metrics
taken from Tsuji et al.: RMSE and PSNR of the event frames with negative,
null and positive events stored as 0, 0.5 and 1; and an F1 score and a
chamfer distance ("PSCD") of signed point clouds, each event becoming a
point (q_x, q_y, t) with its polarity.  Tsuji et al.'s exact thresholds and
normalisation are not given; the readings here are:

* the video is an int8 array [T][H][W] of {-1, 0, +1}; point coordinates
  are lattice units (pixel column, pixel row, frame index);
* MSE is over all T*H*W values of the mapped frames; RMSE = sqrt(MSE),
  PSNR = -10 log10(MSE) (peak 1; +inf for identical videos);
* d(a, B) is the Euclidean distance from point a to the nearest point of B
  with the same polarity; if B has none, the lattice diagonal
  D = sqrt((W-1)^2 + (H-1)^2 + (T-1)^2);
* a point is matched when d^2 <= tau2 (default 3: any of the 26 lattice
  neighbours in space and time); precision = matched A / |A|, recall =
  matched B / |B| (1 for an empty cloud), F1 = 2PR / (P + R) (0 if both 0);
* PSCD = (mean_a d(a, B) + mean_b d(b, A)) / (2 D) (an empty cloud's mean
  is 0; PSCD = 0 when D = 0).

Nearest neighbours are brute force over all same-polarity points.
"""
from __future__ import annotations

import math

import numpy as np


def frame_error(a: np.ndarray, b: np.ndarray):
    """(sum of squared differences of the raw values, MSE, RMSE, PSNR) of
    two event videos after mapping {-1, 0, 1} -> {0, 0.5, 1}."""
    fa = (a.astype(np.float64) + 1.0) / 2.0
    fb = (b.astype(np.float64) + 1.0) / 2.0
    mse = float(np.mean((fa - fb) ** 2))
    sq = int(np.sum((a.astype(np.int64) - b.astype(np.int64)) ** 2))
    rmse = math.sqrt(mse)
    psnr = math.inf if mse == 0.0 else -10.0 * math.log10(mse)
    return sq, mse, rmse, psnr


def signed_points(v: np.ndarray):
    """Points (x, y, t) as int64 [N, 3] and polarities int8 [N], in
    t-major, then row, then column order."""
    idx = np.argwhere(v != 0)                      # (t, y, x)
    pts = idx[:, ::-1].astype(np.int64)            # (x, y, t)
    pol = v[idx[:, 0], idx[:, 1], idx[:, 2]].astype(np.int8)
    return pts, pol


def nearest_sq(pa, qa, pb, qb, chunk: int = 256):
    """Squared distance from every point of (pa, qa) to the nearest point of
    (pb, qb) with the same polarity; -1 where there is none."""
    out = np.full(pa.shape[0], -1, np.int64)
    for pol in (-1, 1):
        ia = np.nonzero(qa == pol)[0]
        B = pb[qb == pol]
        if ia.size == 0 or B.shape[0] == 0:
            continue
        for s in range(0, ia.size, chunk):
            A = pa[ia[s:s + chunk]]
            best = np.full(A.shape[0], np.iinfo(np.int64).max, np.int64)
            for t in range(0, B.shape[0], 8192):
                d = A[:, None, :] - B[None, t:t + 8192, :]
                best = np.minimum(best, np.einsum("ijk,ijk->ij", d, d).min(axis=1))
            out[ia[s:s + chunk]] = best
    return out


def diagonal(shape) -> float:
    T, H, W = shape
    return math.sqrt((W - 1) ** 2 + (H - 1) ** 2 + (T - 1) ** 2)


def quality(a: np.ndarray, b: np.ndarray, tau2: int = 3) -> dict:
    """All four metrics of video `a` (e.g. adaptive) against `b` (e.g. the
    uniform baseline), plus the integer counts and distance sums they come
    from.  d2_a / d2_b: squared distance per point (-1: no same-polarity
    point in the other cloud), in signed_points order."""
    assert a.shape == b.shape and a.ndim == 3
    sq, mse, rmse, psnr = frame_error(a, b)
    D = diagonal(a.shape)
    pa, qa = signed_points(a)
    pb, qb = signed_points(b)
    d2a = nearest_sq(pa, qa, pb, qb)
    d2b = nearest_sq(pb, qb, pa, qa)

    def dist(d2):
        return np.where(d2 >= 0, np.sqrt(np.maximum(d2, 0).astype(np.float64)), D)

    ma = int(np.sum((d2a >= 0) & (d2a <= tau2)))
    mb = int(np.sum((d2b >= 0) & (d2b <= tau2)))
    P = ma / pa.shape[0] if pa.shape[0] else 1.0
    R = mb / pb.shape[0] if pb.shape[0] else 1.0
    f1 = 2.0 * P * R / (P + R) if P + R > 0 else 0.0
    sda = float(dist(d2a).sum())
    sdb = float(dist(d2b).sum())
    mean_a = sda / pa.shape[0] if pa.shape[0] else 0.0
    mean_b = sdb / pb.shape[0] if pb.shape[0] else 0.0
    pscd = (mean_a + mean_b) / (2.0 * D) if D > 0 else 0.0
    return dict(voxels=a.size, n_a=int(pa.shape[0]), n_b=int(pb.shape[0]), matched_a=ma, matched_b=mb,
                sq_diff=sq, sum_dist_a=sda, sum_dist_b=sdb, diag=D, rmse=rmse, psnr=psnr, precision=P,
                recall=R, f1=f1, pscd=pscd, d2_a=d2a, d2_b=d2b)
