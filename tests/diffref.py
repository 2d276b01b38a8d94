"""Reference gradients for the differentiable-rendering tests: central finite
differences of the FP64 oracle's per-pixel mean log luminance (the plain
definition of the derivative of the Monte Carlo estimate with its random
numbers held fixed), and the textured-plane closed form."""
import math

import numpy as np

import oracle as O

Y709 = np.array([0.2126, 0.7152, 0.0722])


def oracle_means(osc, p, t, pixels, spp, eps):
    """FP64 per-pixel mean of ln(L + eps) over samples 0..spp-1."""
    L, _ = O.trace_samples(osc, p, t, np.ascontiguousarray(pixels, np.int32), 0, spp)
    return np.log(L + eps).mean(axis=1)


def texel_fd(osc, texture, loss_of_means, texels, h):
    """Central differences of loss_of_means() with respect to the luminance
    of each texel (iy, ix): all three channels move by +-h, and the step is
    measured on the float32 values the oracle actually sees."""
    out = np.zeros(len(texels))
    for i, (iy, ix) in enumerate(texels):
        vals = []
        lum = []
        for s in (+1.0, -1.0):
            tp = texture.copy()
            tp[iy, ix, :] = (tp[iy, ix, :].astype(np.float64) + s * h).astype(np.float32)
            lum.append(float(Y709 @ tp[iy, ix, :].astype(np.float64)))
            osc.set_texture(tp)
            vals.append(loss_of_means())
        out[i] = (vals[0] - vals[1]) / (lum[0] - lum[1])
    osc.set_texture(texture)
    return out


def emission_fd(osc, emission, loss_of_means, mats, h):
    out = np.zeros(len(mats))
    for i, m in enumerate(mats):
        vals, step = [], []
        for s in (+1.0, -1.0):
            e = np.asarray(emission, np.float32).copy()
            e[m] = np.float32(float(e[m]) + s * h)
            step.append(float(e[m]))
            osc.set_emission(e)
            vals.append(loss_of_means())
        out[i] = (vals[0] - vals[1]) / (step[0] - step[1])
    osc.set_emission(np.asarray(emission, np.float32))
    return out


def plane_hit_texel(o, d, repeat, half, tw, th):
    """Texel (iy, ix) under the camera ray (o, d) on sg.textured_plane."""
    s = -o[1] / d[1]
    x, z = o[0] + s * d[0], o[2] + s * d[2]
    if not (abs(x) < half and abs(z) < half):
        return None                                   # off the plane
    u = repeat * (x + half) / (2.0 * half)
    v = repeat * (z + half) / (2.0 * half)
    u -= math.floor(u)
    v -= math.floor(v)
    return min(int(v * th), th - 1), min(int(u * tw), tw - 1)


def single_texel_pixels(osc, p, width, height, repeat, half, tw, th):
    """Pixels whose whole footprint (the four film corners) lands in one
    texel of sg.textured_plane: pixel index -> (iy, ix)."""
    out = {}
    for y in range(height):
        for x in range(width):
            cells = set()
            for fx, fy in ((x, y), (x + 1, y), (x, y + 1), (x + 1, y + 1)):
                o, d = osc.camera_ray(p, 0.0, fx, fy)
                cells.add(plane_hit_texel(o, d, repeat, half, tw, th))
            if len(cells) == 1 and None not in cells:
                out[y * width + x] = cells.pop()
    return out
