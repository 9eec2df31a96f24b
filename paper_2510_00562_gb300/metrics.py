"""Image-quality metrics of Sec. IV-A: MPSNR (Eq. 29) and MSSIM (Eq. 30).

Cubes are (N3, N1, N2) arrays (band, row, column); both metrics are computed
per band in float64 and averaged over the bands.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["mpsnr", "mssim", "ssim_band"]


def mpsnr(u, u_ref):
    """Eq. 29: mean over bands of 10 log10(N1 N2 / ||u_b - u_ref_b||^2) (peak 1).

    A band that matches exactly has infinite PSNR; such bands are left out of
    the mean, and if every band matches the result is +inf.
    """
    u = np.asarray(u, dtype=np.float64)
    r = np.asarray(u_ref, dtype=np.float64)
    n3 = u.shape[0]
    npix = u.shape[1] * u.shape[2]
    err = ((u - r) ** 2).reshape(n3, -1).sum(axis=1)
    vals = [10.0 * math.log10(npix / e) for e in err if e > 0]
    return float(np.mean(vals)) if vals else math.inf


def _gauss_window(size=11, sigma=1.5):
    ax = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-0.5 * (ax / sigma) ** 2)
    g /= g.sum()
    return g


def _filter_valid(x, g):
    """Separable 'valid' correlation of a 2-D array with the 1-D window g."""
    k = g.size
    rows = np.lib.stride_tricks.sliding_window_view(x, k, axis=0) @ g     # (n1-k+1, n2)
    return np.lib.stride_tricks.sliding_window_view(rows, k, axis=1) @ g  # (n1-k+1, n2-k+1)


def ssim_band(x, y, data_range=1.0, k1=0.01, k2=0.03, size=11, sigma=1.5):
    """SSIM of one band (Wang et al. 2004): Gaussian 11x11 window, sigma 1.5,
    K1 = 0.01, K2 = 0.03, mean over the region where the window fits.

    The paper cites Wang 2004 without its constants; these are the ones of
    that reference.  Bands smaller than the window use the whole band as one
    window.
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    c1 = (k1 * data_range) ** 2
    c2 = (k2 * data_range) ** 2
    if min(x.shape) < size:
        mx, my = x.mean(), y.mean()
        vx, vy = x.var(), y.var()
        cxy = ((x - mx) * (y - my)).mean()
        return float(((2 * mx * my + c1) * (2 * cxy + c2)) / ((mx * mx + my * my + c1) * (vx + vy + c2)))
    g = _gauss_window(size, sigma)
    mx = _filter_valid(x, g)
    my = _filter_valid(y, g)
    sxx = _filter_valid(x * x, g) - mx * mx
    syy = _filter_valid(y * y, g) - my * my
    sxy = _filter_valid(x * y, g) - mx * my
    num = (2 * mx * my + c1) * (2 * sxy + c2)
    den = (mx * mx + my * my + c1) * (sxx + syy + c2)
    return float(np.mean(num / den))


def mssim(u, u_ref, **kw):
    """Eq. 30: mean over bands of SSIM(u_b, u_ref_b)."""
    return float(np.mean([ssim_band(u[b], u_ref[b], **kw) for b in range(u.shape[0])]))
