"""Seeded synthetic hyperspectral cubes shaped like the paper's scenes.

This module only draws inputs; it holds none of the method's arithmetic and
is shared by the tests, the benchmark and the oracle checks.

Observation model (Eq. 14): v = u_bar + s_bar + t_bar + n, with

* u_bar: a clean cube in [0, 1] made of ``n_regions`` polygonal spatial
  regions (Voronoi cells of uniform seeds, so edges run at all angles), each
  region carrying a smooth spectrum that is a sum of three Gaussians over the
  band index (centres U[0, N3), widths U[N3/12, N3/3], amplitudes U[0.2, 1]);
  the whole cube is min-max scaled to [0, 1];
* t_bar: vertical stripes -- on a fraction ``stripe_rate`` of the columns of
  every band, an offset U[-stripe_amp, stripe_amp] constant along the column
  (the noise types of Sec. IV-A, Cases 3 and 5);
* s_bar: sparse noise -- salt-and-pepper voxels (a fraction ``sp_rate``, set to
  0 or 1 with equal odds) and dead lines (in a fraction ``dead_band_rate`` of
  the bands, a dead line starts at a fraction ``dead_col_rate`` of the columns
  and covers a width drawn uniformly from 1..``dead_width_max`` columns, set
  to 0); s_bar is whatever makes v hit those values, so Eq. 14 holds exactly;
* n: Gaussian noise of standard deviation ``sigma`` on every voxel that is not
  replaced by salt-and-pepper or a dead line.

The order of application is not stated in the paper; this one keeps Eq. 14
exact and matches the (1 - p_s) factor of the fidelity radius (Eq. 27).

Arrays are returned C-contiguous in (N3, N1, N2) order (band, row, column),
``v`` and ``u_bar`` as float32 so that the CUDA path and the oracle read the
same bytes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = ["NoiseSpec", "clean_cube", "make_problem", "paper_case", "random_state"]


@dataclass
class NoiseSpec:
    sigma: float = 0.1
    sp_rate: float = 0.05
    stripe_rate: float = 0.05
    stripe_amp: float = 0.25
    dead_col_rate: float = 0.0
    dead_band_rate: float = 0.0
    dead_width_max: int = 1


def paper_case(k: int) -> NoiseSpec:
    """The simulated noise of Sec. IV-A, Cases 1-5: Gaussian sigma 0.1 (all
    cases), salt-and-pepper at rate 0.05 (Cases 2, 5), vertical stripes on 5 %
    of the columns with intensity U[-0.5, 0.5] (Cases 3, 5), dead lines
    starting at 1 % of the columns with widths 1-3 (Cases 4, 5).  Reading: the
    stripes and dead lines affect every band."""
    sp = 0.05 if k in (2, 5) else 0.0
    st = 0.05 if k in (3, 5) else 0.0
    dl = 0.01 if k in (4, 5) else 0.0
    if k not in (1, 2, 3, 4, 5):
        raise ValueError("cases 1..5")
    return NoiseSpec(sigma=0.1, sp_rate=sp, stripe_rate=st, stripe_amp=0.5,
                     dead_col_rate=dl, dead_band_rate=1.0 if dl else 0.0, dead_width_max=3)


def clean_cube(n1: int, n2: int, n3: int, rng: np.random.Generator, n_regions: int = 6):
    """Piecewise-smooth cube: Voronoi regions x 3-Gaussian spectra, in [0, 1]."""
    seeds = rng.uniform(0.0, 1.0, size=(n_regions, 2)) * np.array([n1, n2])
    ii, jj = np.meshgrid(np.arange(n1) + 0.5, np.arange(n2) + 0.5, indexing="ij")
    d2 = (ii[None] - seeds[:, 0, None, None]) ** 2 + (jj[None] - seeds[:, 1, None, None]) ** 2
    label = np.argmin(d2, axis=0)                       # (n1, n2)
    bands = np.arange(n3, dtype=np.float64)
    spectra = np.zeros((n_regions, n3))
    for r in range(n_regions):
        for _ in range(3):
            c = rng.uniform(0.0, n3)
            w = rng.uniform(n3 / 12.0, n3 / 3.0)
            a = rng.uniform(0.2, 1.0)
            spectra[r] += a * np.exp(-0.5 * ((bands - c) / w) ** 2)
    lo, hi = spectra.min(), spectra.max()
    spectra = (spectra - lo) / (hi - lo) if hi > lo else np.zeros_like(spectra)
    # cube[b, i, j] = spectra[label[i, j], b]
    cube = spectra.T.astype(np.float32)[:, label]       # (n3, n1, n2)
    return np.ascontiguousarray(cube)


def make_problem(n1: int, n2: int, n3: int, seed: int = 0, noise: NoiseSpec | None = None,
                 rho_eps: float = 0.95, rho_alpha: float = 0.9, rho_beta: float = 0.9):
    """Clean cube, noisy observation and the radii used by the workloads.

    Radii: eps = rho_eps * sigma * sqrt(N (1 - p_s) (1 - c_d)) with c_d the
    fraction of voxels on dead lines (the Gaussian part only lives on the
    voxels that are not replaced), alpha = rho_alpha ||s_bar||_1 and
    beta = rho_beta ||t_bar||_1.
    """
    noise = noise or NoiseSpec()
    rng = np.random.default_rng(seed)
    u_bar = clean_cube(n1, n2, n3, rng)
    shape = (n3, n1, n2)
    n_vox = n1 * n2 * n3

    # stripes: per band, a subset of columns gets an offset constant along i
    stripe_cols = rng.uniform(size=(n3, n2)) < noise.stripe_rate
    offsets = rng.uniform(-noise.stripe_amp, noise.stripe_amp, size=(n3, n2))
    t_row = np.where(stripe_cols, offsets, 0.0).astype(np.float32)      # (n3, n2)
    t_bar = np.broadcast_to(t_row[:, None, :], shape)

    # salt and pepper
    sp = rng.uniform(size=shape) < noise.sp_rate
    sp_val = (rng.uniform(size=shape) < 0.5).astype(np.float32)
    # dead lines: zeroed columns in a subset of bands
    dead_bands = rng.uniform(size=n3) < noise.dead_band_rate
    dead_cols = (rng.uniform(size=(n3, n2)) < noise.dead_col_rate) & dead_bands[:, None]
    if noise.dead_width_max > 1:
        # each start covers 1..dead_width_max columns (drawn only when widths
        # above 1 are asked for, so the other workloads keep their bytes)
        width = rng.integers(1, noise.dead_width_max + 1, size=(n3, n2))
        starts = dead_cols
        dead_cols = np.zeros_like(starts)
        for w in range(noise.dead_width_max):
            sh = starts & (width > w)
            dead_cols[:, w:] |= sh[:, :n2 - w] if w else sh
    dead = np.broadcast_to(dead_cols[:, None, :], shape)

    gauss = rng.standard_normal(size=shape, dtype=np.float32) * np.float32(noise.sigma)
    replaced = sp | dead
    v = np.where(replaced, 0.0, u_bar + t_bar + gauss).astype(np.float32)
    v = np.where(sp & ~dead, sp_val, v).astype(np.float32)
    # s_bar makes Eq. 14 exact on replaced voxels (n = 0 there)
    s_bar = np.where(replaced, v.astype(np.float64) - u_bar - t_bar, 0.0)
    n_true = np.where(replaced, 0.0, gauss)

    c_d = float(dead.mean()) if dead.any() else 0.0
    p_s = float(sp.mean())
    eps = rho_eps * noise.sigma * math.sqrt(n_vox * (1.0 - noise.sp_rate) * (1.0 - c_d))
    alpha = rho_alpha * float(np.abs(s_bar).sum())
    beta = rho_beta * float(np.abs(t_bar).sum(dtype=np.float64))
    return {
        "v": np.ascontiguousarray(v),
        "u_bar": u_bar,
        "s_bar": s_bar,
        "t_bar": np.ascontiguousarray(t_bar, dtype=np.float32),
        "n": n_true,
        "eps": eps, "alpha": alpha, "beta": beta,
        "p_s_observed": p_s, "c_d": c_d,
        "shape": shape,
    }


def random_state(n1: int, n2: int, n3: int, seed: int = 1, scale: float = 0.1):
    """A random (u, s, t, w1, w2, y1..y4) point, float32, for one-step checks.

    u is drawn in [-0.1, 1.1] so the box clamp is exercised; the other
    variables are centred Gaussian with standard deviation ``scale``.
    """
    rng = np.random.default_rng(seed)
    shp = (n3, n1, n2)
    f = np.float32

    def g(*lead):
        return (rng.standard_normal(size=lead + shp, dtype=np.float32) * f(scale))

    return {
        "u": rng.uniform(-0.1, 1.1, size=shp).astype(f),
        "s": g(), "t": g(),
        "w1": g(3, 2), "w2": g(3, 2),
        "y1": g(2), "y2": g(2),
        "y3": g(), "y4": g(),
    }
