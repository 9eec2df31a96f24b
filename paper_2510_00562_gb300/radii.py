"""Radii of the three constraints as the paper's experiments set them (Sec.
IV-A, Eqs. 25-27), from the noise model and the observation.

    alpha = rho N (0.5 p_s + M c_d)                                  (Eq. 25)
    beta  = rho 0.5 N p_t (1 - p_s) (1 - c_d) / 2                    (Eq. 26)
    eps   = rho sqrt(sigma^2 N (1 - p_s) (1 - c_d))                  (Eq. 27)

N: voxels; M: mean intensity of the observation; p_s, p_t: salt-and-pepper
and stripe rates; c_d = 1 - exp(-w p_d): coverage of dead lines of mean width
w starting at rate p_d (the paper's footnote to Eqs. 25-27); rho = 0.98, 0.95
or 0.90 when one, two or three radii are nonzero.  Eq. 26 assumes stripe
intensities U[-0.5, 0.5] (mean magnitude 0.25), as in the paper's Case 3.
This is experiment set-up, not part of Algorithm 1.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["deadline_coverage", "paper_radii", "RHO_BY_COUNT"]

RHO_BY_COUNT = {1: 0.98, 2: 0.95, 3: 0.90}


def deadline_coverage(rate: float, mean_width: float) -> float:
    """c_d = 1 - exp(-w p_d): the fraction of columns covered by dead lines of
    mean width w that start independently at rate p_d (overlaps counted once)."""
    return 1.0 - math.exp(-mean_width * rate)


def paper_radii(v, sigma: float, sp_rate: float, stripe_rate: float, dead_rate: float = 0.0,
                dead_mean_width: float = 2.0, rho: float | None = None) -> dict:
    """eps, alpha, beta of Eqs. 25-27 for the observation v (any shape)."""
    n = int(np.asarray(v).size)
    m = float(np.asarray(v, dtype=np.float64).mean())
    c_d = deadline_coverage(dead_rate, dead_mean_width) if dead_rate > 0 else 0.0
    alpha_raw = n * (0.5 * sp_rate + m * c_d)
    beta_raw = 0.5 * n * stripe_rate * (1.0 - sp_rate) * (1.0 - c_d) / 2.0
    eps_raw = math.sqrt(sigma * sigma * n * (1.0 - sp_rate) * (1.0 - c_d))
    count = sum(1 for x in (eps_raw, alpha_raw, beta_raw) if x > 0)
    r = rho if rho is not None else RHO_BY_COUNT.get(count, 1.0)
    return {"eps": r * eps_raw, "alpha": r * alpha_raw, "beta": r * beta_raw, "rho": r, "c_d": c_d,
            "mean_v": m}
