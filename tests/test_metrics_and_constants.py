"""Pins of the harness: MPSNR (Eq. 29), MSSIM (Eq. 30), the generator (Eq. 14)
and the constants the paper prints (tests/golden/paper_constants.json)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import ppds as o
from paper_2510_00562_gb300 import metrics, synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def test_mpsnr_closed_form():
    """u = u_ref + delta_b per band gives PSNR_b = 10 log10(1 / delta_b^2)."""
    rng = np.random.default_rng(0)
    ref = rng.uniform(size=(4, 10, 12))
    deltas = np.array([0.1, 0.01, 0.05, 0.2])
    u = ref + deltas[:, None, None]
    want = np.mean([10 * math.log10(1 / d ** 2) for d in deltas])
    assert metrics.mpsnr(u, ref) == pytest.approx(want, rel=1e-12)
    assert metrics.mpsnr(ref, ref) == math.inf


def test_ssim_constant_images():
    """For constant bands a, b: SSIM = (2ab + C1) / (a^2 + b^2 + C1)."""
    c1 = 0.01 ** 2
    a, b = 0.3, 0.6
    x = np.full((20, 24), a)
    y = np.full((20, 24), b)
    assert metrics.ssim_band(x, y) == pytest.approx((2 * a * b + c1) / (a * a + b * b + c1), rel=1e-12)
    rng = np.random.default_rng(1)
    z = rng.uniform(size=(3, 16, 16))
    assert metrics.mssim(z, z) == pytest.approx(1.0, abs=1e-12)
    assert metrics.mssim(z, 1 - z) < 0.5


def test_generator_observation_model():
    pb = synth.make_problem(32, 24, 16, seed=2, noise=synth.NoiseSpec(
        sigma=0.1, sp_rate=0.05, stripe_rate=0.1, dead_col_rate=0.1, dead_band_rate=0.3))
    v = pb["v"].astype(np.float64)
    recon = pb["u_bar"].astype(np.float64) + pb["s_bar"] + pb["t_bar"].astype(np.float64) + pb["n"]
    np.testing.assert_allclose(recon, v, atol=1e-6)     # Eq. 14 (float32 rounding)
    assert pb["u_bar"].min() == 0.0 and pb["u_bar"].max() == pytest.approx(1.0)
    # stripes are constant along each column: D_v t_bar = 0
    assert np.all(np.diff(pb["t_bar"], axis=1) == 0)
    assert v.dtype == np.float64 and pb["v"].dtype == np.float32
    # same seed, same bytes
    pb2 = synth.make_problem(32, 24, 16, seed=2, noise=synth.NoiseSpec(
        sigma=0.1, sp_rate=0.05, stripe_rate=0.1, dead_col_rate=0.1, dead_band_rate=0.3))
    assert pb2["v"].tobytes() == pb["v"].tobytes()


def test_oracle_defaults_are_the_printed_step_sizes():
    g = json.load(open(GOLDEN))
    p = o.Params()
    for k, (num, den) in g["step_sizes"].items():
        assert getattr(p, k) == pytest.approx(num / den, rel=1e-15), k
    assert p.omega in g["omega_set"]
