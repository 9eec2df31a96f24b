"""Radii of the paper's experiments (Sec. IV-A, Eqs. 25-27) and its noise cases."""
import math

import numpy as np
import pytest

from paper_2510_00562_gb300 import radii, synth


def test_case1_only_the_fidelity_radius():
    """Case 1 (Gaussian only): alpha = beta = 0, one nonzero radius so rho =
    0.98, and eps = 0.98 sigma sqrt(N)."""
    v = np.full((4, 8, 8), 0.3, np.float32)
    r = radii.paper_radii(v, sigma=0.1, sp_rate=0.0, stripe_rate=0.0)
    assert r["alpha"] == 0.0 and r["beta"] == 0.0 and r["rho"] == 0.98
    assert r["eps"] == pytest.approx(0.98 * 0.1 * math.sqrt(v.size), rel=1e-15)


def test_case2_closed_form():
    """Case 2: alpha = rho N 0.5 p_s, eps = rho sigma sqrt(N (1 - p_s)), rho = 0.95."""
    v = np.random.default_rng(0).uniform(0, 1, (5, 6, 7)).astype(np.float32)
    n = v.size
    r = radii.paper_radii(v, sigma=0.1, sp_rate=0.05, stripe_rate=0.0)
    assert r["rho"] == 0.95 and r["beta"] == 0.0
    assert r["alpha"] == pytest.approx(0.95 * n * 0.025, rel=1e-15)
    assert r["eps"] == pytest.approx(0.95 * math.sqrt(0.01 * n * 0.95), rel=1e-15)


def test_case5_three_radii_and_the_mean_intensity_term():
    """Case 5: rho = 0.90; alpha carries M c_d with M the observation's mean;
    beta = rho 0.25 N p_t (1 - p_s)(1 - c_d)."""
    v = np.full((3, 10, 10), 0.4, np.float32)
    n = v.size
    c_d = 1.0 - math.exp(-2.0 * 0.01)
    r = radii.paper_radii(v, sigma=0.1, sp_rate=0.05, stripe_rate=0.05, dead_rate=0.01, dead_mean_width=2.0)
    assert r["rho"] == 0.90 and r["c_d"] == pytest.approx(c_d, rel=1e-15)
    m = float(np.float32(0.4))                          # the observation's mean, as stored
    assert r["alpha"] == pytest.approx(0.9 * n * (0.025 + m * c_d), rel=1e-12)
    assert r["beta"] == pytest.approx(0.9 * 0.25 * n * 0.05 * 0.95 * (1 - c_d), rel=1e-12)
    assert r["eps"] == pytest.approx(0.9 * math.sqrt(0.01 * n * 0.95 * (1 - c_d)), rel=1e-12)


def test_deadline_coverage_matches_the_generator():
    """The generator's dead lines (starts at rate 0.01, widths 1..3) cover a
    fraction of the columns close to c_d = 1 - exp(-2 p_d)."""
    pb = synth.make_problem(8, 4096, 64, seed=3, noise=synth.paper_case(4))
    covered = float((pb["v"] == 0).all(axis=1).mean())   # a dead column is zero on every row
    c_d = radii.deadline_coverage(0.01, 2.0)
    assert covered == pytest.approx(c_d, rel=0.08)
    assert pb["c_d"] == pytest.approx(covered, abs=1e-12)


def test_paper_cases_noise_content():
    """Cases 1-5 switch on exactly the noise types of Sec. IV-A, and the
    stripe radius stays below the generated stripes' l1 norm."""
    kinds = {1: (0, 0, 0), 2: (1, 0, 0), 3: (0, 1, 0), 4: (0, 0, 1), 5: (1, 1, 1)}
    for k, (sp, st, dl) in kinds.items():
        c = synth.paper_case(k)
        assert c.sigma == 0.1
        assert (c.sp_rate > 0) == bool(sp) and (c.stripe_rate > 0) == bool(st)
        assert (c.dead_col_rate > 0) == bool(dl)
    pb = synth.make_problem(32, 256, 16, seed=1, noise=synth.paper_case(5))
    r = radii.paper_radii(pb["v"], 0.1, 0.05, 0.05, 0.01, 2.0)
    t1 = float(np.abs(pb["t_bar"]).sum(dtype=np.float64))
    assert r["beta"] < t1
    with pytest.raises(ValueError):
        synth.paper_case(6)
