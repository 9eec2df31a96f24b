"""Pins of the oracle's stopping rule (Eq. 28).

Eq. 28 stops the run after the first pass k+1 with
||u^(k+1) - u^(k)||_2 / ||u^(k)||_2 < tol.  The expected stop is computed
here from passes stepped one at a time, with the ratio summed independently
(math.fsum of the squared entries), at a tol placed between this ratio and
the one taken against u^(k+1), so that the two readings stop at different
passes.  Planted mistakes in the oracle -- the ratio against u^(k+1), and a
check that sees the previous pass's ratio (one pass late) -- must fail.
"""
import math

import numpy as np
import pytest

from oracle import ppds as o
from paper_2510_00562_gb300 import synth


def _ratio_fsum(u_next, u_prev):
    num = math.fsum(((u_next - u_prev) ** 2).ravel().tolist())
    den = math.fsum((u_prev ** 2).ravel().tolist())
    return math.sqrt(num / den)


def _problem():
    pb = synth.make_problem(14, 18, 6, seed=21)
    v = pb["v"].astype(np.float64)
    p = o.Params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=0.03)
    return v, p


def _hand_trajectory(v, p, n):
    """States 0..n stepped one pass at a time, and both readings of the ratio."""
    sts = [o.init_state(v)]
    for _ in range(n):
        sts.append(o.ppds_step(sts[-1], v, p))
    r_prev = [_ratio_fsum(sts[k + 1].u, sts[k].u) for k in range(n)]       # Eq. 28
    r_next = [math.sqrt(math.fsum(((sts[k + 1].u - sts[k].u) ** 2).ravel().tolist())
                        / math.fsum((sts[k + 1].u ** 2).ravel().tolist())) for k in range(n)]
    return sts, r_prev, r_next


def _separating_tol(r_prev, r_next, first=10):
    """(tol, K): tol strictly between the two readings at pass K (0-based), every
    earlier pass above tol under both, so the two readings stop at different
    passes; the tol sits midway, far from either ratio at the float64 level."""
    for K in range(first, len(r_prev)):
        lo, hi = sorted((r_prev[K], r_next[K]))
        if hi - lo < 1e-9 * hi:
            continue
        tol = 0.5 * (lo + hi)
        if all(r_prev[j] > tol and r_next[j] > tol for j in range(K)):
            return tol, K
    raise AssertionError("no separating tol on this trajectory")


N_PASSES = 160


@pytest.fixture(scope="module")
def traj():
    v, p = _problem()
    sts, rp, rn = _hand_trajectory(v, p, N_PASSES)
    tol, K = _separating_tol(rp, rn)
    return v, p, sts, rp, rn, tol, K


def _check_stop(v, p, sts, rp, tol):
    expected = next(k for k in range(len(rp)) if rp[k] < tol) + 1       # passes run
    st, done = o.solve(v, p, N_PASSES, tol=tol)
    assert done == expected, (done, expected)
    for name in o.State.names():
        np.testing.assert_array_equal(getattr(st, name), getattr(sts[done], name), err_msg=name)


def test_stop_pass_matches_hand_stepped_ratio(traj):
    v, p, sts, rp, rn, tol, K = traj
    # the two readings disagree at this tol: the check below can tell them apart
    stop_prev = next(k for k in range(len(rp)) if rp[k] < tol)
    stop_next = next((k for k in range(len(rn)) if rn[k] < tol), None)
    assert stop_prev != stop_next
    _check_stop(v, p, sts, rp, tol)


def test_stop_rule_off_runs_every_pass(traj):
    v, p, sts, rp, rn, tol, K = traj
    st, done = o.solve(v, p, 25, tol=0.0)
    assert done == 25
    np.testing.assert_array_equal(st.u, sts[25].u)
    # a tol no ratio meets also runs to the cap
    st, done = o.solve(v, p, 25, tol=min(rp[:25]) * 0.5)
    assert done == 25


def test_zero_state_never_stops():
    # u^(k) = 0 leaves the ratio undefined: the run goes to its cap
    v = np.zeros((3, 5, 4))
    st, done = o.solve(v, o.Params(eps=0.1, alpha=0.5, beta=0.5), 12, tol=1e-3)
    assert done == 12


def _mistake_ratio_against_next(u_next, u_prev):
    return float(np.linalg.norm(u_next - u_prev) / np.linalg.norm(u_next))


class _LaggedRatio:
    """A check that sees the previous pass's ratio: stops one pass late."""

    def __init__(self, real):
        self.real = real
        self.last = np.inf

    def __call__(self, u_next, u_prev):
        out, self.last = self.last, self.real(u_next, u_prev)
        return out


@pytest.mark.parametrize("mistake", ["ratio_against_next", "one_pass_late"])
def test_planted_mistakes_break_the_stop_pin(traj, monkeypatch, mistake):
    v, p, sts, rp, rn, tol, K = traj
    if mistake == "ratio_against_next":
        monkeypatch.setattr(o, "rel_change", _mistake_ratio_against_next)
    else:
        monkeypatch.setattr(o, "rel_change", _LaggedRatio(o.rel_change))
    with pytest.raises(AssertionError):
        _check_stop(v, p, sts, rp, tol)
