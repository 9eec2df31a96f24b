"""The stopping rule (Eq. 28) on the GPU against the FP64 oracle.

The oracle steps the cube and records the ratio ||u^(k+1) - u^(k)|| / ||u^(k)||
of every pass.  A tol is placed where the ratio crosses it with a clear
margin (the GPU's ratio comes from float32 iterates and compensated float32
sums, so it is close to the oracle's but not equal), and the GPU, testing the
rule every `check_every` passes, must stop at the first tested pass whose
oracle ratio is below tol, with u, s, t there equal to the oracle's state of
that pass.  Single handles and a batch (each cube its own rule) are checked.
"""
import numpy as np
import pytest
import torch

from oracle import ppds as o
from paper_2510_00562_gb300 import synth
from paper_2510_00562_gb300.solver import GeoSSTVBatch, GeoSSTVSolver, make_params

pytestmark = pytest.mark.gpu

MARGIN = 0.05      # relative distance of every tested ratio from tol


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _oracle_run(pb, n):
    v = pb["v"].astype(np.float64)
    p = o.Params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=0.03)
    st = o.init_state(v)
    states, ratios = [st], []
    for _ in range(n):
        nxt = o.ppds_step(st, v, p)
        ratios.append(o.rel_change(nxt.u, st.u))
        st = nxt
        states.append(st)
    return states, ratios


def _tol_for(ratios, every, target):
    """A tol whose first crossing among the tested passes (every `every`-th)
    comes near pass `target`, with every tested ratio up to the crossing at
    least MARGIN away from tol; returns (tol, expected passes)."""
    tested = list(range(every, len(ratios) + 1, every))          # passes (1-based)
    for m in sorted(tested, key=lambda m: abs(m - target)):
        before = [ratios[k - 1] for k in tested if k < m]
        r = ratios[m - 1]
        hi = min(before) if before else np.inf
        if r * (1 + MARGIN) ** 2 < hi:
            tol = r * (1 + MARGIN)
            if all(x > tol * (1 + MARGIN) for x in before):
                return tol, m
    raise AssertionError("no tol with margin on this trajectory")


def _params(pb, **kw):
    return make_params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=0.03, graph_iters=16, **kw)


@pytest.fixture(scope="module")
def case():
    pb = synth.make_problem(24, 40, 10, seed=5)
    states, ratios = _oracle_run(pb, 260)
    return pb, states, ratios


@pytest.mark.parametrize("every,target", [(1, 90), (7, 150), (16, 200)])
def test_gpu_stops_at_the_oracle_pass(case, every, target):
    pb, states, ratios = case
    tol, m = _tol_for(ratios, every, target)
    with GeoSSTVSolver(24, 40, 10, _params(pb, tol=tol, check_every=every, max_iter=len(ratios))) as sol:
        u, s, t, done = sol.solve(torch.from_numpy(pb["v"]).cuda())
    assert done == m, (done, m, tol)
    ref = states[m]
    for name, got, want in (("u", u, ref.u), ("s", s, ref.s), ("t", t, ref.t)):
        e = rel(got.cpu().numpy(), want)
        assert e < 1e-5, (name, e)


def test_gpu_reports_the_ratio_of_the_last_pass(case):
    pb, states, ratios = case
    with GeoSSTVSolver(24, 40, 10, _params(pb, tol=0.0, max_iter=120)) as sol:
        sol.solve(torch.from_numpy(pb["v"]).cuda())
        got = sol.stats()["last_rel_change"]
    assert abs(got - ratios[119]) < 1e-3 * ratios[119], (got, ratios[119])


def test_batch_cubes_stop_at_their_oracle_passes():
    shapes = [(24, 40, 10), (17, 33, 6), (40, 24, 8)]
    runs = []
    for k, (n1, n2, n3) in enumerate(shapes):
        pb = synth.make_problem(n1, n2, n3, seed=30 + k)
        states, ratios = _oracle_run(pb, 200)
        every = (1, 5, 9)[k]
        tol, m = _tol_for(ratios, every, (60, 110, 150)[k])
        runs.append((pb, states, tol, m, every))
    params = [_params(pb, tol=tol, check_every=every, max_iter=200) for pb, _, tol, _, every in runs]
    vs = [torch.from_numpy(pb["v"]).cuda() for pb, *_ in runs]
    with GeoSSTVBatch(shapes, params) as bt:
        us, ss, ts, done = bt.solve(vs)
    for k, (pb, states, tol, m, every) in enumerate(runs):
        assert done[k] == m, (k, done[k], m)
        ref = states[m]
        for name, got, want in (("u", us[k], ref.u), ("s", ss[k], ref.s), ("t", ts[k], ref.t)):
            e = rel(got.cpu().numpy(), want)
            assert e < 1e-5, (k, name, e)
