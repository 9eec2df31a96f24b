"""Batches of independent cubes (gsstv_batch_*): each cube of a batch, with its
own shape, parameters and Eq. 28 stopping rule, gets the result of solving it
alone, and that result matches the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import ppds as o
from paper_2510_00562_gb300 import synth
from paper_2510_00562_gb300.solver import GeoSSTVBatch, GeoSSTVSolver, make_params

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _cube(n1, n2, n3, seed, sigma, sp, st):
    pb = synth.make_problem(n1, n2, n3, seed=seed, noise=synth.NoiseSpec(
        sigma=sigma, sp_rate=sp, stripe_rate=st, stripe_amp=0.25))
    return pb


# shape (N1, N2, N3), noise, and the solver settings of each cube: early
# stopping at different tolerances and check intervals, a fixed count, 16-bit
# storage, a cube of one band
CASES = [
    ((37, 45, 9), (0.10, 0.05, 0.05), dict(tol=1e-4, check_every=10, max_iter=400)),
    ((16, 32, 5), (0.05, 0.00, 0.10), dict(tol=1e-3, check_every=7, max_iter=300)),
    ((64, 48, 31), (0.12, 0.10, 0.05), dict(tol=0.0, max_iter=60)),
    ((20, 20, 12), (0.02, 0.15, 0.00), dict(tol=5e-4, check_every=25, max_iter=500)),
    ((48, 96, 16), (0.08, 0.05, 0.15), dict(tol=1e-4, check_every=20, max_iter=200, storage="bf16")),
    ((33, 17, 1), (0.10, 0.05, 0.05), dict(tol=0.0, max_iter=50)),
]


def _params(pb, kw):
    return make_params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=0.03, graph_iters=16, **kw)


def test_batch_matches_individual_solves():
    pbs = [_cube(*shape, seed=k, sigma=n[0], sp=n[1], st=n[2]) for k, (shape, n, _) in enumerate(CASES)]
    params = [_params(pb, kw) for pb, (_, _, kw) in zip(pbs, CASES)]
    vs = [torch.from_numpy(pb["v"]).cuda() for pb in pbs]
    with GeoSSTVBatch([c[0] for c in CASES], params) as bt:
        us, ss, ts, done = bt.solve(vs)
        # a second solve on the same batch starts afresh and repeats the first
        us2, _, _, done2 = bt.solve(vs)
    assert done == done2
    for k, ((n1, n2, n3), _, kw) in enumerate(CASES):
        with GeoSSTVSolver(n1, n2, n3, _params(pbs[k], kw)) as sol:
            u, s, t, n = sol.solve(vs[k])
        print(f"cube {k} {(n1, n2, n3)} {kw}: {done[k]} passes (alone {n})")
        assert done[k] == n, (k, done[k], n)
        if kw.get("tol", 0.0) == 0.0:
            assert done[k] == kw["max_iter"]
        tol = 1e-6 if kw.get("storage", "fp32") == "fp32" else 1e-3
        for got, ref in ((us[k], u), (ss[k], s), (ts[k], t), (us2[k], u)):
            e = rel(got.cpu().numpy(), ref.cpu().numpy())
            assert e < tol or not ref.any(), (k, e)
    # the early-stopping cubes did stop early, and not all at the same pass
    early = [(done[k], kw["max_iter"]) for k, (_, _, kw) in enumerate(CASES) if kw.get("tol", 0.0) > 0]
    assert any(d < cap for d, cap in early)
    assert len(set(done)) > 2


def test_batch_matches_oracle():
    shapes = [(24, 40, 10), (30, 19, 6)]
    pbs = [_cube(*sh, seed=10 + k, sigma=0.1, sp=0.05, st=0.05) for k, sh in enumerate(shapes)]
    iters = [150, 90]
    params = [_params(pb, dict(max_iter=it)) for pb, it in zip(pbs, iters)]
    vs = [torch.from_numpy(pb["v"]).cuda() for pb in pbs]
    with GeoSSTVBatch(shapes, params) as bt:
        us, ss, ts, done = bt.solve(vs)
        # every cube's fused kernel autotuned: the results stay within parity
        chunks = bt.autotune(vs, passes=3)
        us_t, ss_t, ts_t, done_t = bt.solve(vs)
    assert done == iters and done_t == iters
    for (n1, n2, n3), c in zip(shapes, chunks):
        assert min(8, n3) <= c <= n3, (n3, c)
    for k, pb in enumerate(pbs):
        p = params[k]
        st, _ = o.solve(pb["v"].astype(np.float64), o.Params(eps=p.eps, alpha=p.alpha, beta=p.beta,
                                                             omega=p.omega), iters[k])
        for got, ref in ((us[k], st.u), (ss[k], st.s), (ts[k], st.t), (us_t[k], st.u), (ss_t[k], st.s),
                         (ts_t[k], st.t)):
            e = rel(got.cpu().numpy(), ref)
            print(f"batch cube {k} vs oracle: {e:.3e}")
            assert e < 1e-5


def test_batch_rejects_mismatched_inputs():
    pb = _cube(8, 8, 3, seed=1, sigma=0.1, sp=0.0, st=0.0)
    with GeoSSTVBatch([(8, 8, 3)], [_params(pb, dict(max_iter=5))]) as bt:
        with pytest.raises(ValueError):
            bt.solve([torch.zeros(3, 8, 9, device="cuda")])
        with pytest.raises(ValueError):
            bt.solve([])


def test_fused_batch_equals_stream_batch_and_single_solves(monkeypatch):
    """Float32 cubes run each stage as one launch over all cubes, with the
    stopping rules on the device: every cube must stop at the pass its single
    solve stops at, with the same result; the one-stream-per-cube batch
    (GSSTV_BATCH=streams) too."""
    cases = [c for c in CASES if c[2].get("storage", "fp32") == "fp32"]
    pbs = [_cube(*shape, seed=10 + k, sigma=n[0], sp=n[1], st=n[2]) for k, (shape, n, _) in enumerate(cases)]
    params = [_params(pb, kw) for pb, (_, _, kw) in zip(pbs, cases)]
    vs = [torch.from_numpy(pb["v"]).cuda() for pb in pbs]
    shapes = [c[0] for c in cases]
    with GeoSSTVBatch(shapes, params) as bt:
        us, ss, ts, done = bt.solve(vs)
        us2, _, _, done2 = bt.solve(vs)                 # a second solve repeats the first
        stats = [bt.stats(k) for k in range(len(cases))]
    monkeypatch.setenv("GSSTV_BATCH", "streams")
    with GeoSSTVBatch(shapes, params) as bs:
        us_s, _, _, done_s = bs.solve(vs)
    assert done == done2 == done_s
    for k, ((n1, n2, n3), _, kw) in enumerate(cases):
        with GeoSSTVSolver(n1, n2, n3, _params(pbs[k], kw)) as sol:
            u, s, t, n = sol.solve(vs[k])
        assert done[k] == n, (k, done[k], n)
        for got, ref in ((us[k], u), (ss[k], s), (ts[k], t), (us2[k], u), (us_s[k], u)):
            e = rel(got.cpu().numpy(), ref.cpu().numpy())
            assert e < 1e-6 or not ref.any(), (k, e)
        assert stats[k]["iterations"] >= n
    early = [(done[k], kw["max_iter"]) for k, (_, _, kw) in enumerate(cases) if kw.get("tol", 0.0) > 0]
    assert any(d < cap for d, cap in early)

