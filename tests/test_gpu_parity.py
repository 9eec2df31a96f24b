"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (relative L2 error per variable, ||x_gpu - x_ref|| / ||x_ref||):
  * one pass of Algorithm 1 from a random state: 2e-6 (float32 arithmetic on
    float32 inputs: a few roundings of ~6e-8 each, amplified by the stencil
    sums);
  * after a fixed iteration count from the standard start: 1e-5 on u, s, t and
    |MPSNR_gpu - MPSNR_oracle| <= 0.01 dB (the parity bar of the plain FP32
    method).
Shapes cover several K1 tiles (16 x 32) and band chunks with ragged edges,
N2 not a multiple of the row pitch, and the degenerate N1 = 1, N3 = 1 cubes.
"""
import math
import zlib

import numpy as np
import pytest
import torch

from oracle import ppds as o
from paper_2510_00562_gb300 import metrics, synth
from paper_2510_00562_gb300.solver import GeoSSTVSolver, make_params, project_l1ball

pytestmark = pytest.mark.gpu

KEYS = ("u", "s", "t", "w1", "w2", "y1", "y2", "y3", "y4")


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a - b)


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def oracle_params(p):
    return o.Params(eps=p.eps, alpha=p.alpha, beta=p.beta, omega=p.omega, mu_lo=p.mu_lo, mu_hi=p.mu_hi,
                    gamma_u=p.gamma_u, gamma_w1=p.gamma_w1, gamma_w2=p.gamma_w2, gamma_s=p.gamma_s,
                    gamma_t=p.gamma_t, gamma_y1=p.gamma_y1, gamma_y2=p.gamma_y2, gamma_y3=p.gamma_y3,
                    gamma_y4=p.gamma_y4)


# ---------------------------------------------------------------------------
# l1-ball projection (Sec. III-B)
# ---------------------------------------------------------------------------
def _l1_case(name):
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    if name.startswith("laplace"):
        n = int(name.split("_")[1])
        x = rng.laplace(size=n).astype(np.float32)
        return x, 0.3 * float(np.abs(x.astype(np.float64)).sum())
    if name == "ties":
        x = rng.choice(np.array([-2, -1, -0.5, 0, 0.5, 1, 2], dtype=np.float32), size=50_000)
        return x, 0.2 * float(np.abs(x.astype(np.float64)).sum())
    if name == "sparse_big":
        x = np.zeros(4_000_000, dtype=np.float32)
        idx = rng.choice(x.size, 40_000, replace=False)
        x[idx] = rng.standard_normal(idx.size).astype(np.float32)
        return x, 0.5 * float(np.abs(x.astype(np.float64)).sum())
    if name == "narrow":      # many values within a few ulps: the radix search goes deep
        x = (1.0 + rng.integers(0, 64, size=2_000_000) * 2.0**-23).astype(np.float32)
        return x, 2.0
    raise KeyError(name)


@pytest.mark.parametrize("name", ["laplace_1", "laplace_7", "laplace_1000", "laplace_100000",
                                  "laplace_3000000", "ties", "sparse_big", "narrow"])
def test_l1_projection_matches_oracle(name):
    x, r = _l1_case(name)
    ref, tau_ref = o.proj_l1ball(x.astype(np.float64), r)
    out, tau = project_l1ball(to_dev(x), r)
    out = out.cpu().numpy()
    assert tau == pytest.approx(tau_ref, rel=1e-6, abs=1e-12)
    assert np.abs(out - ref).max() <= 1e-6 * max(1.0, np.abs(x).max())
    # tau is applied in float32: each active entry carries up to half an ulp of max|x|
    n_act = int((ref != 0).sum())
    slack = 1e-5 * r + n_act * 2.0**-24 * float(np.abs(x).max())
    assert abs(np.abs(out.astype(np.float64)).sum() - r) <= slack


def test_l1_projection_edge_cases():
    x = np.array([0.5, -0.25, 0.0, 0.125], dtype=np.float32)
    out, tau = project_l1ball(to_dev(x), 1.0)           # inside: identity
    assert tau == 0.0 and np.array_equal(out.cpu().numpy(), x)
    out, tau = project_l1ball(to_dev(x), 0.875)         # on the sphere: identity
    assert np.array_equal(out.cpu().numpy(), x)
    out, tau = project_l1ball(to_dev(x), 0.0)           # radius 0
    assert np.all(out.cpu().numpy() == 0)
    out, tau = project_l1ball(to_dev(np.zeros(1000, np.float32)), 0.0)
    assert np.all(out.cpu().numpy() == 0)
    y = np.array([1.0, -1.0, 1.0, 0.5, -0.5], dtype=np.float32)
    out, tau = project_l1ball(to_dev(y), 1.5)
    np.testing.assert_allclose(out.cpu().numpy(), [0.5, -0.5, 0.5, 0, 0], atol=1e-7)
    assert tau == pytest.approx(0.5, rel=1e-12)


# ---------------------------------------------------------------------------
# one pass of Algorithm 1 from a random state
# ---------------------------------------------------------------------------
SHAPES = [(37, 45, 9), (16, 32, 1), (1, 7, 3), (5, 3, 2), (70, 100, 20), (33, 64, 17)]


def _random_problem(n1, n2, n3, seed):
    rs = synth.random_state(n1, n2, n3, seed=seed, scale=0.1)
    v = np.random.default_rng(seed + 100).uniform(0, 1, size=(n3, n1, n2)).astype(np.float32)
    s64 = rs["s"].astype(np.float64)
    t64 = rs["t"].astype(np.float64)
    return rs, v, dict(eps=0.2 * math.sqrt(v.size) * 0.1, alpha=0.4 * np.abs(s64).sum(),
                       beta=0.4 * np.abs(t64).sum(), omega=0.05)


@pytest.fixture(params=["tma", "coop"])
def k1_variant(request, monkeypatch):
    """Both implementations of the fused stencil kernel (read at handle creation)."""
    monkeypatch.setenv("GSSTV_K1", request.param)
    return request.param


@pytest.mark.parametrize("tau_mode", ["auto", "exact"])
@pytest.mark.parametrize("shape", SHAPES)
def test_one_pass_matches_oracle(shape, tau_mode, k1_variant):
    n1, n2, n3 = shape
    rs, v, kw = _random_problem(n1, n2, n3, seed=n1 * 7 + n3)
    p = make_params(tau_mode=tau_mode, graph_iters=0, **kw)
    with GeoSSTVSolver(n1, n2, n3, p) as sol:
        sol.load(to_dev(v))
        sol.set_state({k: to_dev(rs[k]) for k in KEYS})
        st_cur = o.State(**{k: rs[k].astype(np.float64) for k in KEYS})
        for it in range(3):
            sol.iterate(1)
            st_cur = o.ppds_step(st_cur, v.astype(np.float64), oracle_params(p))
            got = {k: x.cpu().numpy() for k, x in sol.get_state().items()}
            for k in KEYS:
                e = rel(got[k], getattr(st_cur, k))
                assert e < 2e-6, (it, k, e)


# ---------------------------------------------------------------------------
# fixed iteration counts from the standard start, synthetic noisy cubes
# ---------------------------------------------------------------------------
def _problem(n1, n2, n3, seed=0):
    pb = synth.make_problem(n1, n2, n3, seed=seed, noise=synth.NoiseSpec(
        sigma=0.1, sp_rate=0.05, stripe_rate=0.05, stripe_amp=0.25))
    return pb


def _solve_both(n1, n2, n3, iters, tau_mode="auto", graph_iters=16, omega=0.03):
    pb = _problem(n1, n2, n3)
    p = make_params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=omega,
                    max_iter=iters, tau_mode=tau_mode, graph_iters=graph_iters)
    with GeoSSTVSolver(n1, n2, n3, p) as sol:
        u, s, t, n = sol.solve(to_dev(pb["v"]))
        stats = sol.stats()
    assert n == iters
    st, _ = o.solve(pb["v"].astype(np.float64), oracle_params(p), iters)
    return pb, (u.cpu().numpy(), s.cpu().numpy(), t.cpu().numpy()), st, stats


@pytest.mark.parametrize("tau_mode", ["auto", "exact"])
def test_solve_parity_small(tau_mode, k1_variant):
    pb, (u, s, t), st, stats = _solve_both(40, 36, 12, 300, tau_mode=tau_mode)
    errs = {name: rel(a, b) for name, a, b in (("u", u, st.u), ("s", s, st.s), ("t", t, st.t))}
    print(f"\nparity 40x36x12 300 it {tau_mode} {k1_variant}: {errs}")
    for name, e in errs.items():
        assert e < 1e-5, (name, e)
    d = abs(metrics.mpsnr(u, pb["u_bar"]) - metrics.mpsnr(st.u, pb["u_bar"]))
    assert d <= 0.01
    if tau_mode == "exact":
        assert stats["tau_window_hits"] == 0


def test_solve_parity_64x64x32_2000_iterations():
    """The plain-method parity workload: 64x64x32, sigma 0.1, 5% salt and
    pepper, stripes on 5% of the columns, 2000 iterations."""
    pb, (u, s, t), st, stats = _solve_both(64, 64, 32, 2000)
    errs = {name: rel(a, b) for name, a, b in (("u", u, st.u), ("s", s, st.s), ("t", t, st.t))}
    m_gpu = metrics.mpsnr(u, pb["u_bar"])
    m_ref = metrics.mpsnr(st.u, pb["u_bar"])
    print(f"\nparity 64x64x32 2000 it: {errs} mpsnr gpu {m_gpu:.4f} oracle {m_ref:.4f} "
          f"window hits {stats['tau_window_hits']} exact runs {stats['tau_exact_runs']}")
    assert max(errs.values()) < 1e-5, errs
    assert abs(m_gpu - m_ref) <= 0.01, (m_gpu, m_ref)
    assert m_gpu > metrics.mpsnr(pb["v"], pb["u_bar"]) + 3.0     # it denoises


def test_graph_and_eager_agree():
    pb = _problem(24, 40, 10, seed=3)
    outs = []
    for gi in (0, 4, 16):
        p = make_params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], max_iter=37, graph_iters=gi)
        with GeoSSTVSolver(24, 40, 10, p) as sol:
            outs.append([x.cpu().numpy() for x in sol.solve(to_dev(pb["v"]))[:3]])
    for other in outs[1:]:
        for a, b in zip(outs[0], other):
            assert rel(b, a) < 1e-6


# ---------------------------------------------------------------------------
# exact special cases and invariants at any size
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(9, 7, 6), (100, 70, 12), (512, 512, 224)])
def test_per_band_constant_fixed_point_exact(shape):
    n1, n2, n3 = shape
    levels = np.random.default_rng(1).uniform(0.1, 0.9, size=n3).astype(np.float32)
    v = np.ascontiguousarray(np.broadcast_to(levels[:, None, None], (n3, n1, n2)), dtype=np.float32)
    p = make_params(eps=0.3, alpha=2.0, beta=1.5, omega=0.03, max_iter=20)
    with GeoSSTVSolver(n1, n2, n3, p) as sol:
        dv = to_dev(v)
        u, s, t, _ = sol.solve(dv)
        assert torch.equal(u, dv)
        assert not s.any() and not t.any()
        st = sol.get_state()
        for k in ("w1", "w2", "y1", "y2", "y3", "y4"):
            assert not st[k].any(), k


def test_full_size_one_pass_512x512x224():
    """One pass of Algorithm 1 on the benchmark's 512x512x224 cube from a
    random state, with the kernels and run lengths the benchmark times, against
    one FP64 oracle pass over the whole cube: every variable within the bound
    of the small-cube one-pass test."""
    n1, n2, n3 = 512, 512, 224
    rs, v, kw = _random_problem(n1, n2, n3, seed=2024)
    p = make_params(graph_iters=0, **kw)
    with GeoSSTVSolver(n1, n2, n3, p) as sol:
        sol.load(to_dev(v))
        sol.set_state({k: to_dev(rs[k]) for k in KEYS})
        sol.iterate(1)
        got = sol.get_state()
    ref = o.ppds_step(o.State(**{k: rs[k].astype(np.float64) for k in KEYS}), v.astype(np.float64),
                      oracle_params(p))
    del rs
    for k in KEYS:
        e = rel(got[k].cpu().numpy(), getattr(ref, k))
        print(f"full-size one pass {k}: {e:.3e}")
        assert e < 2e-6, (k, e)


def test_full_size_invariants_512x512x224():
    """The benchmark cube in the benchmark's launch configuration: the
    projected constraints hold after every pass (l1 balls, box)."""
    n1, n2, n3 = 512, 512, 224
    pb = synth.make_problem(n1, n2, n3, seed=0, noise=synth.NoiseSpec(
        sigma=0.1, sp_rate=0.05, stripe_rate=0.1, dead_col_rate=0.02, dead_band_rate=0.1))
    p = make_params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], max_iter=30, graph_iters=16)
    with GeoSSTVSolver(n1, n2, n3, p) as sol:
        u, s, t, n = sol.solve(to_dev(pb["v"]))
        stats = sol.stats()
    assert n == 30
    s1 = s.double().abs().sum().item()
    t1 = t.double().abs().sum().item()
    assert s1 <= pb["alpha"] * (1 + 1e-5)
    assert t1 <= pb["beta"] * (1 + 1e-5)
    assert u.min().item() >= 0.0 and u.max().item() <= 1.0
    assert torch.isfinite(u).all()
    assert stats["iterations"] == 30


# ---------------------------------------------------------------------------
# API behaviour
# ---------------------------------------------------------------------------
def test_solve_host_matches_device():
    pb = _problem(20, 30, 8, seed=5)
    p = make_params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], max_iter=25, graph_iters=0,
                    tau_mode="exact")
    with GeoSSTVSolver(20, 30, 8, p) as sol:
        u, s, t, _ = sol.solve(to_dev(pb["v"]))
        vh = torch.from_numpy(pb["v"]).pin_memory()
        uh = torch.empty_like(vh).pin_memory()
        sh = torch.empty_like(vh).pin_memory()
        th = torch.empty_like(vh).pin_memory()
        sol.solve_host(vh, uh, sh, th)
    assert torch.equal(uh, u.cpu()) and torch.equal(sh, s.cpu()) and torch.equal(th, t.cpu())


def test_state_round_trip_fp32():
    rs = synth.random_state(13, 21, 5, seed=4)
    with GeoSSTVSolver(13, 21, 5, make_params()) as sol:
        sol.set_state({k: to_dev(rs[k]) for k in KEYS})
        got = sol.get_state()
    for k in KEYS:
        assert np.array_equal(got[k].cpu().numpy(), rs[k]), k


def test_nonfinite_observation_is_reported():
    from paper_2510_00562_gb300 import binding as B
    v = np.full((4, 8, 8), 0.5, np.float32)
    v[1, 2, 3] = np.nan
    p = make_params(eps=0.1, alpha=1.0, beta=1.0, max_iter=3, graph_iters=0)
    with GeoSSTVSolver(8, 8, 4, p) as sol:
        with pytest.raises(B.GsstvError) as ei:
            sol.solve(to_dev(v))
        assert ei.value.code == B.GSSTV_ERR_NONFINITE
        # the handle stays usable
        v[1, 2, 3] = 0.5
        u, _, _, n = sol.solve(to_dev(v))
        assert n == 3 and torch.isfinite(u).all()


def test_out_of_memory_is_reported():
    """Handles of the largest accepted cube (8192 x 8192 x 10 voxels, ~115 GB of
    FP32 state each) until the device runs out: the failing create returns
    GSSTV_ERR_OOM, leaks nothing, and the device stays usable."""
    from paper_2510_00562_gb300 import binding as B
    held, code = [], None
    try:
        for _ in range(4):
            try:
                held.append(GeoSSTVSolver(8192, 8192, 10, make_params()))
            except B.GsstvError as e:
                code = e.code
                break
    finally:
        for h in held:
            h.close()
    assert code == B.GSSTV_ERR_OOM
    free, _ = torch.cuda.mem_get_info()
    assert free > 200 * 2**30
    with GeoSSTVSolver(8, 8, 2, make_params(max_iter=2)) as sol:
        sol.solve(to_dev(np.full((2, 8, 8), 0.5, np.float32)))


def test_oversized_cube_is_refused():
    from paper_2510_00562_gb300 import binding as B
    with pytest.raises(B.GsstvError) as ei:
        GeoSSTVSolver(1 << 20, 1 << 14, 4096, make_params())
    assert ei.value.code == B.GSSTV_ERR_ARG


def test_autotune_picks_a_valid_run_length_and_keeps_the_results():
    """gsstv_autotune changes only how the fused kernel's CTAs split the
    bands: the solve afterwards equals the one before up to the summation
    order of the l1 window statistics, and still matches the oracle."""
    n1, n2, n3, iters = 70, 100, 40, 60
    pb = _problem(n1, n2, n3, seed=4)
    v = to_dev(pb["v"])
    p = make_params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=0.03, max_iter=iters)
    with GeoSSTVSolver(n1, n2, n3, p) as sol:
        u0, s0, t0, _ = sol.solve(v)
        before = sol.stats()["iterations"]
        chunk = sol.autotune(v, passes=4)
        assert sol.stats()["iterations"] == before
        assert 8 <= chunk <= n3
        u1, s1, t1, n = sol.solve(v)
    assert n == iters
    for a, b in ((u1, u0), (s1, s0), (t1, t0)):
        assert rel(a.cpu().numpy(), b.cpu().numpy()) < 1e-6
    st, _ = o.solve(pb["v"].astype(np.float64), oracle_params(p), iters)
    assert rel(u1.cpu().numpy(), st.u) < 1e-5
