"""Reverse mode of Algorithm 1 on the GPU (gsstv_vjp_step, gsstv_unrolled_vjp)
against the FP64 reverse mode of the oracle, which is itself pinned to
central finite differences of the forward oracle.

Tolerances (relative L2 error per variable):
  * one pass from a random state: 1e-5 -- float32 arithmetic on float32
    inputs, a few roundings of ~6e-8 per term, amplified by the stencil sums
    and by the cancellation in x_bar = -x'_bar + P'(.)^T (x+_bar + 2 x'_bar);
    the parameter adjoints are global sums: relative 1e-5;
  * K passes from the standard start: 1e-3 on v_bar and on each parameter
    adjoint -- the float32 forward trajectory drifts from the FP64 one by
    ~1e-6 relative per pass and the adjoint sweep adds its own rounding at
    every pass;
  * against central differences of the float32 forward run (step 1e-3 of
    each parameter): 1e-2 -- the secant over that step crosses kinks of the
    box, the shrinkage and the l1 projections, where the derivative jumps.
"""
import math

import numpy as np
import pytest
import torch

from oracle import adjoint as A
from oracle import ppds as o
from paper_2510_00562_gb300 import synth
from paper_2510_00562_gb300.autograd import unrolled_geosstv
from paper_2510_00562_gb300.solver import GRAD_PARAMS, STATE_KEYS, GeoSSTVSolver, make_params

pytestmark = pytest.mark.gpu


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


def _random_point(n1, n2, n3, seed, radii_scale=0.4):
    rs = synth.random_state(n1, n2, n3, seed=seed, scale=0.1)
    v = np.random.default_rng(seed + 100).uniform(0, 1, size=(n3, n1, n2)).astype(np.float32)
    s64 = rs["s"].astype(np.float64)
    t64 = rs["t"].astype(np.float64)
    kw = dict(eps=0.02 * math.sqrt(v.size), alpha=radii_scale * np.abs(s64).sum(),
              beta=radii_scale * np.abs(t64).sum(), omega=0.05)
    return rs, v, kw


# (N1, N2, N3): ragged N2 (not a multiple of the row pitch), one band, one row
STEP_SHAPES = [(37, 45, 9), (16, 32, 1), (1, 7, 3), (70, 100, 20)]


@pytest.mark.parametrize("shape", STEP_SHAPES)
@pytest.mark.parametrize("radii", ["active", "inactive"])
def test_vjp_step_matches_oracle(shape, radii):
    n1, n2, n3 = shape
    rs, v, kw = _random_point(n1, n2, n3, seed=n1 + 3 * n3)
    if radii == "inactive":
        kw.update(eps=1e6, alpha=1e6, beta=1e6)
    p = make_params(graph_iters=0, **kw)
    rng = np.random.default_rng(7)
    bar_next = {k: rng.standard_normal(rs[k].shape).astype(np.float32) for k in STATE_KEYS}
    with GeoSSTVSolver(n1, n2, n3, p) as sol:
        sol.load(to_dev(v))
        x = {k: to_dev(rs[k]) for k in STATE_KEYS}
        sol.set_state(x)
        sol.iterate(1)
        x_next = sol.get_state()
        bar, vbar, pbar = sol.vjp_step(x, x_next, {k: to_dev(bar_next[k]) for k in STATE_KEYS})
        got = {k: t.cpu().numpy() for k, t in bar.items()}
        vbar = vbar.cpu().numpy()
    st = o.State(**{k: rs[k].astype(np.float64) for k in STATE_KEYS})
    ref, vref, pref = A.step_vjp(st, v.astype(np.float64), oracle_params(p),
                                 o.State(**{k: bar_next[k].astype(np.float64) for k in STATE_KEYS}))
    for k in STATE_KEYS:
        e = rel(got[k], getattr(ref, k))
        assert e < 1e-5, (k, e)
    assert rel(vbar, vref) < 1e-5
    for k in GRAD_PARAMS:
        if radii == "inactive" and k != "omega":
            assert pbar[k] == 0.0 and pref[k] == 0.0, k
        else:
            assert pbar[k] == pytest.approx(pref[k], rel=1e-5, abs=1e-9 * np.linalg.norm(vref)), k


def test_vjp_step_in_place_and_accumulating():
    """bar may be bar_next itself; v_bar and the parameter adjoints accumulate."""
    n1, n2, n3 = 24, 19, 5
    rs, v, kw = _random_point(n1, n2, n3, seed=11)
    p = make_params(graph_iters=0, **kw)
    rng = np.random.default_rng(8)
    bn = {k: rng.standard_normal(rs[k].shape).astype(np.float32) for k in STATE_KEYS}
    with GeoSSTVSolver(n1, n2, n3, p) as sol:
        sol.load(to_dev(v))
        x = {k: to_dev(rs[k]) for k in STATE_KEYS}
        sol.set_state(x)
        sol.iterate(1)
        x_next = sol.get_state()
        bar1, vb1, pb1 = sol.vjp_step(x, x_next, {k: to_dev(bn[k]) for k in STATE_KEYS})
        src = {k: to_dev(bn[k]) for k in STATE_KEYS}
        vacc = torch.ones(v.shape, dtype=torch.float32, device="cuda")
        bar2, vb2, pb2 = sol.vjp_step(x, x_next, src, vbar=vacc, in_place=True)
        assert bar2["u"].data_ptr() == src["u"].data_ptr()
        # equal up to the order of the device-wide double sums
        for k in STATE_KEYS:
            torch.testing.assert_close(bar2[k], bar1[k], rtol=1e-6, atol=1e-7)
        torch.testing.assert_close(vb2, vb1 + 1.0, rtol=1e-6, atol=1e-7)
        for k in GRAD_PARAMS:
            assert pb2[k] == pytest.approx(pb1[k], rel=1e-12, abs=1e-300)


def _denoise_problem(n1, n2, n3, seed):
    pb = synth.make_problem(n1, n2, n3, seed=seed, noise=synth.NoiseSpec(
        sigma=0.1, sp_rate=0.05, stripe_rate=0.3, stripe_amp=0.25))
    return pb


@pytest.mark.parametrize("shape,ckpt", [((24, 20, 6), 0), ((24, 20, 6), 1), ((24, 20, 6), 7), ((24, 20, 6), 40),
                                        ((23, 21, 5), 3)])       # odd voxel count
def test_unrolled_gradient_matches_oracle(shape, ckpt):
    (n1, n2, n3), iters = shape, 40
    pb = _denoise_problem(n1, n2, n3, seed=3)
    v = pb["v"].astype(np.float32)
    ub = pb["u_bar"].astype(np.float64)
    # radii that keep all three balls active during the run
    kw = dict(eps=pb["eps"], alpha=0.01 * v.size, beta=0.1 * pb["beta"], omega=0.05)
    p = make_params(graph_iters=16, max_iter=iters, **kw)
    loss, vref, pref = A.unrolled_grad(v.astype(np.float64), ub, oracle_params(p), iters)
    with GeoSSTVSolver(n1, n2, n3, p) as sol:
        u, _, _, _ = sol.solve(to_dev(v))
        seed = 2.0 * (u.double() - torch.from_numpy(ub).cuda()) / v.size
        sol.load(to_dev(v))
        vbar, pbar = sol.unrolled_vjp(iters, seed.float().contiguous(), ckpt_every=ckpt)
        vbar = vbar.cpu().numpy()
    assert float(((u.double().cpu().numpy() - ub) ** 2).mean()) == pytest.approx(loss, rel=1e-4)
    assert rel(vbar, vref) < 1e-3
    for k in GRAD_PARAMS:
        assert abs(pref[k]) > 0, k
        assert pbar[k] == pytest.approx(pref[k], rel=1e-3), k


def test_unrolled_gradient_does_not_depend_on_the_checkpoint_spacing():
    """Equal up to rounding: a re-run from a checkpoint may find an l1
    threshold by another search (window or radix), which rounds differently."""
    n1, n2, n3, iters = 40, 33, 7, 30
    pb = _denoise_problem(n1, n2, n3, seed=5)
    v = to_dev(pb["v"])
    p = make_params(graph_iters=16, eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=0.05)
    g = torch.from_numpy(np.random.default_rng(9).standard_normal(pb["v"].shape).astype(np.float32)).cuda()
    out = []
    with GeoSSTVSolver(n1, n2, n3, p) as sol:
        for ck in (1, 5, 30):
            sol.load(v)
            out.append(sol.unrolled_vjp(iters, g, ckpt_every=ck))
    for vb, pbar in out[1:]:
        assert rel(vb.cpu().numpy(), out[0][0].cpu().numpy()) < 1e-4
        for k in GRAD_PARAMS:
            assert pbar[k] == pytest.approx(out[0][1][k], rel=1e-4, abs=1e-12), k


def test_unrolled_gradient_vs_central_differences():
    """The GPU gradient against central differences of the GPU forward run."""
    n1, n2, n3, iters = 48, 40, 16, 60
    pb = _denoise_problem(n1, n2, n3, seed=6)
    v = to_dev(pb["v"])
    ub = torch.from_numpy(pb["u_bar"].astype(np.float64)).cuda()
    prm = dict(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=0.05)
    with GeoSSTVSolver(n1, n2, n3, make_params(graph_iters=16, max_iter=iters, **prm)) as sol:
        def loss(**over):
            sol.set_params(**{**prm, **over})
            u, _, _, _ = sol.solve(v)
            return float(((u.double() - ub) ** 2).mean()), u

        l0, u = loss()
        sol.load(v)
        _, pbar = sol.unrolled_vjp(iters, ((2.0 / v.numel()) * (u.double() - ub)).float().contiguous())
        for k in GRAD_PARAMS:
            h = 1e-3 * prm[k]
            fd = (loss(**{k: prm[k] + h})[0] - loss(**{k: prm[k] - h})[0]) / (2 * h)
            assert pbar[k] == pytest.approx(fd, rel=1e-2), (k, pbar[k], fd)


def test_zero_iterations_is_the_identity():
    n1, n2, n3 = 8, 9, 3
    v = to_dev(np.random.default_rng(1).uniform(0, 1, (n3, n1, n2)))
    g = to_dev(np.random.default_rng(2).standard_normal((n3, n1, n2)))
    with GeoSSTVSolver(n1, n2, n3, make_params()) as sol:
        sol.load(v)
        vb, pbar = sol.unrolled_vjp(0, g)
    assert torch.equal(vb, g)
    assert all(x == 0.0 for x in pbar.values())


def test_autograd_function():
    n1, n2, n3, iters = 24, 20, 6, 25
    pb = _denoise_problem(n1, n2, n3, seed=4)
    v = to_dev(pb["v"]).requires_grad_(True)
    ub = to_dev(pb["u_bar"])
    eps = torch.tensor(pb["eps"], dtype=torch.float64, requires_grad=True)
    alpha = torch.tensor(0.01 * v.numel(), dtype=torch.float64, requires_grad=True)
    beta = torch.tensor(0.1 * pb["beta"], dtype=torch.float64, requires_grad=True)
    omega = torch.tensor(0.05, dtype=torch.float64, requires_grad=True)
    u = unrolled_geosstv(v, eps, alpha, beta, omega, iters)
    loss = ((u - ub) ** 2).mean()
    loss.backward()
    p = make_params(eps=pb["eps"], alpha=0.01 * v.numel(), beta=0.1 * pb["beta"], omega=0.05)
    lref, vref, pref = A.unrolled_grad(pb["v"].astype(np.float64), pb["u_bar"].astype(np.float64),
                                       oracle_params(p), iters)
    assert float(loss.detach()) == pytest.approx(lref, rel=1e-4)
    assert rel(v.grad.cpu().numpy(), vref) < 1e-3
    for k, t in zip(GRAD_PARAMS, (eps, alpha, beta, omega)):
        assert float(t.grad) == pytest.approx(pref[k], rel=1e-3), k
