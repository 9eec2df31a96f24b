"""The FP64 reverse mode of Algorithm 1 (oracle.adjoint) against central
finite differences of the forward oracle: one pass at generic random points,
and the unrolled gradient of the MSE loss with respect to v and (eps, alpha,
beta, omega)."""
import numpy as np
import pytest

from oracle import adjoint as A
from oracle import ppds as o
from paper_2510_00562_gb300 import synth

KEYS = o.State.names()


def _random_point(shape, seed, scale=0.1):
    rng = np.random.default_rng(seed)
    n3, n1, n2 = shape
    g = lambda *lead: rng.standard_normal(lead + shape) * scale
    st = o.State(u=rng.uniform(-0.1, 1.1, shape), s=g(), t=g(), w1=g(3, 2), w2=g(3, 2), y1=g(2), y2=g(2),
                 y3=g(), y4=g())
    v = rng.uniform(0, 1, shape)
    return st, v


def _params_for(st, v, omega=0.05):
    """Radii that keep both l1 balls and the l2 ball active at this point."""
    p = o.Params(omega=omega)
    a_s = st.s - p.gamma_s * st.y4
    a_t = st.t - p.gamma_t * (o.Dv_T(st.y3) + st.y4)
    p.alpha = 0.5 * float(np.abs(a_s).sum())
    p.beta = 0.6 * float(np.abs(a_t).sum())
    p.eps = 0.02 * np.sqrt(v.size)
    return p


def _with(p, **kw):
    q = o.Params(**p.as_dict())
    for k, x in kw.items():
        setattr(q, k, x)
    return q


def _inner(a: o.State, b: o.State):
    return sum(float(np.sum(getattr(a, k) * getattr(b, k))) for k in KEYS)


def _axpy(st: o.State, h, d: o.State):
    return o.State(**{k: getattr(st, k) + h * getattr(d, k) for k in KEYS})


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_step_vjp_matches_central_differences(seed):
    shape = (4, 6, 5)
    st, v = _random_point(shape, seed)
    p = _params_for(st, v)
    rng = np.random.default_rng(100 + seed)
    out_w = o.State(**{k: rng.standard_normal(getattr(st, k).shape) for k in KEYS})   # weights of the outputs
    d = o.State(**{k: rng.standard_normal(getattr(st, k).shape) for k in KEYS})
    dv = rng.standard_normal(shape)
    dp = {k: float(rng.standard_normal()) for k in A.PARAMS}
    scale = {"eps": p.eps, "alpha": p.alpha, "beta": p.beta, "omega": p.omega}

    def f(h):
        q = _with(p, **{k: getattr(p, k) + h * dp[k] * 1e-2 * scale[k] for k in A.PARAMS})
        return _inner(out_w, o.ppds_step(_axpy(st, h, d), v + h * dv, q))

    h = 1e-6
    fd = (f(h) - f(-h)) / (2 * h)
    bar, vbar, pbar = A.step_vjp(st, v, p, out_w)
    an = _inner(bar, d) + float(np.sum(vbar * dv)) + sum(pbar[k] * dp[k] * 1e-2 * scale[k] for k in A.PARAMS)
    assert an == pytest.approx(fd, rel=1e-6, abs=1e-9)
    # each parameter alone
    for k in A.PARAMS:
        hk = 1e-7 * scale[k]
        fk = lambda s: _inner(out_w, o.ppds_step(st, v, _with(p, **{k: getattr(p, k) + s})))
        assert pbar[k] == pytest.approx((fk(hk) - fk(-hk)) / (2 * hk), rel=1e-5, abs=1e-8), k


def test_step_vjp_inside_the_balls_is_the_identity_part():
    """With radii large enough that no projection is active, the s and t
    adjoints pass through the projections unchanged and the radii get none."""
    shape = (3, 4, 5)
    st, v = _random_point(shape, 7)
    p = o.Params(eps=1e6, alpha=1e6, beta=1e6, omega=0.05)
    bar0 = o.State(**{k: np.zeros_like(getattr(st, k)) for k in KEYS})
    bar0.s = np.ones(shape)
    out, _, pbar = A.step_vjp(st, v, p, bar0)
    assert pbar["alpha"] == 0.0 and pbar["beta"] == 0.0 and pbar["eps"] == 0.0
    # s_bar = P'(.)^T 1 - (nothing from the duals) = 1 for the s path
    assert np.allclose(out.s, 1.0)
    assert np.allclose(out.y4, -p.gamma_s)


def test_unrolled_grad_matches_central_differences():
    """Without salt-and-pepper: those voxels are exactly 0 or 1, on the kinks
    of the box projection at the first pass (u = v, duals zero), where the
    loss has no derivative.  The sparse radius is set directly instead."""
    pb = synth.make_problem(7, 6, 4, seed=2, noise=synth.NoiseSpec(sigma=0.1, sp_rate=0.0, stripe_rate=0.3,
                                                                  stripe_amp=0.25))
    v = pb["v"].astype(np.float64)
    ub = pb["u_bar"].astype(np.float64)
    assert not np.any((v == 0.0) | (v == 1.0))
    # radii small enough that all three balls act within the 8 passes
    p = o.Params(eps=pb["eps"], alpha=0.01 * v.size, beta=0.1 * pb["beta"], omega=0.05)
    iters = 8
    loss, vbar, pbar = A.unrolled_grad(v, ub, p, iters)
    assert all(abs(pbar[k]) > 1e-6 for k in A.PARAMS), pbar

    def L(vv, q):
        return float(np.mean((A.unrolled(vv, q, iters)[-1].u - ub) ** 2))

    assert loss == pytest.approx(L(v, p), rel=1e-14)
    rng = np.random.default_rng(5)
    dv = rng.standard_normal(v.shape)
    h = 1e-6
    fd = (L(v + h * dv, p) - L(v - h * dv, p)) / (2 * h)
    assert float(np.sum(vbar * dv)) == pytest.approx(fd, rel=1e-5)
    for k in A.PARAMS:
        x = getattr(p, k)
        hk = 1e-6 * x
        fk = (L(v, _with(p, **{k: x + hk})) - L(v, _with(p, **{k: x - hk}))) / (2 * hk)
        assert pbar[k] == pytest.approx(fk, rel=1e-4, abs=1e-12), k


def test_unrolled_grad_checkpointing_changes_nothing():
    """Running segments again from checkpoints repeats the same FP64
    arithmetic: the gradient is bit-identical to the one from the kept
    trajectory."""
    pb = synth.make_problem(6, 5, 4, seed=4)
    v = pb["v"].astype(np.float64)
    ub = pb["u_bar"].astype(np.float64)
    p = o.Params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=0.05)
    ref = A.unrolled_grad(v, ub, p, 11)
    for c in (1, 3, 4, 11, 50):
        got = A.unrolled_grad(v, ub, p, 11, ckpt_every=c)
        assert got[0] == ref[0]
        assert np.array_equal(got[1], ref[1])
        assert got[2] == ref[2]


def _bad_l12(x, pbar, g):          # drops the rank-one term of the shrink Jacobian
    nrm = np.sqrt(x[:, 0] ** 2 + x[:, 1] ** 2)
    act = nrm > g
    safe = np.where(act, nrm, 1.0)
    xbar = np.where(act[:, None], (1.0 - g / safe)[:, None] * pbar, 0.0)
    return xbar, -float(np.where(act, ((x / safe[:, None]) * pbar).sum(axis=1), 0.0).sum())


def _bad_l1(x, pbar, r):           # keeps the support but forgets the mean removal
    if np.abs(x).sum() <= r:
        return pbar.copy(), 0.0
    _, tau = o.proj_l1ball(x, r)
    act = np.abs(x) > tau
    return np.where(act, pbar, 0.0), 0.0


def _bad_l2(q, ybar, eps, g):      # treats the l2 step as a plain rescale
    nq = float(np.sqrt(np.sum(q * q)))
    if nq <= eps * g:
        return np.zeros_like(q), 0.0
    return (1.0 - eps * g / nq) * ybar, -g * float(np.sum(q / nq * ybar))


def _bad_box(x, pbar, lo, hi):     # passes the adjoint through the clamp everywhere
    return pbar.copy()


@pytest.mark.parametrize("name,bad", [("_l12_vjp", _bad_l12), ("_l1_vjp", _bad_l1), ("_l2_vjp", _bad_l2),
                                      ("_box_vjp", _bad_box)])
def test_planted_mistakes_fail_the_differences(monkeypatch, name, bad):
    """Each Jacobian of the reverse mode matters: replacing one by a plausible
    wrong version breaks the agreement with central differences."""
    shape = (4, 6, 5)
    st, v = _random_point(shape, 0)
    p = _params_for(st, v)
    rng = np.random.default_rng(100)
    out_w = o.State(**{k: rng.standard_normal(getattr(st, k).shape) for k in KEYS})
    d = o.State(**{k: rng.standard_normal(getattr(st, k).shape) for k in KEYS})
    dv = rng.standard_normal(shape)
    h = 1e-6
    fd = (_inner(out_w, o.ppds_step(_axpy(st, h, d), v + h * dv, p)) -
          _inner(out_w, o.ppds_step(_axpy(st, -h, d), v - h * dv, p))) / (2 * h)

    def an():
        bar, vbar, _ = A.step_vjp(st, v, p, out_w)
        return _inner(bar, d) + float(np.sum(vbar * dv))

    assert an() == pytest.approx(fd, rel=1e-6, abs=1e-9)     # the real one agrees
    monkeypatch.setattr(A, name, bad)
    assert abs(an() - fd) > 1e-4 * abs(fd), name
