"""FP64 reverse mode of the GeoSSTV P-PDS iteration (Algorithm 1), unrolled.

TEST INFRASTRUCTURE ONLY, like ``oracle.ppds`` (same import rules).  It gives
the gradient of a loss of the K-th iterate with respect to the observation v,
the initial state and the parameters (eps, alpha, beta, omega), by running
the transpose of every step of ``ppds_step`` in reverse order.

The operators of Algorithm 1 are not differentiable everywhere; the
derivatives taken here are the ones that hold almost everywhere:

* box projection (Eq. 21): the adjoint passes where mu_lo < x < mu_hi;
* group soft-threshold (Eq. 24) of a 2-vector x with threshold g: for
  ||x|| > g the Jacobian is (1 - g/||x||) I + g x x^T / ||x||^3 and the
  derivative in g is -x/||x||; zero otherwise;
* l1-ball projection (Sec. III-B): inside the ball the identity; otherwise,
  with A = {|x_i| > tau} and sigma = sign(x), P_i = sigma_i (|x_i| - tau) on A
  and tau = (sum_A |x| - r)/|A|, so the adjoint is
  x_bar_i = [i in A] (p_bar_i - sigma_i S/|A|), S = sum_A sigma p_bar, and the
  derivative in the radius is S/|A|;
* l2-ball step (Eq. 23 through Moreau's identity, Eq. 3): y4 = (1 - c) q with
  q = y4' - g v and c = min(1, eps g/||q||): for ||q|| > eps g the Jacobian is
  I - (eps g/||q||)(I - q^ q^^T) (q^ = q/||q||) and the derivative in eps is
  -g q^; zero otherwise.

The linear operators are transposed exactly (D <-> D^T, L <-> L^T, ...).
"""
from __future__ import annotations

import numpy as np

from . import ppds as o

__all__ = ["step_vjp", "unrolled", "unrolled_grad"]

PARAMS = ("eps", "alpha", "beta", "omega")


def _box_vjp(x, pbar, lo, hi):
    return pbar * ((x > lo) & (x < hi))


def _l12_vjp(x, pbar, g):
    """x, pbar: (G, 2, ...); returns (x_bar, g_bar)."""
    nrm = np.sqrt(x[:, 0] ** 2 + x[:, 1] ** 2)
    act = nrm > g
    safe = np.where(act, nrm, 1.0)
    xh = x / safe[:, None]                                  # x / ||x|| on active groups
    dot = (xh * pbar).sum(axis=1)                           # x^ . p_bar
    xbar = (1.0 - g / safe)[:, None] * pbar + (g / safe)[:, None] * xh * dot[:, None]
    xbar = np.where(act[:, None], xbar, 0.0)
    gbar = -float(np.where(act, dot, 0.0).sum())
    return xbar, gbar


def _l1_vjp(x, pbar, r):
    """Adjoint of the l1-ball projection at x (radius r); returns (x_bar, r_bar)."""
    if np.abs(x).sum() <= r:
        return pbar.copy(), 0.0
    _, tau = o.proj_l1ball(x, r)
    act = np.abs(x) > tau
    sg = np.sign(x)
    na = int(act.sum())
    if na == 0:
        return np.zeros_like(x), 0.0
    S = float((sg * pbar)[act].sum())
    xbar = np.where(act, pbar - sg * S / na, 0.0)
    return xbar, S / na


def _l2_vjp(q, ybar, eps, g):
    """Adjoint of y4 = (1 - c) q; returns (q_bar, eps_bar)."""
    nq = float(np.sqrt(np.sum(q * q)))
    if nq <= eps * g:
        return np.zeros_like(q), 0.0
    qh = q / nq
    d = float(np.sum(qh * ybar))
    return ybar - (eps * g / nq) * (ybar - qh * d), -g * d


def step_vjp(st: o.State, v, p: o.Params, bar: o.State):
    """Vector-Jacobian product of ``o.ppds_step`` at (st, v).

    bar: adjoint of the step's output.  Returns (adjoint of st as a State,
    adjoint of v, dict of adjoints of eps, alpha, beta, omega)."""
    v = np.asarray(v, dtype=np.float64)
    # forward intermediates, as in ppds_step
    a_u = st.u - p.gamma_u * (o.D_T(st.y1) + o.Ds_T(o.D_T(st.y2)) + st.y4)
    a_s = st.s - p.gamma_s * st.y4
    a_t = st.t - p.gamma_t * (o.Dv_T(st.y3) + st.y4)
    a_w1 = st.w1 + p.gamma_w1 * o.L(st.y1)
    a_w2 = st.w2 + p.gamma_w2 * o.L(st.y2)
    u1 = o.proj_box(a_u, p.mu_lo, p.mu_hi)
    s1, _ = o.proj_l1ball(a_s, p.alpha)
    t1, _ = o.proj_l1ball(a_t, p.beta)
    ub, sb, tb = 2 * u1 - st.u, 2 * s1 - st.s, 2 * t1 - st.t
    y4p = st.y4 + p.gamma_y4 * (ub + sb + tb)
    q = y4p - p.gamma_y4 * v

    pb = {k: 0.0 for k in PARAMS}
    # y4 = (1 - c) q, q = y4' - g4 v, y4' = y4 + g4 (u' + s' + t')
    qbar, pb["eps"] = _l2_vjp(q, bar.y4, p.eps, p.gamma_y4)
    vbar = -p.gamma_y4 * qbar
    y4bar = qbar.copy()
    ubar_b = p.gamma_y4 * qbar
    sbar_b = p.gamma_y4 * qbar
    tbar_b = p.gamma_y4 * qbar.copy()
    # y3 = y3 + g3 D_v t'
    y3bar = bar.y3.copy()
    tbar_b = tbar_b + p.gamma_y3 * o.Dv_T(bar.y3)
    # y2 = y2 + g2 (D D_s u' - L^T w2')
    y2bar = bar.y2.copy()
    ubar_b = ubar_b + p.gamma_y2 * o.Ds_T(o.D_T(bar.y2))
    w2bar_b = -p.gamma_y2 * o.L(bar.y2)
    # y1 = y1 + g1 (D u' - L^T w1')
    y1bar = bar.y1.copy()
    ubar_b = ubar_b + p.gamma_y1 * o.D_T(bar.y1)
    w1bar_b = -p.gamma_y1 * o.L(bar.y1)
    # extrapolations x' = 2 x+ - x
    u1bar = bar.u + 2 * ubar_b
    s1bar = bar.s + 2 * sbar_b
    t1bar = bar.t + 2 * tbar_b
    w11bar = bar.w1 + 2 * w1bar_b
    w21bar = bar.w2 + 2 * w2bar_b
    ubar, sbar, tbar, w1bar, w2bar = -ubar_b, -sbar_b, -tbar_b, -w1bar_b, -w2bar_b
    # u+ = box(u - g_u (D^T y1 + D_s^T D^T y2 + y4))
    au_bar = _box_vjp(a_u, u1bar, p.mu_lo, p.mu_hi)
    ubar = ubar + au_bar
    gbar = -p.gamma_u * au_bar
    y1bar = y1bar + o.D(gbar)
    y2bar = y2bar + o.D(o.Ds(gbar))
    y4bar = y4bar + gbar
    # s+ = P_alpha(s - g_s y4)
    as_bar, pb["alpha"] = _l1_vjp(a_s, s1bar, p.alpha)
    sbar = sbar + as_bar
    y4bar = y4bar - p.gamma_s * as_bar
    # t+ = P_beta(t - g_t (D_v^T y3 + y4))
    at_bar, pb["beta"] = _l1_vjp(a_t, t1bar, p.beta)
    tbar = tbar + at_bar
    y3bar = y3bar - p.gamma_t * o.Dv(at_bar)
    y4bar = y4bar - p.gamma_t * at_bar
    # w1+ = prox(w1 + g_w1 L y1) with threshold g_w1 omega; w2+ likewise (threshold g_w2)
    aw1_bar, th1 = _l12_vjp(a_w1, w11bar, p.gamma_w1 * p.omega)
    w1bar = w1bar + aw1_bar
    y1bar = y1bar + p.gamma_w1 * o.L_T(aw1_bar)
    pb["omega"] = p.gamma_w1 * th1
    aw2_bar, _ = _l12_vjp(a_w2, w21bar, p.gamma_w2)
    w2bar = w2bar + aw2_bar
    y2bar = y2bar + p.gamma_w2 * o.L_T(aw2_bar)
    out = o.State(u=ubar, s=sbar, t=tbar, w1=w1bar, w2=w2bar, y1=y1bar, y2=y2bar, y3=y3bar, y4=y4bar)
    return out, vbar, pb


def unrolled(v, p: o.Params, iters: int, state: o.State | None = None):
    """The trajectory of ``iters`` passes (states 0..iters)."""
    st = o.init_state(v) if state is None else state.copy()
    traj = [st]
    for _ in range(iters):
        st = o.ppds_step(st, v, p)
        traj.append(st)
    return traj


def unrolled_grad(v, u_ref, p: o.Params, iters: int, ckpt_every: int | None = None):
    """Loss = mean((u_K - u_ref)^2) after ``iters`` passes from the standard
    start (u = v, the rest zero).  Returns (loss, v_bar, params_bar).

    ckpt_every: keep only every ckpt_every-th state and run each segment
    again from it during the reverse sweep (the same arithmetic, less
    memory); None keeps the whole trajectory."""
    v = np.asarray(v, dtype=np.float64)
    C = iters if not ckpt_every else max(1, min(int(ckpt_every), iters))
    # forward: the states at passes 0, C, 2C, ... and the last one
    ckpt = {}
    st = o.init_state(v)
    for k in range(iters):
        if k % C == 0:
            ckpt[k] = st
        st = o.ppds_step(st, v, p)
    last = st
    uk = last.u
    n = uk.size
    loss = float(np.mean((uk - u_ref) ** 2))
    z = lambda x: np.zeros_like(x)
    bar = o.State(u=2.0 * (uk - u_ref) / n, s=z(last.s), t=z(last.t), w1=z(last.w1), w2=z(last.w2),
                  y1=z(last.y1), y2=z(last.y2), y3=z(last.y3), y4=z(last.y4))
    vbar = np.zeros_like(v)
    pbar = {k: 0.0 for k in PARAMS}
    for start in sorted(ckpt, reverse=True):
        seg = [ckpt[start]]                # the segment's states, run again from its checkpoint
        for _ in range(start + 1, min(start + C, iters)):
            seg.append(o.ppds_step(seg[-1], v, p))
        for st_k in reversed(seg):
            bar, vb, pb = step_vjp(st_k, v, p, bar)
            vbar += vb
            for key in PARAMS:
                pbar[key] += pb[key]
    vbar += bar.u                          # the start u = v
    return loss, vbar, pbar
