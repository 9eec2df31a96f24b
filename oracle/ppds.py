"""FP64 CPU oracle of the GeoSSTV P-PDS iteration (Takemoto & Ono, arXiv 2510.00562).

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously-correct
reference that the CUDA path is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline leg and its
``--impl reference`` arm) may import it.  It shares no code with the CUDA path
and imports nothing from the ``paper_2510_00562_gb300`` package.

Every operator is one whole-array NumPy pass in float64, written in the order
and notation of the paper:

* forward differences with Neumann boundary (Sec. II-A);
* Condat's interpolators L_vert, L_hori, L_cent and L (Sec. II-D, Eqs. 10-12;
  Sec. III-A, Eq. 13);
* the proximity operators of Eqs. 21-24 and the l1-ball projection named in
  Sec. III-B;
* one pass of Algorithm 1 (the P-PDS solver of Prob. 20).

Array layout: a cube is indexed ``x[b, i, j]`` with band b in [0, N3), row i in
[0, N1) (vertical) and column j in [0, N2) (horizontal); C-contiguous, so j is
the fastest axis.  A dual pair y in R^{2N} is ``y[c, b, i, j]`` with c = 0 the
vertical component (located at (i+1/2, j)) and c = 1 the horizontal one (at
(i, j+1/2)).  An auxiliary w in R^{6N} is ``w[g, c, b, i, j]`` with g = 0, 1, 2
for the grids (i+1/2, j), (i, j+1/2), (i, j) of L_vert, L_hori, L_cent.

Readings of the paper taken here:

* D_v differentiates along rows i (vertical), D_h along columns j, D_s along
  bands b.  Sec. II-A names them "horizontal, vertical, spectral"; the
  subscripts and the stripe model (D_v t = 0 for stripes constant along a
  column, Eq. 15) fix the reading used here.
* Condat's interpolators are not restated in the paper (it defers to Eqs. 9-14
  of Condat 2017).  Reading: the dual pair is first masked where D is
  structurally zero (vertical component on the last row, horizontal component
  on the last column) and extended by zero outside the image; L_vert averages
  the four horizontal neighbours onto (i+1/2, j) and is zero on the last row;
  L_hori averages the four vertical neighbours onto (i, j+1/2) and is zero on
  the last column; L_cent averages the two neighbours of each component onto
  (i, j).
* L is read as a map R^{2N} -> R^{6N} (Eq. 13 prints its size transposed);
  Algorithm 1 applies L to y and L^T to w.
* The dual steps use "+" (ascent), as Algorithm 1 prints them; the generic
  P-PDS display (Eq. 7) prints "-" for the dual step, read as a typo.
* Initial point: u = v, all other variables (including y4, which Algorithm 1
  does not list) zero.
"""
from __future__ import annotations

from dataclasses import dataclass, field, asdict

import numpy as np

__all__ = [
    "Params", "State",
    "Dv", "Dv_T", "Dh", "Dh_T", "Ds", "Ds_T", "D", "D_T",
    "shift", "L", "L_T",
    "prox_l12", "proj_box", "proj_l1ball", "proj_l2ball",
    "init_state", "ppds_step", "rel_change", "solve",
    "apply_A", "apply_AT", "geosstv_objective",
]


# ---------------------------------------------------------------------------
# Parameters and state
# ---------------------------------------------------------------------------
@dataclass
class Params:
    """Radii, box, balance and step sizes of Prob. 15 / Algorithm 1.

    Defaults for the step sizes are the values Sec. III-B prints after Eq. 24
    (gamma_u = 1/13, gamma_w1 = gamma_w2 = 1/4, gamma_s = 1, gamma_t = 1/3,
    gamma_y1..4 = 1/5).
    """
    eps: float = 1.0          # radius of the l2 fidelity ball B_{2,eps}^v (Eq. 18)
    alpha: float = 1.0        # radius of the l1 ball on s (Eq. 16)
    beta: float = 1.0         # radius of the l1 ball on t (Eq. 17)
    omega: float = 0.03       # balance of the first-order term (Eq. 13)
    mu_lo: float = 0.0        # box [mu_lo, mu_hi] on u (Eq. 19)
    mu_hi: float = 1.0
    gamma_u: float = 1.0 / 13.0
    gamma_w1: float = 1.0 / 4.0
    gamma_w2: float = 1.0 / 4.0
    gamma_s: float = 1.0
    gamma_t: float = 1.0 / 3.0
    gamma_y1: float = 1.0 / 5.0
    gamma_y2: float = 1.0 / 5.0
    gamma_y3: float = 1.0 / 5.0
    gamma_y4: float = 1.0 / 5.0

    def as_dict(self):
        return asdict(self)


@dataclass
class State:
    """Primal (u, s, t, w1, w2) and dual (y1..y4) iterates of Algorithm 1."""
    u: np.ndarray
    s: np.ndarray
    t: np.ndarray
    w1: np.ndarray   # (3, 2, N3, N1, N2)
    w2: np.ndarray   # (3, 2, N3, N1, N2)
    y1: np.ndarray   # (2, N3, N1, N2)
    y2: np.ndarray   # (2, N3, N1, N2)
    y3: np.ndarray   # (N3, N1, N2)
    y4: np.ndarray   # (N3, N1, N2)
    extra: dict = field(default_factory=dict)

    def copy(self) -> "State":
        return State(*(getattr(self, k).copy() for k in State.names()))

    @staticmethod
    def names():
        return ("u", "s", "t", "w1", "w2", "y1", "y2", "y3", "y4")


# ---------------------------------------------------------------------------
# Forward differences, Neumann boundary (Sec. II-A)
# ---------------------------------------------------------------------------
def _fwd(x, axis):
    """x[k+1] - x[k] along ``axis``; the last entry is 0 (Neumann)."""
    out = np.zeros_like(x, dtype=np.float64)
    n = x.shape[axis]
    hi = [slice(None)] * x.ndim
    lo = [slice(None)] * x.ndim
    hi[axis] = slice(1, n)
    lo[axis] = slice(0, n - 1)
    out[tuple(lo)] = x[tuple(hi)] - x[tuple(lo)]
    return out


def _fwd_T(y, axis):
    """Exact transpose of ``_fwd``: out[k] = y[k-1] [k>=1] - y[k] [k<=n-2]."""
    out = np.zeros_like(y, dtype=np.float64)
    n = y.shape[axis]
    a = [slice(None)] * y.ndim
    b = [slice(None)] * y.ndim
    a[axis] = slice(1, n)
    b[axis] = slice(0, n - 1)
    out[tuple(a)] += y[tuple(b)]
    out[tuple(b)] -= y[tuple(b)]
    return out


def Dv(x):
    """Vertical forward difference (along rows i)."""
    return _fwd(x, -2)


def Dv_T(y):
    return _fwd_T(y, -2)


def Dh(x):
    """Horizontal forward difference (along columns j)."""
    return _fwd(x, -1)


def Dh_T(y):
    return _fwd_T(y, -1)


def Ds(x):
    """Spectral forward difference (along bands b)."""
    return _fwd(x, -3)


def Ds_T(y):
    return _fwd_T(y, -3)


def D(x):
    """Spatial difference D = (D_v^T D_h^T)^T : R^N -> R^{2N}."""
    return np.stack([Dv(x), Dh(x)])


def D_T(y):
    return Dv_T(y[0]) + Dh_T(y[1])


# ---------------------------------------------------------------------------
# Condat's interpolators (Sec. II-D, Eqs. 10-12) and L (Sec. III-A, Eq. 13)
# ---------------------------------------------------------------------------
def shift(x, di, dj):
    """out[..., i, j] = x[..., i+di, j+dj], zero outside the image.

    Its transpose is shift(., -di, -dj).
    """
    n1, n2 = x.shape[-2], x.shape[-1]
    out = np.zeros_like(x, dtype=np.float64)
    i_dst = slice(max(0, -di), min(n1, n1 - di))
    i_src = slice(max(0, di), min(n1, n1 + di))
    j_dst = slice(max(0, -dj), min(n2, n2 - dj))
    j_src = slice(max(0, dj), min(n2, n2 + dj))
    out[..., i_dst, j_dst] = x[..., i_src, j_src]
    return out


def _row_mask(shape):
    """1 on rows 0..N1-2, 0 on the last row (where D_v is structurally 0)."""
    m = np.ones(shape)
    m[..., -1, :] = 0.0
    return m


def _col_mask(shape):
    """1 on columns 0..N2-2, 0 on the last column (where D_h is 0)."""
    m = np.ones(shape)
    m[..., :, -1] = 0.0
    return m


def L(y):
    """L = blockdiag over bands of (L_vert; L_hori; L_cent): R^{2N} -> R^{6N}.

    y[0] (vertical differences) lives at (i+1/2, j), y[1] (horizontal) at
    (i, j+1/2).  Each output grid carries a (vertical, horizontal) pair.
    """
    mv = _row_mask(y[0].shape)
    mh = _col_mask(y[1].shape)
    yv = mv * y[0]
    yh = mh * y[1]
    w = np.zeros((3, 2) + y[0].shape)
    # L_vert: grid (i+1/2, j); zero on the last row.
    w[0, 0] = mv * yv
    w[0, 1] = mv * 0.25 * (yh + shift(yh, 0, -1) + shift(yh, 1, 0) + shift(yh, 1, -1))
    # L_hori: grid (i, j+1/2); zero on the last column.
    w[1, 0] = mh * 0.25 * (yv + shift(yv, -1, 0) + shift(yv, 0, 1) + shift(yv, -1, 1))
    w[1, 1] = mh * yh
    # L_cent: grid (i, j).
    w[2, 0] = 0.5 * (yv + shift(yv, -1, 0))
    w[2, 1] = 0.5 * (yh + shift(yh, 0, -1))
    return w


def L_T(w):
    """Exact transpose of ``L``: R^{6N} -> R^{2N}."""
    shp = w.shape[2:]
    mv = _row_mask(shp)
    mh = _col_mask(shp)
    a = mv * w[0, 1]
    b = mh * w[1, 0]
    gv = (mv * w[0, 0]
          + 0.25 * (b + shift(b, 1, 0) + shift(b, 0, -1) + shift(b, 1, -1))
          + 0.5 * (w[2, 0] + shift(w[2, 0], 1, 0)))
    gh = (0.25 * (a + shift(a, 0, 1) + shift(a, -1, 0) + shift(a, -1, 1))
          + mh * w[1, 1]
          + 0.5 * (w[2, 1] + shift(w[2, 1], 0, 1)))
    return np.stack([mv * gv, mh * gh])


# ---------------------------------------------------------------------------
# Proximal tools (Sec. II-B, Eqs. 1-5; Sec. III-B, Eqs. 21-24)
# ---------------------------------------------------------------------------
def prox_l12(x, gamma):
    """Eq. 24: group soft-threshold, groups = the 2-vectors along axis 1.

    ``x`` has shape (G, 2, ...) (G grids); each (vertical, horizontal) pair is
    scaled by max(1 - gamma / ||x_g||_2, 0); a zero group maps to zero.
    """
    nrm = np.sqrt(x[:, 0] ** 2 + x[:, 1] ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        scale = np.where(nrm > 0, np.maximum(1.0 - gamma / nrm, 0.0), 0.0)
    return x * scale[:, None]


def proj_box(x, lo, hi):
    """Eq. 21: projection onto [lo, hi]^N."""
    return np.minimum(np.maximum(x, lo), hi)


def proj_l1ball(x, r):
    """Projection onto {z : ||z||_1 <= r} (Sec. III-B, fast l1-ball projection).

    Returns (P(x), tau).  The projection is sign(x) max(|x| - tau, 0) with
    tau >= 0 the root of sum max(|x_i| - tau, 0) = r, or x itself (tau = 0)
    when x is already inside.  tau is found by the sort-based method: sort |x|
    in decreasing order, take the largest rho with
    a_(rho) > (sum_{k<=rho} a_(k) - r) / rho, then tau = that ratio.
    With r = 0 the ball is {0} and tau = max |x|.
    """
    a = np.abs(x).ravel()
    if a.sum() <= r:
        return x.copy(), 0.0
    if r <= 0:
        return np.zeros_like(x, dtype=np.float64), float(a.max())
    srt = np.sort(a)[::-1]
    cs = np.cumsum(srt)
    k = np.arange(1, srt.size + 1)
    cond = srt - (cs - r) / k > 0
    rho = np.nonzero(cond)[0][-1]
    tau = (cs[rho] - r) / (rho + 1)
    return np.sign(x) * np.maximum(np.abs(x) - tau, 0.0), float(tau)


def proj_l2ball(x, center, eps):
    """Eq. 23: projection onto {z : ||z - center||_2 <= eps}."""
    d = x - center
    nd = np.sqrt(np.sum(d * d))
    if nd <= eps:
        return x.copy()
    return center + (eps / nd) * d


# ---------------------------------------------------------------------------
# Algorithm 1
# ---------------------------------------------------------------------------
def init_state(v):
    """u = v; s, t, w1, w2, y1..y4 = 0 (Algorithm 1 leaves the start open)."""
    v = np.asarray(v, dtype=np.float64)
    z = np.zeros_like(v)
    return State(u=v.copy(), s=z.copy(), t=z.copy(),
                 w1=np.zeros((3, 2) + v.shape), w2=np.zeros((3, 2) + v.shape),
                 y1=np.zeros((2,) + v.shape), y2=np.zeros((2,) + v.shape),
                 y3=z.copy(), y4=z.copy())


def ppds_step(st: State, v, p: Params) -> State:
    """One pass of Algorithm 1: the P-PDS of Eq. 7 applied to Prob. 20.

    Prob. 20 stacks the primal x = (u, w1, w2, s, t) and the dual
    y = (y1, y2, y3, y4) through the operator A of ``apply_A``.  One pass is
    x+ = prox_{Gamma1 f}(x - Gamma1 A^T y) block by block (box, Eq. 21; group
    soft-threshold, Eq. 24; l1-ball projections, Sec. III-B), the
    extrapolation x' = 2 x+ - x, and y+ = prox_{Gamma2 g*}(y + Gamma2 A x').
    The dual blocks: g is the indicator of {0} for y1, y2, y3, so the prox of
    its conjugate is the plain ascent (Eq. 22 through Moreau's identity,
    Eq. 3); for y4 it is the indicator of B_{2,eps}^v, whose conjugate prox
    is z - gamma P_B(z / gamma) (Eq. 23 through Eq. 3).  Dual steps take the
    "+" sign of Algorithm 1.
    """
    v = np.asarray(v, dtype=np.float64)
    # primal blocks: x - Gamma1 A^T y, then the prox of each block of f
    gu, gw1, gw2, gs, gt = apply_AT(st.y1, st.y2, st.y3, st.y4)
    u1 = proj_box(st.u - p.gamma_u * gu, p.mu_lo, p.mu_hi)
    w11 = prox_l12(st.w1 - p.gamma_w1 * gw1, p.gamma_w1 * p.omega)
    w21 = prox_l12(st.w2 - p.gamma_w2 * gw2, p.gamma_w2)
    s1, tau_s = proj_l1ball(st.s - p.gamma_s * gs, p.alpha)
    t1, tau_t = proj_l1ball(st.t - p.gamma_t * gt, p.beta)
    # extrapolated primal x' = 2 x+ - x
    xb = [2 * a - b for a, b in ((u1, st.u), (w11, st.w1), (w21, st.w2), (s1, st.s), (t1, st.t))]
    # dual blocks: y + Gamma2 A x', then the prox of each block of g*
    a1, a2, a3, a4 = apply_A(*xb)
    y11 = st.y1 + p.gamma_y1 * a1
    y21 = st.y2 + p.gamma_y2 * a2
    y31 = st.y3 + p.gamma_y3 * a3
    y4p = st.y4 + p.gamma_y4 * a4
    y41 = y4p - p.gamma_y4 * proj_l2ball(y4p / p.gamma_y4, v, p.eps)
    out = State(u=u1, s=s1, t=t1, w1=w11, w2=w21, y1=y11, y2=y21, y3=y31, y4=y41)
    out.extra = {"tau_s": tau_s, "tau_t": tau_t}
    return out


def rel_change(u_next, u_prev):
    """The ratio of the stopping rule, Eq. 28: ||u^(k+1) - u^(k)||_2 / ||u^(k)||_2.

    +inf when u^(k) = 0 (the ratio is undefined there and never stops the run).
    """
    den = np.linalg.norm(u_prev)
    if den == 0:
        return np.inf
    return float(np.linalg.norm(u_next - u_prev) / den)


def solve(v, p: Params, iters: int, state: State | None = None, tol: float = 0.0):
    """Run Algorithm 1 for ``iters`` passes, or until Eq. 28 holds when tol > 0.

    With tol > 0 the run stops after the first pass k + 1 whose ratio
    ``rel_change(u^(k+1), u^(k))`` is below tol.  Returns (state, passes run).
    """
    st = init_state(v) if state is None else state.copy()
    for k in range(iters):
        nxt = ppds_step(st, v, p)
        stop = tol > 0 and rel_change(nxt.u, st.u) < tol
        st = nxt
        if stop:
            return st, k + 1
    return st, iters


# ---------------------------------------------------------------------------
# The stacked operator A of Prob. 20 (used by ppds_step) and the GeoSSTV objective
# ---------------------------------------------------------------------------
def apply_A(u, w1, w2, s, t):
    """A x = (D u - L^T w1, D D_s u - L^T w2, D_v t, u + s + t)  (Eq. 20)."""
    return (D(u) - L_T(w1), D(Ds(u)) - L_T(w2), Dv(t), u + s + t)


def apply_AT(y1, y2, y3, y4):
    """A^T y, blocks ordered (u, w1, w2, s, t)."""
    gu = D_T(y1) + Ds_T(D_T(y2)) + y4
    return (gu, -L(y1), -L(y2), y4.copy(), Dv_T(y3) + y4)


def geosstv_objective(w1, w2, omega):
    """omega ||w1||_{1,2} + ||w2||_{1,2} (Eq. 13 objective, groups of 2)."""
    n1 = np.sqrt(w1[:, 0] ** 2 + w1[:, 1] ** 2).sum()
    n2 = np.sqrt(w2[:, 0] ** 2 + w2[:, 1] ** 2).sum()
    return omega * n1 + n2
