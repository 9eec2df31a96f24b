"""Pins of the oracle's Algorithm 1 against facts fixed outside it.

* Assembly: Algorithm 1 must equal the generic P-PDS of Eq. 7 run on the
  explicit sparse matrix of Prob. 20 (differences from Kronecker products, L
  from a per-grid-point construction), with the proxes of Eqs. 21-24 and the
  conjugate proxes through Moreau's identity (Eq. 3).
* Optimality: on a tiny noisy cube, the primal objective (Eq. 15) and the
  Fenchel dual objective -f*(-A^T y) - g*(y) of Prob. 20 (conjugates written
  out from their textbook forms) must meet, with the constraints satisfied.
  The dual uses: box* = sum max(mu_lo z, mu_hi z); (w ||.||_{1,2})* = indicator
  of discs of radius w; l1-ball* = r ||.||_inf; l2-ball(v, eps)* = <v, .> +
  eps ||.||_2.  Planted mistakes in the oracle must break this check.
* Exact fixed point: a per-band constant cube in the box, started at u = v,
  never moves (D v = 0, D D_s v = 0, and y4' = gamma v projects back to 0).
* Zero radii: with eps = alpha = beta = 0 the feasible set is {u = v, s = t = 0}.
* Step sizes: the printed values satisfy the P-PDS convergence condition
  ||Gamma2^(1/2) A Gamma1^(1/2)||^2 < 1: exactly (SVD of the explicit matrix)
  on a tiny cube, and at working sizes by Lanczos on the operator applied
  matrix-free through apply_A / apply_AT, checked against the SVD first.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.linalg import LinearOperator, eigsh

from oracle import ppds as o
from paper_2510_00562_gb300 import synth


# ---------------------------------------------------------------------------
# explicit matrices
# ---------------------------------------------------------------------------
def _d1(n):
    m = sp.lil_matrix((n, n))
    for k in range(n - 1):
        m[k, k] = -1.0
        m[k, k + 1] = 1.0
    return m.tocsr()


def _diff_mats(n3, n1, n2):
    i3, i1, i2 = sp.identity(n3), sp.identity(n1), sp.identity(n2)
    dv = sp.kron(sp.kron(i3, _d1(n1)), i2).tocsr()
    dh = sp.kron(sp.kron(i3, i1), _d1(n2)).tocsr()
    ds = sp.kron(sp.kron(_d1(n3), i1), i2).tocsr()
    return dv, dh, ds


def _interp_mat(n3, n1, n2):
    """L as a sparse (6N x 2N) matrix, one grid point at a time.

    Input y = (y_v at (i+1/2, j), y_h at (i, j+1/2)); entries of y_v on the
    last row and of y_h on the last column are never read.
    """
    N = n1 * n2 * n3
    m = sp.lil_matrix((6 * N, 2 * N))

    def yv(b, i, j):
        return None if not (0 <= i < n1 - 1 and 0 <= j < n2) else (b * n1 + i) * n2 + j

    def yh(b, i, j):
        return None if not (0 <= i < n1 and 0 <= j < n2 - 1) else N + (b * n1 + i) * n2 + j

    def row(g, c, b, i, j):
        return (2 * g + c) * N + (b * n1 + i) * n2 + j

    def put(r, col, val):
        if col is not None:
            m[r, col] += val

    for b in range(n3):
        for i in range(n1):
            for j in range(n2):
                if i < n1 - 1:                   # L_vert at (i+1/2, j)
                    put(row(0, 0, b, i, j), yv(b, i, j), 1.0)
                    for (a, c) in ((i, j), (i, j - 1), (i + 1, j), (i + 1, j - 1)):
                        put(row(0, 1, b, i, j), yh(b, a, c), 0.25)
                if j < n2 - 1:                   # L_hori at (i, j+1/2)
                    for (a, c) in ((i, j), (i - 1, j), (i, j + 1), (i - 1, j + 1)):
                        put(row(1, 0, b, i, j), yv(b, a, c), 0.25)
                    put(row(1, 1, b, i, j), yh(b, i, j), 1.0)
                for (a, c) in ((i, j), (i - 1, j)):   # L_cent at (i, j)
                    put(row(2, 0, b, i, j), yv(b, a, c), 0.5)
                for (a, c) in ((i, j), (i, j - 1)):
                    put(row(2, 1, b, i, j), yh(b, a, c), 0.5)
    return m.tocsr()


def _stacked_A(n3, n1, n2):
    """A of Prob. 20: rows (y1, y2, y3, y4), columns (u, w1, w2, s, t)."""
    N = n1 * n2 * n3
    dv, dh, ds = _diff_mats(n3, n1, n2)
    Dm = sp.vstack([dv, dh])
    Lm = _interp_mat(n3, n1, n2)
    I = sp.identity(N)
    Z = lambda r, c: sp.csr_matrix((r, c))
    A = sp.bmat([
        [Dm, -Lm.T, Z(2 * N, 6 * N), Z(2 * N, N), Z(2 * N, N)],
        [Dm @ ds, Z(2 * N, 6 * N), -Lm.T, Z(2 * N, N), Z(2 * N, N)],
        [Z(N, N), Z(N, 6 * N), Z(N, 6 * N), Z(N, N), dv],
        [I, Z(N, 6 * N), Z(N, 6 * N), I, I],
    ]).tocsr()
    return A, Lm


def test_L_matches_per_point_matrix():
    n3, n1, n2 = 2, 5, 4
    N = n1 * n2 * n3
    Lm = _interp_mat(n3, n1, n2)
    rng = np.random.default_rng(0)
    y = rng.standard_normal((2, n3, n1, n2))
    np.testing.assert_allclose(o.L(y).ravel(), Lm @ y.ravel(), atol=1e-14)
    w = rng.standard_normal((3, 2, n3, n1, n2))
    np.testing.assert_allclose(o.L_T(w).ravel(), Lm.T @ w.ravel(), atol=1e-14)


def _generic_ppds(x, y, A, v, p, shape, iters):
    """Eq. 7 on flat vectors, with the conjugate proxes of Eq. 3."""
    N = int(np.prod(shape))
    cuts_x = np.cumsum([N, 6 * N, 6 * N, N])
    cuts_y = np.cumsum([2 * N, 2 * N, N])
    g1 = np.concatenate([np.full(N, p.gamma_u), np.full(6 * N, p.gamma_w1),
                         np.full(6 * N, p.gamma_w2), np.full(N, p.gamma_s), np.full(N, p.gamma_t)])
    g2 = np.concatenate([np.full(2 * N, p.gamma_y1), np.full(2 * N, p.gamma_y2),
                         np.full(N, p.gamma_y3), np.full(N, p.gamma_y4)])
    AT = A.T.tocsr()
    for _ in range(iters):
        z = x - g1 * (AT @ y)
        u, w1, w2, s, t = np.split(z, cuts_x)
        u = np.clip(u, p.mu_lo, p.mu_hi)                                          # Eq. 21
        w1 = o.prox_l12(w1.reshape((3, 2) + shape), p.gamma_w1 * p.omega).ravel()  # Eq. 24
        w2 = o.prox_l12(w2.reshape((3, 2) + shape), p.gamma_w2).ravel()
        s = o.proj_l1ball(s, p.alpha)[0]
        t = o.proj_l1ball(t, p.beta)[0]
        xn = np.concatenate([u, w1, w2, s, t])
        xb = 2 * xn - x
        q = y + g2 * (A @ xb)
        q1, q2, q3, q4 = np.split(q, cuts_y)
        # prox_{g f*}(z) = z - g prox_{f/g}(z/g): f = indicator{0} gives z - 0;
        # f = indicator of the l2 ball gives z - g P_B(z/g).
        g4 = p.gamma_y4
        q4 = q4 - g4 * o.proj_l2ball(q4 / g4, v.ravel(), p.eps)
        y = np.concatenate([q1, q2, q3, q4])
        x = xn
    return x, y


def _flat(st):
    x = np.concatenate([st.u.ravel(), st.w1.ravel(), st.w2.ravel(), st.s.ravel(), st.t.ravel()])
    y = np.concatenate([st.y1.ravel(), st.y2.ravel(), st.y3.ravel(), st.y4.ravel()])
    return x, y


@pytest.mark.parametrize("shape", [(3, 5, 4), (2, 4, 6)])
def test_algorithm1_equals_generic_ppds(shape):
    n3, n1, n2 = shape
    A, _ = _stacked_A(n3, n1, n2)
    rs = synth.random_state(n1, n2, n3, seed=5, scale=0.3)
    st = o.State(**{k: rs[k].astype(np.float64) for k in o.State.names()})
    v = np.random.default_rng(9).uniform(0, 1, size=shape)
    p = o.Params(eps=0.5, alpha=1.0, beta=0.7, omega=0.05)
    x, y = _flat(st)
    xg, yg = _generic_ppds(x, y, A, v, p, shape, 25)
    cur = st
    for _ in range(25):
        cur = o.ppds_step(cur, v, p)
    xo, yo = _flat(cur)
    np.testing.assert_allclose(xo, xg, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(yo, yg, rtol=1e-11, atol=1e-12)


# ---------------------------------------------------------------------------
# optimality through the Fenchel dual
# ---------------------------------------------------------------------------
def _certificate(st, v, p):
    P = o.geosstv_objective(st.w1, st.w2, p.omega)
    a = o.D_T(st.y1) + o.Ds_T(o.D_T(st.y2)) + st.y4
    box_conj = np.maximum(-p.mu_lo * a, -p.mu_hi * a).sum()
    Dd = (-box_conj - p.alpha * np.abs(st.y4).max() - p.beta * np.abs(o.Dv_T(st.y3) + st.y4).max()
          - np.vdot(v, st.y4) - p.eps * np.linalg.norm(st.y4))
    l1, l2 = o.L(st.y1), o.L(st.y2)
    feas1 = np.sqrt(l1[:, 0] ** 2 + l1[:, 1] ** 2).max() / p.omega
    feas2 = np.sqrt(l2[:, 0] ** 2 + l2[:, 1] ** 2).max()
    scale = np.linalg.norm(o.D(st.u)) + 1e-30
    res = {
        "gap": abs(P - Dd) / abs(P),
        "dual_feas": max(feas1, feas2) - 1.0,
        "c1": np.linalg.norm(o.L_T(st.w1) - o.D(st.u)) / scale,
        "c2": np.linalg.norm(o.L_T(st.w2) - o.D(o.Ds(st.u))) / scale,
        "c3": np.linalg.norm(o.Dv(st.t)) / (np.linalg.norm(st.t) + 1e-30),
        "fid": np.linalg.norm(st.u + st.s + st.t - v) / p.eps - 1.0,
        "l1s": np.abs(st.s).sum() / p.alpha - 1.0,
        "l1t": np.abs(st.t).sum() / p.beta - 1.0,
        "box": max(p.mu_lo - st.u.min(), st.u.max() - p.mu_hi),
    }
    return res


def _tiny_problem():
    pb = synth.make_problem(8, 7, 5, seed=3, noise=synth.NoiseSpec(sigma=0.1, sp_rate=0.1, stripe_rate=0.2))
    v = pb["v"].astype(np.float64)
    p = o.Params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=0.05)
    return v, p


def _optimal(st, v, p):
    r = _certificate(st, v, p)
    return (r["gap"] < 5e-4 and r["dual_feas"] < 3e-3 and r["c1"] < 1e-3 and r["c2"] < 3e-3
            and r["c3"] < 1e-3 and r["fid"] < 1e-3 and r["l1s"] < 1e-12 and r["l1t"] < 1e-12
            and r["box"] <= 0), r


N_ITERS_CERT = 6000


def test_duality_gap_closes():
    v, p = _tiny_problem()
    st, _ = o.solve(v, p, N_ITERS_CERT)
    ok, r = _optimal(st, v, p)
    assert ok, r
    # the s and t balls are active for this noise (so the l1 steps matter)
    assert abs(r["l1s"]) < 1e-9 and abs(r["l1t"]) < 1e-9


@pytest.mark.parametrize("mistake", ["drop_Ds_T", "l1_clip", "L_T_swapped", "y3_sign"])
def test_planted_mistakes_break_certificate(mistake, monkeypatch):
    """A plausible mistake planted in the oracle must fail the optimality check."""
    v, p = _tiny_problem()
    if mistake == "drop_Ds_T":
        monkeypatch.setattr(o, "Ds_T", lambda y: np.zeros_like(y))
    elif mistake == "l1_clip":
        def bad(x, r):
            a = np.abs(x).sum()
            return (x * (r / a) if a > r else x.copy()), 0.0
        monkeypatch.setattr(o, "proj_l1ball", bad)
    elif mistake == "L_T_swapped":
        real = o.L_T
        monkeypatch.setattr(o, "L_T", lambda w: real(w)[::-1].copy())
    elif mistake == "y3_sign":
        real = o.Dv
        monkeypatch.setattr(o, "Dv", lambda x: -real(x))
    with np.errstate(all="ignore"):
        try:
            st, _ = o.solve(v, p, N_ITERS_CERT)
        except (IndexError, ValueError):
            return          # the planted mistake made the iteration blow up
    finite = all(np.all(np.isfinite(getattr(st, k))) for k in o.State.names())
    if not finite:
        return
    monkeypatch.undo()
    ok, r = _optimal(st, v, p)
    assert not ok, (mistake, r)


# ---------------------------------------------------------------------------
# exact special cases
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("omega", [0.0, 0.03, 1.0])
def test_per_band_constant_fixed_point(omega):
    n3, n1, n2 = 6, 9, 7
    levels = np.random.default_rng(1).uniform(0.1, 0.9, size=n3)
    v = np.broadcast_to(levels[:, None, None], (n3, n1, n2)).copy()
    p = o.Params(eps=0.3, alpha=2.0, beta=1.5, omega=omega)
    st, _ = o.solve(v, p, 50)
    np.testing.assert_array_equal(st.u, v)
    for k in ("s", "t", "w1", "w2", "y1", "y2", "y3", "y4"):
        assert np.all(getattr(st, k) == 0), k


def test_zero_radii_recover_observation():
    rng = np.random.default_rng(4)
    v = rng.uniform(0.05, 0.95, size=(3, 6, 5))
    p = o.Params(eps=0.0, alpha=0.0, beta=0.0, omega=0.03)
    st, _ = o.solve(v, p, 3000)
    assert np.all(st.s == 0) and np.all(st.t == 0)
    assert np.linalg.norm(st.u - v) / np.linalg.norm(v) < 1e-4


def test_printed_step_sizes_satisfy_convergence_condition():
    shape = (4, 6, 5)
    A, _ = _stacked_A(*shape)
    N = int(np.prod(shape))
    p = o.Params()
    g1 = np.concatenate([np.full(N, p.gamma_u), np.full(6 * N, p.gamma_w1),
                         np.full(6 * N, p.gamma_w2), np.full(N, p.gamma_s), np.full(N, p.gamma_t)])
    g2 = np.concatenate([np.full(2 * N, p.gamma_y1), np.full(2 * N, p.gamma_y2),
                         np.full(N, p.gamma_y3), np.full(N, p.gamma_y4)])
    M = sp.diags(np.sqrt(g2)) @ A @ sp.diags(np.sqrt(g1))
    nrm2 = np.linalg.svd(M.toarray(), compute_uv=False)[0] ** 2
    assert nrm2 < 1.0


# ---------------------------------------------------------------------------
# step-size condition at working sizes
# ---------------------------------------------------------------------------
def p_pds_condition(shape, p=None, tol=1e-4, seed=0):
    """Largest eigenvalue of Gamma1^(1/2) A^T Gamma2 A Gamma1^(1/2), i.e.
    ||Gamma2^(1/2) A Gamma1^(1/2)||^2, by Lanczos (ARPACK) on the operator of
    Prob. 20 applied matrix-free.  Primal blocks (u, w1, w2, s, t)."""
    p = p or o.Params()
    n3, n1, n2 = shape
    N = n1 * n2 * n3
    g1 = (p.gamma_u, p.gamma_w1, p.gamma_w2, p.gamma_s, p.gamma_t)
    g2 = (p.gamma_y1, p.gamma_y2, p.gamma_y3, p.gamma_y4)
    shapes = (shape, (3, 2) + shape, (3, 2) + shape, shape, shape)
    sizes = [int(np.prod(s)) for s in shapes]

    def mv(x):
        x = np.asarray(x).ravel()
        parts, at = [], 0
        for sz, g, sh in zip(sizes, g1, shapes):
            parts.append(math.sqrt(g) * x[at:at + sz].reshape(sh))
            at += sz
        ay = [g * b for g, b in zip(g2, o.apply_A(*parts))]
        return np.concatenate([(math.sqrt(g) * c).ravel() for g, c in zip(g1, o.apply_AT(*ay))])

    op = LinearOperator((15 * N, 15 * N), matvec=mv, dtype=np.float64)
    v0 = np.random.default_rng(seed).standard_normal(15 * N)
    return float(eigsh(op, k=1, which="LA", tol=tol, v0=v0, return_eigenvectors=False)[0])


def test_condition_matches_the_explicit_matrix_on_a_tiny_cube():
    # the matrix-free Lanczos value equals the SVD of the explicit stacked
    # matrix (Kronecker products, per-point L) on the 4x6x5 cube: 0.5838...
    shape = (4, 6, 5)
    A, _ = _stacked_A(*shape)
    N = int(np.prod(shape))
    p = o.Params()
    g1 = np.concatenate([np.full(N, p.gamma_u), np.full(6 * N, p.gamma_w1),
                         np.full(6 * N, p.gamma_w2), np.full(N, p.gamma_s), np.full(N, p.gamma_t)])
    g2 = np.concatenate([np.full(2 * N, p.gamma_y1), np.full(2 * N, p.gamma_y2),
                         np.full(N, p.gamma_y3), np.full(N, p.gamma_y4)])
    M = sp.diags(np.sqrt(g2)) @ A @ sp.diags(np.sqrt(g1))
    exact = np.linalg.svd(M.toarray(), compute_uv=False)[0] ** 2
    assert abs(p_pds_condition(shape, tol=1e-10) - exact) < 1e-8 * exact


@pytest.mark.parametrize("shape", [(8, 16, 16), (16, 32, 32), (32, 64, 64), (64, 128, 128)])
def test_printed_step_sizes_meet_the_condition_at_working_sizes(shape):
    # measured: 0.668 (16x16x8), 0.685 (32x32x16), 0.690 (64x64x32), 0.691
    # (128x128x64, about two minutes on one core): the norm grows with the
    # cube toward its limit and stays well below 1
    lam = p_pds_condition(shape, tol=1e-3)
    assert 0.6 < lam < 0.75, lam
