"""Pins of the oracle's linear operators against facts fixed outside it.

* D_v, D_h, D_s: the Kronecker-product matrices of the 1-D Neumann forward
  difference (Sec. II-A), built here from the textbook definition.
* Operator norms: the closed-form spectrum of the 1-D Neumann difference
  (D1^T D1 is the path-graph Laplacian, eigenvalues 2 - 2 cos(pi k / n)), and
  its Kronecker sums/products for D and D D_s.
* L (Sec. II-D, Eqs. 10-12): interpolation onto the grids (i+1/2, j),
  (i, j+1/2), (i, j) must reproduce affine fields exactly in the interior;
  L_vert / L_hori vanish on the last row / column; each interpolator is an
  average, so has norm <= 1.
* Every adjoint: <Ax, y> = <x, A^T y> on random data.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import ppds as o

SHAPES = [(3, 4, 5), (2, 6, 3), (4, 5, 7)]   # (N3, N1, N2)


def _d1(n):
    """1-D forward difference with Neumann boundary: rows k<n-1 are e_{k+1}-e_k."""
    m = sp.lil_matrix((n, n))
    for k in range(n - 1):
        m[k, k] = -1.0
        m[k, k + 1] = 1.0
    return m.tocsr()


def _dense(op, shape_in, n_out):
    n_in = int(np.prod(shape_in))
    cols = []
    for c in range(n_in):
        e = np.zeros(n_in)
        e[c] = 1.0
        cols.append(np.asarray(op(e.reshape(shape_in))).ravel())
    m = np.stack(cols, axis=1)
    assert m.shape[0] == n_out
    return m


@pytest.mark.parametrize("shape", SHAPES)
def test_differences_match_kronecker(shape):
    n3, n1, n2 = shape
    N = n1 * n2 * n3
    i3, i1, i2 = sp.identity(n3), sp.identity(n1), sp.identity(n2)
    kv = sp.kron(sp.kron(i3, _d1(n1)), i2).toarray()
    kh = sp.kron(sp.kron(i3, i1), _d1(n2)).toarray()
    ks = sp.kron(sp.kron(_d1(n3), i1), i2).toarray()
    np.testing.assert_array_equal(_dense(o.Dv, shape, N), kv)
    np.testing.assert_array_equal(_dense(o.Dh, shape, N), kh)
    np.testing.assert_array_equal(_dense(o.Ds, shape, N), ks)
    np.testing.assert_array_equal(_dense(o.Dv_T, shape, N), kv.T)
    np.testing.assert_array_equal(_dense(o.Dh_T, shape, N), kh.T)
    np.testing.assert_array_equal(_dense(o.Ds_T, shape, N), ks.T)


def _lam(n):
    """Largest eigenvalue of D1^T D1 for the 1-D Neumann difference."""
    return 2.0 - 2.0 * np.cos(np.pi * (n - 1) / n) if n > 1 else 0.0


@pytest.mark.parametrize("shape", SHAPES)
def test_difference_norms_closed_form(shape):
    n3, n1, n2 = shape
    N = n1 * n2 * n3
    mv = _dense(o.Dv, shape, N)
    ms = _dense(o.Ds, shape, N)
    md = _dense(lambda x: o.D(x).ravel(), shape, 2 * N)
    mdds = _dense(lambda x: o.D(o.Ds(x)).ravel(), shape, 2 * N)
    sv = lambda m: np.linalg.svd(m, compute_uv=False)[0] ** 2
    assert sv(mv) == pytest.approx(_lam(n1), rel=1e-12)
    assert sv(ms) == pytest.approx(_lam(n3), rel=1e-12)
    # D^T D = Dv^T Dv + Dh^T Dh acts on different axes: a Kronecker sum
    assert sv(md) == pytest.approx(_lam(n1) + _lam(n2), rel=1e-12)
    # (D Ds)^T (D Ds) = (D^T D)(Ds^T Ds): a Kronecker product
    assert sv(mdds) == pytest.approx((_lam(n1) + _lam(n2)) * _lam(n3), rel=1e-12)
    # all bounded by 4 per axis, as the step-size reading relies on
    assert _lam(n1) < 4 and _lam(n3) < 4


def _affine(a, b, c):
    return lambda x, y: a + b * x + c * y


@pytest.mark.parametrize("shape", [(2, 7, 6), (1, 9, 11)])
def test_L_reproduces_affine_fields(shape):
    """y_v sampled at (i+1/2, j) and y_h at (i, j+1/2) from affine f, g:
    L_vert gives (f, g) at (i+1/2, j), L_hori at (i, j+1/2), L_cent at (i, j)."""
    n3, n1, n2 = shape
    f = _affine(0.3, -1.7, 0.9)
    g = _affine(-0.2, 0.4, 2.3)
    ii, jj = np.meshgrid(np.arange(n1, dtype=float), np.arange(n2, dtype=float), indexing="ij")
    y = np.zeros((2, n3, n1, n2))
    y[0] = f(ii + 0.5, jj)
    y[1] = g(ii, jj + 0.5)
    w = o.L(y)
    inner = (slice(None), slice(1, n1 - 1), slice(1, n2 - 1))
    cases = [(0, ii + 0.5, jj), (1, ii, jj + 0.5), (2, ii, jj)]
    for grid, xi, xj in cases:
        want_v = np.broadcast_to(f(xi, xj), (n3, n1, n2))
        want_h = np.broadcast_to(g(xi, xj), (n3, n1, n2))
        np.testing.assert_allclose(w[grid, 0][inner], want_v[inner], rtol=0, atol=1e-13)
        np.testing.assert_allclose(w[grid, 1][inner], want_h[inner], rtol=0, atol=1e-13)


def test_L_boundary_structure():
    rng = np.random.default_rng(0)
    n3, n1, n2 = 2, 5, 6
    y = rng.standard_normal((2, n3, n1, n2))
    w = o.L(y)
    assert np.all(w[0, :, :, -1, :] == 0)     # L_vert: nothing below the last row
    assert np.all(w[1, :, :, :, -1] == 0)     # L_hori: nothing right of the last column
    # entries where D is structurally zero do not enter L
    y2 = y.copy()
    y2[0, :, -1, :] = rng.standard_normal((n3, n2))
    y2[1, :, :, -1] = rng.standard_normal((n3, n1))
    np.testing.assert_array_equal(o.L(y2), w)
    # and L^T never lands there
    lt = o.L_T(rng.standard_normal((3, 2, n3, n1, n2)))
    assert np.all(lt[0, :, -1, :] == 0) and np.all(lt[1, :, :, -1] == 0)


def test_L_norm_bounded():
    shape = (2, 6, 5)
    N = int(np.prod(shape))
    m = _dense(lambda y: o.L(y).ravel(), (2,) + shape, 6 * N)
    for g in range(3):
        blk = m[g * 2 * N:(g + 1) * 2 * N]
        assert np.linalg.svd(blk, compute_uv=False)[0] <= 1.0 + 1e-12
    assert np.linalg.svd(m, compute_uv=False)[0] ** 2 <= 3.0 + 1e-12


def _rand(rng, *shape):
    return rng.standard_normal(shape)


@pytest.mark.parametrize("shape", SHAPES)
def test_adjoint_identities(shape):
    rng = np.random.default_rng(7)
    pairs = [
        (o.Dv, o.Dv_T, shape, shape),
        (o.Dh, o.Dh_T, shape, shape),
        (o.Ds, o.Ds_T, shape, shape),
        (o.D, o.D_T, shape, (2,) + shape),
        (o.L, o.L_T, (2,) + shape, (3, 2) + shape),
    ]
    for fwd, adj, sin, sout in pairs:
        x = _rand(rng, *sin)
        y = _rand(rng, *sout)
        lhs = np.vdot(fwd(x), y)
        rhs = np.vdot(x, adj(y))
        assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-12)
    # for every shift offset the transpose is the opposite shift
    for di, dj in itertools.product((-1, 0, 1), repeat=2):
        x = _rand(rng, *shape)
        y = _rand(rng, *shape)
        assert np.vdot(o.shift(x, di, dj), y) == pytest.approx(np.vdot(x, o.shift(y, -di, -dj)), rel=1e-12)


@pytest.mark.parametrize("shape", SHAPES)
def test_stacked_operator_adjoint(shape):
    """<A x, y> = <x, A^T y> for the operator of Prob. 20."""
    rng = np.random.default_rng(3)
    x = (_rand(rng, *shape), _rand(rng, 3, 2, *shape), _rand(rng, 3, 2, *shape),
         _rand(rng, *shape), _rand(rng, *shape))
    y = (_rand(rng, 2, *shape), _rand(rng, 2, *shape), _rand(rng, *shape), _rand(rng, *shape))
    ax = o.apply_A(*x)
    aty = o.apply_AT(*y)
    lhs = sum(np.vdot(a, b) for a, b in zip(ax, y))
    rhs = sum(np.vdot(a, b) for a, b in zip(x, aty))
    assert lhs == pytest.approx(rhs, rel=1e-12)
