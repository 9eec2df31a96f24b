"""One cube stored as band slabs (gsstv_slabs_*) against the FP64 oracle.

The slabs split the bands of the cube (each slab in allocations of its own,
with one halo band on each side refreshed by plane copies after every pass;
the global sums of every pass finished over all slabs).  The split changes
nothing in Algorithm 1, so the bars are those of the single handle:
  * one pass from a random state: every variable within 2e-6 of the oracle's
    whole-cube pass (relative L2), for 2, 3 and 4 slabs and both threshold
    searches;
  * 300 passes from the standard start: u, s, t within 1e-5 of the oracle and
    MPSNR within 0.01 dB;
  * against the single handle on the same input: the same passes under the
    stopping rule, and results equal up to the summation order of the global
    sums.
"""
import numpy as np
import pytest
import torch

from oracle import ppds as o
from paper_2510_00562_gb300 import metrics, synth
from paper_2510_00562_gb300.solver import GeoSSTVSlabs, GeoSSTVSolver, make_params

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


def _random_problem(n1, n2, n3, seed):
    rs = synth.random_state(n1, n2, n3, seed=seed, scale=0.1)
    v = np.random.default_rng(seed + 100).uniform(0, 1, size=(n3, n1, n2)).astype(np.float32)
    s64 = rs["s"].astype(np.float64)
    t64 = rs["t"].astype(np.float64)
    return rs, v, dict(eps=0.2 * np.sqrt(v.size) * 0.1, alpha=0.4 * np.abs(s64).sum(),
                       beta=0.4 * np.abs(t64).sum(), omega=0.05)


# shapes: ragged tiles, bands not divisible by the slab count, 1-band slabs
@pytest.mark.parametrize("tau_mode", ["auto", "exact"])
@pytest.mark.parametrize("shape,nslabs", [((37, 45, 9), 2), ((33, 64, 17), 3), ((70, 100, 20), 4),
                                          ((16, 32, 4), 4), ((20, 40, 3), 2)])
def test_one_pass_matches_oracle(shape, nslabs, tau_mode):
    n1, n2, n3 = shape
    rs, v, kw = _random_problem(n1, n2, n3, seed=n1 * 5 + n3)
    p = make_params(tau_mode=tau_mode, graph_iters=0, **kw)
    with GeoSSTVSlabs(n1, n2, n3, nslabs, p) as sl:
        assert len(sl.bands) == nslabs and sum(sl.bands) == n3
        sl.load(to_dev(v))
        sl.set_state({k: to_dev(rs[k]) for k in KEYS})
        st_cur = o.State(**{k: rs[k].astype(np.float64) for k in KEYS})
        for it in range(3):
            sl.iterate(1)
            st_cur = o.ppds_step(st_cur, v.astype(np.float64), oracle_params(p))
            got = {k: x.cpu().numpy() for k, x in sl.get_state().items()}
            for k in KEYS:
                e = rel(got[k], getattr(st_cur, k))
                assert e < 2e-6, (it, k, e)


def _problem(n1, n2, n3, seed=0):
    return synth.make_problem(n1, n2, n3, seed=seed, noise=synth.NoiseSpec(
        sigma=0.1, sp_rate=0.05, stripe_rate=0.05, stripe_amp=0.25))


@pytest.mark.parametrize("nslabs", [2, 3, 4])
def test_300_passes_match_oracle(nslabs):
    n1, n2, n3 = 40, 36, 12
    pb = _problem(n1, n2, n3)
    p = make_params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=0.03, max_iter=300, graph_iters=16)
    with GeoSSTVSlabs(n1, n2, n3, nslabs, p) as sl:
        u, s, t, n = sl.solve(to_dev(pb["v"]))
    assert n == 300
    st, _ = o.solve(pb["v"].astype(np.float64), oracle_params(p), 300)
    for name, a, b in (("u", u, st.u), ("s", s, st.s), ("t", t, st.t)):
        e = rel(a.cpu().numpy(), b)
        assert e < 1e-5, (name, e)
    d = abs(metrics.mpsnr(u.cpu().numpy(), pb["u_bar"]) - metrics.mpsnr(st.u, pb["u_bar"]))
    assert d <= 0.01


@pytest.mark.parametrize("nslabs", [2, 4])
def test_slabs_equal_single_handle(nslabs):
    # a larger cube with several K1 tiles and band runs per slab, the stopping
    # rule on: same passes, results equal up to the order of the global sums
    n1, n2, n3 = 96, 128, 40
    pb = _problem(n1, n2, n3, seed=7)
    p = make_params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=0.03, max_iter=400,
                    tol=1e-3, check_every=10, graph_iters=16)
    v = to_dev(pb["v"])
    with GeoSSTVSolver(n1, n2, n3, p) as sol:
        u1, s1, t1, n1_ = sol.solve(v)
    with GeoSSTVSlabs(n1, n2, n3, nslabs, p) as sl:
        u2, s2, t2, n2_ = sl.solve(v)
        stats = sl.stats()
    assert n1_ == n2_ and n1_ < 400, (n1_, n2_)
    for a, b in ((u2, u1), (s2, s1), (t2, t1)):
        assert rel(a.cpu().numpy(), b.cpu().numpy()) < 1e-6
    assert stats["iterations"] == n2_


def test_slab_arguments_are_checked():
    from paper_2510_00562_gb300 import binding as B
    p = make_params()
    with pytest.raises(B.GsstvError):
        GeoSSTVSlabs(8, 8, 4, 5, p)                   # more slabs than bands
    with pytest.raises(B.GsstvError):
        GeoSSTVSlabs(8, 8, 4, 0, p)
    with pytest.raises(B.GsstvError):
        GeoSSTVSlabs(8, 8, 4, 2, make_params(storage="bf16"))
