"""Precision form: iterates stored in BF16 / FP16 with FP32 arithmetic, then
an FP32 phase warm-started from the 16-bit state (gsstv_get_state ->
gsstv_set_state).  Each result's error against the FP64 oracle is printed;
the claim checked is the one the mixed form must meet to be useful: its
MPSNR against the clean cube is within 0.01 dB of the plain FP32 run's.
"""
import numpy as np
import pytest
import torch

from oracle import ppds as o
from paper_2510_00562_gb300 import metrics, synth
from paper_2510_00562_gb300.solver import GeoSSTVSolver, make_params

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def problem():
    n1, n2, n3, iters = 64, 64, 32, 2000
    pb = synth.make_problem(n1, n2, n3, seed=0, noise=synth.NoiseSpec(
        sigma=0.1, sp_rate=0.05, stripe_rate=0.05, stripe_amp=0.25))
    kw = dict(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=0.03)
    st, _ = o.solve(pb["v"].astype(np.float64), o.Params(**kw), iters)
    with GeoSSTVSolver(n1, n2, n3, make_params(max_iter=iters, **kw)) as sol:
        u32, s32, t32, _ = sol.solve(torch.from_numpy(pb["v"]).cuda())
    return dict(pb=pb, kw=kw, shape=(n1, n2, n3), iters=iters, oracle=st,
                fp32=(u32.cpu().numpy(), s32.cpu().numpy(), t32.cpu().numpy()))


@pytest.mark.parametrize("storage", ["bf16", "fp16"])
def test_mixed_then_fp32_refinement(problem, storage):
    pb, kw, iters = problem["pb"], problem["kw"], problem["iters"]
    n1, n2, n3 = problem["shape"]
    n16 = iters * 4 // 5                     # 16-bit phase, then an FP32 phase
    v = torch.from_numpy(pb["v"]).cuda()
    with GeoSSTVSolver(n1, n2, n3, make_params(max_iter=n16, storage=storage, **kw)) as lo:
        u16, s16, t16, _ = lo.solve(v)
        state = lo.get_state()
    with GeoSSTVSolver(n1, n2, n3, make_params(max_iter=iters - n16, **kw)) as hi:
        hi.load(v, reset=False)
        hi.set_state(state)
        hi.iterate(iters - n16)
        fin = hi.get_state()
    st = problem["oracle"]
    u32 = problem["fp32"][0]
    ub = pb["u_bar"]
    errs16 = {k: rel(x.cpu().numpy(), getattr(st, k)) for k, x in (("u", u16), ("s", s16), ("t", t16))}
    errs = {k: rel(fin[k].cpu().numpy(), getattr(st, k)) for k in ("u", "s", "t")}
    m32 = metrics.mpsnr(u32, ub)
    m16 = metrics.mpsnr(u16.cpu().numpy(), ub)
    mref = metrics.mpsnr(fin["u"].cpu().numpy(), ub)
    print(f"\nprecision {storage}: {n16} 16-bit passes: err vs oracle {errs16}, MPSNR {m16:.4f}; "
          f"+{iters - n16} FP32 passes: err {errs}, MPSNR {mref:.4f}; FP32 alone {m32:.4f}")
    assert abs(mref - m32) <= 0.01
    assert max(errs.values()) < 1e-2


@pytest.mark.parametrize("storage,tol", [("bf16", 2e-2), ("fp16", 3e-3)])
@pytest.mark.parametrize("shape", [(70, 100, 20), (64, 96, 40)])
def test_one_pass_16bit_storage(shape, storage, tol):
    """One pass from a random state with 16-bit storage, on cubes that have
    interior tiles (the stencil kernel's unmasked path) as well as border
    tiles: every variable within the 16-bit rounding of the inputs and outputs
    (BF16 8 bits, FP16 11 bits of mantissa) of the FP64 oracle's pass."""
    n1, n2, n3 = shape
    rs = synth.random_state(n1, n2, n3, seed=3, scale=0.1)
    v = np.random.default_rng(8).uniform(0, 1, size=(n3, n1, n2)).astype(np.float32)
    kw = dict(eps=0.02 * np.sqrt(v.size), alpha=0.4 * float(np.abs(rs["s"].astype(np.float64)).sum()),
              beta=0.4 * float(np.abs(rs["t"].astype(np.float64)).sum()), omega=0.05)
    with GeoSSTVSolver(n1, n2, n3, make_params(storage=storage, graph_iters=0, **kw)) as sol:
        sol.load(torch.from_numpy(v).cuda())
        sol.set_state({k: torch.from_numpy(rs[k]).cuda() for k in rs})
        start = {k: x.cpu().numpy().astype(np.float64) for k, x in sol.get_state().items()}
        sol.iterate(1)
        got = {k: x.cpu().numpy() for k, x in sol.get_state().items()}
    ref = o.ppds_step(o.State(**start), v.astype(np.float64), o.Params(**kw))
    for k in got:
        e = rel(got[k], getattr(ref, k))
        assert e < tol, (k, e)
