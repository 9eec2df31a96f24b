"""Full-size checks against stored FP64 oracle results.  The fixtures in
tests/golden/ are written by the scripts beside them, which call only the
oracle (and the seeded input generator); the GPU side here rebuilds the same
problem from the fixture's recorded recipe.

* The gradient of mean((u_K - u_bar)^2) after K = 200 passes on the
  128x128x64 differentiation workload: each parameter adjoint and v_bar (on
  2048 sampled voxels, and its norm) within 1e-3 relative of the oracle.
* 5000 passes on a 64x64x200 cube, and 1000 passes on the 256x256x200 crop,
  of the precision-study recipe: the float32
  path within 1e-5 relative L2 of the oracle on u, s, t (sampled voxels) and
  within 0.01 dB of its MPSNR either way (the parity bar of the plain
  method); the mixed forms (4/5 of the passes with 16-bit iterates, then
  float32 passes warm-started from them) lose at most 0.01 dB of MPSNR
  against the oracle (their bar is a loss: ending above it is allowed), their
  errors printed.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

from paper_2510_00562_gb300 import synth
from paper_2510_00562_gb300.solver import GRAD_PARAMS, GeoSSTVSolver, make_params

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _fixture(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _problem(fx):
    n1, n2, n3 = fx["shape_n1_n2_n3"]
    pb = synth.make_problem(n1, n2, n3, seed=fx["seed"], noise=synth.NoiseSpec(**fx["noise"]))
    for k in ("eps", "alpha", "beta"):      # the same recipe gives the same radii
        assert pb[k] == pytest.approx(fx["params"][k], rel=1e-9), k
    return (n1, n2, n3), pb


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _mpsnr_from_band_errors(err, npix):
    return float(np.mean([10.0 * math.log10(npix / e) for e in err if e > 0]))


def test_unrolled_gradient_full_size_matches_oracle():
    fx = _fixture("grad_128x128x64_k200.json")
    (n1, n2, n3), pb = _problem(fx)
    K = fx["iters"]
    v = torch.from_numpy(pb["v"]).cuda()
    ub = torch.from_numpy(pb["u_bar"].astype(np.float64)).cuda()
    p = make_params(max_iter=K, graph_iters=16, **fx["params"])
    with GeoSSTVSolver(n1, n2, n3, p) as sol:
        u, _, _, _ = sol.solve(v)
        loss = float(((u.double() - ub) ** 2).mean())
        seed = ((2.0 / v.numel()) * (u.double() - ub)).float().contiguous()
        sol.load(v)
        vbar, pbar = sol.unrolled_vjp(K, seed, ckpt_every=20)
    idx = np.asarray(fx["sample_flat_index"])
    vb = vbar.cpu().numpy().reshape(-1)
    print("loss", loss, fx["loss"], "vbar sample rel", _rel(vb[idx], fx["vbar_sample"]),
          "norm", float(np.linalg.norm(vb)), fx["vbar_norm"],
          {k: (pbar[k], fx["params_bar"][k]) for k in GRAD_PARAMS})
    assert loss == pytest.approx(fx["loss"], rel=1e-4)
    assert _rel(vb[idx], fx["vbar_sample"]) < 1e-3
    assert float(np.linalg.norm(vb)) == pytest.approx(fx["vbar_norm"], rel=1e-3)
    for k in GRAD_PARAMS:
        assert pbar[k] == pytest.approx(fx["params_bar"][k], rel=1e-3), k


def _precision_forms_against_fixture(name):
    fx = _fixture(name)
    (n1, n2, n3), pb = _problem(fx)
    K = fx["iters"]
    n16 = (4 * K) // 5
    idx = np.asarray(fx["sample_flat_index"])
    m_or = _mpsnr_from_band_errors(fx["u_band_sq_err"], n1 * n2)
    v = torch.from_numpy(pb["v"]).cuda()
    kw = dict(graph_iters=16, **fx["params"])
    ub = pb["u_bar"]

    def errs(st):
        out = {k: _rel(st[k].cpu().numpy().reshape(-1)[idx], fx[f"{k}_sample"]) for k in ("u", "s", "t")}
        u = st["u"].cpu().numpy().astype(np.float64)
        band = ((u - ub) ** 2).reshape(n3, -1).sum(axis=1)
        out["mpsnr_delta_db"] = _mpsnr_from_band_errors(band, n1 * n2) - m_or
        return out

    with GeoSSTVSolver(n1, n2, n3, make_params(max_iter=K, **kw)) as s32:
        s32.load(v)
        s32.iterate(K)
        e32 = errs(s32.get_state())
        res = {"fp32": e32}
        for storage in ("bf16", "fp16"):
            with GeoSSTVSolver(n1, n2, n3, make_params(max_iter=n16, storage=storage, **kw)) as lo:
                lo.load(v)
                lo.iterate(n16)
                st = lo.get_state()
            s32.load(v, reset=False)
            s32.set_state(st)
            s32.iterate(K - n16)
            res[storage] = errs(s32.get_state())
    print(name, "oracle MPSNR", m_or, json.dumps(res))
    for k in ("u", "s", "t"):
        assert e32[k] < 1e-5, (k, e32[k])
    assert abs(e32["mpsnr_delta_db"]) <= 0.01
    for form in ("bf16", "fp16"):
        assert res[form]["mpsnr_delta_db"] >= -0.01, (form, res[form])
    return res


def test_precision_forms_5000_passes_against_oracle():
    _precision_forms_against_fixture("precision_64x64x200_5000.json")


@pytest.mark.skipif(not os.path.exists(os.path.join(GOLD, "precision_256x256x200_1000.json")),
                    reason="fixture not written (tests/golden/make_precision_256x256x200.py)")
def test_precision_forms_256x256x200_crop_against_oracle():
    """The precision form's error reference on the 256x256x200 crop of the
    precision-study recipe: 1000 passes (800 with 16-bit iterates, then 200
    float32 passes; the 4:1 split of 4000 + 1000), against the FP64 oracle's
    1000 passes on the same crop."""
    _precision_forms_against_fixture("precision_256x256x200_1000.json")
