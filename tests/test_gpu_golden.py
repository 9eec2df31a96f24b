"""Full-size checks against stored FP64 oracle results.  The fixtures in
tests/golden/ are written by the scripts beside them, which call only the
oracle (and the seeded input generator); the GPU side here rebuilds the same
problem from the fixture's recorded recipe.

* The gradient of mean((u_K - u_bar)^2) after K = 200 passes on the
  128x128x64 differentiation workload: each parameter adjoint and v_bar (on
  2048 sampled voxels, and its norm) within 1e-3 relative of the oracle.
"""
import json
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
