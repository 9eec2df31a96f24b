"""Timed passes (gsstv_set_timing) against untimed ones.

With timing on, whole blocks of passes still run as CUDA graphs (each built
for its launch, with a pair of timing events captured around every K1), the
rest eagerly; the passes must be the same computation as with timing off, and
every K1 launch must be timed.  The search gate's count (`search_passes`) is
bounded by the graph passes run.
"""
import numpy as np
import pytest
import torch

from paper_2510_00562_gb300 import synth
from paper_2510_00562_gb300.solver import GeoSSTVSolver, make_params

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a - b)


@pytest.mark.parametrize("passes", [37, 48])
def test_timed_passes_equal_untimed(passes):
    n1, n2, n3 = 48, 64, 20
    pb = synth.make_problem(n1, n2, n3, seed=3)
    p = make_params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=0.03, graph_iters=16)
    v = torch.from_numpy(pb["v"]).cuda()
    with GeoSSTVSolver(n1, n2, n3, p) as a, GeoSSTVSolver(n1, n2, n3, p) as b:
        a.load(v)
        b.load(v)
        a.reset_stats()
        a.set_timing(True)
        a.iterate(passes)
        st = a.stats()
        a.set_timing(False)
        b.reset_stats()
        b.iterate(passes)
        sa, sb = a.get_state(), b.get_state()
        stb = b.stats()
    for k in ("u", "s", "t", "w1", "w2", "y1", "y2", "y3", "y4"):
        assert rel(sa[k], sb[k]) < 1e-6, k
    assert st["iterations"] == passes
    assert st["k1_launches"] == passes and st["k1_ms"] > 0.0
    graph_passes = (passes // 16) * 16
    assert 0 <= st["search_passes"] <= graph_passes
    assert 0 <= stb["search_passes"] <= graph_passes
