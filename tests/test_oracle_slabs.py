"""The oracle split into band slabs over gloo ranks (CPU) reproduces the
whole-cube oracle bit for bit.

Each rank holds its bands plus one halo band on each side, exchanges the
halos (u' of its first band down, y2 of its last band up) and takes the l1-
and l2-ball projections on the gathered whole vectors (oracle/slabs.py).  Every
operation on an owned band is then the same float64 operation as in the
whole-cube pass, so the assembled state must equal the whole-cube oracle's
exactly, from the standard start and from a random state, for 2 and 3 ranks
and for bands that do not divide evenly.  Planted mistakes (no halo exchange;
one l1 ball per slab) must break it.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import numpy as np
import torch.distributed as dist
from oracle import ppds as o
from oracle import slabs
from paper_2510_00562_gb300 import synth

rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
plant = os.environ.get("PLANT", "")
if plant == "no_halo":          # skip both halo exchanges
    slabs._send_recv = lambda *a, **k: None
if plant == "local_l1":         # each slab projects onto its own l1 ball
    def _local_l1(dist_, x, r, n3_, rank_, world_):
        b0, b1, l0, l1 = slabs.slab_bands(rank_, world_, n3_)
        out = np.zeros_like(x)
        out[b0 - l0:b1 - l0], tau = o.proj_l1ball(x[b0 - l0:b1 - l0], r / world_)
        return out, tau
    slabs._global_l1 = _local_l1
n1, n2, n3, iters = {n1}, {n2}, {n3}, {iters}
pb = synth.make_problem(n1, n2, n3, seed=4)
v = pb["v"].astype(np.float64)
p = o.Params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=0.03)
out = {{}}
# from the standard start
got = slabs.solve_slabs(dist, v, p, iters, rank, world)
ref, _ = o.solve(v, p, iters)
out["start"] = {{k: bool(np.array_equal(getattr(got, k), getattr(ref, k))) for k in o.State.names()}}
# from a random state (every variable nonzero, the box and both balls active)
rs = synth.random_state(n1, n2, n3, seed=9, scale=0.1)
st0 = o.State(**{{k: rs[k].astype(np.float64) for k in o.State.names()}})
q = o.Params(eps=0.2 * np.sqrt(v.size) * 0.1, alpha=0.4 * np.abs(st0.s).sum(),
             beta=0.4 * np.abs(st0.t).sum(), omega=0.05)
got = slabs.solve_slabs(dist, v, q, 3, rank, world, state=st0)
ref, _ = o.solve(v, q, 3, state=st0)
out["random"] = {{k: bool(np.array_equal(getattr(got, k), getattr(ref, k))) for k in o.State.names()}}
out["rank"] = rank
print(json.dumps(out))
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _run(world, shape, iters, plant=""):
    n1, n2, n3 = shape
    port = _free_port()
    procs = []
    for rank in range(world):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="", PLANT=plant)
        code = WORKER.format(root=ROOT, n1=n1, n2=n2, n3=n3, iters=iters)
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    results = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err[-3000:]
        results.append(json.loads(out.strip().splitlines()[-1]))
    return results


@pytest.mark.parametrize("world,shape,iters", [(2, (12, 10, 7), 40), (3, (9, 11, 8), 25), (2, (6, 8, 2), 10)])
def test_slab_split_is_bit_exact(world, shape, iters):
    for res in _run(world, shape, iters):
        for case in ("start", "random"):
            assert all(res[case].values()), (res["rank"], case, res[case])


@pytest.mark.parametrize("plant", ["no_halo", "local_l1"])
def test_planted_mistakes_break_bit_exactness(plant):
    # a split without the halo exchanges, or with one l1 ball per slab, must
    # not reproduce the whole cube
    for res in _run(2, (12, 10, 7), 10, plant=plant):
        assert not all(res["start"].values()) or not all(res["random"].values()), (plant, res)


def test_slab_bands_partition_the_cube():
    from oracle import slabs
    for n3 in (1, 2, 7, 224):
        for world in range(1, min(n3, 6) + 1):
            owned = []
            for r in range(world):
                b0, b1, l0, l1 = slabs.slab_bands(r, world, n3)
                assert b1 > b0 and l0 == max(b0 - 1, 0) and l1 == min(b1 + 1, n3)
                owned.extend(range(b0, b1))
            assert owned == list(range(n3))
