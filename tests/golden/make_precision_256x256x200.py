"""Writes precision_256x256x200_1000.json: the FP64 oracle's u, s, t after
1000 passes of Algorithm 1 from the standard start on the 256x256x200 crop of
the precision-study recipe (13.1 M voxels), at 4096 seeded voxels, with the
norms of u, s, t and the per-band squared errors of u against the clean cube
(for MPSNR, Eq. 29).  It is the error reference of the precision form on that
crop: 800 passes with 16-bit iterates, then 200 float32 passes (the 4:1 split
of 4000 + 1000).

Calls only the oracle -- its band-slab split over spawned gloo processes
(oracle/slabs.py, bit-identical to the whole-cube oracle) -- and the seeded
input generator, which holds none of the method's arithmetic.  About an hour
with 6 processes:

    python tests/golden/make_precision_256x256x200.py [nprocs]
"""
import json
import os
import socket
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

SHAPE = (256, 256, 200)                  # N1, N2, N3
ITERS = 1000
NOISE = dict(sigma=0.1, sp_rate=0.05, stripe_rate=0.1, stripe_amp=0.25, dead_col_rate=0.02,
             dead_band_rate=0.1)
OMEGA = 0.03
SAMPLES = 4096
OUT = os.path.join(HERE, "precision_256x256x200_1000.json")


def _worker(rank, world, port):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS="1")
    import torch.distributed as dist
    from oracle import ppds as o
    from oracle import slabs
    from paper_2510_00562_gb300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n1, n2, n3 = SHAPE
    pb = synth.make_problem(n1, n2, n3, seed=0, noise=synth.NoiseSpec(**NOISE))
    v = pb["v"].astype(np.float64)
    p = o.Params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=OMEGA)
    st = slabs.solve_slabs(dist, v, p, ITERS, rank, world)
    if rank == 0:
        ub = pb["u_bar"].astype(np.float64)
        idx = np.sort(np.random.default_rng(2026).choice(v.size, SAMPLES, replace=False))
        flat = lambda x: [float(y) for y in x.reshape(-1)[idx]]
        out = {
            "what": "FP64 oracle u, s, t after K passes of Algorithm 1 from u = v",
            "shape_n1_n2_n3": list(SHAPE), "iters": ITERS, "seed": 0, "noise": NOISE,
            "params": {"eps": p.eps, "alpha": p.alpha, "beta": p.beta, "omega": OMEGA},
            "norms": {k: float(np.linalg.norm(getattr(st, k))) for k in ("u", "s", "t")},
            "u_band_sq_err": [float(x) for x in ((st.u - ub) ** 2).reshape(n3, -1).sum(axis=1)],
            "sample_flat_index": idx.tolist(),
            "u_sample": flat(st.u), "s_sample": flat(st.s), "t_sample": flat(st.t),
            "processes": world,
        }
        with open(OUT, "w") as f:
            json.dump(out, f)
    dist.destroy_process_group()


def main():
    import torch.multiprocessing as mp
    world = int(sys.argv[1]) if len(sys.argv) > 1 else 6
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mp.spawn(_worker, args=(world, port), nprocs=world, join=True)


if __name__ == "__main__":
    main()
