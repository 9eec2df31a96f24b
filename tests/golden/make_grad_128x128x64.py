"""Writes grad_128x128x64_k200.json: the FP64 oracle's gradient of the loss
mean((u_K - u_bar)^2) after K = 200 passes of Algorithm 1 from the standard
start, on the 128x128x64 differentiation workload, with respect to v (at 2048
seeded voxels, and its norm) and to eps, alpha, beta, omega.

Calls only the oracle (and the seeded input generator, which holds none of
the method's arithmetic).  About 15 minutes on one host core:

    python tests/golden/make_grad_128x128x64.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import adjoint as A          # noqa: E402
from oracle import ppds as o             # noqa: E402
from paper_2510_00562_gb300 import synth  # noqa: E402

SHAPE = (128, 128, 64)                   # N1, N2, N3
ITERS = 200
NOISE = dict(sigma=0.1, sp_rate=0.05, stripe_rate=0.1, stripe_amp=0.25, dead_col_rate=0.02,
             dead_band_rate=0.1)
OMEGA = 0.03
SAMPLES = 2048


def main():
    n1, n2, n3 = SHAPE
    pb = synth.make_problem(n1, n2, n3, seed=0, noise=synth.NoiseSpec(**NOISE))
    v = pb["v"].astype(np.float64)
    ub = pb["u_bar"].astype(np.float64)
    p = o.Params(eps=pb["eps"], alpha=pb["alpha"], beta=pb["beta"], omega=OMEGA)
    loss, vbar, pbar = A.unrolled_grad(v, ub, p, ITERS, ckpt_every=20)
    idx = np.sort(np.random.default_rng(2024).choice(v.size, SAMPLES, replace=False))
    out = {
        "what": "FP64 oracle gradient of mean((u_K - u_bar)^2), K passes of Algorithm 1 from u = v",
        "shape_n1_n2_n3": list(SHAPE), "iters": ITERS, "seed": 0, "noise": NOISE,
        "params": {"eps": p.eps, "alpha": p.alpha, "beta": p.beta, "omega": OMEGA},
        "loss": loss, "params_bar": pbar, "vbar_norm": float(np.linalg.norm(vbar)),
        "sample_flat_index": idx.tolist(), "vbar_sample": [float(x) for x in vbar.reshape(-1)[idx]],
    }
    with open(os.path.join(HERE, "grad_128x128x64_k200.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()
