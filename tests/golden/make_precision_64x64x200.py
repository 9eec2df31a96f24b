"""Writes precision_64x64x200_5000.json: the FP64 oracle's u, s, t after 5000
passes of Algorithm 1 from the standard start on a 64x64x200 cube of the
precision-study recipe, at 2048 seeded voxels, with the norms of u, s, t and
the per-band squared errors of u against the clean cube (for MPSNR, Eq. 29).

Calls only the oracle (and the seeded input generator, which holds none of
the method's arithmetic).  About an hour on one host core:

    python tests/golden/make_precision_64x64x200.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ppds as o             # noqa: E402
from paper_2510_00562_gb300 import synth  # noqa: E402

SHAPE = (64, 64, 200)                    # N1, N2, N3
ITERS = 5000
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
    st = o.init_state(v)
    for _ in range(ITERS):
        st = o.ppds_step(st, v, p)
    idx = np.sort(np.random.default_rng(2025).choice(v.size, SAMPLES, replace=False))
    flat = lambda x: [float(y) for y in x.reshape(-1)[idx]]
    out = {
        "what": "FP64 oracle u, s, t after K passes of Algorithm 1 from u = v",
        "shape_n1_n2_n3": list(SHAPE), "iters": ITERS, "seed": 0, "noise": NOISE,
        "params": {"eps": p.eps, "alpha": p.alpha, "beta": p.beta, "omega": OMEGA},
        "norms": {k: float(np.linalg.norm(getattr(st, k))) for k in ("u", "s", "t")},
        "u_band_sq_err": [float(x) for x in ((st.u - ub) ** 2).reshape(n3, -1).sum(axis=1)],
        "sample_flat_index": idx.tolist(),
        "u_sample": flat(st.u), "s_sample": flat(st.s), "t_sample": flat(st.t),
    }
    with open(os.path.join(HERE, "precision_64x64x200_5000.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()
