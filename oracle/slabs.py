"""Algorithm 1 on one cube split into band slabs over processes (FP64, CPU).

TEST INFRASTRUCTURE ONLY, like ``oracle/ppds.py``: imported by ``tests/``
(and usable from ``bench.py``'s CPU legs), never by the
``paper_2510_00562_gb300`` package, and sharing no code with the CUDA path.

The only couplings between bands in a pass of Algorithm 1 are the spectral
difference D_s and its transpose (Sec. II-A) and the two global projections:
onto the l1 balls (Sec. III-B) and onto the l2 ball (Eq. 23).  So a rank
holding bands [B0, B1) plus one halo band on each side runs the pass of
``ppds_step`` on its local arrays, with

* the l1-ball projections of s~ and t~ and the l2-ball projection of
  y4'/gamma taken on the whole vectors gathered from every rank (in band
  order, so the projections see exactly the whole-cube vectors);
* one halo exchange inside the pass: the extrapolated u' of a slab's first
  band goes to the slab below (D D_s u' at its last band needs it);
* one after the pass: y2 of a slab's last band goes to the slab above
  (D_s^T D^T y2 at its first band needs it).

The owned bands then hold, bit for bit, what the whole-cube oracle computes.
Communication uses torch.distributed (any backend that moves CPU tensors,
e.g. gloo).
"""
from __future__ import annotations

import numpy as np

from . import ppds as o

__all__ = ["slab_bands", "scatter_state", "gather_state", "slab_step", "solve_slabs"]


def slab_bands(rank: int, world: int, n3: int):
    """(B0, B1, L0, L1): owned bands [B0, B1) and stored bands [L0, L1)."""
    b0 = rank * n3 // world
    b1 = (rank + 1) * n3 // world
    return b0, b1, max(b0 - 1, 0), min(b1 + 1, n3)


def _cut(x, lo, hi):
    """Bands [lo, hi) of a cube, or of each cube of a stack (bands axis -3)."""
    return x[..., lo:hi, :, :].copy()


def scatter_state(st: o.State, rank: int, world: int) -> o.State:
    """The local (stored) bands of a whole-cube state."""
    n3 = st.u.shape[0]
    _, _, l0, l1 = slab_bands(rank, world, n3)
    return o.State(*(_cut(getattr(st, k), l0, l1) for k in o.State.names()))


def _owned(x, rank, world, n3):
    b0, b1, l0, _ = slab_bands(rank, world, n3)
    return x[..., b0 - l0:b1 - l0, :, :]


def _gather_bands(dist, x_owned, n3, rank, world):
    """All ranks' owned bands of x (bands axis -3) concatenated in band order."""
    import torch
    counts = [slab_bands(r, world, n3)[1] - slab_bands(r, world, n3)[0] for r in range(world)]
    width = max(counts)
    lead = x_owned.shape[:-3]
    tail = x_owned.shape[-2:]
    pad = np.zeros(lead + (width,) + tail)
    pad[..., :x_owned.shape[-3], :, :] = x_owned
    bufs = [torch.zeros(pad.shape, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(bufs, torch.from_numpy(pad))
    parts = [b.numpy()[..., :c, :, :] for b, c in zip(bufs, counts)]
    return np.concatenate(parts, axis=-3)


def gather_state(dist, st_local: o.State, n3: int, rank: int, world: int) -> o.State:
    """The whole-cube state assembled from every rank's owned bands."""
    return o.State(*(_gather_bands(dist, _owned(getattr(st_local, k), rank, world, n3), n3, rank, world)
                     for k in o.State.names()))


def _send_recv(dist, send, dst, recv_shape, src):
    """Sends `send` to rank dst (if not None) and receives from src (if not None)."""
    import torch
    reqs = []
    out = None
    if send is not None:
        reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(send)), dst))
    if src is not None:
        out = torch.zeros(recv_shape, dtype=torch.float64)
        reqs.append(dist.irecv(out, src))
    for r in reqs:
        r.wait()
    return None if out is None else out.numpy()


def _global_l1(dist, x_local, r, n3, rank, world):
    """Projection of the owned part of x onto the l1 ball of the whole vector."""
    whole = _gather_bands(dist, _owned(x_local, rank, world, n3), n3, rank, world)
    p_whole, tau = o.proj_l1ball(whole, r)
    b0, b1, l0, l1 = slab_bands(rank, world, n3)
    out = np.zeros_like(x_local)
    out[b0 - l0:b1 - l0] = p_whole[b0:b1]
    return out, tau


def slab_step(dist, st: o.State, v_local, p: o.Params, n3: int, rank: int, world: int,
              v_whole=None) -> o.State:
    """One pass of Algorithm 1 on this rank's slab (see the module docstring).

    st, v_local: the stored bands [L0, L1); v_whole (optional): the whole
    observation, gathered here when not given.  Returns the next local state,
    with the halo bands refreshed from the neighbours."""
    v_local = np.asarray(v_local, dtype=np.float64)
    b0, b1, l0, l1 = slab_bands(rank, world, n3)
    lo_nb = rank - 1 if b0 > 0 else None          # the rank holding the band below
    hi_nb = rank + 1 if b1 < n3 else None         # the rank holding the band above
    # primal blocks (the same steps as ppds_step, on the stored bands)
    gu, gw1, gw2, gs, gt = o.apply_AT(st.y1, st.y2, st.y3, st.y4)
    u1 = o.proj_box(st.u - p.gamma_u * gu, p.mu_lo, p.mu_hi)
    w11 = o.prox_l12(st.w1 - p.gamma_w1 * gw1, p.gamma_w1 * p.omega)
    w21 = o.prox_l12(st.w2 - p.gamma_w2 * gw2, p.gamma_w2)
    s1, tau_s = _global_l1(dist, st.s - p.gamma_s * gs, p.alpha, n3, rank, world)
    t1, tau_t = _global_l1(dist, st.t - p.gamma_t * gt, p.beta, n3, rank, world)
    xb = [2 * a - b for a, b in ((u1, st.u), (w11, st.w1), (w21, st.w2), (s1, st.s), (t1, st.t))]
    # halo: u' of the first owned band goes down, the band above comes up
    plane = st.u.shape[1:]
    got = _send_recv(dist, xb[0][b0 - l0] if lo_nb is not None else None, lo_nb, plane, hi_nb)
    if got is not None:
        xb[0][b1 - l0] = got
    # dual blocks
    a1, a2, a3, a4 = o.apply_A(*xb)
    y11 = st.y1 + p.gamma_y1 * a1
    y21 = st.y2 + p.gamma_y2 * a2
    y31 = st.y3 + p.gamma_y3 * a3
    y4p = st.y4 + p.gamma_y4 * a4
    # the l2-ball step on the whole vector: y4 = y4' - g P_B(y4' / g)
    z_whole = _gather_bands(dist, _owned(y4p / p.gamma_y4, rank, world, n3), n3, rank, world)
    if v_whole is None:
        v_whole = _gather_bands(dist, _owned(v_local, rank, world, n3), n3, rank, world)
    pz = o.proj_l2ball(z_whole, v_whole, p.eps)
    y41 = np.zeros_like(y4p)
    y41[b0 - l0:b1 - l0] = y4p[b0 - l0:b1 - l0] - p.gamma_y4 * pz[b0:b1]
    out = o.State(u=u1, s=s1, t=t1, w1=w11, w2=w21, y1=y11, y2=y21, y3=y31, y4=y41)
    # halo: y2 of the last owned band goes up, the band below comes down
    got = _send_recv(dist, y21[:, b1 - 1 - l0] if hi_nb is not None else None, hi_nb, (2,) + plane, lo_nb)
    if got is not None:
        out.y2[:, 0] = got
    out.extra = {"tau_s": tau_s, "tau_t": tau_t}
    return out


def solve_slabs(dist, v, p: o.Params, iters: int, rank: int, world: int, state: o.State | None = None):
    """`iters` passes from the standard start (or `state`, a whole-cube
    state), split over the ranks of `dist`; returns the whole-cube state
    (every rank gets it)."""
    v = np.asarray(v, dtype=np.float64)
    n3 = v.shape[0]
    whole = o.init_state(v) if state is None else state
    st = scatter_state(whole, rank, world)
    _, _, l0, l1 = slab_bands(rank, world, n3)
    v_local = v[l0:l1]
    for _ in range(iters):
        st = slab_step(dist, st, v_local, p, n3, rank, world, v_whole=v)
    return gather_state(dist, st, n3, rank, world)
