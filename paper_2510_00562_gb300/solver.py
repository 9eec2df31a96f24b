"""PyTorch-facing wrapper of the C ABI: device memory and streams from torch,
every computation in libgsstv.

Cubes are float32 tensors of shape (N3, N1, N2) -- band, row (vertical),
column (horizontal) -- contiguous, the layout of include/gsstv.h.
"""
from __future__ import annotations

import torch

from . import binding as B

STORAGE = {"fp32": B.GSSTV_FP32, "bf16": B.GSSTV_BF16, "fp16": B.GSSTV_FP16}
STATE_KEYS = ("u", "s", "t", "w1", "w2", "y1", "y2", "y3", "y4")
STATE_LEAD = {"u": (), "s": (), "t": (), "w1": (3, 2), "w2": (3, 2), "y1": (2,), "y2": (2,),
              "y3": (), "y4": ()}
# the parameters the reverse mode differentiates, in the order of the C ABI
GRAD_PARAMS = ("eps", "alpha", "beta", "omega")


def make_params(**kw) -> B.GsstvParams:
    """gsstv_default_params() with fields overridden by keyword; ``storage``
    may be given as "fp32" / "bf16" / "fp16"."""
    p = B.gsstv_default_params()
    for k, v in kw.items():
        if k == "storage" and isinstance(v, str):
            v = STORAGE[v]
        if k == "tau_mode" and isinstance(v, str):
            v = {"auto": B.GSSTV_TAU_AUTO, "exact": B.GSSTV_TAU_EXACT}[v]
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


class GeoSSTVSolver:
    """One libgsstv handle for N1 x N2 x N3 cubes on the current CUDA device."""

    def __init__(self, n1: int, n2: int, n3: int, params: B.GsstvParams | None = None,
                 stream: torch.cuda.Stream | None = None, **kw):
        if not torch.cuda.is_available():
            raise RuntimeError("GeoSSTVSolver needs a CUDA device")
        B.load()
        self.shape = (n3, n1, n2)
        self.params = params if params is not None else make_params(**kw)
        self.stream = stream or torch.cuda.current_stream()
        self.h = B.gsstv_create(n1, n2, n3, self.params, self.stream.cuda_stream)

    # -- lifetime ------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None) is not None:
            B.gsstv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- helpers ---------------------------------------------------------------
    def _dev(self, x: torch.Tensor, lead=()) -> torch.Tensor:
        want = tuple(lead) + self.shape
        if tuple(x.shape) != want:
            raise ValueError(f"expected shape {want}, got {tuple(x.shape)}")
        if x.dtype != torch.float32 or not x.is_cuda or not x.is_contiguous():
            raise ValueError("expected a contiguous float32 CUDA tensor")
        return x

    def _empty(self, lead=()):
        return torch.empty(tuple(lead) + self.shape, dtype=torch.float32, device="cuda")

    # -- API -------------------------------------------------------------------
    def set_params(self, params: B.GsstvParams | None = None, **kw):
        if params is None:
            params = self.params
            for k, v in kw.items():
                setattr(params, k, STORAGE.get(v, v) if k == "storage" else v)
        B.gsstv_set_params(self.h, params)
        self.params = params

    def solve(self, v: torch.Tensor):
        """Runs max_iter passes from the standard start; returns (u, s, t, iters)."""
        self._dev(v)
        u, s, t = self._empty(), self._empty(), self._empty()
        n = B.gsstv_solve(self.h, v.data_ptr(), u.data_ptr(), s.data_ptr(), t.data_ptr())
        return u, s, t, n

    def solve_host(self, v_host: torch.Tensor, u_host: torch.Tensor, s_host=None, t_host=None) -> int:
        """End to end from host memory (pinned tensors give the fastest copies)."""
        for x in (v_host, u_host, s_host, t_host):
            if x is not None and (x.is_cuda or x.dtype != torch.float32 or tuple(x.shape) != self.shape
                                  or not x.is_contiguous()):
                raise ValueError("expected contiguous float32 host tensors of the cube shape")
        return B.gsstv_solve_host(self.h, v_host.data_ptr(), u_host.data_ptr(),
                                  s_host.data_ptr() if s_host is not None else None,
                                  t_host.data_ptr() if t_host is not None else None)

    def load(self, v: torch.Tensor, reset: bool = True):
        B.gsstv_load_observation(self.h, self._dev(v).data_ptr())
        if reset:
            B.gsstv_reset_state(self.h)

    def reset(self):
        B.gsstv_reset_state(self.h)

    def iterate(self, n: int) -> int:
        return B.gsstv_iterate(self.h, n)

    def get_state(self) -> dict:
        st = {k: self._empty(STATE_LEAD[k]) for k in STATE_KEYS}
        B.gsstv_get_state(self.h, {k: v.data_ptr() for k, v in st.items()})
        return st

    def set_state(self, st: dict):
        tens = {k: self._dev(st[k], STATE_LEAD[k]) for k in STATE_KEYS}
        B.gsstv_set_state(self.h, {k: v.data_ptr() for k, v in tens.items()})

    def vjp_step(self, x: dict, x_next: dict, bar_next: dict, vbar: torch.Tensor | None = None,
                 in_place: bool = False, want_params: bool = True):
        """Transpose of one pass (gsstv_vjp_step): x the state before it,
        x_next the state after it, bar_next the adjoint of x_next.  Returns
        (adjoint of x, adjoint of v, adjoints of eps/alpha/beta/omega); vbar,
        if given, is accumulated into; in_place reuses bar_next's buffers;
        want_params=False skips the parameter adjoints (None) and the
        synchronisation."""
        views = [{k: self._dev(d[k], STATE_LEAD[k]) for k in STATE_KEYS} for d in (x, x_next, bar_next)]
        bar = views[2] if in_place else {k: self._empty(STATE_LEAD[k]) for k in STATE_KEYS}
        vbar = torch.zeros(self.shape, dtype=torch.float32, device="cuda") if vbar is None else self._dev(vbar)
        ptr = lambda d: {k: t.data_ptr() for k, t in d.items()}
        pb = B.gsstv_vjp_step(self.h, ptr(views[0]), ptr(views[1]), ptr(views[2]), ptr(bar), vbar.data_ptr(),
                              want_params=want_params)
        return bar, vbar, (dict(zip(GRAD_PARAMS, pb)) if want_params else None)

    def unrolled_vjp(self, iters: int, ubar: torch.Tensor, ckpt_every: int = 0):
        """Adjoint of `iters` passes from the standard start on the loaded
        observation (gsstv_unrolled_vjp): ubar is the adjoint of u after the
        last pass; returns (adjoint of v, adjoints of eps/alpha/beta/omega)."""
        vbar = self._empty()
        pb = B.gsstv_unrolled_vjp(self.h, int(iters), int(ckpt_every), self._dev(ubar).data_ptr(),
                                  vbar.data_ptr())
        return vbar, dict(zip(GRAD_PARAMS, pb))

    def stats(self) -> dict:
        s = B.gsstv_get_stats(self.h)
        return {k: getattr(s, k) for k, _ in B.GsstvStats._fields_}

    def reset_stats(self):
        B.gsstv_reset_stats(self.h)

    def set_timing(self, on: bool):
        B.gsstv_set_timing(self.h, on)

    def device_bytes(self) -> int:
        return B.gsstv_device_bytes(self.h)

    def autotune(self, v: torch.Tensor | None = None, passes: int = 20) -> int:
        """Measures the fused stencil kernel's band-run lengths on v (or the
        loaded observation) and keeps the fastest; the state is reset.
        Returns the bands per CTA chosen (0: nothing to tune)."""
        if v is not None:
            B.gsstv_load_observation(self.h, self._dev(v).data_ptr())
        return B.gsstv_autotune(self.h, passes)


class GeoSSTVBatch:
    """Independent cubes of different shapes solved together (libgsstv batch):
    each with its own parameters and Eq. 28 stopping rule; each result equals
    GeoSSTVSolver.solve on that cube alone."""

    def __init__(self, shapes, params, stream: torch.cuda.Stream | None = None):
        """shapes: list of (N1, N2, N3); params: one GsstvParams per cube."""
        if not torch.cuda.is_available():
            raise RuntimeError("GeoSSTVBatch needs a CUDA device")
        if len(shapes) != len(params) or not shapes:
            raise ValueError("one parameter set per cube, at least one cube")
        B.load()
        self.shapes = [(int(n3), int(n1), int(n2)) for n1, n2, n3 in shapes]
        self.stream = stream or torch.cuda.current_stream()
        self.b = B.gsstv_batch_create([tuple(s) for s in shapes], list(params), self.stream.cuda_stream)

    def close(self):
        if getattr(self, "b", None) is not None:
            B.gsstv_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def solve(self, vs):
        """vs: one contiguous float32 CUDA tensor (N3, N1, N2) per cube.
        Returns lists u, s, t and the passes each cube ran."""
        if len(vs) != len(self.shapes):
            raise ValueError("one observation per cube")
        for v, shp in zip(vs, self.shapes):
            if tuple(v.shape) != shp or v.dtype != torch.float32 or not v.is_cuda or not v.is_contiguous():
                raise ValueError(f"expected a contiguous float32 CUDA tensor of shape {shp}")
        us = [torch.empty_like(v) for v in vs]
        ss = [torch.empty_like(v) for v in vs]
        ts = [torch.empty_like(v) for v in vs]
        done = B.gsstv_batch_solve(self.b, [v.data_ptr() for v in vs], [u.data_ptr() for u in us],
                                   [s.data_ptr() for s in ss], [t.data_ptr() for t in ts])
        return us, ss, ts, done

    def autotune(self, vs, passes: int = 20) -> list:
        """Autotunes every cube's fused stencil kernel on its observation
        (GeoSSTVSolver.autotune); returns the bands per CTA chosen."""
        if len(vs) != len(self.shapes):
            raise ValueError("one observation per cube")
        out = []
        for c, (v, shp) in enumerate(zip(vs, self.shapes)):
            if tuple(v.shape) != shp or v.dtype != torch.float32 or not v.is_cuda or not v.is_contiguous():
                raise ValueError(f"expected a contiguous float32 CUDA tensor of shape {shp}")
            h = B.gsstv_batch_handle(self.b, c)
            B.gsstv_load_observation(h, v.data_ptr())
            out.append(B.gsstv_autotune(h, passes))
        return out

    def stats(self, c: int) -> dict:
        s = B.gsstv_get_stats(B.gsstv_batch_handle(self.b, c))
        return {k: getattr(s, k) for k, _ in B.GsstvStats._fields_}


class GeoSSTVSlabs:
    """One N1 x N2 x N3 cube stored as `nslabs` band slabs (gsstv_slabs_*):
    each slab in allocations of its own with one halo band on each side, the
    global sums of every pass finished over all slabs, the halo planes copied
    after every pass.  The same calls as GeoSSTVSolver for solves and states."""

    def __init__(self, n1: int, n2: int, n3: int, nslabs: int, params: B.GsstvParams | None = None,
                 stream: torch.cuda.Stream | None = None, **kw):
        if not torch.cuda.is_available():
            raise RuntimeError("GeoSSTVSlabs needs a CUDA device")
        B.load()
        self.shape = (n3, n1, n2)
        self.params = params if params is not None else make_params(**kw)
        self.stream = stream or torch.cuda.current_stream()
        self.h = B.gsstv_slabs_create(n1, n2, n3, nslabs, self.params, self.stream.cuda_stream)
        self.bands = B.gsstv_slabs_count(self.h)

    def close(self):
        if getattr(self, "h", None) is not None:
            B.gsstv_slabs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _empty(self, lead=()):
        return torch.empty(tuple(lead) + self.shape, dtype=torch.float32, device="cuda")

    def solve(self, v: torch.Tensor):
        """Runs max_iter passes from the standard start; returns (u, s, t, iters)."""
        if tuple(v.shape) != self.shape or v.dtype != torch.float32 or not v.is_cuda or not v.is_contiguous():
            raise ValueError("expected a contiguous float32 CUDA tensor of the cube shape")
        u, s, t = self._empty(), self._empty(), self._empty()
        n = B.gsstv_slabs_solve(self.h, v.data_ptr(), u.data_ptr(), s.data_ptr(), t.data_ptr())
        return u, s, t, n

    def load(self, v: torch.Tensor, reset: bool = True):
        B.gsstv_slabs_load_observation(self.h, v.data_ptr())
        if reset:
            B.gsstv_slabs_reset_state(self.h)

    def iterate(self, n: int) -> int:
        return B.gsstv_slabs_iterate(self.h, n)

    def get_state(self) -> dict:
        st = {k: self._empty(STATE_LEAD[k]) for k in STATE_KEYS}
        B.gsstv_slabs_get_state(self.h, {k: st[k].data_ptr() for k in STATE_KEYS})
        return st

    def set_state(self, st: dict):
        for k in STATE_KEYS:
            want = tuple(STATE_LEAD[k]) + self.shape
            x = st[k]
            if tuple(x.shape) != want or x.dtype != torch.float32 or not x.is_cuda or not x.is_contiguous():
                raise ValueError(f"state {k}: expected a contiguous float32 CUDA tensor of shape {want}")
        B.gsstv_slabs_set_state(self.h, {k: st[k].data_ptr() for k in STATE_KEYS})

    def stats(self) -> dict:
        s = B.gsstv_slabs_get_stats(self.h)
        return {k: getattr(s, k) for k, _ in B.GsstvStats._fields_}


def project_l1ball(x: torch.Tensor, radius: float, out: torch.Tensor | None = None):
    """Projection of a float32 CUDA vector onto the l1 ball; returns (out, tau)."""
    if x.dtype != torch.float32 or not x.is_cuda or not x.is_contiguous():
        raise ValueError("expected a contiguous float32 CUDA tensor")
    out = torch.empty_like(x) if out is None else out
    tau = B.gsstv_project_l1ball(x.data_ptr(), x.numel(), float(radius), out.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    return out, tau
