"""Thin ctypes binding of libgsstv's C ABI (include/gsstv.h).

Argument marshalling only: every step of the solver runs in the CUDA library.
Device buffers are passed as raw pointers (``tensor.data_ptr()`` of CUDA
tensors), streams as ``cudaStream_t`` values (``torch.cuda.current_stream()
.cuda_stream``).  The library is the in-tree ``libgsstv.so`` built by
``paper_2510_00562_gb300.build``; if it is missing or fails to load, every
entry point raises -- there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgsstv.so")

GSSTV_OK = 0
GSSTV_ERR_ARG = -1
GSSTV_ERR_OOM = -2
GSSTV_ERR_CUDA = -3
GSSTV_ERR_NONFINITE = -4
GSSTV_ERR_TIMEOUT = -5
GSSTV_ERR_INTERNAL = -6

GSSTV_FP32, GSSTV_BF16, GSSTV_FP16 = 0, 1, 2
GSSTV_TAU_AUTO, GSSTV_TAU_EXACT = 0, 1

c_double, c_int, c_void_p, c_int64 = ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64


class GsstvParams(ctypes.Structure):
    _fields_ = [
        ("eps", c_double), ("alpha", c_double), ("beta", c_double), ("omega", c_double),
        ("mu_lo", c_double), ("mu_hi", c_double),
        ("gamma_u", c_double), ("gamma_w1", c_double), ("gamma_w2", c_double),
        ("gamma_s", c_double), ("gamma_t", c_double),
        ("gamma_y1", c_double), ("gamma_y2", c_double), ("gamma_y3", c_double), ("gamma_y4", c_double),
        ("max_iter", c_int), ("tol", c_double), ("check_every", c_int),
        ("storage", c_int), ("tau_mode", c_int), ("graph_iters", c_int),
    ]


class GsstvStats(ctypes.Structure):
    _fields_ = [
        ("iterations", c_int64), ("tau_window_hits", c_int64), ("tau_exact_runs", c_int64),
        ("k1_ms", c_double), ("k1_launches", c_int64),
        ("last_rel_change", c_double), ("last_tau_s", c_double), ("last_tau_t", c_double),
        ("last_l2_scale", c_double), ("tau_retry_hits", c_int64), ("search_passes", c_int64),
    ]


class GsstvStateView(ctypes.Structure):
    _fields_ = [(k, c_void_p) for k in ("u", "s", "t", "w1", "w2", "y1", "y2", "y3", "y4")]


_lib = None

_SIGS = {
    "gsstv_default_params": (None, [ctypes.POINTER(GsstvParams)]),
    "gsstv_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_int, c_int,
                             ctypes.POINTER(GsstvParams), c_void_p]),
    "gsstv_set_params": (c_int, [c_void_p, ctypes.POINTER(GsstvParams)]),
    "gsstv_destroy": (c_int, [c_void_p]),
    "gsstv_load_observation": (c_int, [c_void_p, c_void_p]),
    "gsstv_reset_state": (c_int, [c_void_p]),
    "gsstv_iterate": (c_int, [c_void_p, c_int, ctypes.POINTER(c_int)]),
    "gsstv_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_int)]),
    "gsstv_solve_host": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_int)]),
    "gsstv_get_state": (c_int, [c_void_p, ctypes.POINTER(GsstvStateView)]),
    "gsstv_set_state": (c_int, [c_void_p, ctypes.POINTER(GsstvStateView)]),
    "gsstv_get_stats": (c_int, [c_void_p, ctypes.POINTER(GsstvStats)]),
    "gsstv_reset_stats": (c_int, [c_void_p]),
    "gsstv_set_timing": (c_int, [c_void_p, c_int]),
    "gsstv_device_bytes": (c_int64, [c_void_p]),
    "gsstv_autotune": (c_int, [c_void_p, c_int, ctypes.POINTER(c_int)]),
    "gsstv_project_l1ball": (c_int, [c_void_p, c_int64, c_double, c_void_p,
                                     ctypes.POINTER(c_double), c_void_p]),
    "gsstv_project_l1ball_noalloc": (c_int, [c_void_p, c_int64, c_double, c_void_p,
                                             ctypes.POINTER(c_double), c_void_p]),
    "gsstv_batch_create": (c_int, [ctypes.POINTER(c_void_p), c_int, ctypes.POINTER(c_int),
                                   ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                   ctypes.POINTER(GsstvParams), c_void_p]),
    "gsstv_batch_solve": (c_int, [c_void_p, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                  ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                  ctypes.POINTER(c_int)]),
    "gsstv_batch_size": (c_int, [c_void_p]),
    "gsstv_batch_handle": (c_int, [c_void_p, c_int, ctypes.POINTER(c_void_p)]),
    "gsstv_batch_destroy": (c_int, [c_void_p]),
    "gsstv_vjp_step": (c_int, [c_void_p] + [ctypes.POINTER(GsstvStateView)] * 4 +
                       [c_void_p, ctypes.POINTER(c_double)]),
    "gsstv_unrolled_vjp": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, ctypes.POINTER(c_double)]),
    "gsstv_slabs_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_int, c_int, c_int,
                                   ctypes.POINTER(GsstvParams), c_void_p]),
    "gsstv_slabs_destroy": (c_int, [c_void_p]),
    "gsstv_slabs_load_observation": (c_int, [c_void_p, c_void_p]),
    "gsstv_slabs_reset_state": (c_int, [c_void_p]),
    "gsstv_slabs_iterate": (c_int, [c_void_p, c_int, ctypes.POINTER(c_int)]),
    "gsstv_slabs_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_int)]),
    "gsstv_slabs_get_state": (c_int, [c_void_p, ctypes.POINTER(GsstvStateView)]),
    "gsstv_slabs_set_state": (c_int, [c_void_p, ctypes.POINTER(GsstvStateView)]),
    "gsstv_slabs_get_stats": (c_int, [c_void_p, ctypes.POINTER(GsstvStats)]),
    "gsstv_slabs_count": (c_int, [c_void_p, ctypes.POINTER(c_int)]),
    "gsstv_strerror": (ctypes.c_char_p, [c_int]),
}

# largest n accepted by gsstv_project_l1ball_noalloc (include/gsstv.h)
GSSTV_NOALLOC_MAX_N = 262144

EXPORTED = tuple(_SIGS)


class GsstvError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


def load(path: str | None = None) -> ctypes.CDLL:
    """Loads libgsstv.so (once) and declares the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libgsstv.so not found at {p}; build it with "
                           "`python -m paper_2510_00562_gb300.build`")
    lib = ctypes.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().gsstv_strerror(code).decode()


def _check(code, where):
    if code != GSSTV_OK:
        raise GsstvError(code, where)


# ---- entry points under their C names ------------------------------------
def gsstv_default_params() -> GsstvParams:
    p = GsstvParams()
    load().gsstv_default_params(ctypes.byref(p))
    return p


def gsstv_create(n1: int, n2: int, n3: int, params: GsstvParams, stream: int | None = None):
    h = c_void_p()
    _check(load().gsstv_create(ctypes.byref(h), n1, n2, n3, ctypes.byref(params), stream or None),
           "gsstv_create")
    return h


def gsstv_set_params(h, params: GsstvParams):
    _check(load().gsstv_set_params(h, ctypes.byref(params)), "gsstv_set_params")


def gsstv_destroy(h):
    _check(load().gsstv_destroy(h), "gsstv_destroy")


def gsstv_load_observation(h, d_v: int):
    _check(load().gsstv_load_observation(h, d_v), "gsstv_load_observation")


def gsstv_reset_state(h):
    _check(load().gsstv_reset_state(h), "gsstv_reset_state")


def gsstv_iterate(h, n: int) -> int:
    done = c_int(0)
    _check(load().gsstv_iterate(h, n, ctypes.byref(done)), "gsstv_iterate")
    return done.value


def gsstv_solve(h, d_v: int, d_u: int, d_s: int | None = None, d_t: int | None = None) -> int:
    done = c_int(0)
    _check(load().gsstv_solve(h, d_v, d_u, d_s, d_t, ctypes.byref(done)), "gsstv_solve")
    return done.value


def gsstv_solve_host(h, h_v: int, h_u: int, h_s: int | None = None, h_t: int | None = None) -> int:
    done = c_int(0)
    _check(load().gsstv_solve_host(h, h_v, h_u, h_s, h_t, ctypes.byref(done)), "gsstv_solve_host")
    return done.value


def _view(ptrs: dict) -> GsstvStateView:
    return GsstvStateView(**{k: ptrs[k] for k in ("u", "s", "t", "w1", "w2", "y1", "y2", "y3", "y4")})


def gsstv_get_state(h, ptrs: dict):
    v = _view(ptrs)
    _check(load().gsstv_get_state(h, ctypes.byref(v)), "gsstv_get_state")


def gsstv_set_state(h, ptrs: dict):
    v = _view(ptrs)
    _check(load().gsstv_set_state(h, ctypes.byref(v)), "gsstv_set_state")


def gsstv_get_stats(h) -> GsstvStats:
    s = GsstvStats()
    _check(load().gsstv_get_stats(h, ctypes.byref(s)), "gsstv_get_stats")
    return s


def gsstv_reset_stats(h):
    _check(load().gsstv_reset_stats(h), "gsstv_reset_stats")


def gsstv_set_timing(h, on: bool):
    _check(load().gsstv_set_timing(h, 1 if on else 0), "gsstv_set_timing")


def gsstv_autotune(h, passes: int = 20) -> int:
    """Times the fused stencil kernel for a few band-run lengths and keeps the
    fastest; returns the bands per CTA chosen (0: nothing to tune)."""
    chunk = c_int(0)
    _check(load().gsstv_autotune(h, passes, ctypes.byref(chunk)), "gsstv_autotune")
    return chunk.value


def gsstv_device_bytes(h) -> int:
    return int(load().gsstv_device_bytes(h))


def gsstv_project_l1ball(d_x: int, n: int, radius: float, d_out: int, stream: int | None = None) -> float:
    tau = c_double(0.0)
    _check(load().gsstv_project_l1ball(d_x, n, radius, d_out, ctypes.byref(tau), stream or None),
           "gsstv_project_l1ball")
    return tau.value


def gsstv_project_l1ball_noalloc(d_x: int, n: int, radius: float, d_out: int,
                                 stream: int | None = None) -> float:
    """Same as gsstv_project_l1ball, for callers that may not allocate device
    memory: the scratch is a static device array, n <= GSSTV_NOALLOC_MAX_N, and
    calls whose GPU work overlaps race on that array."""
    tau = c_double(0.0)
    _check(load().gsstv_project_l1ball_noalloc(d_x, n, radius, d_out, ctypes.byref(tau), stream or None),
           "gsstv_project_l1ball_noalloc")
    return tau.value


def gsstv_batch_create(shapes, params, stream: int | None = None):
    """shapes: list of (n1, n2, n3); params: list of GsstvParams (same length)."""
    n = len(shapes)
    arr = lambda k: (c_int * n)(*[int(sh[k]) for sh in shapes])
    ps = (GsstvParams * n)(*params)
    b = c_void_p()
    _check(load().gsstv_batch_create(ctypes.byref(b), n, arr(0), arr(1), arr(2), ps, stream or None),
           "gsstv_batch_create")
    return b


def gsstv_batch_solve(b, d_v, d_u, d_s=None, d_t=None) -> list:
    """d_v, d_u, d_s, d_t: lists of device addresses (d_s, d_t may be None)."""
    n = len(d_v)
    vec = lambda xs: (c_void_p * n)(*xs) if xs is not None else None
    done = (c_int * n)()
    _check(load().gsstv_batch_solve(b, vec(d_v), vec(d_u), vec(d_s), vec(d_t), done), "gsstv_batch_solve")
    return list(done)


def gsstv_batch_size(b) -> int:
    return int(load().gsstv_batch_size(b))


def gsstv_batch_handle(b, c: int):
    h = c_void_p()
    _check(load().gsstv_batch_handle(b, c, ctypes.byref(h)), "gsstv_batch_handle")
    return h


def gsstv_batch_destroy(b):
    _check(load().gsstv_batch_destroy(b), "gsstv_batch_destroy")


def gsstv_vjp_step(h, x: dict, x_next: dict, bar_next: dict, bar: dict, d_vbar: int, pbar=None,
                   want_params: bool = True):
    """One pass transposed; x, x_next, bar_next, bar: dicts of device
    addresses.  Adds to d_vbar and to pbar (4 floats, returned as a list);
    want_params=False passes NULL (no parameter adjoints, no synchronisation)
    and returns None."""
    acc = (c_double * 4)(*(pbar or [0.0] * 4)) if want_params else None
    vs = [_view(d) for d in (x, x_next, bar_next, bar)]
    _check(load().gsstv_vjp_step(h, *[ctypes.byref(v) for v in vs], d_vbar, acc), "gsstv_vjp_step")
    return list(acc) if want_params else None


def gsstv_unrolled_vjp(h, iters: int, ckpt_every: int, d_ubar: int, d_vbar: int) -> list:
    """Adjoint of `iters` passes from the standard start; returns the adjoints
    of (eps, alpha, beta, omega)."""
    acc = (c_double * 4)()
    _check(load().gsstv_unrolled_vjp(h, iters, ckpt_every, d_ubar, d_vbar, acc), "gsstv_unrolled_vjp")
    return list(acc)


def gsstv_strerror(code: int) -> str:
    return strerror(code)


# ---- one cube split into band slabs -----------------------------------------
def gsstv_slabs_create(n1: int, n2: int, n3: int, nslabs: int, params: GsstvParams, stream: int | None = None):
    h = c_void_p()
    _check(load().gsstv_slabs_create(ctypes.byref(h), n1, n2, n3, nslabs, ctypes.byref(params), stream or None),
           "gsstv_slabs_create")
    return h


def gsstv_slabs_destroy(h):
    _check(load().gsstv_slabs_destroy(h), "gsstv_slabs_destroy")


def gsstv_slabs_load_observation(h, d_v: int):
    _check(load().gsstv_slabs_load_observation(h, d_v), "gsstv_slabs_load_observation")


def gsstv_slabs_reset_state(h):
    _check(load().gsstv_slabs_reset_state(h), "gsstv_slabs_reset_state")


def gsstv_slabs_iterate(h, n: int) -> int:
    done = c_int(0)
    _check(load().gsstv_slabs_iterate(h, n, ctypes.byref(done)), "gsstv_slabs_iterate")
    return done.value


def gsstv_slabs_solve(h, d_v: int, d_u: int, d_s: int | None = None, d_t: int | None = None) -> int:
    done = c_int(0)
    _check(load().gsstv_slabs_solve(h, d_v, d_u, d_s, d_t, ctypes.byref(done)), "gsstv_slabs_solve")
    return done.value


def gsstv_slabs_get_state(h, ptrs: dict):
    v = _view(ptrs)
    _check(load().gsstv_slabs_get_state(h, ctypes.byref(v)), "gsstv_slabs_get_state")


def gsstv_slabs_set_state(h, ptrs: dict):
    v = _view(ptrs)
    _check(load().gsstv_slabs_set_state(h, ctypes.byref(v)), "gsstv_slabs_set_state")


def gsstv_slabs_get_stats(h) -> GsstvStats:
    s = GsstvStats()
    _check(load().gsstv_slabs_get_stats(h, ctypes.byref(s)), "gsstv_slabs_get_stats")
    return s


def gsstv_slabs_count(h) -> list:
    n = load().gsstv_slabs_count(h, None)
    arr = (c_int * max(n, 1))()
    load().gsstv_slabs_count(h, arr)
    return list(arr[:n])
