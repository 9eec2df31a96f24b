"""The C-ABI library builds, loads and exports what include/gsstv.h declares
(no GPU needed: only calls that never reach the device)."""
import ctypes
import json
import os
import re

import pytest

from paper_2510_00562_gb300 import binding as B
from paper_2510_00562_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gsstv.h")
GOLDEN = os.path.join(ROOT, "tests", "golden", "paper_constants.json")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return B.load()


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gsstv_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    # the binding covers the same set, under the same names
    assert sorted(B.EXPORTED) == names


def test_strerror_and_defaults(lib):
    assert B.strerror(0) == "ok"
    assert "non-finite" in B.strerror(B.GSSTV_ERR_NONFINITE)
    assert B.strerror(12345) == "unknown error code"
    g = json.load(open(GOLDEN))
    p = B.gsstv_default_params()
    for k, (num, den) in g["step_sizes"].items():
        assert getattr(p, k) == pytest.approx(num / den, rel=1e-15), k
    assert p.mu_lo == 0.0 and p.mu_hi == 1.0 and p.storage == B.GSSTV_FP32


@pytest.mark.parametrize("bad", [
    dict(shape=(0, 4, 4)), dict(shape=(4, -1, 4)), dict(shape=(4, 4, 0)),
    dict(eps=-1.0), dict(alpha=float("nan")), dict(beta=-0.1), dict(omega=-1.0),
    dict(mu_lo=1.0, mu_hi=1.0), dict(gamma_u=0.0), dict(gamma_y4=-0.2), dict(gamma_t=float("inf")),
    dict(max_iter=-1), dict(check_every=0), dict(storage=7), dict(tau_mode=3), dict(tol=-1.0),
])
def test_create_rejects_bad_arguments_before_touching_the_device(lib, bad):
    p = B.gsstv_default_params()
    shape = bad.pop("shape", (4, 4, 4))
    for k, v in bad.items():
        setattr(p, k, v)
    h = ctypes.c_void_p()
    rc = lib.gsstv_create(ctypes.byref(h), shape[0], shape[1], shape[2], ctypes.byref(p), None)
    assert rc == B.GSSTV_ERR_ARG
    assert not h.value


def test_null_arguments(lib):
    assert lib.gsstv_create(None, 4, 4, 4, None, None) == B.GSSTV_ERR_ARG
    assert lib.gsstv_destroy(None) == B.GSSTV_OK
    assert lib.gsstv_iterate(None, 1, None) == B.GSSTV_ERR_ARG
    assert lib.gsstv_project_l1ball(None, 4, 1.0, None, None, None) == B.GSSTV_ERR_ARG
    assert lib.gsstv_device_bytes(None) == 0
    acc = (ctypes.c_double * 4)()
    assert lib.gsstv_vjp_step(None, None, None, None, None, None, acc) == B.GSSTV_ERR_ARG
    assert lib.gsstv_unrolled_vjp(None, 1, 0, None, None, acc) == B.GSSTV_ERR_ARG
    assert lib.gsstv_autotune(None, 1, None) == B.GSSTV_ERR_ARG


def test_batch_rejects_bad_arguments_before_touching_the_device(lib):
    """The batch entry points check every cube's shape and parameters first
    (no CUDA call is made, so this runs without a GPU)."""
    p = B.gsstv_default_params()
    b = ctypes.c_void_p()
    n = (ctypes.c_int * 2)(4, 4)
    ps = (B.GsstvParams * 2)(p, p)
    assert lib.gsstv_batch_create(None, 2, n, n, n, ps, None) == B.GSSTV_ERR_ARG
    assert lib.gsstv_batch_create(ctypes.byref(b), 0, n, n, n, ps, None) == B.GSSTV_ERR_ARG
    assert lib.gsstv_batch_create(ctypes.byref(b), 2, None, n, n, ps, None) == B.GSSTV_ERR_ARG
    bad_shape = (ctypes.c_int * 2)(4, 0)
    assert lib.gsstv_batch_create(ctypes.byref(b), 2, n, bad_shape, n, ps, None) == B.GSSTV_ERR_ARG
    huge = (ctypes.c_int * 2)(4, 1 << 14)
    sides = (ctypes.c_int * 2)(4, 1 << 20)
    assert lib.gsstv_batch_create(ctypes.byref(b), 2, sides, huge, n, ps, None) == B.GSSTV_ERR_ARG
    q = B.gsstv_default_params()
    q.eps = -1.0
    bad_params = (B.GsstvParams * 2)(p, q)
    assert lib.gsstv_batch_create(ctypes.byref(b), 2, n, n, n, bad_params, None) == B.GSSTV_ERR_ARG
    assert not b.value
    assert lib.gsstv_batch_solve(None, None, None, None, None, None) == B.GSSTV_ERR_ARG
    assert lib.gsstv_batch_destroy(None) == B.GSSTV_OK
    assert lib.gsstv_batch_size(None) == 0
    assert lib.gsstv_batch_handle(None, 0, ctypes.byref(b)) == B.GSSTV_ERR_ARG


def test_noalloc_limit_in_binding_matches_header():
    # the binding checks sizes against its own copy of GSSTV_NOALLOC_MAX_N;
    # it must be the header's value
    src = open(HEADER).read()
    m = re.search(r"#define\s+GSSTV_NOALLOC_MAX_N\s+(\d+)", src)
    assert m is not None
    assert int(m.group(1)) == B.GSSTV_NOALLOC_MAX_N
