"""The allocation-free l1-ball projection against the allocating one and the
FP64 oracle.

gsstv_project_l1ball_noalloc serves callers that must not allocate device
memory (their memory belongs to another allocator, or cudaFree's device-wide
synchronisation is not acceptable where they run): it keeps its scratch in a
static device array.  It must give the same projection as
gsstv_project_l1ball and as the oracle's sort-based projection (Sec. III-B),
call after call, since every call reuses (and must first clear) that shared
array.  The largest accepted size is run with every value equal and with
values a few ulps apart, so that the radix search's bracket holds the whole
input.  This file is collected last, so a failure here comes after every
other test has run; it also passes on its own in a fresh process, where its
first call is the one that sets the array up.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import ppds as o
from paper_2510_00562_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def _both(x, r):
    d = _dev(x)
    out_ref = torch.empty_like(d)
    out_na = torch.empty_like(d)
    st = torch.cuda.current_stream().cuda_stream
    tau_ref = B.gsstv_project_l1ball(d.data_ptr(), d.numel(), r, out_ref.data_ptr(), st)
    tau_na = B.gsstv_project_l1ball_noalloc(d.data_ptr(), d.numel(), r, out_na.data_ptr(), st)
    return tau_ref, out_ref.cpu().numpy(), tau_na, out_na.cpu().numpy()


def _check(x, r):
    tau_ref, out_ref, tau_na, out_na = _both(x, r)
    # the tolerances of the l1-projection parity tests, against the allocating
    # projection and against the oracle
    scale = 1e-6 * max(1.0, float(np.abs(x).max()))
    assert tau_na == pytest.approx(tau_ref, rel=1e-6, abs=1e-12)
    assert np.abs(out_na - out_ref).max() <= scale
    ref, tau_o = o.proj_l1ball(x.astype(np.float64), r)
    if r > 0:
        assert tau_na == pytest.approx(tau_o, rel=1e-6, abs=1e-12)
    else:
        # the ball is {0}: every tau >= max |x| is a valid threshold (the
        # oracle reports max |x|, the library +inf); the projection is unique
        assert tau_na >= float(np.abs(x).max())
    assert np.abs(out_na - ref).max() <= scale


def test_noalloc_matches_allocating_projection_two_calls_in_a_row():
    rng = np.random.default_rng(2024)
    # first call: a large vector whose radix search gathers a bracket bin
    x1 = rng.laplace(size=B.GSSTV_NOALLOC_MAX_N).astype(np.float32)
    _check(x1, 0.3 * float(np.abs(x1.astype(np.float64)).sum()))
    # second call right after: different size, values and radius; nothing of
    # the first call may leak through the shared scratch
    x2 = (rng.standard_normal(77_777) * 3.0).astype(np.float32)
    _check(x2, 0.05 * float(np.abs(x2.astype(np.float64)).sum()))
    # and the degenerate cases: inside the ball, radius 0
    x3 = rng.uniform(-1, 1, size=1000).astype(np.float32)
    _check(x3, 10.0 * float(np.abs(x3.astype(np.float64)).sum()))
    _check(x3, 0.0)


def test_noalloc_bracket_holding_the_whole_input():
    # n = the maximum, every |x| equal to a = 0.8f, which lies strictly inside
    # its radix bins (0.8f = 0x3f4ccccd): with r = 0.01 n the level-0 bracket
    # holds the whole input, with r = 1e-6 n the level-1 bracket does too; the
    # exact threshold is a - r / n
    n = B.GSSTV_NOALLOC_MAX_N
    sign = np.where(np.random.default_rng(5).random(n) < 0.5, -1.0, 1.0)
    a = float(np.float32(0.8))
    x = (a * sign).astype(np.float32)
    for r in (0.01 * n, 1e-6 * n):
        _check(x, r)
        _, _, tau_na, _ = _both(x, r)
        assert tau_na == pytest.approx(a - r / n, rel=1e-12)
    # values a few ulps apart: the bracket narrows through every level
    k = np.random.default_rng(6).integers(0, 6, size=n)
    y = (sign * a * (1.0 + k * 2.0**-23)).astype(np.float32)
    for frac in (0.01, 1e-6):
        _check(y, frac * n)


def test_noalloc_rejects_sizes_beyond_its_maximum():
    lib = B.load()
    n = B.GSSTV_NOALLOC_MAX_N + 1
    d = torch.zeros(n, dtype=torch.float32, device="cuda")
    tau = ctypes.c_double(0.0)
    rc = lib.gsstv_project_l1ball_noalloc(d.data_ptr(), n, 1.0, d.data_ptr(), ctypes.byref(tau), None)
    assert rc == B.GSSTV_ERR_ARG
