"""The allocation-free l1-ball projection against the allocating one.

gsstv_project_l1ball_noalloc serves callers that must not allocate device
memory (their memory belongs to another allocator, or cudaFree's device-wide
synchronisation is not acceptable where they run): it keeps its scratch in a
static device array.  It must give the same projection as
gsstv_project_l1ball, call after call, since every call reuses (and must
first clear) that shared array.  This file is collected last, so a failure
here comes after every other test has run; it also passes on its own in a
fresh process, where its first call is the one that sets the array up.
"""
import ctypes

import numpy as np
import pytest
import torch

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
    # the tolerances of the l1-projection parity tests
    assert tau_na == pytest.approx(tau_ref, rel=1e-6, abs=1e-12)
    assert np.abs(out_na - out_ref).max() <= 1e-6 * max(1.0, float(np.abs(x).max()))


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


def test_noalloc_rejects_sizes_beyond_its_maximum():
    lib = B.load()
    n = B.GSSTV_NOALLOC_MAX_N + 1
    d = torch.zeros(n, dtype=torch.float32, device="cuda")
    tau = ctypes.c_double(0.0)
    rc = lib.gsstv_project_l1ball_noalloc(d.data_ptr(), n, 1.0, d.data_ptr(), ctypes.byref(tau), None)
    assert rc == B.GSSTV_ERR_ARG
