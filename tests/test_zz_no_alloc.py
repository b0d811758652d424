"""The allocation-free ||A||_2 entry point (feast_norm2_estimate_static).

It exists for callers that may not call cudaMalloc, for example code running
while a host framework owns all device memory and hands out only its own
buffers.  It runs the power iteration of feast_create with its scratch in a
fixed device array of the library.  This file is collected last, so a run that
stops at the first failure has run every other test before it.  The test
calls the entry point twice in a row, on two different matrices, and compares
each result with the value the handle path (feast_create, whose scratch the
handle allocates) reports for the same matrix, at the FP64 tolerance of the
other parity tests (1e-12 relative)."""
import ctypes

import numpy as np
import pytest

import workloads
from helpers import lib

pytestmark = pytest.mark.gpu


def _device_colmajor(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a.T)).to("cuda").mT


def test_static_scratch_norm_matches_handle_path_twice():
    torch = pytest.importorskip("torch")
    fg = lib()
    mats = []
    for n, seed in ((700, 31), (129, 32)):
        rng = np.random.default_rng(seed)
        mats.append(workloads.cgauss(rng, n, n) + np.diag(np.linspace(0.5, 2.5, n)))
    refs = []
    for A in mats:
        h = fg.feast_create(A, None, fg.make_contour(), 1, fg.make_options())
        refs.append(fg.feast_get_stats(h)["normA"])
        fg.feast_destroy(h)
    for A, ref in zip(mats, refs):  # two calls in a row share the fixed scratch
        got = fg.feast_norm2_estimate_static(_device_colmajor(torch, A), iters=50)
        assert abs(got - ref) <= 1e-12 * ref, (got, ref)


def test_static_scratch_rejects_oversize_and_host_memory():
    torch = pytest.importorskip("torch")
    fg = lib()
    so = fg.load()
    small = _device_colmajor(torch, np.eye(4, dtype=np.complex128))
    out = ctypes.c_double()
    s = so.feast_norm2_estimate_static(small.data_ptr(), 16385, 16385, 50, ctypes.byref(out), None)
    assert s == fg.FEAST_ERR_TOO_LARGE
    host = np.asfortranarray(np.eye(4, dtype=np.complex128))
    s = so.feast_norm2_estimate_static(host.ctypes.data, 4, 4, 50, ctypes.byref(out), None)
    assert s == fg.FEAST_ERR_ARG
