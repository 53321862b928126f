"""The no-allocation fine smoother (mg_smooth_fine_noalloc) against the context smoother.

Callers that cannot allocate device memory when they smooth (inside a stream
capture, or under a framework that owns the whole memory pool) use
mg_smooth_fine_noalloc, whose scratch is a fixed device array. Its result must
equal mg_smooth at level 0 of a set-up context (same U, m, b, nu, omega) on
two calls in a row: the second call reuses the array the first one left behind.
"""
import ctypes

import numpy as np
import pytest

import inputs
from tests._util import rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu


def test_no_alloc_smoother_matches_context_smoother_twice():
    import torch
    import paper_0707_4018_gb300 as mg
    dims, m, nu = (64, 64), 0.03, 4
    theta, _ = inputs.metropolis_u1_2d(64, 64, 6.0, 100, seed=inputs.workload_seed(5, 64, 6.0))
    U = to_dev(inputs.links_from_angles(theta))
    b = to_dev(inputs.gaussian_source(64, 64, seed=11))
    ctx = mg.Context.setup(U, m, dims, mg.mg_default_params(n_pass=1, nu_setup=2))
    x_ref = torch.empty_like(b)
    ctx.smooth(0, b, x_ref, nu)
    ref = to_host(x_ref)
    for _ in range(2):
        x = torch.full_like(b, float("nan"))
        mg.mg_smooth_fine_noalloc(U, b, x, m, dims, nu, omega=ctx.params.omega)
        torch.cuda.synchronize()
        got = to_host(x)
        assert np.all(np.isfinite(got))
        assert rel_err(got, ref) <= 1e-14
    ctx.close()


def test_no_alloc_smoother_rejects_lattices_beyond_its_limit():
    import paper_0707_4018_gb300 as mg
    from paper_0707_4018_gb300 import binding
    lib = binding.load()
    g = binding.make_geom((512, 256))
    code = lib.mg_smooth_fine_noalloc(ctypes.byref(g), ctypes.c_void_p(16), 0.1, ctypes.c_void_p(32),
                                      ctypes.c_void_p(64), 4, 0.8, None)
    assert code == 1
    assert b"65536" in lib.mg_last_error()
    del mg
