"""Failure detection on the GPU without a fault: bounded waits, NaN inputs, breakdown.

The persistent kernels wait at grid barriers with a bounded number of polls. A
test makes such a wait run out (a barrier whose last arrival never comes) and
checks that the kernel returned, the status says so, and the GPU context keeps
working. Bad inputs (NaN) must be reported as MG_ERR_NAN, not hang or fault.
"""
import numpy as np
import pytest

import inputs
from tests._util import to_dev, to_host

pytestmark = pytest.mark.gpu


def test_bounded_barrier_reports_timeout_and_context_survives():
    import torch
    import paper_0707_4018_gb300 as mg
    mg.mg_selftest_barrier(0)  # complete barrier: no error
    with pytest.raises(mg.MGError) as e:
        mg.mg_selftest_barrier(1)  # one arrival missing: the wait gives up
    assert e.value.code == 8
    # the context is still usable afterwards
    U = to_dev(inputs.hot_links(16, 16, seed=1))
    psi = to_dev(inputs.gaussian_source(16, 16, seed=2))
    out = torch.empty_like(psi)
    mg.mg_dslash(U, psi, out, 0.1, (16, 16))
    torch.cuda.synchronize()
    assert np.all(np.isfinite(to_host(out)))


def test_nan_source_is_reported():
    import torch
    import paper_0707_4018_gb300 as mg
    L = 16
    U = to_dev(inputs.hot_links(L, L, seed=1))
    ctx = mg.Context.setup(U, 0.2, (L, L), mg.mg_default_params(n_pass=1))
    chi = inputs.gaussian_source(L, L, seed=3)
    chi[5, 0] = np.nan
    psi = torch.empty((L * L, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(mg.MGError) as e:
        ctx.solve(to_dev(chi), psi, 1e-10)
    assert e.value.code == 5
    # a good source still solves on the same context
    st = ctx.solve(to_dev(inputs.gaussian_source(L, L, seed=4)), psi, 1e-10)
    assert st["converged"]


def test_nan_links_are_reported_by_setup():
    import paper_0707_4018_gb300 as mg
    L = 16
    U = inputs.hot_links(L, L, seed=1)
    U[7, 1] = np.nan
    with pytest.raises(mg.MGError) as e:
        mg.Context.setup(to_dev(U), 0.2, (L, L), mg.mg_default_params(n_pass=2))
    assert e.value.code in (5,)


def test_4d_nan_source_and_links_are_reported():
    import torch
    import paper_0707_4018_gb300 as mg
    dims = (4, 4, 4, 4)
    V = 256
    U = inputs.su3_links(dims, seed=2)
    p = mg.mg_default_params(levels=2, blocks=[(2, 2, 2, 2)], Nv=[4], chiral_split=1, n_pass=1)
    ctx = mg.Context.setup(to_dev(U), 0.1, dims, p)
    chi = inputs.gaussian_spinor(V, 12, 3, 0)
    chi[9, 4] = np.nan
    psi = torch.empty((V, 12), dtype=torch.complex128, device="cuda")
    with pytest.raises(mg.MGError) as e:
        ctx.solve(to_dev(chi), psi, 1e-10)
    assert e.value.code == 5
    assert ctx.solve(to_dev(inputs.gaussian_spinor(V, 12, 3, 1)), psi, 1e-10)["converged"]
    ctx.close()
    Ubad = U.copy()
    Ubad[17, 2, 1, 1] = np.nan
    with pytest.raises(mg.MGError) as e:
        mg.Context.setup(to_dev(Ubad), 0.1, dims, p)
    assert e.value.code == 5
