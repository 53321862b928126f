"""mg_clone: a context for another mass that reuses a setup must behave exactly like
mg_update_mass applied to an identical context (same Galerkin operators, same solves, bit
for bit), and leave its source untouched."""
import numpy as np
import pytest

import inputs
from oracle import wilson
from oracle.lattice import Lattice
from tests._util import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_clone_equals_update_mass(precision):
    import torch
    import paper_0707_4018_gb300 as mg
    dims = (64, 64)
    lat = Lattice(dims)
    U, _, _ = inputs.schwinger_links(64, 6.0, sweeps=100, workload_id=11)
    p = mg.mg_default_params(levels=3, blocks=[(4, 4), (2, 2)], Nv=[8, 8], precision=precision, n_pass=2,
                             coarsest_tol=0.2)
    m1, m2 = 0.05, 0.12
    a = mg.Context.setup(to_dev(U), m1, dims, p)
    b = mg.Context.setup(to_dev(U), m1, dims, p)
    c = a.clone(m2)
    b.update_mass(m2)
    for lvl in (1, 2):
        assert torch.equal(c.coarse_op(lvl), b.coarse_op(lvl))
    chi = to_dev(inputs.gaussian_source(64, 64, seed=3))
    out = [torch.empty_like(chi) for _ in range(3)]
    st_c = c.solve(chi, out[0], 1e-10)
    st_b = b.solve(chi, out[1], 1e-10)
    assert st_c["converged"] and st_c["iters"] == st_b["iters"]
    assert torch.equal(out[0], out[1])
    # the source still solves at m1
    a.solve(chi, out[2], 1e-10)
    res = np.linalg.norm(to_host(chi) - wilson.apply_D(U, to_host(out[2]), m1, lat)) / np.linalg.norm(to_host(chi))
    assert res <= 1e-10
    for ctx in (a, b, c):
        ctx.close()
