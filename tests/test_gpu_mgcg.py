"""MG-preconditioned CG on the normal equations (the paper's own experiment) on the GPU against the
oracle: the 9-point Galerkin operators of the adaptive hierarchy, the MG-CG and plain CG solves
(iteration counts and solutions), and the paper's cost measure of 6 fine D^dagger D applications
per MG-CG iteration."""
import numpy as np
import pytest

import inputs
from oracle import normal, wilson
from oracle.lattice import Lattice
from tests._util import rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu


def _params(levels, Nv=8, n_pass=1, nu_setup=4, seed=20070704):
    import paper_0707_4018_gb300 as mg
    return mg.mg_default_params(levels=levels, blocks=[(4, 4)] * (levels - 1), Nv=[Nv] * (levels - 1),
                                n_pass=n_pass, nu_setup=nu_setup, seed=seed)


def test_coarse_operators_match_oracle():
    import paper_0707_4018_gb300 as mg
    L = 48
    U, _, _ = inputs.schwinger_links(L, 6.0, sweeps=200, workload_id=5)
    m = 0.1
    ctx = mg.CgContext.setup(to_dev(U), m, (L, L), _params(3, n_pass=2))
    h = normal.adaptive_setup(U, m, Lattice((L, L)), [(4, 4), (4, 4)], [8, 8], n_pass=2, nu_setup=4)
    for level, side in ((1, 12), (2, 3)):
        got = to_host(ctx.coarse_op(level, side * side, 8))
        assert rel_err(got, h.ops[level].Y) < 1e-10, level
    ctx.close()


@pytest.mark.parametrize("precondition", [True, False])
def test_solves_match_oracle(precondition):
    import torch
    import paper_0707_4018_gb300 as mg
    L = 48
    U, _, _ = inputs.schwinger_links(L, 6.0, sweeps=200, workload_id=5)
    m = 0.1
    lat = Lattice((L, L))
    ctx = mg.CgContext.setup(to_dev(U), m, (L, L), _params(3, n_pass=2))
    chi = np.zeros((L * L, 2), dtype=np.complex128)
    chi[0, 0] = 1.0  # point source, as in the paper
    psi = torch.empty((L * L, 2), dtype=torch.complex128, device="cuda")
    st = ctx.solve(to_dev(chi), psi, 1e-12, precondition=precondition)
    if precondition:
        h = normal.adaptive_setup(U, m, lat, [(4, 4), (4, 4)], [8, 8], n_pass=2, nu_setup=4)
        want, info = normal.mgcg_solve(h, chi, 1e-12)
        # the paper's cost: 1 A in CG and 5 in the V-cycle per iteration (and 5 for the first V-cycle)
        assert st["fine_apps"] == 6 * st["iters"] + 5
    else:
        op = normal.NormalOperator(U, m, lat)
        want, info = normal.cg(op.apply, wilson.apply_Ddag(U, chi, m, lat), 1e-12, 100000)
        assert st["fine_apps"] == st["iters"]
    assert st["converged"] and st["rel_residual"] <= 2e-12
    assert abs(st["iters"] - info["iters"]) <= (1 if precondition else 3), (st["iters"], info["iters"])
    got = to_host(psi)
    assert rel_err(got, want) < 1e-8
    res = np.linalg.norm(chi - wilson.apply_D(U, got, m, lat)) / np.linalg.norm(chi)
    assert res < 1e-9
    ctx.close()


def test_rejects_coarse_extents_below_three():
    import paper_0707_4018_gb300 as mg
    U = inputs.hot_links(32, 32, seed=2)
    with pytest.raises(mg.MGError) as e:
        mg.CgContext.setup(to_dev(U), 0.1, (32, 32), _params(3))  # 32 -> 8 -> 2
    assert e.value.code == 1
