"""Near-critical solves at the largest 2d size: the 1024^2 beta = 6 thermal field of the mass sweep
(2000 Metropolis sweeps from the GPU twin of the generator, checked by its stored digest), at
m = m_c + 0.005 with m_c from the 256^2 calibration. This is where the condition number is largest
(the paper's mass-gap scans approach m_c), and at 1M sites the oracle cannot solve the system; the
property that holds at any size is checked instead: the solution's true residual, recomputed by the
oracle's FP64 Wilson operator, meets the tolerance, for the mixed-precision and the all-FP64
solver, and the solver's own closing residual is that same number."""
import numpy as np
import pytest

import inputs
from oracle import wilson
from oracle.lattice import Lattice
from tests._util import mcrit_table, to_dev, to_host

pytestmark = pytest.mark.gpu


def test_1024_beta6_near_critical_true_residual():
    import torch
    import paper_0707_4018_gb300 as mg
    row = mcrit_table()["w1_L1024_b6"]
    L = row["L"]
    th, acc = inputs.metropolis_u1_2d_gpu(L, L, [row["beta"]], [row["seed"]], row["sweeps"])
    assert inputs.field_digest(th[0]) == row["theta_digest"] and abs(acc[0] - row["acceptance"]) < 1e-15
    U = inputs.links_from_angles(th[0])
    m = row["m_crit"] + 0.005
    chi = inputs.gaussian_source(L, L, seed=row["seed"], index=0)
    lat = Lattice((L, L))
    for prec in (mg.MG_FP32, mg.MG_FP64):
        p = mg.mg_default_params(levels=3, blocks=[(4, 4), (2, 2)], Nv=[8, 8], precision=prec,
                                 coarsest_tol=0.2, coarsest_restart=16, max_iter=3000)
        ctx = mg.Context.setup(to_dev(U), m, (L, L), p)
        psi = torch.empty((L * L, 2), dtype=torch.complex128, device="cuda")
        st = ctx.solve(to_dev(chi), psi, 1e-10)
        x = to_host(psi)
        res = np.linalg.norm(chi - wilson.apply_D(U, x, m, lat)) / np.linalg.norm(chi)
        assert st["converged"] and res <= 1.05e-10, (prec, st, res)
        assert abs(res - st["true_rel_residual"]) <= 1e-12, (res, st["true_rel_residual"])
        ctx.close()
