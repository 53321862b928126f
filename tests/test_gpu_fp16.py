"""MG_FP16 contexts: FP32 V-cycles whose fine level keeps the links and the MR smoother's vectors
r and A r in half precision with per-site FP32 norms, inside the FP64 flexible GCR (the mixed-
precision scheme with FP16 storage). The cycle is checked against the oracle's FP64 V-cycle on the
same hierarchy (its error is that of half storage: well above the FP32 cycle's, well below what the
outer loop tolerates), and the solves against the oracle's FP64 true residual."""
import os

import numpy as np
import pytest

import inputs
from oracle import solvers, wilson
from oracle.lattice import Lattice
from tests._util import rel_err, to_dev, to_host
from tests.test_gpu_mg import make_pair

pytestmark = pytest.mark.gpu


def test_fp16_vcycle_error_is_that_of_half_storage():
    import torch
    dims = (64, 64)
    U, _, _ = inputs.schwinger_links(64, 6.0, sweeps=200, workload_id=5)
    lat = Lattice(dims)
    b = inputs.gaussian_source(*dims, seed=21)
    errs = {}
    for prec in (1, 2):
        hier, ctx, _ = make_pair(dims, 0.05, [(4, 4), (2, 2)], [8, 8], U, precision=prec, coarsest_lu_max=4096,
                                 coarsest_tol=1e-13)
        x = torch.empty((lat.volume, 2), dtype=torch.complex128, device="cuda")
        ctx.vcycle(to_dev(b), x)
        errs[prec] = rel_err(to_host(x), solvers.vcycle(hier, 0, b))
        ctx.close()
    # FP32 cycle: ~1e-6; half storage (11-bit significands, per-site scaling): ~1e-3
    assert errs[1] < 1e-5, errs
    assert 20 * errs[1] < errs[2] < 1e-2, errs


def test_fp16_solve_reaches_true_residual_with_fp32_iteration_counts():
    import torch
    import paper_0707_4018_gb300 as mg
    L = 128
    U, _, _ = inputs.schwinger_links(L, 6.0, sweeps=500, workload_id=5)
    lat = Lattice((L, L))
    chi = inputs.gaussian_source(L, L, seed=31)
    its = {}
    for prec in (mg.MG_FP32, mg.MG_FP16):
        p = mg.mg_default_params(levels=3, blocks=[(4, 4), (2, 2)], Nv=[8, 8], precision=prec, coarsest_tol=0.2,
                                 coarsest_lu_max=0)
        ctx = mg.Context.setup(to_dev(U), 0.02, (L, L), p)
        assert ctx.info()["precision"] == prec
        psi = torch.empty((L * L, 2), dtype=torch.complex128, device="cuda")
        st = ctx.solve(to_dev(chi), psi, 1e-10)
        res = np.linalg.norm(chi - wilson.apply_D(U, to_host(psi), 0.02, lat)) / np.linalg.norm(chi)
        assert st["converged"] and res <= 1.05e-10, (prec, st, res)
        its[prec] = st["iters"]
        ctx.close()
    assert its[mg.MG_FP16] <= its[mg.MG_FP32] + max(3, its[mg.MG_FP32] // 4), its


def test_fp16_batched_multi_clone_and_saved_setup(tmp_path):
    # the half-storage cycles in lockstep batches (host-driven and device-driven), in a clone and in
    # a context reloaded from a saved setup; the precision survives clone, save and load
    import torch
    import paper_0707_4018_gb300 as mg
    L = 64
    dims = (L, L)
    U, _, _ = inputs.schwinger_links(L, 6.0, sweeps=200, workload_id=5)
    lat = Lattice(dims)
    p = mg.mg_default_params(levels=3, blocks=[(4, 4), (2, 2)], Nv=[8, 8], precision=mg.MG_FP16, coarsest_tol=0.2,
                             coarsest_lu_max=0, max_rhs=8)
    ctx = mg.Context.setup(to_dev(U), 0.03, dims, p)
    chi = torch.stack([to_dev(inputs.gaussian_source(L, L, seed=50 + v)) for v in range(8)])

    def check(psi, m, stats):
        for v in range(psi.shape[0]):
            b = to_host(chi[v])
            res = np.linalg.norm(b - wilson.apply_D(U, to_host(psi[v]), m, lat)) / np.linalg.norm(b)
            assert stats[v]["converged"] and res <= 1.05e-10, (v, stats[v], res)

    psi = torch.empty_like(chi)
    check(psi, 0.03, ctx.solve_batch(chi, psi, 1e-10))
    psi2 = torch.empty_like(chi)
    check(psi2, 0.03, mg.solve_multi([ctx], [chi], [psi2], 1e-10, nrhs=[8]))
    other = ctx.clone(0.06)
    assert other.info()["precision"] == mg.MG_FP16
    psi3 = torch.empty_like(chi[:1])
    check(psi3, 0.06, [other.solve(chi[0], psi3[0], 1e-10)])
    path = os.path.join(str(tmp_path), "fp16.mgs")
    ctx.save(path)
    back = mg.Context.load(path, to_dev(U), dims)
    assert back.info()["precision"] == mg.MG_FP16
    psi4 = torch.empty_like(chi[:1])
    psi5 = torch.empty_like(chi[:1])
    s4 = back.solve(chi[0], psi4[0], 1e-10)
    s5 = ctx.solve(chi[0], psi5[0], 1e-10)
    assert s4["iters"] == s5["iters"] and torch.equal(psi4, psi5)
    for c in (ctx, other, back):
        c.close()
