"""Batched solves (mg_solve_batch): several right-hand sides, each with its own mass,
through one hierarchy set up at the lightest mass.

Each vector's solution is compared with the exact psi_v = D(m_v)^{-1} chi_v from the
oracle's dense Wilson matrix (small lattices, |dpsi|/|psi| <= 1e-8 at a 1e-13 solve),
and every true residual is recomputed in FP64 by the oracle's D. The coarse
operators of a shifted vector are P^dagger D(m) P + (m_v - m), which equals
P^dagger D(m_v) P for the block-orthonormal P; the dense comparison checks that end
to end. Both coarsest paths are covered: dense LU per mass and the batched
persistent GCR kernel (up to four vectors per launch, per-mass block-Jacobi).
"""
import numpy as np
import pytest

import inputs
from oracle import wilson
from oracle.lattice import Lattice
from tests._util import mcrit_for, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu

DIMS = (32, 32)
BLOCKS = [(4, 4), (2, 2)]


def _mg():
    import paper_0707_4018_gb300 as mg
    return mg


def _field():
    U, _, _ = inputs.schwinger_links(32, 6.0, sweeps=300, workload_id=7)
    return U


def _sources(nrhs, seed=31):
    return np.stack([inputs.gaussian_source(*DIMS, seed=seed, index=i) for i in range(nrhs)])


def _ctx(U, m0, precision, max_rhs, **kw):
    mg = _mg()
    p = mg.mg_default_params(levels=3, blocks=BLOCKS, Nv=[8, 8], precision=precision, max_rhs=max_rhs, **kw)
    return mg.Context.setup(to_dev(U), m0, DIMS, p)


def _exact(U, m, chi):
    lat = Lattice(DIMS)
    return np.linalg.solve(wilson.dense_D(U, m, lat), chi.reshape(-1)).reshape(chi.shape)


def _true_rel(U, m, psi, chi):
    lat = Lattice(DIMS)
    return np.linalg.norm(chi - wilson.apply_D(U, psi, m, lat)) / np.linalg.norm(chi)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("lu_max", [100000, 0])
def test_batch_of_masses_matches_dense_solutions(precision, lu_max):
    import torch
    U = _field()
    m0 = 0.02
    masses = [m0, 0.05, 0.3]
    chi = _sources(3)
    ctx = _ctx(U, m0, precision, 3, coarsest_lu_max=lu_max, coarsest_tol=1e-2 if lu_max == 0 else 1e-12)
    psi = torch.empty((3, DIMS[0] * DIMS[1], 2), dtype=torch.complex128, device="cuda")
    st = ctx.solve_batch(to_dev(chi), psi, 1e-13, masses)
    out = to_host(psi)
    for v, m in enumerate(masses):
        assert st[v]["converged"], (v, st[v])
        assert _true_rel(U, m, out[v], chi[v]) <= 1e-12
        assert rel_err(out[v], _exact(U, m, chi[v])) <= 1e-8, v
    assert st[0]["graphs"]


def test_batch_matches_single_solves_per_mass():
    # the same three systems one at a time (mg_update_mass between them): same solutions,
    # and the batch needs no more outer iterations than the slowest single solve plus one
    import torch
    U = _field()
    m0 = 0.02
    masses = [m0, 0.05, 0.3]
    chi = _sources(3, seed=5)
    ctx = _ctx(U, m0, 1, 3, coarsest_lu_max=0, coarsest_tol=0.2)
    psi = torch.empty((3, DIMS[0] * DIMS[1], 2), dtype=torch.complex128, device="cuda")
    st = ctx.solve_batch(to_dev(chi), psi, 1e-10, masses)
    single = _ctx(U, m0, 1, 1, coarsest_lu_max=0, coarsest_tol=0.2)
    one = torch.empty((DIMS[0] * DIMS[1], 2), dtype=torch.complex128, device="cuda")
    its = []
    for v, m in enumerate(masses):
        if v:
            single.update_mass(m)
        s1 = single.solve(to_dev(chi[v]), one, 1e-10)
        its.append(s1["iters"])
        assert rel_err(to_host(psi)[v], to_host(one)) <= 1e-8
        assert _true_rel(U, m, to_host(psi)[v], chi[v]) <= 1e-10
        assert abs(st[v]["iters"] - s1["iters"]) <= 1, (v, st[v]["iters"], s1["iters"])


def test_batch_of_one_and_default_mass():
    import torch
    U = _field()
    chi = _sources(1, seed=9)
    ctx = _ctx(U, 0.1, 0, 1)  # max_rhs 1: the batch buffers are made on the first batched call
    psi = torch.empty((1, DIMS[0] * DIMS[1], 2), dtype=torch.complex128, device="cuda")
    st = ctx.solve_batch(to_dev(chi), psi, 1e-13)
    assert st[0]["converged"]
    assert rel_err(to_host(psi)[0], _exact(U, 0.1, chi[0])) <= 1e-8


def test_five_vectors_span_two_coarsest_launches_and_a_zero_source():
    # five right-hand sides: the batched coarsest kernel runs in chunks of four; vector 2 is zero
    import torch
    U = _field()
    masses = [0.02, 0.02, 0.05, 0.1, 0.2]
    chi = _sources(5, seed=13)
    chi[2] = 0.0
    ctx = _ctx(U, 0.02, 1, 5, coarsest_lu_max=0, coarsest_tol=0.2)
    psi = torch.empty((5, DIMS[0] * DIMS[1], 2), dtype=torch.complex128, device="cuda")
    st = ctx.solve_batch(to_dev(chi), psi, 1e-10, masses)
    out = to_host(psi)
    assert st[2]["converged"] and st[2]["iters"] == 0 and np.all(out[2] == 0)
    for v in (0, 1, 3, 4):
        assert st[v]["converged"]
        assert _true_rel(U, masses[v], out[v], chi[v]) <= 1e-10


def test_batch_rejects_bad_arguments():
    import torch
    mg = _mg()
    U = _field()
    ctx = _ctx(U, 0.1, 1, 2)
    chi = torch.zeros((3, DIMS[0] * DIMS[1], 2), dtype=torch.complex128, device="cuda")
    psi = torch.empty_like(chi)
    with pytest.raises(mg.MGError) as e:
        ctx.solve_batch(chi, psi, 1e-10)  # three vectors, max_rhs 2
    assert e.value.code == 1
    chi2 = chi[:2].contiguous()
    with pytest.raises(mg.MGError) as e:
        ctx.solve_batch(chi2, psi[:2].contiguous(), 1e-10, [0.1, float("nan")])
    assert e.value.code == 1


@pytest.mark.parametrize("beta", [3.0, 10.0])
def test_batch_full_size_256(beta):
    # the 256^2 three-level workload: one setup at m_c + 0.005, the three masses as one batch
    import torch
    L = 256
    U, theta, _ = inputs.schwinger_links(L, beta, sweeps=2000, workload_id=1)
    mc = mcrit_for(L, beta, 1, U, theta)
    assert mc is not None
    masses = [mc + 0.005, mc + 0.02, mc + 0.1]
    mg = _mg()
    p = mg.mg_default_params(levels=3, blocks=BLOCKS, Nv=[8, 8], precision=1, max_rhs=3, coarsest_tol=0.2)
    ctx = mg.Context.setup(to_dev(U), masses[0], (L, L), p)
    chi = np.stack([inputs.gaussian_source(L, L, seed=inputs.workload_seed(1, L, beta), index=i) for i in range(3)])
    psi = torch.empty((3, L * L, 2), dtype=torch.complex128, device="cuda")
    st = ctx.solve_batch(to_dev(chi), psi, 1e-10, masses)
    lat = Lattice((L, L))
    for v in range(3):
        assert st[v]["converged"]
        r = np.linalg.norm(chi[v] - wilson.apply_D(U, to_host(psi)[v], masses[v], lat)) / np.linalg.norm(chi[v])
        assert r <= 1e-10
