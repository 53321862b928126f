"""Pins of the oracle's MR smoother, V-cycle, coarsest solve and outer GCR."""
import numpy as np
import pytest

import inputs
from oracle import coarse, setup, solvers, transfer, wilson
from oracle.lattice import Lattice


def _thermal(L, beta=6.0, sweeps=150, wid=9):
    U, theta, _ = inputs.schwinger_links(L, beta, sweeps=sweeps, workload_id=wid)
    return U


def test_mr_step_is_residual_minimising():
    lat = Lattice((8, 8))
    U = inputs.hot_links(8, 8, seed=1)
    A = lambda v: wilson.apply_D(U, v, 0.3, lat)
    b = inputs.gaussian_complex(lat.volume * 2, 1, 1).reshape(-1, 2)
    # omega = 1: the new residual is orthogonal to A r and no line search does better
    x, r = solvers.mr(A, b, 1, 1.0)
    Ab = A(b)
    assert abs(np.vdot(Ab, r)) < 1e-12 * np.linalg.norm(Ab) * np.linalg.norm(r)
    for t in (0.9, 1.1, 1.0 + 0.05j):
        alpha = np.vdot(Ab, b) / np.vdot(Ab, Ab) * t
        assert np.linalg.norm(b - alpha * Ab) >= np.linalg.norm(r) * (1 - 1e-14)
    # the recursively updated residual equals b - A x
    x, r = solvers.mr(A, b, 4, 0.8)
    np.testing.assert_allclose(r, b - A(x), atol=1e-12)
    assert np.linalg.norm(r) < np.linalg.norm(b)


def _hier(U, m, dims, params):
    lat = Lattice(dims)
    return setup.adaptive_setup(U, m, lat, params), lat


def test_vcycle_operator_form_with_linear_smoother():
    # With a fixed polynomial smoother S (pre = post = S), the five steps give
    #   V = S + S - S A S + (1 - S A) P A_c^{-1} P^dagger (1 - A S)
    # (the operator form with the sign of the R A R^dagger term that the five steps imply)
    dims = (8, 8)
    lat = Lattice(dims)
    U = inputs.hot_links(*dims, seed=5)
    m = 0.4
    p = setup.MGParams(levels=2, blocks=((4, 4),), Nv=(4,), n_pass=1, nu_setup=2)
    hier = setup.adaptive_setup(U, m, lat, p)
    n = lat.volume * 2
    Ad = wilson.dense_D(U, m, lat)
    om = 0.3
    Sd = om * np.eye(n) + om * (np.eye(n) - om * Ad)  # two Richardson steps from x = 0

    def lin(level, b):
        return (Sd @ np.asarray(b).reshape(-1)).reshape(np.shape(b))

    hier.linear_smoother = lin
    Pd = transfer.dense_P(hier.P[0], hier.blk[0], 2)
    Ac = Pd.conj().T @ Ad @ Pd
    I = np.eye(n)
    want = Sd + Sd - Sd @ Ad @ Sd + (I - Sd @ Ad) @ Pd @ np.linalg.inv(Ac) @ Pd.conj().T @ (I - Ad @ Sd)
    got = np.zeros((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for c in range(n):
        e[:] = 0
        e[c] = 1
        got[:, c] = solvers.vcycle(hier, 0, e.reshape(-1, 2)).reshape(-1)
    np.testing.assert_allclose(got, want, atol=1e-11)


def test_full_rank_two_grid_is_exact():
    # Nv = block dimension (4x4 sites x 2 spins = 32): P is unitary and with the exact
    # coarsest solve one V-cycle inverts D, whatever the smoother does.
    dims = (8, 8)
    lat = Lattice(dims)
    U = inputs.hot_links(*dims, seed=6)
    p = setup.MGParams(levels=2, blocks=((4, 4),), Nv=(32,), n_pass=1, nu_setup=1, coarsest_lu_max=4096)
    hier = setup.adaptive_setup(U, 0.2, lat, p)
    b = inputs.gaussian_complex(lat.volume * 2, 3, 3).reshape(-1, 2)
    x = solvers.vcycle(hier, 0, b)
    xd = np.linalg.solve(wilson.dense_D(U, 0.2, lat), b.reshape(-1))
    assert np.linalg.norm(x.reshape(-1) - xd) < 1e-11 * np.linalg.norm(xd)


def test_coarse_correction_galerkin_orthogonality():
    # after steps 1-4 with an exact coarse solve, P^dagger (b - A x) = 0
    dims = (16, 16)
    lat = Lattice(dims)
    U = _thermal(16)
    p = setup.MGParams(levels=2, blocks=((4, 4),), Nv=(6,), n_pass=2)
    hier = setup.adaptive_setup(U, 0.1, lat, p)
    A = hier.ops[0].apply
    b = inputs.gaussian_complex(lat.volume * 2, 4, 4).reshape(-1, 2)
    x, _ = solvers.mr(A, b, 4, 0.8)
    ec = hier.coarsest.solve(hier.restrict(0, b - A(x)))
    x = x + hier.prolong(0, ec)
    rc = hier.restrict(0, b - A(x))
    assert np.linalg.norm(rc) < 1e-12 * np.linalg.norm(b)


def test_coarsest_lu_and_gcr_agree():
    dims = (16, 16)
    lat = Lattice(dims)
    U = _thermal(16)
    p = setup.MGParams(levels=2, blocks=((4, 4),), Nv=(8,), n_pass=1)
    hier = setup.adaptive_setup(U, 0.2, lat, p)
    op = hier.ops[1]
    b = inputs.gaussian_complex(op.lat.volume * 8, 5, 5).reshape(-1, 8)
    lu = solvers.CoarsestSolver(op, 10 ** 9, 1e-13, 64, 5000)
    it = solvers.CoarsestSolver(op, 0, 1e-13, 64, 5000)
    xl, xi = lu.solve(b), it.solve(b)
    xd = np.linalg.solve(coarse.dense_operator(op, b.size), b.reshape(-1))
    assert np.linalg.norm(xl.reshape(-1) - xd) < 1e-12 * np.linalg.norm(xd)
    assert np.linalg.norm(xi.reshape(-1) - xd) < 1e-9 * np.linalg.norm(xd)


def test_gcr_unpreconditioned_matches_dense_solve():
    dims = (8, 8)
    lat = Lattice(dims)
    U = inputs.hot_links(*dims, seed=7)
    A = lambda v: wilson.apply_D(U, v, 0.5, lat)
    b = inputs.gaussian_complex(lat.volume * 2, 6, 6).reshape(-1, 2)
    x, info = solvers.gcr(A, b, 1e-13, 10, 5000)
    assert info["converged"]
    xd = np.linalg.solve(wilson.dense_D(U, 0.5, lat), b.reshape(-1))
    assert np.linalg.norm(x.reshape(-1) - xd) < 1e-11 * np.linalg.norm(xd)


@pytest.mark.parametrize("levels,dims", [(2, (16, 16)), (3, (32, 32))])
def test_mg_solve_matches_dense_lu(levels, dims):
    lat = Lattice(dims)
    U = _thermal(dims[0])
    from oracle import spectrum
    mc = spectrum.critical_mass_arnoldi(U, lat)
    m = mc + 0.02
    blocks = ((4, 4), (2, 2))[:levels - 1]
    p = setup.MGParams(levels=levels, blocks=blocks, Nv=(8,) * (levels - 1))
    hier = setup.adaptive_setup(U, m, lat, p)
    chi = inputs.gaussian_source(*dims, seed=8)
    x, info = solvers.mg_solve(hier, chi, 1e-12)
    assert info["converged"] and info["true_rel_residual"] <= 1e-12
    xd = np.linalg.solve(wilson.dense_D(U, m, lat), chi.reshape(-1))
    assert np.linalg.norm(x.reshape(-1) - xd) < 1e-8 * np.linalg.norm(xd)


def test_vcycle_cost_is_2nu_plus_2_per_level():
    dims = (16, 16)
    lat = Lattice(dims)
    U = _thermal(16)
    p = setup.MGParams(levels=2, blocks=((4, 4),), Nv=(8,), n_pass=1)
    hier = setup.adaptive_setup(U, 0.2, lat, p)
    cnt = solvers.OpCounter()
    solvers.vcycle(hier, 0, inputs.gaussian_source(*dims, seed=2), counter=cnt)
    assert cnt.counts[0] == 2 * p.nu_pre + 2
