"""Pins of the oracle's 4d SU(3) multigrid: chirality-split prolongator, Galerkin operator and
two-level solves (DeGrand-Rossi basis, gamma_5 = diag(1, 1, -1, -1))."""
import numpy as np
import pytest

import inputs
from oracle import coarse, setup, solvers, transfer, wilson
from oracle.lattice import Blocking, Lattice


def _params(block, nv, **kw):
    base = dict(levels=2, blocks=(block,), Nv=(nv,), n_pass=2, nu_setup=6, chiral_split=True, coarsest_lu_max=4096)
    base.update(kw)
    return setup.MGParams(**base)


def test_chirality_split_halves_are_chiral_and_complete():
    dims = (2, 2, 2, 4)
    lat = Lattice(dims)
    v = [inputs.gaussian_spinor(lat.volume, 12, 3, k) for k in range(3)]
    parts = setup.chirality_split(v, lat, 3)
    assert len(parts) == 6
    for k in range(3):
        p, q = parts[k].reshape(-1, 4, 3), parts[3 + k].reshape(-1, 4, 3)
        np.testing.assert_array_equal(p[:, 2:], 0)   # P+ keeps spins 0, 1
        np.testing.assert_array_equal(q[:, :2], 0)   # P- keeps spins 2, 3
        np.testing.assert_allclose(parts[k] + parts[3 + k], v[k], atol=0)


def test_split_prolongator_is_block_orthonormal_and_chiral():
    dims = (4, 4, 2, 2)
    U = inputs.su3_links(dims, seed=4, ape_steps=2)
    hier = setup.adaptive_setup(U, 0.2, Lattice(dims), _params((2, 2, 2, 2), 3), Nc=3)
    P = hier.P[0]                                 # (n_blocks, 16 * 12, 6)
    assert P.shape == (4, 192, 6)
    G = np.einsum("bik,bil->bkl", P.conj(), P)
    np.testing.assert_allclose(G, np.broadcast_to(np.eye(6), G.shape), atol=1e-13)
    Ps = P.reshape(4, 16, 4, 3, 6)
    np.testing.assert_array_equal(Ps[:, :, 2:, :, :3], 0)
    np.testing.assert_array_equal(Ps[:, :, :2, :, 3:], 0)


def test_split_coarse_operator_gamma5_hermitian():
    # columns of one chirality: P^dagger gamma_5 = Gamma_5 P^dagger with Gamma_5 = diag(1 x Nv, -1 x Nv)
    # per coarse site, so gamma_5-hermiticity of D carries over to the coarse matrix
    dims = (4, 2, 2, 4)
    lat = Lattice(dims)
    U = inputs.su3_random(lat.volume * 4, 5, 1).reshape(-1, 4, 3, 3)
    hier = setup.adaptive_setup(U, -0.1, lat, _params((2, 2, 2, 2), 2, n_pass=1), Nc=3)
    Ac = solvers.stencil_matrix(hier.ops[1])
    nc = hier.ops[1].lat.volume
    G5 = np.kron(np.eye(nc), np.diag([1.0, 1.0, -1.0, -1.0]))
    np.testing.assert_allclose(G5 @ Ac @ G5, Ac.conj().T, atol=1e-13)


def test_split_galerkin_matches_dense_PdagDP():
    dims = (4, 2, 2, 2)
    lat = Lattice(dims)
    U = inputs.su3_links(dims, seed=8, ape_steps=1)
    m = 0.15
    hier = setup.adaptive_setup(U, m, lat, _params((2, 2, 1, 2), 2, n_pass=1), Nc=3)
    Pd = transfer.dense_P(hier.P[0], hier.blk[0], 12)
    want = Pd.conj().T @ wilson.dense_D(U, m, lat, 3) @ Pd
    np.testing.assert_allclose(solvers.stencil_matrix(hier.ops[1]), want, atol=1e-13)


def test_full_rank_split_two_grid_is_exact():
    # Nv per chirality = half the block dimension (2 x 1 x 1 x 1 blocks: 2 sites x 6 dofs):
    # P is unitary, so one V-cycle without smoothing solves exactly
    dims = (4, 2, 2, 2)
    lat = Lattice(dims)
    U = inputs.su3_random(lat.volume * 4, 6, 2).reshape(-1, 4, 3, 3)
    p = _params((2, 1, 1, 1), 12, n_pass=1, nu_pre=0, nu_post=0)
    hier = setup.adaptive_setup(U, 0.3, lat, p, Nc=3)
    b = inputs.gaussian_spinor(lat.volume, 12, 7, 0)
    x = solvers.vcycle(hier, 0, b)
    r = b - wilson.apply_D(U, x, 0.3, lat)
    assert np.linalg.norm(r) < 1e-12 * np.linalg.norm(b)


def test_4d_mg_solve_matches_dense_lu():
    dims = (4, 4, 4, 4)
    lat = Lattice(dims)
    U = inputs.su3_links(dims, seed=11)
    m = 0.05
    p = _params((2, 2, 2, 2), 4, n_pass=2, gcr_restart=16, max_iter=200)
    hier = setup.adaptive_setup(U, m, lat, p, Nc=3)
    chi = inputs.gaussian_spinor(lat.volume, 12, 12, 0)
    psi, info = solvers.mg_solve(hier, chi, 1e-12)
    assert info["converged"]
    ref = np.linalg.solve(wilson.dense_D(U, m, lat, 3), chi.reshape(-1)).reshape(chi.shape)
    assert np.linalg.norm(psi - ref) <= 1e-10 * np.linalg.norm(ref)
    # and MG beats plain GCR by a wide margin in outer iterations
    _, plain = solvers.gcr(lambda v: wilson.apply_D(U, v, m, lat), chi, 1e-12, 16, 2000)
    assert info["iters"] * 3 < plain["iters"], (info["iters"], plain["iters"])
