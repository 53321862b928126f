"""Invariants of the oracle's adaptive setup and critical-mass scan.

Individual near-null vectors after the first pass have no closed form
(parity unpinned); they are checked through invariants: block orthonormality,
the decrease of ||A v|| / ||v|| over the passes, the removal of critical slowing
down against plain GCR, gauge covariance of the solution.
"""
import numpy as np
import pytest

import inputs
from oracle import coarse, setup, solvers, spectrum, wilson
from oracle.lattice import Lattice


def _thermal(L, beta=6.0, sweeps=150, wid=9):
    U, theta, _ = inputs.schwinger_links(L, beta, sweeps=sweeps, workload_id=wid)
    return U


def test_setup_orthonormal_on_every_level():
    dims = (32, 32)
    lat = Lattice(dims)
    U = _thermal(32)
    p = setup.MGParams(levels=3, blocks=((4, 4), (2, 2)), Nv=(8, 8), n_pass=2)
    hier = setup.adaptive_setup(U, 0.0, lat, p)
    for level in range(2):
        P = hier.P[level]
        eye = np.eye(P.shape[2])
        for b in range(0, P.shape[0], 5):
            np.testing.assert_allclose(P[b].conj().T @ P[b], eye, atol=1e-13)


def _rayleigh(hier, level=0):
    A = hier.ops[level].apply
    return np.mean([np.linalg.norm(A(v)) / np.linalg.norm(v) for v in hier.vecs[level]])


def test_adaptive_passes_lower_the_vectors_residual():
    dims = (16, 16)
    lat = Lattice(dims)
    U = _thermal(16)
    mc = spectrum.critical_mass_dense(U, lat)
    vals = []
    for n_pass in (1, 2, 4):
        p = setup.MGParams(levels=2, blocks=((4, 4),), Nv=(8,), n_pass=n_pass)
        vals.append(_rayleigh(setup.adaptive_setup(U, mc + 0.01, lat, p)))
    assert vals[0] > vals[1] > vals[2]
    # random vectors relaxed only: clearly above the lowest singular value scale
    smin = np.linalg.svd(wilson.dense_D(U, mc + 0.01, lat), compute_uv=False).min()
    assert vals[2] < 20 * vals[0] and vals[2] > smin * 0.999


def test_mg_removes_critical_slowing_down():
    dims = (32, 32)
    lat = Lattice(dims)
    U = _thermal(32)
    mc = spectrum.critical_mass_arnoldi(U, lat)
    m = mc + 0.01
    p = setup.MGParams(levels=2, blocks=((4, 4),), Nv=(8,))
    hier = setup.adaptive_setup(U, m, lat, p)
    chi = inputs.gaussian_source(*dims, seed=3)
    _, info_mg = solvers.mg_solve(hier, chi, 1e-10)
    _, info_plain = solvers.gcr(hier.ops[0].apply, chi, 1e-10, 16, 100000)
    assert info_mg["converged"] and info_plain["converged"]
    assert info_mg["iters"] * 10 < info_plain["iters"]


def test_mg_solution_is_gauge_covariant():
    dims = (16, 16)
    lat = Lattice(dims)
    U = _thermal(16)
    omega = inputs.u1_phases(lat.volume, 3, 3)
    Ug = wilson.gauge_transform(U, omega, lat)[:, :, 0, 0]
    chi = inputs.gaussian_source(*dims, seed=4)
    p = setup.MGParams(levels=2, blocks=((4, 4),), Nv=(8,), n_pass=2)
    m = 0.05
    x, _ = solvers.mg_solve(setup.adaptive_setup(U, m, lat, p), chi, 1e-12)
    xg, _ = solvers.mg_solve(setup.adaptive_setup(Ug, m, lat, p), wilson.transform_spinor(chi, omega, lat), 1e-12)
    want = wilson.transform_spinor(x, omega, lat)
    assert np.linalg.norm(xg - want) < 1e-9 * np.linalg.norm(want)


def test_update_mass_equals_fresh_galerkin():
    dims = (16, 16)
    lat = Lattice(dims)
    U = _thermal(16)
    p = setup.MGParams(levels=3, blocks=((4, 4), (2, 2)), Nv=(8, 8), n_pass=1)
    hier = setup.adaptive_setup(U, 0.01, lat, p)
    Y1_old = hier.ops[1].Y.copy()
    Y2_old = hier.ops[2].Y.copy()
    setup.update_mass(hier, 0.11)
    # P^dagger P = I on every level, so a mass shift moves only the coarse self blocks
    np.testing.assert_allclose(hier.ops[1].Y[:, 0] - Y1_old[:, 0], np.broadcast_to(0.1 * np.eye(8), Y1_old[:, 0].shape),
                               atol=1e-13)
    np.testing.assert_allclose(hier.ops[2].Y[:, 0] - Y2_old[:, 0], np.broadcast_to(0.1 * np.eye(8), Y2_old[:, 0].shape),
                               atol=1e-13)


def test_critical_mass_free_field_is_zero():
    lat = Lattice((8, 8))
    assert abs(spectrum.critical_mass_dense(inputs.free_links(8, 8), lat)) < 1e-12


def test_critical_mass_twisted_free_field():
    # constant twist phi: min over p of (d - sum cos(p + phi)) is at the lattice momentum nearest -phi
    dims, phi = (8, 6), (0.4, -0.2)
    lat = Lattice(dims)
    p0 = 2 * np.pi * np.arange(8) / 8 + phi[0]
    p1 = 2 * np.pi * np.arange(6) / 6 + phi[1]
    want = -min(2 - np.cos(a) - np.cos(b) for a in p0 for b in p1)
    got = spectrum.critical_mass_dense(inputs.free_links(*dims, phi=phi), lat)
    assert abs(got - want) < 1e-12


def test_critical_mass_arnoldi_matches_dense():
    lat = Lattice((16, 16))
    U = _thermal(16)
    assert abs(spectrum.critical_mass_arnoldi(U, lat) - spectrum.critical_mass_dense(U, lat)) < 1e-8
