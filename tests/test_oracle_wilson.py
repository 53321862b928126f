"""Pins of the oracle's Wilson-Dirac operator against what the mathematics fixes.

* gamma algebra of the chosen bases;
* closed-form free-field spectrum (U = 1) and its constant-U(1)-twist shift;
* gamma_5-hermiticity gamma_5 D gamma_5 = D^dagger;
* gauge covariance D[U^Omega] Omega psi = Omega D[U] psi.
A dropped hopping term, a wrong projector sign, a swapped U / U^dagger or a
wrong diagonal fails at least one of them.
"""
import numpy as np
import pytest

import inputs
from oracle import wilson
from oracle.lattice import Lattice


def _sorted(ev):
    ev = np.asarray(ev)
    return ev[np.lexsort((np.round(ev.imag, 8), np.round(ev.real, 8)))]


@pytest.mark.parametrize("d", [2, 4])
def test_gamma_algebra(d):
    g, g5 = wilson.gammas(d)
    ns = wilson.n_spin(d)
    for mu in range(d):
        np.testing.assert_allclose(g[mu], g[mu].conj().T)
        for nu in range(d):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            np.testing.assert_allclose(anti, 2 * np.eye(ns) * (mu == nu), atol=1e-15)
        np.testing.assert_allclose(g5 @ g[mu] + g[mu] @ g5, 0, atol=1e-15)
    # gamma_5 is diagonal in both bases: sigma_3 (2d), diag(1,1,-1,-1) (DeGrand-Rossi)
    want = np.diag([1, -1]) if d == 2 else np.diag([1, 1, -1, -1])
    np.testing.assert_allclose(g5, want, atol=1e-15)
    if d == 2:  # gamma_5 = -i gamma_1 gamma_2
        np.testing.assert_allclose(-1j * g[0] @ g[1], g5, atol=1e-15)


def free_spectrum(dims, m, phi=None):
    d = len(dims)
    phi = np.zeros(d) if phi is None else np.asarray(phi)
    grids = np.meshgrid(*[2 * np.pi * np.arange(L) / L for L in dims], indexing="ij")
    ps = [g.reshape(-1) + phi[mu] for mu, g in enumerate(grids)]
    re = d + m - sum(np.cos(p) for p in ps)
    im = np.sqrt(sum(np.sin(p) ** 2 for p in ps))
    mult = wilson.n_spin(d) // 2
    ev = np.concatenate([re + 1j * im, re - 1j * im] * mult)
    return ev


@pytest.mark.parametrize("dims,m", [((4, 4), 0.1), ((6, 4), -0.3), ((5, 3), 0.0)])
def test_free_spectrum_2d(dims, m):
    lat = Lattice(dims)
    U = inputs.free_links(*dims)
    ev = np.linalg.eigvals(wilson.dense_D(U, m, lat))
    np.testing.assert_allclose(_sorted(ev), _sorted(free_spectrum(dims, m)), atol=1e-12)


@pytest.mark.parametrize("phi", [(0.3, -1.1), (np.pi / 4, 0.0)])
def test_twisted_free_spectrum_2d(phi):
    dims, m = (4, 6), 0.05
    lat = Lattice(dims)
    U = inputs.free_links(*dims, phi=phi)
    ev = np.linalg.eigvals(wilson.dense_D(U, m, lat))
    np.testing.assert_allclose(_sorted(ev), _sorted(free_spectrum(dims, m, phi)), atol=1e-12)


def test_free_spectrum_4d():
    dims, m = (3, 2, 2, 4), 0.2
    lat = Lattice(dims)
    U = np.ones((lat.volume, 4), dtype=np.complex128)
    ev = np.linalg.eigvals(wilson.dense_D(U, m, lat))
    np.testing.assert_allclose(_sorted(ev), _sorted(free_spectrum(dims, m)), atol=1e-12)


def test_plane_wave_eigenvector():
    # D e^{ipx} u = [(d + m - sum cos p) + i sum sin p gamma_mu] e^{ipx} u
    dims, m = (8, 4), 0.3
    lat = Lattice(dims)
    U = inputs.free_links(*dims)
    x0, x1 = lat.coords(np.arange(lat.volume))
    p = (2 * np.pi * 3 / 8, 2 * np.pi * 1 / 4)
    u = np.array([0.3 - 0.2j, 1.1 + 0.5j])
    psi = np.exp(1j * (p[0] * x0 + p[1] * x1))[:, None] * u[None, :]
    g, _ = wilson.gammas(2)
    Dp = (2 + m - np.cos(p[0]) - np.cos(p[1])) * np.eye(2) + 1j * (np.sin(p[0]) * g[0] + np.sin(p[1]) * g[1])
    want = np.exp(1j * (p[0] * x0 + p[1] * x1))[:, None] * (Dp @ u)[None, :]
    np.testing.assert_allclose(wilson.apply_D(U, psi, m, lat), want, atol=1e-13)


@pytest.mark.parametrize("dims", [(8, 8), (6, 10)])
def test_gamma5_hermiticity(dims):
    lat = Lattice(dims)
    U = inputs.hot_links(*dims, seed=3)
    m = -0.2
    phi = inputs.gaussian_complex(lat.volume * 2, 11, 1).reshape(-1, 2)
    psi = inputs.gaussian_complex(lat.volume * 2, 11, 2).reshape(-1, 2)
    g5Dg5psi = wilson.apply_gamma5(wilson.apply_D(U, wilson.apply_gamma5(psi, lat), m, lat), lat)
    lhs = np.vdot(phi, g5Dg5psi)
    rhs = np.vdot(wilson.apply_D(U, phi, m, lat), psi)
    assert abs(lhs - rhs) <= 1e-14 * abs(rhs) * 10


def test_gamma5_hermiticity_dense():
    lat = Lattice((4, 4))
    U = inputs.hot_links(4, 4, seed=8)
    M = wilson.dense_D(U, 0.1, lat)
    G5 = np.kron(np.eye(lat.volume), np.diag([1.0, -1.0]))
    np.testing.assert_allclose(G5 @ M @ G5, M.conj().T, atol=1e-14)


def test_gauge_covariance():
    dims = (8, 6)
    lat = Lattice(dims)
    U = inputs.hot_links(*dims, seed=21)
    omega = inputs.u1_phases(lat.volume, 5, 9)
    Ug = wilson.gauge_transform(U, omega, lat)[:, :, 0, 0]
    psi = inputs.gaussian_complex(lat.volume * 2, 12, 3).reshape(-1, 2)
    lhs = wilson.apply_D(Ug, wilson.transform_spinor(psi, omega, lat), 0.07, lat)
    rhs = wilson.transform_spinor(wilson.apply_D(U, psi, 0.07, lat), omega, lat)
    np.testing.assert_allclose(lhs, rhs, atol=1e-13)


def test_each_hop_is_nearest_neighbour():
    # the matrix of D has nonzeros only on (x, x) and (x, x +- mu)
    lat = Lattice((5, 4))
    U = inputs.hot_links(5, 4, seed=2)
    M = wilson.dense_D(U, 0.0, lat).reshape(lat.volume, 2, lat.volume, 2)
    allowed = np.zeros((lat.volume, lat.volume), dtype=bool)
    xs = np.arange(lat.volume)
    allowed[xs, xs] = True
    for mu in range(2):
        for s in (+1, -1):
            allowed[xs, lat.neighbour(xs, mu, s)] = True
    blk = np.abs(M).sum(axis=(1, 3))
    assert np.all(blk[~allowed] == 0)


def test_sampled_apply_matches_whole_field_apply():
    lat = Lattice((12, 10))
    U = inputs.hot_links(12, 10, seed=13)
    psi = inputs.gaussian_complex(lat.volume * 2, 1, 5).reshape(-1, 2)
    sites = np.array([0, 5, 11, 12, 59, 119])
    np.testing.assert_allclose(wilson.apply_D_at(U, psi, 0.3, lat, sites),
                               wilson.apply_D(U, psi, 0.3, lat)[sites], atol=1e-14)


def test_gamma5_hermiticity_4d_su3():
    dims = (4, 2, 4, 6)
    lat = Lattice(dims)
    U = inputs.su3_random(lat.volume * 4, 4, 0x11).reshape(-1, 4, 3, 3)
    m = -0.3
    phi = inputs.gaussian_spinor(lat.volume, 12, 11, 1)
    psi = inputs.gaussian_spinor(lat.volume, 12, 11, 2)
    g5Dg5psi = wilson.apply_gamma5(wilson.apply_D(U, wilson.apply_gamma5(psi, lat, 3), m, lat), lat, 3)
    lhs = np.vdot(phi, g5Dg5psi)
    rhs = np.vdot(wilson.apply_D(U, phi, m, lat), psi)
    assert abs(lhs - rhs) <= 1e-13 * abs(rhs)


def test_gauge_covariance_4d_su3():
    dims = (4, 4, 2, 4)
    lat = Lattice(dims)
    U = inputs.su3_links(dims, seed=6, ape_steps=1)
    omega = inputs.su3_random(lat.volume, 5, 9)
    Ug = wilson.gauge_transform(U, omega, lat)
    psi = inputs.gaussian_spinor(lat.volume, 12, 12, 3)
    lhs = wilson.apply_D(Ug, wilson.transform_spinor(psi, omega, lat, 3), 0.07, lat)
    rhs = wilson.transform_spinor(wilson.apply_D(U, psi, 0.07, lat), omega, lat, 3)
    np.testing.assert_allclose(lhs, rhs, atol=1e-13)


def test_4d_projector_rank_two():
    # every (1 -+ gamma_mu) of the DeGrand-Rossi basis is twice a rank-2 projector: the
    # property that lets a 4d hop carry a half spinor
    g, _ = wilson.gammas(4)
    for gm in g:
        for sgn in (+1, -1):
            Pm = (np.eye(4) + sgn * gm) / 2
            np.testing.assert_allclose(Pm @ Pm, Pm, atol=1e-15)
            assert np.linalg.matrix_rank(Pm) == 2
