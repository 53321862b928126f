"""Wilson-Dirac operator (oracle).

Paper, definition of D following Eq. 1 (the Wilson discretisation):

    D_{x,y} = -1/2 sum_mu [ (1 - gamma_mu) U_x^mu delta_{x+mu,y}
                          + (1 + gamma_mu) U_{x-mu}^{mu dagger} delta_{x-mu,y} ]
              + (diag) delta_{x,y}

Readings taken here (the paper is silent or ambiguous):
  * diagonal: the paper prints (2d + m); we use (d + m), the r = 1 Wilson
    normalisation under which the free field has D(p = 0) = m and the free
    critical mass is 0. The two differ by a constant shift of m only
    (m_paper = m - d); every workload sets m relative to m_c.
  * gamma basis: 2d gamma_1 = sigma_1, gamma_2 = sigma_2 (gamma_5 = sigma_3);
    4d DeGrand-Rossi (gamma_5 = diag(1, 1, -1, -1)).
  * fermion boundary conditions: periodic in every direction (the paper states
    periodic boundaries for the gauge field).

Field layouts: U[x, mu, a, b] (Nc x Nc link from x to x + mu-hat), psi[x, s, c].
For U(1), Nc = 1.
"""
from __future__ import annotations

import numpy as np

from .lattice import Lattice

SIGMA1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SIGMA2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
SIGMA3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def gammas(d: int):
    """(gamma_0, ..., gamma_{d-1}, gamma_5) in the basis fixed above."""
    if d == 2:
        return [SIGMA1, SIGMA2], SIGMA3
    if d == 4:
        i = 1j
        g1 = np.array([[0, 0, 0, i], [0, 0, i, 0], [0, -i, 0, 0], [-i, 0, 0, 0]], dtype=np.complex128)
        g2 = np.array([[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]], dtype=np.complex128)
        g3 = np.array([[0, 0, i, 0], [0, 0, 0, -i], [-i, 0, 0, 0], [0, i, 0, 0]], dtype=np.complex128)
        g4 = np.array([[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]], dtype=np.complex128)
        g5 = g1 @ g2 @ g3 @ g4
        return [g1, g2, g3, g4], g5
    raise ValueError("only d = 2 and d = 4 are defined")


def n_spin(d: int) -> int:
    return 2 if d == 2 else 4


def _as_links(U, lat: Lattice):
    U = np.asarray(U, dtype=np.complex128)
    if U.ndim == 2:  # U(1): U[x, mu]
        U = U[:, :, None, None]
    assert U.shape[:2] == (lat.volume, lat.d)
    return U


def _as_spinor(psi, lat: Lattice, Nc: int):
    psi = np.asarray(psi, dtype=np.complex128)
    Ns = n_spin(lat.d)
    return psi.reshape(lat.volume, Ns, Nc)


def hop(U, psi, lat: Lattice, mu: int, sign: int):
    """One hopping term H_{sign*mu} psi (with its -1/2):

    sign = +1:  (H psi)_x = -1/2 (1 - gamma_mu) U_x^mu        psi_{x+mu}
    sign = -1:  (H psi)_x = -1/2 (1 + gamma_mu) U_{x-mu}^mu^+ psi_{x-mu}
    """
    U = _as_links(U, lat)
    Nc = U.shape[-1]
    shape = np.shape(psi)
    p = _as_spinor(psi, lat, Nc)
    g, _ = gammas(lat.d)
    one = np.eye(n_spin(lat.d), dtype=np.complex128)
    if sign > 0:
        src = lat.shift(p, mu, +1)                      # psi_{x+mu}
        link = U[:, mu]                                 # U_x^mu
        t = np.einsum("xab,xsb->xsa", link, src)
        proj = one - g[mu]
    else:
        src = lat.shift(p, mu, -1)                      # psi_{x-mu}
        link = lat.shift(U[:, mu], mu, -1)              # U_{x-mu}^mu
        t = np.einsum("xba,xsb->xsa", link.conj(), src)  # U^dagger
        proj = one + g[mu]
    out = -0.5 * np.einsum("st,xta->xsa", proj, t)
    return out.reshape(shape)


def diag_value(lat: Lattice, m: float) -> float:
    return lat.d + m


def apply_D(U, psi, m: float, lat: Lattice):
    """D psi with D as defined above (diagonal d + m)."""
    out = diag_value(lat, m) * np.asarray(psi, dtype=np.complex128)
    for mu in range(lat.d):
        out = out + hop(U, psi, lat, mu, +1) + hop(U, psi, lat, mu, -1)
    return out


def apply_Ddag(U, psi, m: float, lat: Lattice):
    """D^dagger psi = gamma_5 D gamma_5 psi (gamma_5-hermiticity; tested separately)."""
    _, g5 = gammas(lat.d)
    U = _as_links(U, lat)
    Nc = U.shape[-1]
    shape = np.shape(psi)
    p = _as_spinor(psi, lat, Nc)
    t = np.einsum("st,xta->xsa", g5, p)
    t = _as_spinor(apply_D(U, t, m, lat), lat, Nc)
    return np.einsum("st,xta->xsa", g5, t).reshape(shape)


def apply_gamma5(psi, lat: Lattice, Nc: int = 1):
    _, g5 = gammas(lat.d)
    shape = np.shape(psi)
    p = _as_spinor(psi, lat, Nc)
    return np.einsum("st,xta->xsa", g5, p).reshape(shape)


def dense_D(U, m: float, lat: Lattice, Nc: int = 1):
    """The matrix of D, column by column from unit vectors (tiny lattices only)."""
    n = lat.volume * n_spin(lat.d) * Nc
    M = np.zeros((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for col in range(n):
        e[:] = 0
        e[col] = 1
        M[:, col] = apply_D(U, e.reshape(lat.volume, -1), m, lat).reshape(-1)
    return M


def gauge_transform(U, omega, lat: Lattice):
    """U'_x^mu = Omega_x U_x^mu Omega_{x+mu}^dagger (Omega[x, a, b], or U(1) phases Omega[x])."""
    U = _as_links(U, lat)
    om = np.asarray(omega, dtype=np.complex128)
    if om.ndim == 1:
        om = om[:, None, None]
    out = np.empty_like(U)
    for mu in range(lat.d):
        om_fwd = lat.shift(om, mu, +1)
        out[:, mu] = np.einsum("xab,xbc,xdc->xad", om, U[:, mu], om_fwd.conj())
    return out


def transform_spinor(psi, omega, lat: Lattice, Nc: int = 1):
    """psi'_x = Omega_x psi_x."""
    om = np.asarray(omega, dtype=np.complex128)
    if om.ndim == 1:
        om = om[:, None, None]
    shape = np.shape(psi)
    p = _as_spinor(psi, lat, Nc)
    return np.einsum("xab,xsb->xsa", om, p).reshape(shape)


def apply_D_at(U, psi, m: float, lat: Lattice, sites):
    """(D psi)_x at the given sites only, from the same definition (for sampled checks
    of fields too large to apply D to as a whole)."""
    U = _as_links(U, lat)
    Nc = U.shape[-1]
    p = _as_spinor(psi, lat, Nc)
    sites = np.asarray(sites, dtype=np.int64)
    g, _ = gammas(lat.d)
    one = np.eye(n_spin(lat.d), dtype=np.complex128)
    out = diag_value(lat, m) * p[sites]
    for mu in range(lat.d):
        fwd = lat.neighbour(sites, mu, +1)
        bwd = lat.neighbour(sites, mu, -1)
        t = np.einsum("xab,xsb->xsa", U[sites, mu], p[fwd])
        out = out - 0.5 * np.einsum("st,xta->xsa", one - g[mu], t)
        t = np.einsum("xba,xsb->xsa", U[bwd, mu].conj(), p[bwd])
        out = out - 0.5 * np.einsum("st,xta->xsa", one + g[mu], t)
    return out.reshape((len(sites),) + np.shape(psi)[1:])
