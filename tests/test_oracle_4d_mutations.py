"""Planted mistakes in the oracle's 4d SU(3) Wilson operator (on the CPU) must be caught by its pins.

Each case replaces the hopping term (or the diagonal) of `oracle/wilson.py` with a plausible
error (the backward link without its dagger, a transposed forward link, the backward link taken
at x instead of x - mu, a 2d + m diagonal) and asserts that one of the 4d pins fails: the
closed-form free spectrum (U = 1), gamma_5-hermiticity and gauge covariance on SU(3) links.
"""
import numpy as np
import pytest

import inputs
from oracle import wilson
from oracle.lattice import Lattice
from tests.test_oracle_wilson import _sorted, free_spectrum


def _pins_pass():
    ok = []
    # free spectrum (closed form)
    dims, m = (3, 2, 2, 4), 0.2
    lat = Lattice(dims)
    U1 = np.ones((lat.volume, 4), dtype=np.complex128)
    ev = np.linalg.eigvals(wilson.dense_D(U1, m, lat))
    ok.append(np.allclose(_sorted(ev), _sorted(free_spectrum(dims, m)), atol=1e-12))
    # gamma_5-hermiticity on random SU(3) links
    lat = Lattice((4, 2, 4, 6))
    U = inputs.su3_random(lat.volume * 4, 4, 0x11).reshape(-1, 4, 3, 3)
    phi = inputs.gaussian_spinor(lat.volume, 12, 11, 1)
    psi = inputs.gaussian_spinor(lat.volume, 12, 11, 2)
    lhs = np.vdot(phi, wilson.apply_gamma5(wilson.apply_D(U, wilson.apply_gamma5(psi, lat, 3), -0.3, lat), lat, 3))
    rhs = np.vdot(wilson.apply_D(U, phi, -0.3, lat), psi)
    ok.append(abs(lhs - rhs) <= 1e-13 * abs(rhs))
    # gauge covariance
    dims = (4, 4, 2, 4)
    lat = Lattice(dims)
    U = inputs.su3_links(dims, seed=6, ape_steps=1)
    omega = inputs.su3_random(lat.volume, 5, 9)
    Ug = wilson.gauge_transform(U, omega, lat)
    psi = inputs.gaussian_spinor(lat.volume, 12, 12, 3)
    lhs = wilson.apply_D(Ug, wilson.transform_spinor(psi, omega, lat, 3), 0.07, lat)
    rhs = wilson.transform_spinor(wilson.apply_D(U, psi, 0.07, lat), omega, lat, 3)
    ok.append(np.allclose(lhs, rhs, atol=1e-13))
    return ok


def _mutant_hop(kind):
    original = wilson.hop

    def hop(U, psi, lat, mu, sign):
        if lat.d != 4:
            return original(U, psi, lat, mu, sign)
        U = wilson._as_links(U, lat)
        Nc = U.shape[-1]
        shape = np.shape(psi)
        p = wilson._as_spinor(psi, lat, Nc)
        g, _ = wilson.gammas(lat.d)
        one = np.eye(wilson.n_spin(lat.d), dtype=np.complex128)
        if sign > 0:
            src = lat.shift(p, mu, +1)
            link = U[:, mu]
            if kind == "transposed_forward":
                t = np.einsum("xba,xsb->xsa", link, src)
            else:
                t = np.einsum("xab,xsb->xsa", link, src)
            proj = one - g[mu]
        else:
            src = lat.shift(p, mu, -1)
            link = U[:, mu] if kind == "backward_link_at_x" else lat.shift(U[:, mu], mu, -1)
            if kind == "no_dagger":
                t = np.einsum("xab,xsb->xsa", link, src)
            else:
                t = np.einsum("xba,xsb->xsa", link.conj(), src)
            proj = one + g[mu]
        return (-0.5 * np.einsum("st,xta->xsa", proj, t)).reshape(shape)

    return hop


def test_unmutated_4d_oracle_passes_all():
    assert all(_pins_pass())


@pytest.mark.parametrize("kind", ["no_dagger", "transposed_forward", "backward_link_at_x"])
def test_planted_4d_hop_mistake_is_caught(kind, monkeypatch):
    monkeypatch.setattr(wilson, "hop", _mutant_hop(kind))
    assert not all(_pins_pass()), kind


def test_planted_4d_diagonal_mistake_is_caught(monkeypatch):
    monkeypatch.setattr(wilson, "diag_value", lambda lat, m: 2 * lat.d + m)
    assert not all(_pins_pass())
