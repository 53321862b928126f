"""Pins of the seeded input generators (shared by the oracle and the GPU path)."""
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy.special import iv

import inputs
from oracle import rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(t, 16) for t in line.split()]
        rows.append((w[:4], w[4:6], w[6:]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_kat_inputs_module(ctr, key, out):
    assert list(inputs.philox4x32_10(ctr, key)) == out


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_kat_oracle(ctr, key, out):
    got = rng.philox4x32_10(*[np.array([c], dtype=np.uint64) for c in ctr], key[0], key[1])
    assert [int(g[0]) for g in got] == out


def test_gaussian_two_implementations_agree():
    # the C generator with tag = k + 2^32 * level and the oracle's numpy draw are
    # two independent implementations of the same published definition
    n, seed = 5000, 987654321012345
    for k, level in [(0, 0), (3, 1), (7, 2)]:
        a = inputs.gaussian_complex(n, seed, k + (level << 32))
        b = rng.gaussian_vector(n, seed, k, level)
        np.testing.assert_allclose(a, b, rtol=1e-14, atol=1e-14)


def test_gaussian_moments():
    z = inputs.gaussian_complex(400000, 42, 7)
    assert abs(z.real.mean()) < 0.01 and abs(z.imag.mean()) < 0.01
    assert abs(z.real.var() - 1) < 0.01 and abs(z.imag.var() - 1) < 0.01
    assert abs(np.mean(z.real * z.imag)) < 0.01


@pytest.mark.parametrize("beta", [3.0, 6.0])
def test_metropolis_plaquette_closed_form(beta):
    # 2d U(1) with the plaquette action: <Re U_p> = I1(beta)/I0(beta) in infinite volume
    L = 32
    theta, acc = inputs.metropolis_u1_2d(L, L, beta, 600, seed=1234 + int(beta))
    assert 0.2 < acc < 0.95
    # measure over the second half of a longer run for statistics
    samples = []
    th = theta
    for i in range(20):
        th, _ = inputs.metropolis_u1_2d(L, L, beta, 10, seed=99 + i, theta0=th)
        samples.append(np.cos(inputs.plaquette_angles(th, L, L)).mean())
    mean = np.mean(samples)
    err = np.std(samples) / np.sqrt(len(samples)) + 2.0 / (L * L)  # statistics + finite volume
    exact = iv(1, beta) / iv(0, beta)
    assert abs(mean - exact) < 5 * err, (mean, exact, err)


def test_topological_charge_integer():
    L = 16
    theta, _ = inputs.metropolis_u1_2d(L, L, 3.0, 300, seed=5)
    q = inputs.topological_charge(theta, L, L)
    assert abs(q - round(q)) < 1e-9


def test_metropolis_thread_count_independent():
    code = ("import inputs, sys; t,_ = inputs.metropolis_u1_2d(16, 8, 6.0, 30, seed=77); "
            "sys.stdout.write(inputs.field_digest(t))")
    env = dict(os.environ)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env["PYTHONPATH"] = root + os.pathsep + env.get("PYTHONPATH", "")
    outs = []
    for nt in ("1", "3"):
        env["OMP_NUM_THREADS"] = nt
        outs.append(subprocess.check_output([sys.executable, "-c", code], env=env, cwd=root).decode())
    assert outs[0] == outs[1]


def test_cold_start_zero_sweeps():
    theta, _ = inputs.metropolis_u1_2d(8, 8, 6.0, 0, seed=1)
    assert np.all(theta == 0)
    U = inputs.links_from_angles(theta)
    assert np.all(U == 1)


def test_su3_fields_are_special_unitary():
    for U in (inputs.su3_near_identity(500, 0.4, 3, 1), inputs.su3_random(500, 3, 2),
              inputs.su3_links((4, 2, 2, 4), seed=8).reshape(-1, 3, 3)):
        np.testing.assert_allclose(U @ np.conj(np.swapaxes(U, 1, 2)), np.broadcast_to(np.eye(3), U.shape), atol=1e-14)
        np.testing.assert_allclose(np.linalg.det(U), 1.0, atol=1e-14)


def test_su3_near_identity_distribution():
    # projection of 1 + eps H: to first order U = 1 + eps (H_offdiag-antihermitian part); the
    # off-diagonal entries have mean 0 and E|U_01|^2 = eps^2 E|H_01|^2 = eps^2 (1/2 + 1/2) to O(eps^4)
    U = inputs.su3_near_identity(200000, 0.01, 5, 1)
    assert abs(U[:, 0, 1].mean()) < 5 * 0.01 / np.sqrt(len(U))  # five standard errors
    np.testing.assert_allclose(np.mean(np.abs(U[:, 0, 1]) ** 2) / 0.01 ** 2, 1.0, rtol=0.02)


def _plaquette_4d(U, dims):
    L0, L1, L2, L3 = dims
    G = U.reshape(L3, L2, L1, L0, 4, 3, 3)
    tot = []
    for mu in range(4):
        for nu in range(mu + 1, 4):
            Un = np.roll(G[..., nu, :, :], -1, axis=3 - mu)   # U_{x+mu}^nu
            Um = np.roll(G[..., mu, :, :], -1, axis=3 - nu)   # U_{x+nu}^mu
            P = G[..., mu, :, :] @ Un @ np.conj(np.swapaxes(Um, -1, -2)) @ np.conj(np.swapaxes(G[..., nu, :, :], -1, -2))
            tot.append(np.trace(P, axis1=-2, axis2=-1).real.mean() / 3)
    return float(np.mean(tot))


def test_ape_leaves_pure_gauge_field_unchanged():
    # U_x^mu = Omega_x Omega_{x+mu}^dagger: every staple equals the link, so V = U and the
    # projection of a special unitary matrix returns it
    dims = (4, 2, 4, 2)
    V = int(np.prod(dims))
    om = inputs.su3_random(V, 9, 3)
    from oracle.lattice import Lattice
    lat = Lattice(dims)
    U = np.empty((V, 4, 3, 3), dtype=np.complex128)
    for mu in range(4):
        U[:, mu] = om @ np.conj(np.swapaxes(lat.shift(om, mu, +1), 1, 2))
    np.testing.assert_allclose(inputs.ape_smear(U, dims, 0.5, 2), U, atol=1e-13)
    assert abs(_plaquette_4d(U, dims) - 1.0) < 1e-13


def test_ape_smoothing_raises_plaquette():
    dims = (4, 4, 2, 4)
    U0 = inputs.su3_links(dims, seed=2, ape_steps=0)
    p = [_plaquette_4d(inputs.ape_smear(U0, dims, 0.5, k), dims) for k in range(4)]
    assert all(b > a for a, b in zip(p, p[1:])), p


def test_su3_generators_thread_count_independent():
    code = ("import inputs, sys; U = inputs.su3_links((4, 4, 2, 6), seed=7); "
            "sys.stdout.write(inputs.field_digest(U))")
    env = dict(os.environ)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env["PYTHONPATH"] = root + os.pathsep + env.get("PYTHONPATH", "")
    outs = []
    for nt in ("1", "3"):
        env["OMP_NUM_THREADS"] = nt
        outs.append(subprocess.check_output([sys.executable, "-c", code], env=env, cwd=root).decode())
    assert outs[0] == outs[1]
