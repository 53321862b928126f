"""Planted mistakes in the oracle (on the CPU) must be caught by its pins.

Each case monkeypatches one oracle function with a plausible error (a dropped
term, a wrong sign, a wrong link, a transposed block) and asserts that at least
one of the closed-form / invariant checks used by the pin tests fails.
"""
import numpy as np
import pytest

import inputs
from oracle import coarse, transfer, wilson
from oracle.lattice import Blocking, Lattice


def _pins_pass(apply_D):
    """The Wilson pins (free spectrum, plane wave, gamma_5-hermiticity, covariance) as booleans."""
    ok = []
    dims, m = (4, 6), 0.1
    lat = Lattice(dims)
    # free spectrum (closed form)
    n = lat.volume * 2
    M = np.zeros((n, n), dtype=np.complex128)
    U1 = inputs.free_links(*dims)
    for c in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[c] = 1
        M[:, c] = apply_D(U1, e.reshape(-1, 2), m, lat).reshape(-1)
    ev = np.linalg.eigvals(M)
    ps = np.meshgrid(2 * np.pi * np.arange(4) / 4, 2 * np.pi * np.arange(6) / 6, indexing="ij")
    re = 2 + m - np.cos(ps[0]).reshape(-1) - np.cos(ps[1]).reshape(-1)
    im = np.sqrt(np.sin(ps[0]).reshape(-1) ** 2 + np.sin(ps[1]).reshape(-1) ** 2)
    want = np.concatenate([re + 1j * im, re - 1j * im])
    srt = lambda v: v[np.lexsort((np.round(v.imag, 8), np.round(v.real, 8)))]
    ok.append(np.allclose(srt(ev), srt(want), atol=1e-10))
    # plane wave
    x0, x1 = lat.coords(np.arange(lat.volume))
    p = (2 * np.pi / 4, 2 * np.pi * 2 / 6)
    u = np.array([0.3 - 0.2j, 1.1 + 0.5j])
    ph = np.exp(1j * (p[0] * x0 + p[1] * x1))[:, None]
    g, _ = wilson.gammas(2)
    Dp = (2 + m - np.cos(p[0]) - np.cos(p[1])) * np.eye(2) + 1j * (np.sin(p[0]) * g[0] + np.sin(p[1]) * g[1])
    ok.append(np.allclose(apply_D(U1, ph * u[None, :], m, lat), ph * (Dp @ u)[None, :], atol=1e-12))
    # gamma_5-hermiticity and covariance on a random field
    U = inputs.hot_links(*dims, seed=3)
    a = inputs.gaussian_complex(n, 1, 1).reshape(-1, 2)
    b = inputs.gaussian_complex(n, 1, 2).reshape(-1, 2)
    g5 = np.array([1.0, -1.0])
    lhs = np.vdot(a, g5 * apply_D(U, g5 * b, m, lat))
    rhs = np.vdot(apply_D(U, a, m, lat), b)
    ok.append(abs(lhs - rhs) < 1e-12 * abs(rhs))
    om = inputs.u1_phases(lat.volume, 5, 9)
    Ug = wilson.gauge_transform(U, om, lat)[:, :, 0, 0]
    ok.append(np.allclose(apply_D(Ug, om[:, None] * b, m, lat), om[:, None] * apply_D(U, b, m, lat), atol=1e-12))
    return ok


def test_unmutated_oracle_passes_all():
    assert all(_pins_pass(wilson.apply_D))


def _mutant(kind):
    def apply_D(U, psi, m, lat):
        psi = np.asarray(psi, dtype=np.complex128)
        diag = (2 * lat.d + m) if kind == "diag_2d" else (lat.d + m)
        out = diag * psi
        g, _ = wilson.gammas(lat.d)
        one = np.eye(2)
        for mu in range(lat.d):
            fwd_proj = one + g[mu] if kind == "proj_sign" else one - g[mu]
            bwd_proj = one - g[mu] if kind == "proj_sign" else one + g[mu]
            f = U[:, mu][:, None] * lat.shift(psi, mu, +1)
            out = out - 0.5 * f @ fwd_proj.T
            if kind == "drop_backward" and mu == 1:
                continue
            if kind == "no_conj":
                link = lat.shift(U[:, mu], mu, -1)
            elif kind == "wrong_site":
                link = U[:, mu].conj()
            else:
                link = lat.shift(U[:, mu], mu, -1).conj()
            bk = link[:, None] * lat.shift(psi, mu, -1)
            out = out - 0.5 * bk @ bwd_proj.T
        return out
    return apply_D


@pytest.mark.parametrize("kind", ["diag_2d", "proj_sign", "drop_backward", "no_conj", "wrong_site"])
def test_planted_wilson_mistake_is_caught(kind):
    assert not all(_pins_pass(_mutant(kind))), kind


def test_planted_galerkin_transpose_is_caught(monkeypatch):
    dims = (8, 8)
    lat = Lattice(dims)
    blk = Blocking(lat, (4, 4))
    U = inputs.hot_links(*dims, seed=4)
    op = coarse.WilsonOperator(U, 0.1, lat)
    vecs = np.stack([inputs.gaussian_complex(lat.volume * 2, 4, 100 + k).reshape(-1, 2) for k in range(3)])
    P, _ = transfer.block_gram_schmidt(vecs, blk)
    Pd = transfer.dense_P(P, blk, 2)
    want = Pd.conj().T @ wilson.dense_D(U, 0.1, lat) @ Pd
    Yc = coarse.galerkin(op, P, blk)
    n = Pd.shape[1]
    good = coarse.dense_operator(coarse.StencilOperator(Yc, blk.coarse), n)
    assert np.allclose(good, want, atol=1e-13)
    bad = coarse.dense_operator(coarse.StencilOperator(np.swapaxes(Yc, 2, 3).copy(), blk.coarse), n)
    assert not np.allclose(bad, want, atol=1e-6)
    # swapping the +mu and -mu blocks: on a 2x2 coarse lattice those neighbours coincide, so use 4x2
    lat4 = Lattice((16, 8))
    blk4 = Blocking(lat4, (4, 4))
    U4 = inputs.hot_links(16, 8, seed=4)
    vec4 = np.stack([inputs.gaussian_complex(lat4.volume * 2, 4, 100 + k).reshape(-1, 2) for k in range(3)])
    P4, _ = transfer.block_gram_schmidt(vec4, blk4)
    Y4 = coarse.galerkin(coarse.WilsonOperator(U4, 0.1, lat4), P4, blk4)
    Y4[:, [1, 2]] = Y4[:, [2, 1]]
    Pd4 = transfer.dense_P(P4, blk4, 2)
    want4 = Pd4.conj().T @ wilson.dense_D(U4, 0.1, lat4) @ Pd4
    assert not np.allclose(coarse.dense_operator(coarse.StencilOperator(Y4, blk4.coarse), Pd4.shape[1]), want4,
                           atol=1e-6)
