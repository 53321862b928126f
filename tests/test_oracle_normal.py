"""Pins of the oracle's MG-CG on the normal equations (the paper's own experiment): each function is
checked against a dense construction of what it stands for on tiny lattices, so a dropped term, a
wrong adjoint, a transposed block or a wrong neighbour fails here."""
import numpy as np
import pytest
import scipy.linalg

import inputs
from oracle import normal, wilson
from oracle.lattice import Blocking, Lattice
from oracle.rng import gaussian_vector
from oracle.transfer import block_gram_schmidt, dense_P


def _setup(L=12, m=0.1, seed=3):
    lat = Lattice((L, L))
    U = inputs.hot_links(L, L, seed=seed)
    return lat, U, normal.NormalOperator(U, m, lat)


def test_normal_operator_is_dense_DdagD_and_positive():
    lat, U, op = _setup(L=6)
    D = wilson.dense_D(U, 0.1, lat)
    A = normal.dense_matrix(op)
    assert np.abs(A - D.conj().T @ D).max() < 1e-13
    assert np.abs(A - A.conj().T).max() < 1e-13
    assert np.linalg.eigvalsh(A).min() > 0


def test_galerkin9_equals_dense_PdagAP_on_two_levels():
    # 12^2 -> 6^2 -> 3^2 with 2 x 2 blocks: the fine D^dagger D, then a 9-point stencil coarsened again
    lat, U, op = _setup()
    A = normal.dense_matrix(op)
    for level, (n_int, nv) in enumerate([(2, 4), (4, 3)]):
        blk = Blocking(op.lat, (2, 2))
        vecs = [gaussian_vector(op.lat.volume * n_int, 5, k, level).reshape(op.lat.volume, n_int) for k in range(nv)]
        P, _ = block_gram_schmidt(vecs, blk)
        Y = normal.galerkin9(op, P, blk)
        Pd = dense_P(P, blk, n_int)
        want = Pd.conj().T @ A @ Pd
        coarse = normal.Stencil9(Y, blk.coarse)
        got = normal.dense_matrix(coarse)
        assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max(), level
        op, A = coarse, got


def test_colour_period_needs_three_coarse_sites():
    assert normal.colour_period(8) == 4 and normal.colour_period(9) == 3 and normal.colour_period(5) == 5
    with pytest.raises(ValueError):
        normal.colour_period(2)


def test_frozen_smoother_is_the_real_polynomial():
    lat, U, op = _setup(L=6)
    A = normal.dense_matrix(op)
    b = gaussian_vector(lat.volume * 2, 9, 0, 0).reshape(lat.volume, 2)
    a1, a2 = normal.mr_coefficients(op.apply, b, 0.8)
    # the step lengths are those of two MR steps: alpha = omega <A r, r> / |A r|^2
    r = b.reshape(-1)
    Ar = A @ r
    assert abs(a1 - 0.8 * np.vdot(Ar, r).real / np.vdot(Ar, Ar).real) < 1e-14
    R = (a1 + a2) * np.eye(len(A)) - a1 * a2 * A
    x, res = normal.frozen_smooth(op.apply, [a1, a2], b)
    assert np.abs(x.reshape(-1) - R @ b.reshape(-1)).max() < 1e-13
    assert np.abs(res.reshape(-1) - (b.reshape(-1) - A @ x.reshape(-1))).max() < 1e-12


def test_vcycle_is_the_hermitian_two_grid_formula():
    # two levels with an exact coarse solve: V = 2R - R A R + (1 - R A) P A_c^-1 P^dagger (1 - A R)
    lat, U, op = _setup(L=12)
    h = normal.NormalHierarchy(U, 0.1, lat, [(2, 2)], [4])
    vecs = [gaussian_vector(lat.volume * 2, 7, k, 0).reshape(lat.volume, 2) for k in range(4)]
    h.build_level(0, vecs)
    h.prepare()
    A = normal.dense_matrix(op)
    n = len(A)
    a1, a2 = h.alphas[0]
    R = (a1 + a2) * np.eye(n) - a1 * a2 * A
    Pd = dense_P(h.P[0], h.blk[0], 2)
    Ac = Pd.conj().T @ A @ Pd
    I = np.eye(n)
    want = 2 * R - R @ A @ R + (I - R @ A) @ Pd @ np.linalg.solve(Ac, Pd.conj().T) @ (I - A @ R)
    V = np.zeros((n, n), dtype=complex)
    for i in range(n):
        e = np.zeros(n, dtype=complex)
        e[i] = 1
        V[:, i] = h.vcycle(0, e.reshape(lat.volume, 2)).reshape(-1)
    assert np.abs(V - want).max() <= 1e-11 * np.abs(want).max()
    assert np.abs(V - V.conj().T).max() <= 1e-12 * np.abs(V).max()
    assert np.linalg.eigvalsh((V + V.conj().T) / 2).min() > 0


def test_mgcg_and_cg_solve_the_wilson_system():
    lat, U, op = _setup(L=12)
    h = normal.adaptive_setup(U, 0.1, lat, [(2, 2), (2, 2)], [4, 3], n_pass=2, nu_setup=4)
    chi = np.zeros((lat.volume, 2), dtype=complex)
    chi[0, 0] = 1
    want = scipy.linalg.solve(wilson.dense_D(U, 0.1, lat), chi.reshape(-1))
    x, info = normal.mgcg_solve(h, chi, 1e-12)
    assert np.linalg.norm(x.reshape(-1) - want) <= 1e-9 * np.linalg.norm(want), info
    rhs = wilson.apply_Ddag(U, chi, 0.1, lat)
    x2, info2 = normal.cg(op.apply, rhs, 1e-12, 5000)
    assert np.linalg.norm(x2.reshape(-1) - want) <= 1e-9 * np.linalg.norm(want)
    # the V-cycle preconditioner cuts the CG iterations, and an exact inverse needs one
    assert info["iters"] < info2["iters"]
    Ainv = np.linalg.inv(normal.dense_matrix(op))
    _, info3 = normal.cg(op.apply, rhs, 1e-12, 10, precond=lambda r: (Ainv @ r.reshape(-1)).reshape(r.shape))
    assert info3["iters"] == 1
