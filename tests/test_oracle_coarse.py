"""Pins of the oracle's Galerkin coarse operator P^dagger D P (Eq. Galerkin)."""
import numpy as np
import pytest

import inputs
from oracle import coarse, solvers, transfer, wilson
from oracle.lattice import Blocking, Lattice


def _hier2(dims, block, nv, seed=4, U=None, m=0.1):
    lat = Lattice(dims)
    blk = Blocking(lat, block)
    U = inputs.hot_links(*dims, seed=seed) if U is None else U
    op = coarse.WilsonOperator(U, m, lat)
    vecs = np.stack([inputs.gaussian_complex(lat.volume * 2, seed, 100 + k).reshape(-1, 2) for k in range(nv)])
    P, _ = transfer.block_gram_schmidt(vecs, blk)
    return lat, blk, op, P


@pytest.mark.parametrize("dims,block,nv", [((8, 8), (4, 4), 4), ((16, 16), (4, 4), 8), ((8, 4), (4, 4), 3),
                                           ((8, 8), (2, 4), 5), ((4, 8), (1, 2), 2)])
def test_galerkin_matches_dense_PdagDP(dims, block, nv):
    lat, blk, op, P = _hier2(dims, block, nv)
    Yc = coarse.galerkin(op, P, blk)
    Pd = transfer.dense_P(P, blk, 2)
    Dd = wilson.dense_D(op.U, op.m, lat)
    want = Pd.conj().T @ Dd @ Pd
    got = coarse.dense_operator(coarse.StencilOperator(Yc, blk.coarse), Pd.shape[1])
    np.testing.assert_allclose(got, want, atol=1e-13)
    # the block assembly of the stencil agrees with its unit-vector assembly
    np.testing.assert_allclose(solvers.stencil_matrix(coarse.StencilOperator(Yc, blk.coarse)), got, atol=1e-14)


def test_galerkin_beyond_nearest_neighbours_is_zero():
    lat, blk, op, P = _hier2((16, 16), (4, 4), 4)
    Pd = transfer.dense_P(P, blk, 2)
    Ac = Pd.conj().T @ wilson.dense_D(op.U, op.m, lat) @ Pd
    cl = blk.coarse
    nv = 4
    A4 = Ac.reshape(cl.volume, nv, cl.volume, nv)
    js = np.arange(cl.volume)
    near = np.zeros((cl.volume, cl.volume), dtype=bool)
    near[js, js] = True
    for mu in range(2):
        for s in (+1, -1):
            near[js, cl.neighbour(js, mu, s)] = True
    assert np.abs(A4).sum(axis=(1, 3))[~near].max() < 1e-14


def test_three_level_galerkin_matches_dense():
    dims = (16, 16)
    lat, blk1, op, P1 = _hier2(dims, (4, 4), 4)
    Y1 = coarse.galerkin(op, P1, blk1)
    op2 = coarse.StencilOperator(Y1, blk1.coarse)
    blk2 = Blocking(blk1.coarse, (2, 2))
    vecs2 = np.stack([inputs.gaussian_complex(blk1.coarse.volume * 4, 7, 200 + k).reshape(-1, 4) for k in range(3)])
    P2, _ = transfer.block_gram_schmidt(vecs2, blk2)
    Y2 = coarse.galerkin(op2, P2, blk2)
    Pd1 = transfer.dense_P(P1, blk1, 2)
    Pd2 = transfer.dense_P(P2, blk2, 4)
    want = Pd2.conj().T @ Pd1.conj().T @ wilson.dense_D(op.U, op.m, lat) @ Pd1 @ Pd2
    got = solvers.stencil_matrix(coarse.StencilOperator(Y2, blk2.coarse))
    np.testing.assert_allclose(got, want, atol=1e-13)


def test_free_field_constant_vectors_give_scaled_wilson_stencil():
    # U = 1 and block-constant spin vectors v_s = e_s / 4 on 4x4 blocks: 4 of the 16
    # sites sit on each face, 12 hop inside. So the coarse operator is a Wilson stencil
    #   X = (d + m - 2 * (12/16)) I,  Y_{+mu} = -(4/16)/2 (1 - gamma_mu),  Y_{-mu} = -(4/16)/2 (1 + gamma_mu)
    dims, m = (16, 8), 0.13
    lat = Lattice(dims)
    blk = Blocking(lat, (4, 4))
    U = inputs.free_links(*dims)
    op = coarse.WilsonOperator(U, m, lat)
    vecs = np.zeros((2, lat.volume, 2), dtype=np.complex128)
    vecs[0, :, 0] = 1.0
    vecs[1, :, 1] = 1.0
    P, _ = transfer.block_gram_schmidt(vecs, blk)
    Yc = coarse.galerkin(op, P, blk)
    g, _ = wilson.gammas(2)
    one = np.eye(2)
    np.testing.assert_allclose(Yc[:, 0], np.broadcast_to((2 + m - 1.5) * one, Yc[:, 0].shape), atol=1e-14)
    for mu in range(2):
        np.testing.assert_allclose(Yc[:, 1 + 2 * mu], np.broadcast_to(-0.125 * (one - g[mu]), Yc[:, 0].shape),
                                   atol=1e-14)
        np.testing.assert_allclose(Yc[:, 2 + 2 * mu], np.broadcast_to(-0.125 * (one + g[mu]), Yc[:, 0].shape),
                                   atol=1e-14)


def test_mass_shift_moves_only_self_blocks():
    # P^dagger (D + dm) P = P^dagger D P + dm I because P^dagger P = I
    lat, blk, op, P = _hier2((8, 8), (4, 4), 4)
    Y0 = coarse.galerkin(op, P, blk)
    Y1 = coarse.galerkin(op.with_mass(op.m + 0.37), P, blk)
    np.testing.assert_allclose(Y1[:, 0] - Y0[:, 0], np.broadcast_to(0.37 * np.eye(4), Y0[:, 0].shape), atol=1e-14)
    np.testing.assert_allclose(Y1[:, 1:], Y0[:, 1:], atol=1e-15)


def test_coarse_gamma5_hermiticity_with_chirality_blocked_vectors():
    # if every v_k is an eigenvector of gamma_5 (chirality split), the coarse operator is
    # gamma_5^c-hermitian with gamma_5^c = diag(chirality of v_k)
    dims = (8, 8)
    lat = Lattice(dims)
    blk = Blocking(lat, (4, 4))
    U = inputs.hot_links(*dims, seed=31)
    op = coarse.WilsonOperator(U, 0.2, lat)
    raw = [inputs.gaussian_complex(lat.volume * 2, 2, 300 + k).reshape(-1, 2) for k in range(2)]
    vecs = []
    chir = []
    for v in raw:
        for s, c in ((0, 1.0), (1, -1.0)):
            w = np.zeros_like(v)
            w[:, s] = v[:, s]
            vecs.append(w)
            chir.append(c)
    P, _ = transfer.block_gram_schmidt(np.stack(vecs), blk)
    Yc = coarse.galerkin(op, P, blk)
    Ac = solvers.stencil_matrix(coarse.StencilOperator(Yc, blk.coarse))
    G5 = np.kron(np.eye(blk.n_blocks), np.diag(chir))
    np.testing.assert_allclose(G5 @ Ac @ G5, Ac.conj().T, atol=1e-13)
