"""Pins of the oracle's index maps, block Gram-Schmidt, P and P^dagger."""
import os

import numpy as np
import pytest

import inputs
from oracle import transfer
from oracle.lattice import Blocking, Lattice

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_index_maps_hand_worked_example():
    lat = Lattice((8, 4))
    blk = Blocking(lat, (4, 2))
    for line in open(os.path.join(GOLDEN, "index_maps_8x4_b4x2.txt")):
        if line.startswith("#") or not line.strip():
            continue
        x0, x1, x, b, s = (int(t) for t in line.split())
        assert lat.index((x0, x1)) == x
        assert blk.block_of(x) == b
        assert blk.site_in_block(x) == s
        assert blk.fine_site(b, s) == x


@pytest.mark.parametrize("dims,block", [((64, 64), (4, 4)), ((16, 16), (2, 2)), ((8, 12), (4, 3)),
                                        ((4, 4, 4, 8), (2, 2, 2, 4))])
def test_index_maps_round_trip(dims, block):
    lat = Lattice(dims)
    blk = Blocking(lat, block)
    x = np.arange(lat.volume)
    b, s = blk.block_of(x), blk.site_in_block(x)
    assert np.array_equal(blk.fine_site(b, s), x)
    # every (b, s) pair appears exactly once
    assert len(set(zip(b.tolist(), s.tolist()))) == lat.volume
    assert b.max() == blk.n_blocks - 1 and s.max() == blk.block_volume - 1
    # the block of a site is its coarse-lattice site
    cc = [c // B for c, B in zip(lat.coords(x), block)]
    assert np.array_equal(blk.coarse.index(cc), b)


def _setup_vectors(dims, block, nv, n_int, seed=3):
    lat = Lattice(dims)
    blk = Blocking(lat, block)
    vecs = np.stack([inputs.gaussian_complex(lat.volume * n_int, seed, k).reshape(lat.volume, n_int)
                     for k in range(nv)])
    return lat, blk, vecs


@pytest.mark.parametrize("dims,block,nv,n_int", [((16, 16), (4, 4), 8, 2), ((8, 8), (2, 2), 8, 8)])
def test_block_gram_schmidt_orthonormal_and_span(dims, block, nv, n_int):
    lat, blk, vecs = _setup_vectors(dims, block, nv, n_int)
    P, min_norm = transfer.block_gram_schmidt(vecs, blk)
    assert min_norm > 1e-3
    for b in range(blk.n_blocks):
        np.testing.assert_allclose(P[b].conj().T @ P[b], np.eye(nv), atol=1e-14)
    # span preserved: every original block vector lies in span(P_b)
    vb = np.stack([transfer.to_blocks(vecs[k], blk) for k in range(nv)], axis=-1)
    for b in range(blk.n_blocks):
        resid = vb[b] - P[b] @ (P[b].conj().T @ vb[b])
        assert np.linalg.norm(resid) < 1e-12 * np.linalg.norm(vb[b])
    # Gram-Schmidt is triangular: P_b[:, k] lies in span of the first k+1 inputs
    for b in range(0, blk.n_blocks, 7):
        for k in range(nv):
            Q, _ = np.linalg.qr(vb[b][:, :k + 1])
            r = P[b][:, k] - Q @ (Q.conj().T @ P[b][:, k])
            assert np.linalg.norm(r) < 1e-12


def test_block_gram_schmidt_keeps_orthonormal_input():
    lat = Lattice((8, 8))
    blk = Blocking(lat, (4, 4))
    # block-orthonormal input: unit vectors on distinct dofs of each block
    nv = 4
    vecs = np.zeros((nv, lat.volume, 2), dtype=np.complex128)
    table = blk.site_table()
    for k in range(nv):
        vecs[k, table[:, k], 0] = np.exp(0.3j * k)
    P, _ = transfer.block_gram_schmidt(vecs, blk)
    for k in range(nv):
        np.testing.assert_allclose(transfer.from_blocks(P[:, :, k], blk, 2), vecs[k], atol=1e-15)


def test_restrict_is_adjoint_of_prolong():
    lat, blk, vecs = _setup_vectors((16, 8), (4, 4), 6, 2)
    P, _ = transfer.block_gram_schmidt(vecs, blk)
    r = inputs.gaussian_complex(lat.volume * 2, 9, 1).reshape(-1, 2)
    e = inputs.gaussian_complex(blk.n_blocks * 6, 9, 2).reshape(-1, 6)
    lhs = np.vdot(transfer.restrict(P, r, blk), e)
    rhs = np.vdot(r, transfer.prolong(P, e, blk, 2))
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)
    # P^dagger P = I on coarse vectors
    np.testing.assert_allclose(transfer.restrict(P, transfer.prolong(P, e, blk, 2), blk), e, atol=1e-13)


def test_dense_P_is_block_local():
    lat, blk, vecs = _setup_vectors((8, 8), (4, 4), 3, 2)
    P, _ = transfer.block_gram_schmidt(vecs, blk)
    M = transfer.dense_P(P, blk, 2)
    np.testing.assert_allclose(M.conj().T @ M, np.eye(M.shape[1]), atol=1e-14)
    b_of_row = np.repeat(blk.block_of(np.arange(lat.volume)), 2)
    b_of_col = np.repeat(np.arange(blk.n_blocks), 3)
    mask = b_of_row[:, None] != b_of_col[None, :]
    assert np.all(M[mask] == 0)
