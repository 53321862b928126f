"""Block-local prolongation and restriction (oracle).

Paper, Eq. P1 and the adaptive step: a vector e' is cut into the pieces e'_j
that agree with e' on block S_j and vanish elsewhere; v_1j = e'_j / |e'_j| and
P_{i,j} = v_{1j,i}. Each further vector e'' is restricted to the blocks, made
orthogonal to the earlier v_sj and normalised, giving P_{i,sj} = v_{sj,i}
(s an intrinsic index on the coarse site). Restriction is P^dagger.

Reading (the paper fixes neither order nor re-orthogonalisation): modified
Gram-Schmidt over the vectors in their given order k = 0..Nv-1, run twice, in
FP64, separately in every block.

A level's field has shape (n_sites, n_int): n_int internal dofs per site
(Ns*Nc on the fine level, Nv of the finer level on coarse levels). A block's
dofs are ordered (in-block position s, internal dof a) -> s*n_int + a.
"""
from __future__ import annotations

import numpy as np

from .lattice import Blocking


def to_blocks(v, blk: Blocking):
    """(n_sites, n_int) -> (n_blocks, block_volume * n_int)."""
    v = np.asarray(v)
    table = blk.site_table()
    return v[table].reshape(blk.n_blocks, -1)


def from_blocks(vb, blk: Blocking, n_int: int):
    """Inverse of to_blocks."""
    table = blk.site_table()
    out = np.empty((blk.lat.volume, n_int), dtype=vb.dtype)
    out[table.reshape(-1)] = vb.reshape(blk.n_blocks * blk.block_volume, n_int)
    return out


def block_gram_schmidt(vectors, blk: Blocking, passes: int = 2):
    """Block-orthonormal basis from Nv level vectors.

    vectors: (Nv, n_sites, n_int). Returns P with shape (n_blocks, N_b, Nv)
    whose columns in every block are orthonormal (P_b^dagger P_b = I).
    Also returns the smallest pre-normalisation norm seen (a degeneracy flag).
    """
    vecs = np.asarray(vectors, dtype=np.complex128)
    nv = vecs.shape[0]
    blocks = np.stack([to_blocks(vecs[k], blk) for k in range(nv)], axis=-1)  # (nb, Nb, Nv)
    P = blocks.copy()
    min_norm = np.inf
    for _ in range(passes):
        for k in range(nv):
            for j in range(k):
                proj = np.einsum("bi,bi->b", P[:, :, j].conj(), P[:, :, k])
                P[:, :, k] -= proj[:, None] * P[:, :, j]
            nrm = np.sqrt(np.einsum("bi,bi->b", P[:, :, k].conj(), P[:, :, k]).real)
            min_norm = min(min_norm, float(nrm.min()))
            P[:, :, k] /= nrm[:, None]
    return P, min_norm


def restrict(P, r, blk: Blocking):
    """Coarse vector r_c[b, k] = sum_i conj(P[b, i, k]) r_b[i]  (P^dagger r)."""
    rb = to_blocks(r, blk)
    return np.einsum("bik,bi->bk", P.conj(), rb)


def prolong(P, e, blk: Blocking, n_int: int):
    """Fine vector (P e)_b[i] = sum_k P[b, i, k] e[b, k]."""
    xb = np.einsum("bik,bk->bi", P, np.asarray(e).reshape(blk.n_blocks, -1))
    return from_blocks(xb, blk, n_int)


def dense_P(P, blk: Blocking, n_int: int):
    """The prolongator as a dense (n_fine_dofs, n_coarse_dofs) matrix (tiny lattices only)."""
    nb, Nb, nv = P.shape
    n_f = blk.lat.volume * n_int
    M = np.zeros((n_f, nb * nv), dtype=np.complex128)
    e = np.zeros((nb, nv), dtype=np.complex128)
    for col in range(nb * nv):
        e[:] = 0
        e.reshape(-1)[col] = 1
        M[:, col] = prolong(P, e, blk, n_int).reshape(-1)
    return M
