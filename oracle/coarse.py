"""Level operators and the Galerkin coarse operator (oracle).

Paper, Eq. Galerkin: A^(l+1) = P^(l,l+1)dagger A^(l) P^(l,l+1). Here (as in the
solver this oracle checks) the operator coarsened is D itself, so the coarse
operator is P^dagger D P. Because D couples nearest neighbours only and every
column of P lives on one block, P^dagger D P couples a coarse site only to
itself and its nearest coarse neighbours. It is stored as a stencil

    y_j = sum_dir Y[j, dir] x_{j + offset(dir)}

with dir 0 = self, dir 1 + 2 mu = +mu (source j + mu-hat), dir 2 + 2 mu = -mu
(source j - mu-hat); each Y[j, dir] is an (Nv x Nv) complex block.

Every level operator exposes ``part(dir, x)``: the contribution to (A x) that
comes from direction dir (dir 0: the site-local term), so that A x is the sum
of the parts. The Galerkin blocks split the fine hops of direction dir into
those that stay inside a block (they belong to the coarse self term) and those
that cross into the neighbouring block (they belong to the coarse dir term).
"""
from __future__ import annotations

import numpy as np

from . import wilson
from .lattice import Blocking, Lattice
from .transfer import from_blocks, to_blocks


def n_dirs(d: int) -> int:
    return 2 * d + 1


def dir_of(mu: int, sign: int) -> int:
    return 1 + 2 * mu + (0 if sign > 0 else 1)


class WilsonOperator:
    """Fine-level D as a level operator (fields (V, Ns*Nc))."""

    def __init__(self, U, m: float, lat: Lattice, Nc: int = 1):
        self.U = np.asarray(U, dtype=np.complex128)
        self.m = float(m)
        self.lat = lat
        self.Nc = Nc
        self.n_int = wilson.n_spin(lat.d) * Nc

    def part(self, dirn: int, x):
        x = np.asarray(x, dtype=np.complex128).reshape(self.lat.volume, self.n_int)
        if dirn == 0:
            return wilson.diag_value(self.lat, self.m) * x
        mu, back = divmod(dirn - 1, 2)
        return wilson.hop(self.U, x, self.lat, mu, -1 if back else +1)

    def apply(self, x):
        x = np.asarray(x, dtype=np.complex128).reshape(self.lat.volume, self.n_int)
        return wilson.apply_D(self.U, x, self.m, self.lat)

    def with_mass(self, m: float):
        return WilsonOperator(self.U, m, self.lat, self.Nc)


class StencilOperator:
    """Coarse-level operator given by its stencil blocks Y[j, dir, a, b]."""

    def __init__(self, Y, lat: Lattice):
        self.Y = np.asarray(Y, dtype=np.complex128)
        self.lat = lat
        self.n_int = self.Y.shape[-1]
        assert self.Y.shape == (lat.volume, n_dirs(lat.d), self.n_int, self.n_int)

    def part(self, dirn: int, x):
        x = np.asarray(x, dtype=np.complex128).reshape(self.lat.volume, self.n_int)
        if dirn == 0:
            src = x
        else:
            mu, back = divmod(dirn - 1, 2)
            src = self.lat.shift(x, mu, -1 if back else +1)
        return np.einsum("jab,jb->ja", self.Y[:, dirn], src)

    def apply(self, x):
        out = self.part(0, x)
        for dirn in range(1, n_dirs(self.lat.d)):
            out = out + self.part(dirn, x)
        return out


def galerkin(op, P, blk: Blocking):
    """Coarse stencil Y_c of P^dagger A P for a level operator A and block-orthonormal P.

    P: (n_blocks, N_b, Nv) as returned by transfer.block_gram_schmidt.
    Returns Y_c with shape (n_blocks, 2d+1, Nv, Nv).
    """
    lat = op.lat
    d = lat.d
    nb, Nb, nv = P.shape
    n_int = op.n_int
    Yc = np.zeros((nb, n_dirs(d), nv, nv), dtype=np.complex128)
    sites = np.arange(lat.volume)
    for k in range(nv):
        # the field equal to column k of P_b in every block b
        W = from_blocks(P[:, :, k], blk, n_int)
        self_part = op.part(0, W)
        cross = {}
        for mu in range(d):
            for sign in (+1, -1):
                dirn = dir_of(mu, sign)
                h = op.part(dirn, W)
                face = blk.on_forward_face(sites, mu) if sign > 0 else blk.on_backward_face(sites, mu)
                self_part = self_part + np.where(face[:, None], 0, h)
                cross[dirn] = np.where(face[:, None], h, 0)
        Yc[:, 0, :, k] = np.einsum("bia,bi->ba", P.conj(), to_blocks(self_part, blk))
        for dirn, h in cross.items():
            Yc[:, dirn, :, k] = np.einsum("bia,bi->ba", P.conj(), to_blocks(h, blk))
    return Yc


def dense_operator(op, n_dofs: int):
    """Matrix of a level operator from unit vectors (tiny lattices only)."""
    M = np.zeros((n_dofs, n_dofs), dtype=np.complex128)
    e = np.zeros(n_dofs, dtype=np.complex128)
    for col in range(n_dofs):
        e[:] = 0
        e[col] = 1
        M[:, col] = op.apply(e.reshape(op.lat.volume, op.n_int)).reshape(-1)
    return M
