"""Lattice geometry and index maps (oracle).

Paper: the fine lattice is partitioned geometrically into fixed blocks S_j of
neighbouring sites (4x4 squares in 2d), which keeps a regular coarse lattice
(section on blocking, after Eq. P1). Conventions (stated here, also used by the
library's boundary):

  site        x = x0 + L0*(x1 + L1*(x2 + L2*x3))            x0 fastest
  block       b = sum_mu (x_mu // B_mu) * prod_{nu<mu} (L_nu/B_nu)
  in-block    s = sum_mu (x_mu %  B_mu) * prod_{nu<mu} B_nu
  coarse site j = b   (coarse coordinates x_mu // B_mu)

Fields are numpy arrays whose first axis is the site index; for stencil work
they are reshaped to (L_{d-1}, ..., L_1, L_0, ...) so that axis d-1-mu is the
mu direction.
"""
from __future__ import annotations

import numpy as np


class Lattice:
    """A periodic d-dimensional lattice with extents dims = (L0, L1, ...)."""

    def __init__(self, dims):
        self.dims = tuple(int(L) for L in dims)
        self.d = len(self.dims)
        self.volume = int(np.prod(self.dims))

    # -- coordinates -------------------------------------------------------
    def coords(self, x):
        """Coordinates (x0, x1, ...) of site index x (array or int)."""
        x = np.asarray(x, dtype=np.int64)
        out = []
        for L in self.dims:
            out.append(x % L)
            x = x // L
        return tuple(out)

    def index(self, coords):
        """Site index from coordinates (each taken modulo the extent)."""
        x = np.zeros_like(np.asarray(coords[0], dtype=np.int64))
        stride = 1
        for mu, L in enumerate(self.dims):
            x = x + (np.asarray(coords[mu], dtype=np.int64) % L) * stride
            stride *= L
        return x

    def neighbour(self, x, mu, sign):
        """Index of x + sign * mu-hat with periodic wrap."""
        c = list(self.coords(x))
        c[mu] = c[mu] + sign
        return self.index(c)

    # -- stencil views -----------------------------------------------------
    def grid_shape(self):
        return tuple(reversed(self.dims))

    def axis(self, mu):
        """numpy axis of direction mu in the grid view."""
        return self.d - 1 - mu

    def to_grid(self, field):
        return field.reshape(self.grid_shape() + field.shape[1:])

    def from_grid(self, grid):
        return grid.reshape((self.volume,) + grid.shape[self.d:])

    def shift(self, field, mu, sign):
        """Returns g with g[x] = field[x + sign*mu-hat] (periodic)."""
        g = self.to_grid(field)
        return self.from_grid(np.roll(g, -sign, axis=self.axis(mu)))


class Blocking:
    """Geometric blocking of a lattice into blocks of extents B = (B0, B1, ...)."""

    def __init__(self, lat: Lattice, block):
        self.lat = lat
        self.block = tuple(int(b) for b in block)
        if len(self.block) != lat.d:
            raise ValueError("block rank must equal lattice rank")
        for L, B in zip(lat.dims, self.block):
            if B <= 0 or L % B:
                raise ValueError(f"lattice extent {L} not divisible by block {B}")
        self.coarse = Lattice([L // B for L, B in zip(lat.dims, self.block)])
        self.block_volume = int(np.prod(self.block))
        self.n_blocks = self.coarse.volume

    def block_of(self, x):
        """Block (= coarse site) index b of fine site x."""
        c = self.lat.coords(x)
        b = np.zeros_like(np.asarray(c[0]))
        stride = 1
        for mu in range(self.lat.d):
            b = b + (c[mu] // self.block[mu]) * stride
            stride *= self.lat.dims[mu] // self.block[mu]
        return b

    def site_in_block(self, x):
        """Position s of fine site x inside its block."""
        c = self.lat.coords(x)
        s = np.zeros_like(np.asarray(c[0]))
        stride = 1
        for mu in range(self.lat.d):
            s = s + (c[mu] % self.block[mu]) * stride
            stride *= self.block[mu]
        return s

    def fine_site(self, b, s):
        """Inverse map: fine site index of (block b, in-block position s)."""
        b = np.asarray(b, dtype=np.int64)
        s = np.asarray(s, dtype=np.int64)
        coords = []
        for mu in range(self.lat.d):
            nb = self.lat.dims[mu] // self.block[mu]
            coords.append((b % nb) * self.block[mu] + (s % self.block[mu]))
            b = b // nb
            s = s // self.block[mu]
        return self.lat.index(coords)

    def site_table(self):
        """table[b, s] = fine site index; shape (n_blocks, block_volume)."""
        b = np.arange(self.n_blocks)[:, None]
        s = np.arange(self.block_volume)[None, :]
        return self.fine_site(b, s)

    def on_forward_face(self, x, mu):
        """True where x + mu-hat lies in a different block position (x_mu % B_mu == B_mu - 1)."""
        return (self.lat.coords(x)[mu] % self.block[mu]) == self.block[mu] - 1

    def on_backward_face(self, x, mu):
        """True where x - mu-hat lies in a different block position (x_mu % B_mu == 0)."""
        return (self.lat.coords(x)[mu] % self.block[mu]) == 0
