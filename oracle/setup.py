"""Adaptive multigrid setup and the level hierarchy (oracle).

Paper, adaptive procedure (Eq. relax, Eq. P1 and the passes that follow):
  * pass 1: relax the homogeneous problem A e = 0 from a random e (nu steps),
    cut e' into blocks, normalise -> v_1j, P_{i,j} = v_{1j,i};
  * later passes: run the V-cycle built from the current P on the homogeneous
    problem; the error e'' that survives is cut into blocks, orthogonalised
    against the earlier v_sj and normalised -> v_2j, ...; P_{i,sj} = v_{sj,i};
  * the procedure is recursive: the coarse operator P^dagger A P is coarsened
    the same way.

Readings taken here (the paper fixes neither nu, the stopping rule nor the
order of recursion):
  * Nv random vectors are drawn at once (rng.gaussian_vector) and relaxed
    with nu_setup MR iterations (omega) on A x = 0 starting from x = v;
  * a fixed number n_pass of passes; passes 2..n_pass replace every vector by
    v - V(A v), one V-cycle error-propagation step on A x = 0 with the
    hierarchy of the previous pass, before block Gram-Schmidt and the
    Galerkin rebuild;
  * chirality split (params.chiral_split, the 4d SU(3) hierarchy): before the
    Gram-Schmidt of the fine level every vector v_k is replaced by the pair
    (1 + gamma_5) v_k / 2, (1 - gamma_5) v_k / 2, giving 2 Nv coarse dofs per site;
  * recursion: after every pass on level l the next level is rebuilt from
    the new coarse operator; it receives only its first pass (relaxation,
    Gram-Schmidt, Galerkin) except after the last pass on level l, when it
    receives its full n_pass passes. The coarsest level is then prepared
    for its exact solve.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import coarse, rng, transfer, wilson
from .lattice import Blocking, Lattice
from .solvers import CoarsestSolver, OpCounter, mr, vcycle


@dataclasses.dataclass
class MGParams:
    levels: int = 2
    blocks: tuple = ((4, 4),)
    Nv: tuple = (8,)
    nu_pre: int = 4
    nu_post: int = 4
    omega: float = 0.8
    n_pass: int = 5
    nu_setup: int = 8
    gcr_restart: int = 16
    max_iter: int = 500
    coarsest_lu_max: int = 2048
    coarsest_tol: float = 1e-12
    coarsest_restart: int = 16
    coarsest_max_iter: int = 20000
    seed: int = 20070704
    chiral_split: bool = False


class Hierarchy:
    """Operators, blockings and prolongators of all levels (0 = finest)."""

    def __init__(self, fine_op, params: MGParams):
        self.params = params
        self.n_levels = params.levels
        self.ops = [fine_op] + [None] * (params.levels - 1)
        self.blk = [None] * (params.levels - 1)
        self.P = [None] * (params.levels - 1)
        self.vecs = [None] * (params.levels - 1)
        self.coarsest = None
        lat = fine_op.lat
        for l in range(params.levels - 1):
            self.blk[l] = Blocking(lat, params.blocks[l])
            lat = self.blk[l].coarse

    def n_int(self, level: int) -> int:
        if level == 0:
            return self.ops[0].n_int
        return self.params.Nv[level - 1] * (2 if self.split(level - 1) else 1)

    def split(self, level: int) -> bool:
        """Chirality split of the vectors that build level + 1 (the fine level only)."""
        return bool(self.params.chiral_split) and level == 0

    def restrict(self, level: int, r):
        return transfer.restrict(self.P[level], r, self.blk[level])

    def prolong(self, level: int, e):
        return transfer.prolong(self.P[level], e, self.blk[level], self.n_int(level))

    def build_level(self, level: int, vectors):
        """Block Gram-Schmidt of ``vectors`` (after the chirality split where it applies) and
        the Galerkin coarse operator of the next level."""
        self.vecs[level] = [np.array(v) for v in vectors]
        if self.split(level):
            vectors = chirality_split(vectors, self.ops[level].lat, self.ops[level].Nc)
        self.P[level], _ = transfer.block_gram_schmidt(np.stack(vectors), self.blk[level])
        Yc = coarse.galerkin(self.ops[level], self.P[level], self.blk[level])
        self.ops[level + 1] = coarse.StencilOperator(Yc, self.blk[level].coarse)

    def prepare_coarsest(self):
        p = self.params
        self.coarsest = CoarsestSolver(self.ops[-1], p.coarsest_lu_max, p.coarsest_tol, p.coarsest_restart,
                                       p.coarsest_max_iter)


def chirality_split(vectors, lat: Lattice, Nc: int):
    """[P+ v_0, ..., P+ v_{Nv-1}, P- v_0, ..., P- v_{Nv-1}] with P+- = (1 +- gamma_5) / 2.

    Applied to the fine near-null vectors before block Gram-Schmidt (a reading: the paper
    has one vector set; the split doubles the coarse dofs, each coarse dof of one
    chirality, so that the coarse operator inherits gamma_5-hermiticity with the coarse
    gamma_5 = diag(1, ..., 1, -1, ..., -1)).
    """
    plus, minus = [], []
    for v in vectors:
        v = np.asarray(v, dtype=np.complex128)
        g5v = wilson.apply_gamma5(v, lat, Nc).reshape(v.shape)
        plus.append(0.5 * (v + g5v))
        minus.append(0.5 * (v - g5v))
    return plus + minus


def initial_vectors(hier: Hierarchy, level: int):
    p = hier.params
    lat = hier.ops[level].lat
    n_int = hier.n_int(level)
    n = lat.volume * n_int
    return [rng.gaussian_vector(n, p.seed, k, level).reshape(lat.volume, n_int) for k in range(p.Nv[level])]


def relax_null(hier: Hierarchy, level: int, v, counter=None):
    """nu_setup MR iterations on A x = 0 from x = v (paper, Eq. relax, with MR as relaxation)."""
    p = hier.params
    A = hier.ops[level].apply
    x, _ = mr(A, np.zeros_like(v), p.nu_setup, p.omega, x0=v, counter=counter, level=level)
    return x


def adapt_vector(hier: Hierarchy, level: int, v, counter=None):
    """v - V(A v): one V-cycle on the homogeneous problem A x = 0 from x = v."""
    Av = hier.ops[level].apply(v)
    if counter is not None:
        counter.add(level)
    return v - vcycle(hier, level, Av, counter=counter)


def setup_level(hier: Hierarchy, level: int, full: bool, counter=None):
    p = hier.params
    vecs = [relax_null(hier, level, v, counter) for v in initial_vectors(hier, level)]
    n_pass = p.n_pass if full else 1
    for pss in range(1, n_pass + 1):
        if pss > 1:
            vecs = [adapt_vector(hier, level, v, counter) for v in vecs]
        hier.build_level(level, vecs)
        if level + 1 == hier.n_levels - 1:
            hier.prepare_coarsest()
        else:
            setup_level(hier, level + 1, full=(full and pss == n_pass), counter=counter)


def adaptive_setup(U, m: float, lat: Lattice, params: MGParams, Nc: int = 1, counter=None) -> Hierarchy:
    """The full adaptive setup for D(U) with mass m."""
    hier = Hierarchy(coarse.WilsonOperator(U, m, lat, Nc), params)
    if counter is None:
        counter = OpCounter()
    setup_level(hier, 0, full=True, counter=counter)
    hier.setup_counter = counter
    return hier


def update_mass(hier: Hierarchy, m_new: float):
    """Reuse the near-null vectors for another mass (paper: setup at the lightest mass only,
    reused for the heavier ones). The Galerkin operators are rebuilt from the kept P."""
    hier.ops[0] = hier.ops[0].with_mass(m_new)
    for level in range(hier.n_levels - 1):
        Yc = coarse.galerkin(hier.ops[level], hier.P[level], hier.blk[level])
        hier.ops[level + 1] = coarse.StencilOperator(Yc, hier.blk[level].coarse)
    hier.prepare_coarsest()
    return hier
