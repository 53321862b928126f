"""MG-preconditioned CG on the normal equations (oracle): the paper's own experiment.

Test infrastructure: only tests/, the bench's CPU baseline and smoke checks use this module.

Paper, numerical-results section: the operator is A = D^dagger D (hermitian positive definite);
4 x 4 blocks, M = 8 vectors, coarsened twice and solved exactly on the coarsest lattice; the
relaxation is a degree-2 polynomial smoother whose coefficients come from two iterations of
under-relaxed minimum residual (omega = 0.8) and are then held fixed, so that R = R^dagger; the
V-cycle (Eq. vcycle) preconditions conjugate gradients; the setup is done at the lightest mass
only. Cost: 6 fine A applications per MG-CG iteration (1 in CG, 2 pre- and 2 post-smoothing, 1 for
the residual); the coarse levels are not counted.

Readings (the paper fixes none of these):
- the Galerkin operator P^dagger A P of the fine D^dagger D couples a coarse site to its 8
  neighbours, diagonal ones included (D^dagger D reaches x +- 2 mu-hat and x +- mu-hat +- nu-hat,
  and a block is at least 2 sites wide), so coarse levels are 9-point stencils
  y_j = sum_o Y[j, o] x_{j + o}, o in {-1, 0, 1}^2 (index 3 (o1 + 1) + (o0 + 1); 4 is the site);
- the frozen coefficients of level l come from two MR steps on A x = b_l from x = 0, b_l Gaussian
  (Philox key seed, vector index 0x2C, level l); with A hermitian the step lengths are real, and
  the smoother R b = alpha1 b + alpha2 (b - alpha1 A b) is a real polynomial in A;
- the adaptive setup runs on A as on D: Nv random vectors relaxed by nu_setup MR iterations on
  A x = 0, block Gram-Schmidt, then passes v <- v - V(A v) with the hierarchy built so far, level
  by level, each followed by a rebuild of that level and the ones below from their vectors;
- the CG residual is the residual of the normal equations, |D^dagger chi - A psi| / |D^dagger chi|.
"""
from __future__ import annotations

import numpy as np

from . import solvers, wilson
from .lattice import Blocking, Lattice
from .rng import gaussian_vector
from .transfer import block_gram_schmidt, prolong, restrict

OFFSETS = [(o0, o1) for o1 in (-1, 0, 1) for o0 in (-1, 0, 1)]
SMOOTHER_VECTOR = 0x2C


def shift2(lat: Lattice, x, o):
    """Field with value x_{j + o} at site j (periodic), o = (o0, o1)."""
    y = x
    for mu in range(2):
        for _ in range(abs(o[mu])):
            y = lat.shift(y, mu, 1 if o[mu] > 0 else -1)
    return y


class NormalOperator:
    """Fine level: A = D^dagger D on 2d U(1) spinor fields (V, 2)."""

    def __init__(self, U, m: float, lat: Lattice):
        self.U, self.m, self.lat, self.n_int = U, float(m), lat, 2

    def apply(self, x):
        x = np.asarray(x, dtype=np.complex128).reshape(self.lat.volume, 2)
        return wilson.apply_Ddag(self.U, wilson.apply_D(self.U, x, self.m, self.lat), self.m, self.lat)


class Stencil9:
    """Coarse level: y_j = sum_o Y[j, o] x_{j + o} with (N x N) complex blocks."""

    def __init__(self, Y, lat: Lattice):
        self.Y = np.asarray(Y, dtype=np.complex128)
        self.lat = lat
        self.n_int = self.Y.shape[-1]
        assert self.Y.shape == (lat.volume, 9, self.n_int, self.n_int)

    def apply(self, x):
        x = np.asarray(x, dtype=np.complex128).reshape(self.lat.volume, self.n_int)
        out = np.zeros_like(x)
        for o_idx, o in enumerate(OFFSETS):
            out += np.einsum("jab,jb->ja", self.Y[:, o_idx], shift2(self.lat, x, o))
        return out


def colour_period(n: int) -> int:
    """Smallest period >= 3 dividing a coarse extent n (n >= 3): neighbours -1, 0, +1 differ."""
    if n < 3:
        raise ValueError("coarse extents must be at least 3 for the 9-point Galerkin probe")
    for p in range(3, n + 1):
        if n % p == 0:
            return p
    return n


def galerkin9(op, P, blk: Blocking):
    """Y[j, o] = P_j^dagger A P_{j+o} for a level operator A coupling a block only to its 8
    neighbouring blocks. Probing: blocks are coloured by (b0 mod p0, b1 mod p1); for a colour c and
    column k, A applied to the prolongation of the unit vectors (block b of colour c, dof k) and
    restricted gives, on block j, P_j^dagger A P_b e_k for the one neighbour b = j + o of colour c."""
    coarse = blk.coarse
    nb, Nb, nv = P.shape
    n0, n1 = coarse.dims
    p0, p1 = colour_period(n0), colour_period(n1)
    c = coarse.coords(np.arange(coarse.volume))
    colour = (c[0] % p0) + p0 * (c[1] % p1)
    Y = np.zeros((nb, 9, nv, nv), dtype=np.complex128)
    for col in range(p0 * p1):
        for k in range(nv):
            e = np.zeros((nb, nv), dtype=np.complex128)
            e[colour == col, k] = 1.0
            y = restrict(P, op.apply(prolong(P, e, blk, op.n_int)), blk)
            for o_idx, o in enumerate(OFFSETS):
                src = coarse.index([(c[0] + o[0]) % n0, (c[1] + o[1]) % n1])
                sel = colour[src] == col
                Y[sel, o_idx, :, k] = y[sel]
    return Y


def mr_coefficients(apply_A, b, omega: float = 0.8, steps: int = 2):
    """Step lengths of `steps` MR iterations on A x = b from x = 0 (real for hermitian A)."""
    r = np.asarray(b, dtype=np.complex128).copy()
    alphas = []
    for _ in range(steps):
        Ar = apply_A(r)
        a = omega * np.vdot(Ar, r).real / np.vdot(Ar, Ar).real
        alphas.append(float(a))
        r = r - a * Ar
    return alphas


def frozen_smooth(apply_A, alphas, b):
    """x = R b with the frozen MR polynomial; returns (x, b - A x)."""
    x = np.zeros_like(b)
    r = np.asarray(b, dtype=np.complex128).copy()
    for a in alphas:
        x = x + a * r
        r = r - a * apply_A(r)
    return x, r


class NormalHierarchy:
    """Levels of the MG-CG preconditioner: operators, blockings, prolongators, frozen coefficients."""

    def __init__(self, U, m: float, lat: Lattice, blocks, Nv, seed: int = 20070704, omega: float = 0.8):
        self.ops = [NormalOperator(U, m, lat)]
        self.blocks = [tuple(b) for b in blocks]
        self.Nv = list(Nv)
        self.levels = len(self.blocks) + 1
        self.seed, self.omega = seed, omega
        self.blk, self.P, self.alphas = [], [], []
        self.lu = None

    def build_level(self, level: int, vectors):
        op = self.ops[level]
        blk = Blocking(op.lat, self.blocks[level])
        P, _ = block_gram_schmidt(vectors, blk)
        Y = galerkin9(op, P, blk)
        del self.blk[level:], self.P[level:], self.ops[level + 1:]
        self.blk.append(blk)
        self.P.append(P)
        self.ops.append(Stencil9(Y, blk.coarse))

    def prepare(self):
        """Frozen smoother coefficients of every non-coarsest level, and the coarsest factorisation."""
        self.alphas = []
        for level in range(self.levels - 1):
            op = self.ops[level]
            b = gaussian_vector(op.lat.volume * op.n_int, self.seed, SMOOTHER_VECTOR, level)
            self.alphas.append(mr_coefficients(op.apply, b.reshape(op.lat.volume, op.n_int), self.omega))
        import scipy.linalg
        A = dense_matrix(self.ops[-1])
        self.lu = scipy.linalg.lu_factor(A)

    def vcycle(self, level: int, b):
        """Eq. vcycle with R = R^dagger: pre-smoothing, coarse correction, residual, post-smoothing."""
        op = self.ops[level]
        if level == self.levels - 1:
            import scipy.linalg
            return scipy.linalg.lu_solve(self.lu, b.reshape(-1)).reshape(b.shape)
        x, r = frozen_smooth(op.apply, self.alphas[level], b)
        e = self.vcycle(level + 1, restrict(self.P[level], r, self.blk[level]))
        x = x + prolong(self.P[level], e, self.blk[level], op.n_int)
        r = b - op.apply(x)
        x2, _ = frozen_smooth(op.apply, self.alphas[level], r)
        return x + x2


def dense_matrix(op):
    n = op.lat.volume * op.n_int
    M = np.zeros((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for col in range(n):
        e[:] = 0
        e[col] = 1
        M[:, col] = op.apply(e.reshape(op.lat.volume, op.n_int)).reshape(-1)
    return M


def adaptive_setup(U, m: float, lat: Lattice, blocks, Nv, n_pass: int = 5, nu_setup: int = 8,
                   omega: float = 0.8, seed: int = 20070704) -> NormalHierarchy:
    """The adaptive setup on A = D^dagger D. Pass 1, level by level: Nv Philox vectors (key seed,
    vector k, level l) relaxed by nu_setup MR iterations on A x = 0, block Gram-Schmidt, Galerkin.
    Passes 2..n_pass, level by level: every vector v of level l becomes v - V_l(A v) with the
    current hierarchy, and levels l, l+1, ... are rebuilt from their current vectors."""
    h = NormalHierarchy(U, m, lat, blocks, Nv, seed, omega)

    def relax(level):
        op = h.ops[level]
        n = op.lat.volume * op.n_int
        out = []
        for k in range(h.Nv[level]):
            v = gaussian_vector(n, seed, k, level).reshape(op.lat.volume, op.n_int)
            x, _ = solvers.mr(op.apply, np.zeros_like(v), nu_setup, omega, x0=v)
            out.append(x)
        return out

    vecs = []
    for level in range(h.levels - 1):
        vecs.append(relax(level))
        h.build_level(level, vecs[level])
    h.prepare()
    for _ in range(1, n_pass):
        for level in range(h.levels - 1):
            op = h.ops[level]
            vecs[level] = [v - h.vcycle(level, op.apply(v)) for v in vecs[level]]
            for l in range(level, h.levels - 1):
                h.build_level(l, vecs[l])
            h.prepare()
    return h


def cg(apply_A, b, tol: float, max_iter: int, precond=None):
    """(Preconditioned) conjugate gradients from x = 0; stops when |r| <= tol |b| (recurrence
    residual). Returns x and (iterations, true relative residual)."""
    b = np.asarray(b, dtype=np.complex128)
    x = np.zeros_like(b)
    r = b.copy()
    bn = np.linalg.norm(b)
    z = precond(r) if precond else r
    p = z.copy()
    rz = np.vdot(r, z).real
    it = 0
    while it < max_iter and np.linalg.norm(r) > tol * bn:
        q = apply_A(p)
        alpha = rz / np.vdot(p, q).real
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        z = precond(r) if precond else r
        rz_new = np.vdot(r, z).real
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, dict(iters=it, true_rel_residual=float(np.linalg.norm(b - apply_A(x)) / bn))


def mgcg_solve(h: NormalHierarchy, chi, tol: float, max_iter: int = 1000):
    """psi with D psi = chi through A psi = D^dagger chi, CG preconditioned by the V-cycle."""
    op = h.ops[0]
    rhs = wilson.apply_Ddag(op.U, np.asarray(chi, dtype=np.complex128).reshape(op.lat.volume, 2), op.m, op.lat)
    return cg(op.apply, rhs, tol, max_iter, precond=lambda r: h.vcycle(0, r))
