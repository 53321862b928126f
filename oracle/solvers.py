"""Smoother, V-cycle, coarsest solve and outer Krylov loop (oracle).

Paper, the five V-cycle steps (section after Eq. Galerkin) and Eq. vcycle:
  1. relax on the input:           x = R^dagger b
  2. restrict the residual:        r_c = P^dagger (b - A x)
  3. coarse V-cycle:               e_c = V^(l+1) r_c   (exact solve on the coarsest level)
  4. coarse-grid correction:       x = x + P e_c
  5. relax on the final residual:  x = x + R (b - A x)
Reading of the printed cycle: steps 1 and 5 are additive corrections (the
printed "x = R(b - Ax)" means x += R(b - Ax)), and the operator form then reads
V = R + R^dagger - R A R^dagger + (1 - R A) P V_c P^dagger (1 - A R^dagger);
the printed "+RAR^dagger" cannot hold for the five steps. The cost is 2 nu + 2
applications of A per level.

Smoother: minimum-residual (MR) iterations with under-relaxation omega = 0.8,
the paper's choice of relaxation (it freezes two MR iterations into a degree-2
polynomial; here MR is iterated nu_pre = nu_post = 4 times on D directly).

Outer loop: flexible GCR with the V-cycle as right preconditioner and a true
FP64 residual at every restart (the paper uses V-cycle-preconditioned CG on
the normal equations; GCR works on the non-hermitian D directly).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def vdot(a, b) -> complex:
    """<a, b> = sum conj(a) b."""
    return complex(np.vdot(np.asarray(a).reshape(-1), np.asarray(b).reshape(-1)))


def norm2(a) -> float:
    a = np.asarray(a).reshape(-1)
    return float(np.vdot(a, a).real)


class OpCounter:
    """Counts operator applications per level (the paper's cost metric)."""

    def __init__(self):
        self.counts = {}

    def add(self, level: int, n: int = 1):
        self.counts[level] = self.counts.get(level, 0) + n


def mr(apply_A, b, nu: int, omega: float, x0=None, counter=None, level=0):
    """nu minimum-residual iterations for A x = b.

    r = b - A x;  per iteration: alpha = omega <A r, r> / <A r, A r>,
    x += alpha r, r -= alpha A r. Starts from x0 (zero when None, with no
    operator application needed for the initial residual).
    Returns (x, r) with r the recursively updated residual.
    """
    b = np.asarray(b, dtype=np.complex128)
    if x0 is None:
        x = np.zeros_like(b)
        r = b.copy()
    else:
        x = np.array(x0, dtype=np.complex128)
        r = b - apply_A(x)
        if counter is not None:
            counter.add(level)
    for _ in range(nu):
        Ar = apply_A(r)
        if counter is not None:
            counter.add(level)
        den = norm2(Ar)
        if den == 0.0:
            break
        alpha = omega * vdot(Ar, r) / den
        x = x + alpha * r
        r = r - alpha * Ar
    return x, r


def gcr(apply_A, b, tol: float, restart: int, max_iter: int, precond=None, x0=None, counter=None, level=0):
    """(Flexible) GCR for A x = b with right preconditioner ``precond`` (identity if None).

    Each iteration: z = M(r), w = A z; w and z are orthogonalised against the
    earlier (w_j, z_j) of the cycle by modified Gram-Schmidt on w, scaled so
    that |w| = 1; then alpha = <w, r>, x += alpha z, r -= alpha w. After each
    cycle of ``restart`` iterations (or convergence of the updated residual)
    the residual is recomputed as b - A x.
    Returns (x, info) with info = dict(iters, true_rel_residual, converged).
    """
    b = np.asarray(b, dtype=np.complex128)
    bnorm = np.sqrt(norm2(b))
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    if bnorm == 0.0:
        return x, dict(iters=0, true_rel_residual=0.0, converged=True)
    if x0 is None:
        r = b.copy()
    else:
        r = b - apply_A(x)
        if counter is not None:
            counter.add(level)
    it = 0
    converged = False
    history = []
    while it < max_iter:
        Z, W = [], []
        for _ in range(restart):
            z = r.copy() if precond is None else precond(r)
            w = apply_A(z)
            if counter is not None:
                counter.add(level)
            for wj, zj in zip(W, Z):
                beta = vdot(wj, w)
                w = w - beta * wj
                z = z - beta * zj
            nw = np.sqrt(norm2(w))
            if nw == 0.0:
                break
            w = w / nw
            z = z / nw
            alpha = vdot(w, r)
            x = x + alpha * z
            r = r - alpha * w
            W.append(w)
            Z.append(z)
            it += 1
            rel = np.sqrt(norm2(r)) / bnorm
            history.append(rel)
            if rel <= tol or it >= max_iter:
                break
        r = b - apply_A(x)
        if counter is not None:
            counter.add(level)
        true_rel = np.sqrt(norm2(r)) / bnorm
        if true_rel <= tol:
            converged = True
            break
        if not W:
            break
    true_rel = np.sqrt(norm2(r)) / bnorm
    return x, dict(iters=it, true_rel_residual=float(true_rel), converged=converged, history=history)


class CoarsestSolver:
    """Exact solve on the coarsest level.

    n <= lu_max: dense LU with partial pivoting (LAPACK via scipy) of the
    assembled stencil matrix. Otherwise GCR to relative residual ``tol`` with
    restart ``restart`` (an iterative stand-in for the exact solve; the outer
    flexible GCR absorbs the remaining inexactness).
    """

    def __init__(self, op, lu_max: int, tol: float, restart: int, max_iter: int):
        self.op = op
        self.n = op.lat.volume * op.n_int
        self.tol, self.restart, self.max_iter = tol, restart, max_iter
        self.lu = None
        if self.n <= lu_max:
            self.lu = scipy.linalg.lu_factor(stencil_matrix(op))

    def solve(self, b, counter=None, level=0):
        b = np.asarray(b, dtype=np.complex128)
        if self.lu is not None:
            return scipy.linalg.lu_solve(self.lu, b.reshape(-1)).reshape(b.shape)
        x, _ = gcr(self.op.apply, b, self.tol, self.restart, self.max_iter, counter=counter, level=level)
        return x


def stencil_matrix(op):
    """Dense matrix of a StencilOperator assembled block by block from Y[j, dir]."""
    lat = op.lat
    nv = op.n_int
    n = lat.volume * nv
    M = np.zeros((n, n), dtype=np.complex128)
    sites = np.arange(lat.volume)
    for dirn in range(op.Y.shape[1]):
        if dirn == 0:
            src = sites
        else:
            mu, back = divmod(dirn - 1, 2)
            src = lat.neighbour(sites, mu, -1 if back else +1)
        for j in range(lat.volume):
            s = int(src[j])
            M[j * nv:(j + 1) * nv, s * nv:(s + 1) * nv] += op.Y[j, dirn]
    return M


def smooth(hier, level: int, b, nu: int, counter=None):
    """Relaxation x = R b from x = 0: nu MR iterations, or a fixed linear smoother
    ``hier.linear_smoother(level, b)`` when one is installed (used to check the
    operator form of the V-cycle, which needs a linear R)."""
    lin = getattr(hier, "linear_smoother", None)
    if lin is not None:
        return lin(level, b)
    x, _ = mr(hier.ops[level].apply, b, nu, hier.params.omega, counter=counter, level=level)
    return x


def vcycle(hier, level: int, b, counter=None):
    """One V-cycle V^(level) applied to b (levels numbered from 0 = finest)."""
    if level == hier.n_levels - 1:
        return hier.coarsest.solve(b, counter=counter, level=level)
    A = hier.ops[level].apply
    p = hier.params
    # 1. pre-relaxation from x = 0
    x = smooth(hier, level, b, p.nu_pre, counter)
    # 2. restrict the residual
    r = b - A(x)
    if counter is not None:
        counter.add(level)
    rc = hier.restrict(level, r)
    # 3. coarse V-cycle (or exact coarsest solve)
    ec = vcycle(hier, level + 1, rc, counter=counter)
    # 4. coarse-grid correction
    x = x + hier.prolong(level, ec)
    # 5. post-relaxation on the final residual
    r = b - A(x)
    if counter is not None:
        counter.add(level)
    return x + smooth(hier, level, r, p.nu_post, counter)


def mg_solve(hier, chi, tol: float, counter=None):
    """psi with D psi = chi by flexible GCR preconditioned with the V-cycle."""
    p = hier.params
    A = hier.ops[0].apply
    return gcr(A, chi, tol, p.gcr_restart, p.max_iter, precond=lambda r: vcycle(hier, 0, r, counter=counter),
               counter=counter, level=0)
