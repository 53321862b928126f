"""Critical mass from the low edge of the spectrum of D (oracle).

The workloads set the mass relative to the critical mass m_c, where the
smallest real part of the spectrum of D(m) reaches zero (the paper's mass gap
m_hat = m - m_crit). With the diagonal d + m, D(m) = D(0) + m, so

    m_c = - min Re lambda(D(0)).

Small lattices: all eigenvalues of the dense matrix (LAPACK). Larger lattices:
ARPACK's implicitly restarted Arnoldi for the eigenvalues of smallest real
part (an extremal part of the spectrum, so no inversion is needed).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as sla

from . import wilson
from .lattice import Lattice


def eigenvalues_dense(U, m: float, lat: Lattice, Nc: int = 1):
    return np.linalg.eigvals(wilson.dense_D(U, m, lat, Nc))


def critical_mass_dense(U, lat: Lattice, Nc: int = 1) -> float:
    return float(-eigenvalues_dense(U, 0.0, lat, Nc).real.min())


def critical_mass_arnoldi(U, lat: Lattice, Nc: int = 1, k: int = 6, ncv: int = 64, tol: float = 1e-8,
                          maxiter: int = 20000, seed: int = 1) -> float:
    n = lat.volume * wilson.n_spin(lat.d) * Nc

    def mv(v):
        return wilson.apply_D(U, v.reshape(lat.volume, -1), 0.0, lat).reshape(-1)

    op = sla.LinearOperator((n, n), matvec=mv, dtype=np.complex128)
    v0 = np.random.default_rng(seed).standard_normal(n) + 0j
    vals = sla.eigs(op, k=k, which="SR", ncv=ncv, tol=tol, maxiter=maxiter, v0=v0, return_eigenvectors=False)
    return float(-np.min(vals.real))


def critical_mass(U, lat: Lattice, Nc: int = 1, dense_max: int = 2048) -> float:
    n = lat.volume * wilson.n_spin(lat.d) * Nc
    if n <= dense_max:
        return critical_mass_dense(U, lat, Nc)
    return critical_mass_arnoldi(U, lat, Nc)
