"""Planted mistakes in the MG-CG oracle (normal equations, on the CPU) must be caught by its pins.

Each case replaces one piece of `oracle/normal.py` with a plausible error (the wrong operator
product, coarse blocks stored under the opposite offset or transposed, aliased probe colours, a
wrong MR step length, a V-cycle that skips the residual before post-smoothing) and asserts that the matching dense
check of `tests/test_oracle_normal.py` fails, while the unmutated oracle passes it.
"""
import numpy as np
import pytest

import inputs
from oracle import normal, wilson
from oracle.lattice import Blocking, Lattice
from oracle.rng import gaussian_vector
from oracle.transfer import block_gram_schmidt, dense_P


def _operator_pin(op_cls) -> bool:
    """A equals the dense D^dagger D and is hermitian positive definite."""
    lat = Lattice((6, 6))
    U = inputs.hot_links(6, 6, seed=3)
    D = wilson.dense_D(U, 0.1, lat)
    A = normal.dense_matrix(op_cls(U, 0.1, lat))
    return (np.abs(A - D.conj().T @ D).max() < 1e-13 and np.abs(A - A.conj().T).max() < 1e-13
            and np.linalg.eigvalsh((A + A.conj().T) / 2).min() > 0)


def _galerkin_pin() -> bool:
    """The 9-point stencil equals the dense P^dagger A P (12^2 -> 6^2, 2 x 2 blocks)."""
    lat = Lattice((12, 12))
    U = inputs.hot_links(12, 12, seed=3)
    op = normal.NormalOperator(U, 0.1, lat)
    blk = Blocking(lat, (2, 2))
    vecs = [gaussian_vector(lat.volume * 2, 5, k, 0).reshape(lat.volume, 2) for k in range(4)]
    P, _ = block_gram_schmidt(vecs, blk)
    Pd = dense_P(P, blk, 2)
    want = Pd.conj().T @ normal.dense_matrix(op) @ Pd
    got = normal.dense_matrix(normal.Stencil9(normal.galerkin9(op, P, blk), blk.coarse))
    return np.abs(got - want).max() <= 1e-13 * np.abs(want).max()


def _smoother_pin() -> bool:
    """The frozen step lengths are those of MR, and the smoother is the real polynomial in A."""
    lat = Lattice((6, 6))
    U = inputs.hot_links(6, 6, seed=3)
    op = normal.NormalOperator(U, 0.1, lat)
    A = normal.dense_matrix(op)
    b = gaussian_vector(lat.volume * 2, 9, 0, 0).reshape(lat.volume, 2)
    a1, a2 = normal.mr_coefficients(op.apply, b, 0.8)
    r = b.reshape(-1)
    Ar = A @ r
    ok = abs(a1 - 0.8 * np.vdot(Ar, r).real / np.vdot(Ar, Ar).real) < 1e-14
    R = (a1 + a2) * np.eye(len(A)) - a1 * a2 * A
    x, _ = normal.frozen_smooth(op.apply, [a1, a2], b)
    return ok and np.abs(x.reshape(-1) - R @ b.reshape(-1)).max() < 1e-13


def _vcycle_pin() -> bool:
    """Two levels with an exact coarse solve: V = 2R - R A R + (1 - R A) P A_c^-1 P^dagger (1 - A R)."""
    lat = Lattice((12, 12))
    U = inputs.hot_links(12, 12, seed=3)
    h = normal.NormalHierarchy(U, 0.1, lat, [(2, 2)], [4])
    h.build_level(0, [gaussian_vector(lat.volume * 2, 7, k, 0).reshape(lat.volume, 2) for k in range(4)])
    h.prepare()
    A = normal.dense_matrix(h.ops[0])
    n = len(A)
    a1, a2 = h.alphas[0]
    R = (a1 + a2) * np.eye(n) - a1 * a2 * A
    Pd = dense_P(h.P[0], h.blk[0], 2)
    I = np.eye(n)
    want = 2 * R - R @ A @ R + (I - R @ A) @ Pd @ np.linalg.solve(Pd.conj().T @ A @ Pd, Pd.conj().T) @ (I - A @ R)
    V = np.zeros((n, n), dtype=complex)
    for i in range(n):
        e = np.zeros(n, dtype=complex)
        e[i] = 1
        V[:, i] = h.vcycle(0, e.reshape(lat.volume, 2)).reshape(-1)
    return np.abs(V - want).max() <= 1e-11 * np.abs(want).max()


def test_unmutated_normal_oracle_passes_its_pins():
    assert _operator_pin(normal.NormalOperator)
    assert _galerkin_pin() and _smoother_pin() and _vcycle_pin()


def test_planted_operator_without_adjoint_is_caught():
    class DD(normal.NormalOperator):  # D D in place of D^dagger D
        def apply(self, x):
            x = np.asarray(x, dtype=np.complex128).reshape(self.lat.volume, 2)
            return wilson.apply_D(self.U, wilson.apply_D(self.U, x, self.m, self.lat), self.m, self.lat)

    assert not _operator_pin(DD)


def test_planted_operator_with_wrong_mass_is_caught():
    class WrongMass(normal.NormalOperator):  # D^dagger at m, D at m + 0.1
        def apply(self, x):
            x = np.asarray(x, dtype=np.complex128).reshape(self.lat.volume, 2)
            y = wilson.apply_D(self.U, x, self.m + 0.1, self.lat)
            return wilson.apply_Ddag(self.U, y, self.m, self.lat)

    assert not _operator_pin(WrongMass)


@pytest.mark.parametrize("kind", ["offset_sign", "transposed_block", "colour_alias"])
def test_planted_galerkin9_mistake_is_caught(kind, monkeypatch):
    original = normal.galerkin9
    if kind == "offset_sign":  # each block stored under the opposite offset (o where -o belongs)
        monkeypatch.setattr(normal, "galerkin9", lambda op, P, blk: original(op, P, blk)[:, ::-1].copy())
    elif kind == "transposed_block":  # rows and columns of every block exchanged
        monkeypatch.setattr(normal, "galerkin9", lambda op, P, blk: np.swapaxes(original(op, P, blk), 2, 3).copy())
    else:  # period 2: the neighbours -1 and +1 of a coarse site share a colour
        monkeypatch.setattr(normal, "colour_period", lambda n: 2)
    assert not _galerkin_pin(), kind


def test_planted_mr_step_length_is_caught(monkeypatch):
    def wrong(apply_A, b, omega=0.8, steps=2):  # <Ar, r> / |r|^2 in place of <Ar, r> / |Ar|^2
        r = np.asarray(b, dtype=np.complex128).copy()
        out = []
        for _ in range(steps):
            Ar = apply_A(r)
            a = omega * np.vdot(Ar, r).real / np.vdot(r, r).real
            out.append(float(a))
            r = r - a * Ar
        return out

    monkeypatch.setattr(normal, "mr_coefficients", wrong)
    assert not _smoother_pin()


def test_planted_vcycle_without_residual_update_is_caught(monkeypatch):
    def vcycle(self, level, b):  # post-smoothing on the pre-smoothing residual, not b - A x
        op = self.ops[level]
        if level == self.levels - 1:
            import scipy.linalg
            return scipy.linalg.lu_solve(self.lu, b.reshape(-1)).reshape(b.shape)
        x, r = normal.frozen_smooth(op.apply, self.alphas[level], b)
        e = self.vcycle(level + 1, normal.restrict(self.P[level], r, self.blk[level]))
        x = x + normal.prolong(self.P[level], e, self.blk[level], op.n_int)
        x2, _ = normal.frozen_smooth(op.apply, self.alphas[level], r)
        return x + x2

    monkeypatch.setattr(normal.NormalHierarchy, "vcycle", vcycle)
    assert not _vcycle_pin()
