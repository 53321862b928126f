"""Pins of the oracle's learned near-null network (oracle/nullnet.py) against what the
mathematics fixes: gauge covariance and translation equivariance of the network, the
closed-form values of the rotation-invariant loss, its invariance under per-block changes
of basis, central finite differences of the loss for the analytic gradients, and the
bfloat16 rounding rule."""
import numpy as np
import pytest

import inputs
from oracle import nullnet, transfer
from oracle.lattice import Blocking, Lattice


def _weights(cin, ch, nv, seed, scale=0.6):
    rs = np.random.default_rng(seed)
    ws = []
    for co, ci in nullnet.shapes(cin, ch, nv):
        w = (rs.standard_normal((5, 2 * co, 2 * ci)) + 1j * rs.standard_normal((5, 2 * co, 2 * ci)))
        ws.append(w * scale / np.sqrt(10 * ci))
    return ws


def _field(L0, L1, seed):
    theta, _ = inputs.metropolis_u1_2d(L0, L1, 3.0, 20, seed=seed)
    return inputs.links_from_angles(theta)


def test_bf16_rounding_rule():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -9, -2.5, 3.0e-3, 1.0 + 2.0 ** -7])
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -6, 1.0, -2.5, 197 * 2.0 ** -16, 1.0 + 2.0 ** -7])
    assert np.array_equal(nullnet.bf16_round(x), want)


def test_network_is_gauge_covariant():
    L = 8
    lat = Lattice((L, L))
    U = _field(L, L, 3)
    ws = _weights(3, 4, 2, 1)
    x0 = nullnet.noise(lat, 3, seed=11)
    g = inputs.u1_phases(lat.volume, 5, 0)
    xs = np.arange(lat.volume)
    Ug = np.empty_like(U)
    for mu in range(2):
        Ug[:, mu] = g * U[:, mu] * np.conj(g[lat.neighbour(xs, mu, +1)])
    out = nullnet.forward(ws, x0, U, lat)[2]
    outg = nullnet.forward(ws, g[:, None] * x0, Ug, lat)[2]
    assert np.abs(outg - g[:, None] * out).max() < 1e-13 * np.abs(out).max()


def test_network_is_translation_equivariant():
    L0, L1 = 8, 6
    lat = Lattice((L0, L1))
    U = _field(L0, L1, 4)
    ws = _weights(2, 4, 2, 2)
    x0 = nullnet.noise(lat, 2, seed=12)
    out = nullnet.forward(ws, x0, U, lat)[2]
    Us = lat.shift(U, 0, +1)
    xs0 = lat.shift(x0, 0, +1)
    outs = nullnet.forward(ws, xs0, Us, lat)[2]
    assert np.abs(outs - lat.shift(out, 0, +1)).max() < 1e-13 * np.abs(out).max()


def _orthonormal_target(lat, blk, nv, seed):
    rs = np.random.default_rng(seed)
    raw = rs.standard_normal((nv, lat.volume, 2)) + 1j * rs.standard_normal((nv, lat.volume, 2))
    P, _ = transfer.block_gram_schmidt([raw[k] for k in range(nv)], blk, 2)
    return np.stack([transfer.from_blocks(P[:, :, k], blk, 2) for k in range(nv)])


def test_loss_closed_forms_and_rotation_invariance():
    L, nv = 8, 3
    lat = Lattice((L, L))
    blk = Blocking(lat, (4, 4))
    T = _orthonormal_target(lat, blk, nv, 1)
    rows = nullnet.block_rows(np.transpose(T, (1, 0, 2)).reshape(-1, 2 * nv), blk)
    rs = np.random.default_rng(2)
    # predictions spanning the target on every block: loss 0
    M = rs.standard_normal((blk.n_blocks, nv, nv)) + 1j * rs.standard_normal((blk.n_blocks, nv, nv))
    same = nullnet.unblock_rows(rows @ M, blk, lat.volume)
    assert nullnet.loss_and_grad(same, T, blk)[0] < 1e-12
    # predictions orthogonal to the target on every block: loss 1
    R = rs.standard_normal(rows.shape) + 1j * rs.standard_normal(rows.shape)
    R -= rows @ (np.conj(np.transpose(rows, (0, 2, 1))) @ R)
    perp = nullnet.unblock_rows(R, blk, lat.volume)
    assert abs(nullnet.loss_and_grad(perp, T, blk)[0] - 1.0) < 1e-12
    # a generic prediction: the loss does not change under a per-block change of basis
    G = rs.standard_normal(rows.shape) + 1j * rs.standard_normal(rows.shape)
    l1 = nullnet.loss_and_grad(nullnet.unblock_rows(G, blk, lat.volume), T, blk)[0]
    l2 = nullnet.loss_and_grad(nullnet.unblock_rows(G @ M, blk, lat.volume), T, blk)[0]
    assert 0.1 < l1 < 0.99 and abs(l1 - l2) < 1e-12
    # one block's vectors replaced by its target: that block's share of the loss vanishes
    G2 = G.copy()
    G2[0] = rows[0]
    l3 = nullnet.loss_and_grad(nullnet.unblock_rows(G2, blk, lat.volume), T, blk)[0]
    lb = [nullnet.loss_and_grad(nullnet.unblock_rows(G, blk, lat.volume), T, blk)[0]]
    assert l3 < lb[0]


@pytest.mark.parametrize("layer", [0, 1, 2, 3])
def test_weight_gradients_match_finite_differences(layer):
    L, nv, cin, ch = 8, 2, 2, 3
    lat = Lattice((L, L))
    blk = Blocking(lat, (4, 4))
    U = _field(L, L, 6)
    ws = _weights(cin, ch, nv, 3 + layer, scale=1.5)
    x0 = nullnet.noise(lat, cin, seed=13)
    T = _orthonormal_target(lat, blk, nv, 7)

    def loss(wl):
        return nullnet.loss_and_grad(nullnet.forward(wl, x0, U, lat)[2], T, blk)[0]

    hs, As, out = nullnet.forward(ws, x0, U, lat)
    l0, gout = nullnet.loss_and_grad(out, T, blk)
    grads = nullnet.backward(ws, hs, As, gout, U, lat)
    rs = np.random.default_rng(layer)
    h = 1e-6
    for _ in range(6):
        idx = tuple(rs.integers(0, n) for n in ws[layer].shape)
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            wp = [w.copy() for w in ws]
            wm = [w.copy() for w in ws]
            wp[layer][idx] += unit * h
            wm[layer][idx] -= unit * h
            fd = (loss(wp) - loss(wm)) / (2 * h)
            an = 2.0 * part(grads[layer][idx])
            assert abs(fd - an) <= 1e-6 * max(1e-3, abs(an)), (idx, fd, an)


def test_bf16_forward_stays_close_to_fp64_forward():
    L = 8
    lat = Lattice((L, L))
    U = _field(L, L, 8)
    ws = _weights(4, 4, 2, 9)
    x0 = nullnet.noise(lat, 4, seed=14)
    a = nullnet.forward(ws, x0, U, lat)[2]
    b = nullnet.forward(ws, x0, U, lat, bf16=True)[2]
    err = np.abs(a - b).max() / np.abs(a).max()
    assert 1e-6 < err < 3e-2


def _covariance_ok():
    L = 8
    lat = Lattice((L, L))
    U = _field(L, L, 3)
    ws = _weights(3, 4, 2, 1)
    x0 = nullnet.noise(lat, 3, seed=11)
    g = inputs.u1_phases(lat.volume, 5, 0)
    xs = np.arange(lat.volume)
    Ug = np.empty_like(U)
    for mu in range(2):
        Ug[:, mu] = g * U[:, mu] * np.conj(g[lat.neighbour(xs, mu, +1)])
    out = nullnet.forward(ws, x0, U, lat)[2]
    outg = nullnet.forward(ws, g[:, None] * x0, Ug, lat)[2]
    return np.abs(outg - g[:, None] * out).max() < 1e-13 * np.abs(out).max()


def _gradients_ok():
    L, nv, cin, ch = 8, 2, 2, 3
    lat = Lattice((L, L))
    blk = Blocking(lat, (4, 4))
    U = _field(L, L, 6)
    ws = _weights(cin, ch, nv, 5, scale=1.5)
    x0 = nullnet.noise(lat, cin, seed=13)
    T = _orthonormal_target(lat, blk, nv, 7)
    hs, As, out = nullnet.forward(ws, x0, U, lat)
    _, gout = nullnet.loss_and_grad(out, T, blk)
    grads = nullnet.backward(ws, hs, As, gout, U, lat)
    rs = np.random.default_rng(0)
    h = 1e-6
    for layer in range(4):
        for _ in range(3):
            idx = tuple(rs.integers(0, n) for n in ws[layer].shape)
            wp = [w.copy() for w in ws]
            wm = [w.copy() for w in ws]
            wp[layer][idx] += h
            wm[layer][idx] -= h
            fd = (nullnet.loss_and_grad(nullnet.forward(wp, x0, U, lat)[2], T, blk)[0] -
                  nullnet.loss_and_grad(nullnet.forward(wm, x0, U, lat)[2], T, blk)[0]) / (2 * h)
            an = 2.0 * grads[layer][idx].real
            if abs(fd - an) > 1e-6 * max(1e-3, abs(an)):
                return False
    return True


def _mut_transport_wrong_link(h, U, lat):
    T = _orig_transport(h, U, lat)
    xs = np.arange(lat.volume)
    T[1] = U[lat.neighbour(xs, 0, -1), 0, None] * h[lat.neighbour(xs, 0, +1)]  # link of x - 0 instead of x
    return T


def _mut_adjoint_no_conj(G, U, lat):
    out = G[0].copy()
    xs = np.arange(lat.volume)
    for mu in range(2):
        fwd, bwd = lat.neighbour(xs, mu, +1), lat.neighbour(xs, mu, -1)
        out[fwd] += U[:, mu][:, None] * G[1 + 2 * mu]  # conj dropped
        out[bwd] += U[bwd, mu][:, None] * G[2 + 2 * mu]
    return out


def _mut_gate_backward_dropped_term(a, gh):
    s = np.abs(a[:, 0::2]) ** 2 + np.abs(a[:, 1::2]) ** 2
    return gh * np.repeat(1.0 / np.sqrt(1.0 + s), 2, axis=1)


def _mut_gate_not_channelwise(a):
    s = np.abs(a) ** 2  # per spin component instead of per channel: still covariant, different map
    return a / np.sqrt(1.0 + s)


_orig_transport = nullnet.transport


@pytest.mark.parametrize("name,fn,check", [
    ("transport", _mut_transport_wrong_link, _covariance_ok),
    ("transport_adjoint", _mut_adjoint_no_conj, _gradients_ok),
    ("gate_backward", _mut_gate_backward_dropped_term, _gradients_ok),
    ("gate", _mut_gate_not_channelwise, _gradients_ok),
])
def test_planted_network_mistakes_are_caught(monkeypatch, name, fn, check):
    assert check()
    monkeypatch.setattr(nullnet, name, fn)
    assert not check()
