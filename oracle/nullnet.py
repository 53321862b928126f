"""Learned near-null vectors: a gauge-covariant parallel-transport network (oracle side).

Test infrastructure, like all of ``oracle/``: only the tests, the smoke check and the
bench's CPU-baseline leg use it.

The paper finds its near-null vectors by relaxation on the homogeneous problem (Eq. relax)
and refines them with the adaptive passes. The learned setup replaces most of that work by
a network that maps random spinor fields to Nv vectors and is trained on vectors the plain
setup produced. Everything it does to a spinor must commute with a gauge transformation,
so that the vectors it predicts for a gauge-transformed field are the transformed vectors:

  * parallel-transport convolution (one layer): per site x, channel-spin index l = 2 c + s,
        a_x = sum_dir W_dir T_dir(h)_x,
        T_self(h)_x = h_x,  T_{+mu}(h)_x = U_x^mu h_{x+mu},  T_{-mu}(h)_x = conj(U_{x-mu}^mu) h_{x-mu},
    with complex weights W_dir[l_out][l_in] acting only on channel and spin indices, directions
    ordered (self, +0, -0, +1, -1) as the coarse stencil;
  * gate on each hidden channel (the two spin components of channel c at x):
        h = a g(|a_c|^2),  g(s) = 1 / sqrt(1 + s),
    a function of the gauge-invariant |a_c|^2 times a, so it is covariant; no biases (a bias
    would not be);
  * the last layer is linear; its output channel k is the predicted vector v_k (2 spins).

Loss (rotation invariant): for block b with rows r = (site in block, spin), W_b the
predicted vectors cut to the block (rows x Nv) and V_b the plain setup's block-orthonormal
prolongator columns there, Q_b an orthonormal basis of span W_b:
    L_b = sum_k |(1 - Q_b Q_b^dagger) V_b e_k|^2 = Nv - tr(C^dagger G^{-1} C),
    G = W_b^dagger W_b, C = W_b^dagger V_b;  loss = mean_b L_b / Nv, in [0, 1].
It depends only on the span of each block's predicted vectors, which is all the prolongator
keeps after block Gram-Schmidt. Its conjugate cogradient is
    dL_b / dW_b^* = -(V_b - W_b A) A^dagger,  A = G^{-1} C.

Backpropagation (conjugate cogradients g = dL/dz^* throughout):
    dL/dW_dir^* = sum_x g_a(x) T_dir(h)_x^dagger,
    dL/dh^*_z   = W_self^dagger g_a(z) + conj(U_{z-mu}^mu) W_{+mu}^dagger g_a(z-mu) + U_z^mu W_{-mu}^dagger g_a(z+mu),
    gate:       dL/da^* = g gh + 2 g'(s) Re(a_c^dagger gh_c) a_c.
For real parameters, d loss / d Re W = 2 Re(dL/dW^*) and d loss / d Im W = 2 Im(dL/dW^*).

Inputs: noise channel c (of Cin) is the complex Gaussian field of the setup's generator
(``rng.gaussian_vector`` with vector index c and level tag NOISE_TAG) over the dofs (x, s).
With ``bf16`` set, every layer's output (and the noise) is rounded to bfloat16 before the next
layer reads it, as the GPU stores its activations; arithmetic is otherwise FP64.
"""
from __future__ import annotations

import numpy as np

from . import rng
from .lattice import Lattice

NDIR = 5
NOISE_TAG = 0x4E4E  # level field of the noise draws (distinct from the setup's levels)


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float64 values to the nearest bfloat16 (ties to even), returned as float64.
    Goes through float32 first (exact for the float32 values the GPU rounds)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16c(z: np.ndarray) -> np.ndarray:
    return bf16_round(z.real) + 1j * bf16_round(z.imag)


def shapes(cin: int, ch: int, nv: int, layers: int = 4):
    """(out channels, in channels) of each layer: cin -> ch -> ... -> ch -> nv."""
    dims = [cin] + [ch] * (layers - 1) + [nv]
    return [(dims[i + 1], dims[i]) for i in range(layers)]


def noise(lat: Lattice, cin: int, seed: int) -> np.ndarray:
    """Noise input [x][2 cin] (l = 2 c + s) from the setup's Philox + Box-Muller generator."""
    V = lat.volume
    out = np.empty((V, 2 * cin), dtype=np.complex128)
    for c in range(cin):
        out[:, 2 * c:2 * c + 2] = rng.gaussian_vector(2 * V, seed, c, NOISE_TAG).reshape(V, 2)
    return out


def transport(h: np.ndarray, U: np.ndarray, lat: Lattice) -> np.ndarray:
    """T_dir(h) for the five directions: [5][x][l]."""
    T = np.empty((NDIR,) + h.shape, dtype=np.complex128)
    T[0] = h
    for mu in range(2):
        xs = np.arange(lat.volume)
        fwd = lat.neighbour(xs, mu, +1)
        bwd = lat.neighbour(xs, mu, -1)
        T[1 + 2 * mu] = U[:, mu, None] * h[fwd]
        T[2 + 2 * mu] = np.conj(U[bwd, mu])[:, None] * h[bwd]
    return T


def transport_adjoint(G: np.ndarray, U: np.ndarray, lat: Lattice) -> np.ndarray:
    """Adjoint of transport: sum_dir T_dir^dagger G[dir] ([5][x][l] -> [x][l])."""
    out = G[0].copy()
    for mu in range(2):
        xs = np.arange(lat.volume)
        fwd = lat.neighbour(xs, mu, +1)
        bwd = lat.neighbour(xs, mu, -1)
        # T_{+mu} moves h_{x+mu} to x with U_x^mu: its adjoint moves g_x to x + mu with conj(U_x^mu)
        out[fwd] += np.conj(U[:, mu])[:, None] * G[1 + 2 * mu]
        # T_{-mu} moves h_{x-mu} to x with conj(U_{x-mu}^mu): adjoint moves g_x to x - mu with U_{x-mu}^mu
        out[bwd] += U[bwd, mu][:, None] * G[2 + 2 * mu]
    return out


def gate(a: np.ndarray) -> np.ndarray:
    s = np.abs(a[:, 0::2]) ** 2 + np.abs(a[:, 1::2]) ** 2
    g = 1.0 / np.sqrt(1.0 + s)
    return a * np.repeat(g, 2, axis=1)


def gate_backward(a: np.ndarray, gh: np.ndarray) -> np.ndarray:
    s = np.abs(a[:, 0::2]) ** 2 + np.abs(a[:, 1::2]) ** 2
    g = 1.0 / np.sqrt(1.0 + s)
    dg = -0.5 * (1.0 + s) ** -1.5
    re = (np.conj(a) * gh).real
    proj = re[:, 0::2] + re[:, 1::2]
    return gh * np.repeat(g, 2, axis=1) + a * np.repeat(2.0 * dg * proj, 2, axis=1)


def forward(weights, x0: np.ndarray, U: np.ndarray, lat: Lattice, bf16: bool = False):
    """Layer by layer: returns (inputs h_l of each layer, pre-activations a_l, output).

    weights[l]: complex [5][2 cout][2 cin]; x0: [x][2 cin0]; output [x][2 nv]."""
    h = bf16c(x0) if bf16 else x0
    hs, As = [], []
    for li, W in enumerate(weights):
        hs.append(h)
        T = transport(h, U, lat)
        a = np.einsum("dol,dxl->xo", W, T)
        As.append(a)
        last = li == len(weights) - 1
        h = a if last else gate(a)
        if bf16 and not last:
            h = bf16c(h)
    return hs, As, h


def block_rows(out: np.ndarray, blk) -> np.ndarray:
    """[x][2 nv] -> [block][rows = bvol * 2][nv] with row = 2 * (site in block) + s."""
    nv = out.shape[1] // 2
    V3 = out.reshape(-1, nv, 2)  # [x][k][s]
    rows = V3[blk.site_table()]  # [b][i][k][s]
    return np.transpose(rows, (0, 1, 3, 2)).reshape(blk.n_blocks, -1, nv)


def unblock_rows(R: np.ndarray, blk, V: int) -> np.ndarray:
    nb, nr, nv = R.shape
    out = np.zeros((V, nv, 2), dtype=np.complex128)
    r4 = R.reshape(nb, nr // 2, 2, nv)
    out[blk.site_table()] = np.transpose(r4, (0, 1, 3, 2))
    return out.reshape(V, 2 * nv)


def loss_and_grad(out: np.ndarray, target: np.ndarray, blk):
    """Loss (mean over blocks of L_b / Nv) of the predicted vectors out[x][2 nv] against the
    target block-orthonormal columns target[k][x][s], and dloss/dout^*."""
    nv = out.shape[1] // 2
    W = block_rows(out, blk)
    Vt = block_rows(np.transpose(target, (1, 0, 2)).reshape(-1, 2 * nv), blk)
    nb = W.shape[0]
    total = 0.0
    grad = np.empty_like(W)
    for b in range(nb):
        Wb, Vb = W[b], Vt[b]
        G = Wb.conj().T @ Wb
        C = Wb.conj().T @ Vb
        A = np.linalg.solve(G, C)
        total += nv - np.trace(C.conj().T @ A).real
        R = Vb - Wb @ A
        grad[b] = -(R @ A.conj().T)
    scale = 1.0 / (nb * nv)
    return total * scale, unblock_rows(grad * scale, blk, out.shape[0])


def backward(weights, hs, As, gout: np.ndarray, U: np.ndarray, lat: Lattice):
    """Conjugate cogradients dloss/dW_l^* of every layer, given dloss/dout^* = gout."""
    grads = [None] * len(weights)
    ga = gout
    for li in range(len(weights) - 1, -1, -1):
        T = transport(hs[li], U, lat)
        grads[li] = np.einsum("xo,dxl->dol", ga, np.conj(T))
        if li == 0:
            break
        gT = np.einsum("dol,xo->dxl", np.conj(weights[li]), ga)
        gh = transport_adjoint(gT, U, lat)
        ga = gate_backward(As[li - 1], gh)
    return grads


def predict_vectors(weights, x0, U, lat, bf16=False) -> np.ndarray:
    """The predicted near-null vectors v[k][x][s] from the network output."""
    _, _, out = forward(weights, x0, U, lat, bf16)
    nv = out.shape[1] // 2
    return np.transpose(out.reshape(-1, nv, 2), (1, 0, 2)).copy()
