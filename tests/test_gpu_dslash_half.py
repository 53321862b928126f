"""The fine Wilson operator on half-precision storage with per-site norms (mg_dslash with MG_FP16,
mg_half_convert) against the FP64 oracle. The half fields are encoded and decoded on the host by
this test's own numpy code (IEEE half, round to nearest even); the GPU encoder must produce the same
bytes, and the GPU operator on the host-encoded input must match the oracle's FP64 operator on the
decoded input to the rounding of its half output (2^-11 of the site's largest component)."""
import numpy as np
import pytest

import inputs
from oracle import wilson
from oracle.lattice import Lattice
from tests._util import to_dev, to_host

pytestmark = pytest.mark.gpu


def encode_spinor(psi):
    """[V][2] complex -> bytes of [V][2] half pairs + [V] float32 norms (FP32 scaling as specified)."""
    p = psi.astype(np.complex64)
    comp = np.stack([p.real, p.imag], axis=-1).reshape(len(p), 4).astype(np.float32)
    nu = np.abs(comp).max(axis=1).astype(np.float32)
    inv = np.where(nu > 0, np.float32(1.0) / np.where(nu > 0, nu, np.float32(1.0)), np.float32(0.0)).astype(np.float32)
    h = (comp * inv[:, None]).astype(np.float32).astype(np.float16)
    return np.concatenate([h.view(np.uint8).reshape(-1), nu.view(np.uint8).reshape(-1)]), h, nu


def decode_spinor(raw, V):
    h = raw[: 8 * V].view(np.float16).reshape(V, 4).astype(np.float64)
    nu = raw[8 * V:].view(np.float32).astype(np.float64)
    c = h * nu[:, None]
    return (c[:, 0::2] + 1j * c[:, 1::2]).reshape(V, 2)


def encode_links(U):
    u = U.astype(np.complex64).reshape(-1)
    h = np.stack([u.real, u.imag], axis=-1).astype(np.float16)
    return h.view(np.uint8).reshape(-1), (h[:, 0].astype(np.float64) + 1j * h[:, 1].astype(np.float64)).reshape(U.shape)


# even L0: two sites per thread; odd L0 (15, 3): one site per thread
@pytest.mark.parametrize("dims", [(2, 2), (16, 12), (130, 66), (256, 256), (15, 12), (3, 2)])
def test_half_dslash_matches_oracle(dims):
    import torch
    import paper_0707_4018_gb300 as mg
    lat = Lattice(dims)
    V = lat.volume
    U = inputs.hot_links(*dims, seed=19)
    psi = inputs.gaussian_complex(V * 2, 5, 1).reshape(-1, 2) * np.exp(np.linspace(-3, 3, V))[:, None]
    m = 0.13
    raw_in, _, _ = encode_spinor(psi)
    raw_U, U_dec = encode_links(U)
    psi_dec = decode_spinor(raw_in, V)
    out = mg.half_spinor(V)
    mg.mg_dslash_half(to_dev(raw_U), to_dev(raw_in), out, m, dims)
    torch.cuda.synchronize()
    got = decode_spinor(to_host(out), V)
    want = wilson.apply_D(U_dec, psi_dec, m, lat)
    # per-site scale: |diag psi_x| + 1/2 sum of the hop magnitudes (bounds the cancellation)
    hop = np.zeros(V)
    for mu in range(2):
        for sgn in (+1, -1):
            nb = lat.neighbour(np.arange(V), mu, sgn)
            hop += np.abs(psi_dec[nb]).sum(axis=1)
    scale = (2 + m) * np.abs(psi_dec).sum(axis=1) + hop
    err = np.abs(got - want).max(axis=1) / scale
    assert err.max() < 1e-3, err.max()
    # the output rounding is the error: most sites sit well inside the bound, none far below FP32 noise
    assert np.median(err) < 3e-4


def test_half_conversions_match_host_encoding():
    import torch
    import paper_0707_4018_gb300 as mg
    dims = (64, 48)
    V = dims[0] * dims[1]
    psi = inputs.gaussian_complex(V * 2, 6, 2).reshape(-1, 2)
    U = inputs.hot_links(*dims, seed=3)
    for dt in (torch.complex128, torch.complex64):
        h = mg.half_spinor(V)
        mg.mg_half_convert(0, to_dev(psi, dt), h, V)
        hl = mg.half_links(V)
        mg.mg_half_convert(2, to_dev(U, dt), hl, V)
        back = torch.empty((V, 2), dtype=dt, device="cuda")
        mg.mg_half_convert(1, h, back, V)
        torch.cuda.synchronize()
        raw, _, _ = encode_spinor(psi)
        assert np.array_equal(to_host(h), raw)
        assert np.array_equal(to_host(hl), encode_links(U)[0])
        # the decoder scales in FP32: the exact products rounded to FP32 (then widened for complex128)
        assert np.array_equal(to_host(back).astype(np.complex64), decode_spinor(raw, V).astype(np.complex64))
