"""GPU parity of the 4d SU(3) Wilson operator (DeGrand-Rossi basis; CUDA kernel through
the C ABI) with the oracle's D, on APE-smeared and rough SU(3) fields."""
import numpy as np
import pytest

import inputs
from oracle import wilson
from oracle.lattice import Lattice
from tests._util import to_dev, to_host

pytestmark = pytest.mark.gpu


def _gpu_D(U, psi, m, dims, precision=0):
    import torch
    import paper_0707_4018_gb300 as mg
    dt = torch.complex128 if precision == 0 else torch.complex64
    Ud, pd = to_dev(U, dt), to_dev(psi, dt)
    out = torch.empty_like(pd)
    mg.mg_dslash(Ud, pd, out, m, dims, precision)
    torch.cuda.synchronize()
    return to_host(out)


def _field(dims, seed, smooth=True):
    if smooth:
        return inputs.su3_links(dims, seed=seed)
    return inputs.su3_random(int(np.prod(dims)) * 4, seed, 0x7F).reshape(-1, 4, 3, 3)


@pytest.mark.parametrize("dims,smooth", [((2, 2, 2, 2), False), ((4, 4, 4, 4), True), ((6, 4, 2, 8), False),
                                         ((5, 3, 7, 2), True), ((8, 8, 8, 16), True), ((8, 4, 4, 2), False),
                                         ((16, 8, 4, 6), False)])
def test_dslash4d_fp64_matches_oracle(dims, smooth):
    lat = Lattice(dims)
    U = _field(dims, 31, smooth)
    psi = inputs.gaussian_spinor(lat.volume, 12, 3, 1).reshape(lat.volume, 4, 3)
    m = -0.41
    want = wilson.apply_D(U, psi, m, lat)
    got = _gpu_D(U, psi, m, dims).reshape(want.shape)
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err < 1e-14, err


def test_dslash4d_free_plane_wave_closed_form():
    # U = 1: D e^{ipx} u = [(4 + m - sum cos p) + i sum sin p_mu gamma_mu] e^{ipx} u (colour-diagonal)
    dims = (4, 6, 2, 8)
    lat = Lattice(dims)
    coords = lat.coords(np.arange(lat.volume))
    n = (1, 5, 1, 3)
    p = [2 * np.pi * n[mu] / dims[mu] for mu in range(4)]
    ph = np.exp(1j * sum(p[mu] * coords[mu] for mu in range(4)))
    u = (np.arange(12) * (0.3 + 0.7j) + 1).reshape(4, 3)
    g, _ = wilson.gammas(4)
    m = 0.03
    Dp = (4 + m - sum(np.cos(q) for q in p)) * np.eye(4) + 1j * sum(np.sin(p[mu]) * g[mu] for mu in range(4))
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (lat.volume, 4, 3, 3)).copy()
    got = _gpu_D(U, ph[:, None, None] * u[None], m, dims).reshape(lat.volume, 4, 3)
    np.testing.assert_allclose(got, ph[:, None, None] * (Dp @ u)[None], atol=1e-13)


# (8, 2, 2, 2): one 8x2x2x2 tile of the tiled FP32 kernel (every face wraps onto the tile itself);
# (8, 4, 4, 2), (16, 8, 4, 8), (16, 16, 16, 32): several tiles; (4, 4, 4, 4), (6, 10, 4, 2): the
# warp-gather kernel
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (16, 16, 16, 32), (6, 10, 4, 2), (8, 4, 4, 2), (16, 8, 4, 8),
                                  (8, 2, 2, 2)])
def test_dslash4d_fp32_per_site_error_below_1e6(dims):
    # reference: FP64 D on the same FP32-rounded inputs; per-site error relative to
    # |diag psi_x| + 1/2 sum |hop terms_x| (bounds the cancellation at that site)
    lat = Lattice(dims)
    U = _field(dims, 7, smooth=dims[0] != 6)
    psi = inputs.gaussian_spinor(lat.volume, 12, 5, 2)
    U32 = U.astype(np.complex64).astype(np.complex128)
    p32 = psi.astype(np.complex64).astype(np.complex128)
    m = 0.01
    ref = wilson.apply_D(U32, p32, m, lat).reshape(lat.volume, 12)
    scale = (4 + m) * np.abs(p32).sum(axis=1)
    for mu in range(4):
        for s in (+1, -1):
            scale += np.abs(wilson.hop(U32, p32, lat, mu, s)).reshape(lat.volume, 12).sum(axis=1)
    got = _gpu_D(U32.astype(np.complex64), p32.astype(np.complex64), m, dims, precision=1).reshape(lat.volume, 12)
    err = np.abs(got - ref).sum(axis=1) / scale
    assert err.max() < 1e-6, err.max()


def test_dslash4d_gauge_covariance_on_gpu():
    # D[U^Omega] (Omega psi) = Omega D[U] psi for a random SU(3) gauge transformation
    dims = (4, 4, 6, 4)
    lat = Lattice(dims)
    U = _field(dims, 11)
    om = inputs.su3_random(lat.volume, 12, 0x47)
    psi = inputs.gaussian_spinor(lat.volume, 12, 13, 0)
    m = 0.2
    Ug = wilson.gauge_transform(U, om, lat)
    lhs = _gpu_D(Ug, wilson.transform_spinor(psi, om, lat, 3), m, dims)
    rhs = wilson.transform_spinor(_gpu_D(U, psi, m, dims), om, lat, 3)
    assert np.abs(lhs - rhs).max() < 1e-13


def test_dslash4d_large_sampled_fp32():
    # the size of the 4d bandwidth measurement (32^3 x 64), checked on sampled sites
    dims = (32, 32, 32, 64)
    lat = Lattice(dims)
    U = inputs.su3_near_identity(lat.volume * 4, 0.4, 21, 0x535533).reshape(lat.volume, 4, 3, 3)
    psi = inputs.gaussian_spinor(lat.volume, 12, 9, 1)
    U32 = U.astype(np.complex64)
    p32 = psi.astype(np.complex64)
    got = _gpu_D(U32, p32, 0.01, dims, precision=1).reshape(lat.volume, 12)
    rng = np.random.default_rng(0)
    sites = np.concatenate([rng.integers(0, lat.volume, 3000), [0, lat.volume - 1, 31, 32 * 32 * 32 * 63]])
    want = wilson.apply_D_at(U32.astype(np.complex128), p32.astype(np.complex128).reshape(lat.volume, 4, 3), 0.01,
                             lat, sites).reshape(len(sites), 12)
    assert np.abs(got[sites] - want).max() / np.abs(want).max() < 1e-6


@pytest.mark.parametrize("variant", ["0", "1", "2", "3", "4", "5", "6", "7"])
def test_dslash4d_fp32_tiled_and_gather_kernels_agree(variant, monkeypatch):
    # the FP32 kernels (every tile shape, and the warp-gather kernel) form the same hop sums in the
    # same order: they agree to rounding
    dims = (16, 8, 8, 8)
    lat = Lattice(dims)
    U = _field(dims, 17)
    psi = inputs.gaussian_spinor(lat.volume, 12, 19, 0)
    U32, p32 = U.astype(np.complex64), psi.astype(np.complex64)
    monkeypatch.setenv("MG_DSLASH4_TILE", variant)
    tiled = _gpu_D(U32, p32, 0.05, dims, precision=1)
    monkeypatch.setenv("MG_DSLASH4_GATHER", "1")
    gather = _gpu_D(U32, p32, 0.05, dims, precision=1)
    assert np.abs(tiled - gather).max() <= 1e-6 * np.abs(gather).max()
