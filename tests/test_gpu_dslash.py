"""GPU parity of the fine Wilson operator (CUDA kernel through the C ABI) with the oracle."""
import numpy as np
import pytest

import inputs
from oracle import wilson
from oracle.lattice import Lattice
from tests._util import rel_err, to_dev, to_host

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


@pytest.mark.parametrize("dims", [(2, 2), (8, 8), (16, 12), (130, 66), (64, 64)])
def test_dslash_fp64_matches_oracle(dims):
    lat = Lattice(dims)
    U = inputs.hot_links(*dims, seed=17)
    psi = inputs.gaussian_complex(lat.volume * 2, 3, 1).reshape(-1, 2)
    m = -0.37
    want = wilson.apply_D(U, psi, m, lat)
    got = _gpu_D(U, psi, m, dims)
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err < 1e-14, err


def test_dslash_thermal_field_fp64():
    dims = (64, 64)
    lat = Lattice(dims)
    U, _, _ = inputs.schwinger_links(64, 6.0, sweeps=100, workload_id=7)
    psi = inputs.gaussian_complex(lat.volume * 2, 3, 2).reshape(-1, 2)
    assert rel_err(_gpu_D(U, psi, 0.1, dims), wilson.apply_D(U, psi, 0.1, lat)) < 1e-15


def test_dslash_free_plane_wave_closed_form():
    dims = (32, 16)
    lat = Lattice(dims)
    x0, x1 = lat.coords(np.arange(lat.volume))
    p = (2 * np.pi * 5 / 32, 2 * np.pi * 3 / 16)
    u = np.array([0.7 + 0.1j, -0.2 + 0.9j])
    ph = np.exp(1j * (p[0] * x0 + p[1] * x1))[:, None]
    g, _ = wilson.gammas(2)
    m = 0.05
    Dp = (2 + m - np.cos(p[0]) - np.cos(p[1])) * np.eye(2) + 1j * (np.sin(p[0]) * g[0] + np.sin(p[1]) * g[1])
    got = _gpu_D(inputs.free_links(*dims), ph * u[None, :], m, dims)
    np.testing.assert_allclose(got, ph * (Dp @ u)[None, :], atol=1e-14)


@pytest.mark.parametrize("dims", [(64, 64), (256, 256), (98, 34)])
def test_dslash_fp32_per_site_error_below_1e6(dims):
    # reference: FP64 D on the same FP32-rounded inputs; per-site error relative to
    # |diag psi_x| + 1/2 sum |hop terms_x| (bounds the cancellation at that site)
    lat = Lattice(dims)
    if dims[0] == dims[1]:
        U, _, _ = inputs.schwinger_links(dims[0], 6.0, sweeps=50, workload_id=8)
    else:
        U = inputs.hot_links(*dims, seed=4)
    psi = inputs.gaussian_complex(lat.volume * 2, 5, 1).reshape(-1, 2)
    U32 = U.astype(np.complex64).astype(np.complex128)
    p32 = psi.astype(np.complex64).astype(np.complex128)
    m = 0.02
    ref = wilson.apply_D(U32, p32, m, lat)
    scale = (2 + m) * np.abs(p32).sum(axis=1)
    for mu in range(2):
        for s in (+1, -1):
            scale += np.abs(wilson.hop(U32, p32, lat, mu, s)).sum(axis=1)
    got = _gpu_D(U32.astype(np.complex64), p32.astype(np.complex64), m, dims, precision=1)
    err = np.abs(got - ref).sum(axis=1) / scale
    assert err.max() < 1e-6, err.max()


def test_dslash_large_sampled_fp64():
    # full size of the bandwidth measurement: 4096^2, checked on sampled sites
    dims = (4096, 4096)
    lat = Lattice(dims)
    U = inputs.hot_links(*dims, seed=99)
    psi = inputs.gaussian_complex(lat.volume * 2, 9, 1).reshape(-1, 2)
    got = _gpu_D(U, psi, 0.01, dims)
    rng = np.random.default_rng(0)
    sites = np.concatenate([rng.integers(0, lat.volume, 4000), [0, lat.volume - 1, 4095, 4096 * 4095]])
    want = wilson.apply_D_at(U, psi, 0.01, lat, sites)
    assert np.abs(got[sites] - want).max() / np.abs(want).max() < 1e-14
