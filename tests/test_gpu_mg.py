"""GPU parity of the multigrid steps with the oracle, through the C ABI.

Hierarchies are fixed by near-null vectors taken from the seeded input
generator, handed to both sides (mg_build_level / Hierarchy.build_level), so
block Gram-Schmidt, the Galerkin operators, restriction, prolongation, the
smoother, the V-cycle and the coarsest solve are compared on identical inputs.
The random draws of the adaptive setup are compared separately (both sides
implement Philox4x32-10 + Box-Muller; they differ only by libm rounding).
"""
import numpy as np
import pytest

import inputs
from oracle import coarse, setup, solvers, transfer, wilson
from oracle.lattice import Lattice
from tests._util import rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu


def _mg():
    import paper_0707_4018_gb300 as mg
    return mg


def _vectors(lat_volume, n_int, nv, seed, tag0=500):
    return np.stack([inputs.gaussian_complex(lat_volume * n_int, seed, tag0 + k).reshape(lat_volume, n_int)
                     for k in range(nv)])


def make_pair(dims, m, blocks, Nv, U, seed=11, precision=0, **kw):
    """Oracle hierarchy and GPU context built from the same seeded vectors."""
    mg = _mg()
    lat = Lattice(dims)
    levels = len(blocks) + 1
    p = setup.MGParams(levels=levels, blocks=tuple(blocks), Nv=tuple(Nv), **kw)
    hier = setup.Hierarchy(coarse.WilsonOperator(U, m, lat), p)
    gp = mg.mg_default_params(levels=levels, blocks=blocks, Nv=Nv, n_pass=1, nu_setup=0, precision=precision,
                              **{k: v for k, v in kw.items() if k in ("coarsest_lu_max", "coarsest_tol",
                                                                      "coarsest_restart", "nu_pre", "nu_post")})
    ctx = mg.Context.setup(to_dev(U), m, dims, gp)
    vecs_all = []
    n_sites, n_int = lat.volume, 2
    for l in range(levels - 1):
        v = _vectors(n_sites, n_int, Nv[l], seed + l)
        vecs_all.append(v)
        hier.build_level(l, list(v))
        ctx.build_level(l, to_dev(v))
        n_sites = hier.blk[l].coarse.volume
        n_int = Nv[l]
    hier.prepare_coarsest()
    return hier, ctx, vecs_all


def _U(dims, seed=5):
    return inputs.hot_links(*dims, seed=seed)


@pytest.mark.parametrize("dims,blocks,Nv", [((16, 16), [(4, 4)], [8]), ((8, 8), [(4, 4)], [8]),
                                            ((4, 8), [(4, 4)], [3]), ((32, 32), [(4, 4), (2, 2)], [8, 8]),
                                            ((24, 16), [(4, 2), (3, 2)], [5, 6])])
def test_prolongator_and_galerkin_match_oracle(dims, blocks, Nv):
    hier, ctx, _ = make_pair(dims, 0.1, blocks, Nv, _U(dims), coarsest_lu_max=100000)
    for l in range(len(blocks)):
        P = to_host(ctx.prolongator(l))
        want = np.stack([transfer.from_blocks(hier.P[l][:, :, k], hier.blk[l], hier.n_int(l)) for k in range(Nv[l])])
        assert np.abs(P - want).max() < 1e-13
        Y = to_host(ctx.coarse_op(l + 1))
        Yw = hier.ops[l + 1].Y
        assert np.abs(Y - Yw).max() / np.abs(Yw).max() < 1e-13, l


def test_restrict_prolong_apply_match_oracle():
    dims = (32, 32)
    hier, ctx, _ = make_pair(dims, 0.05, [(4, 4), (2, 2)], [8, 8], _U(dims), coarsest_lu_max=100000)
    import torch
    for l in range(2):
        n_f, k_f = ctx.level_size(l)
        n_c, k_c = ctx.level_size(l + 1)
        r = inputs.gaussian_complex(n_f * k_f, 3, 10 + l).reshape(n_f, k_f)
        e = inputs.gaussian_complex(n_c * k_c, 3, 20 + l).reshape(n_c, k_c)
        rc = torch.empty((n_c, k_c), dtype=torch.complex128, device="cuda")
        ctx.restrict(l, to_dev(r), rc)
        assert rel_err(to_host(rc), hier.restrict(l, r)) < 1e-14
        f = torch.empty((n_f, k_f), dtype=torch.complex128, device="cuda")
        ctx.prolong(l, to_dev(e), f)
        assert rel_err(to_host(f), hier.prolong(l, e)) < 1e-14
    for l in range(3):
        n, k = ctx.level_size(l)
        x = inputs.gaussian_complex(n * k, 4, 30 + l).reshape(n, k)
        y = torch.empty_like(to_dev(x))
        ctx.level_apply(l, to_dev(x), y)
        assert rel_err(to_host(y), hier.ops[l].apply(x)) < 1e-14


@pytest.mark.parametrize("level", [0, 1])
def test_mr_smoother_matches_oracle(level):
    dims = (32, 32)
    hier, ctx, _ = make_pair(dims, 0.05, [(4, 4), (2, 2)], [8, 8], _U(dims), coarsest_lu_max=100000)
    import torch
    n, k = ctx.level_size(level)
    b = inputs.gaussian_complex(n * k, 5, 40).reshape(n, k)
    x = torch.empty((n, k), dtype=torch.complex128, device="cuda")
    ctx.smooth(level, to_dev(b), x, 4)
    want, _ = solvers.mr(hier.ops[level].apply, b, 4, 0.8)
    assert rel_err(to_host(x), want) < 1e-13


@pytest.mark.parametrize("dims,blocks,Nv,lu_max", [((16, 16), [(4, 4)], [8], 2048), ((32, 32), [(4, 4), (2, 2)], [8, 8], 4096),
                                                   ((32, 32), [(4, 4), (2, 2)], [8, 8], 0)])
def test_vcycle_matches_oracle(dims, blocks, Nv, lu_max):
    U, _, _ = inputs.schwinger_links(dims[0], 6.0, sweeps=100, workload_id=5)
    hier, ctx, _ = make_pair(dims, 0.0, blocks, Nv, U, coarsest_lu_max=lu_max, coarsest_tol=1e-13)
    import torch
    lat = Lattice(dims)
    b = inputs.gaussian_source(*dims, seed=6)
    x = torch.empty((lat.volume, 2), dtype=torch.complex128, device="cuda")
    ctx.vcycle(to_dev(b), x)
    want = solvers.vcycle(hier, 0, b)
    assert rel_err(to_host(x), want) < 1e-10


def test_setup_first_pass_matches_oracle():
    # pass 1 only: Philox draws relaxed by MR on A x = 0; both sides draw with their own
    # Philox4x32-10 + Box-Muller implementation
    mg = _mg()
    dims = (32, 32)
    lat = Lattice(dims)
    U, _, _ = inputs.schwinger_links(32, 6.0, sweeps=100, workload_id=5)
    p = setup.MGParams(levels=3, blocks=((4, 4), (2, 2)), Nv=(8, 8), n_pass=1, seed=12345)
    hier = setup.adaptive_setup(U, 0.02, lat, p)
    gp = mg.mg_default_params(levels=3, blocks=[(4, 4), (2, 2)], Nv=[8, 8], n_pass=1, seed=12345)
    ctx = mg.Context.setup(to_dev(U), 0.02, dims, gp)
    for l in range(2):
        v = to_host(ctx.null_vectors(l))
        want = np.stack(hier.vecs[l])
        assert rel_err(v, want) < 1e-12, l
        assert rel_err(to_host(ctx.coarse_op(l + 1)), hier.ops[l + 1].Y) < 1e-12


@pytest.mark.parametrize("levels", [2, 3])
def test_full_adaptive_setup_matches_oracle(levels):
    mg = _mg()
    dims = (32, 32)
    lat = Lattice(dims)
    U, _, _ = inputs.schwinger_links(32, 6.0, sweeps=200, workload_id=5)
    blocks = [(4, 4), (2, 2)][:levels - 1]
    p = setup.MGParams(levels=levels, blocks=tuple(blocks), Nv=(8,) * (levels - 1), n_pass=3, seed=777,
                       coarsest_lu_max=4096)
    hier = setup.adaptive_setup(U, 0.0, lat, p)
    gp = mg.mg_default_params(levels=levels, blocks=blocks, Nv=[8] * (levels - 1), n_pass=3, seed=777,
                              coarsest_lu_max=4096)
    ctx = mg.Context.setup(to_dev(U), 0.0, dims, gp)
    for l in range(levels - 1):
        assert rel_err(to_host(ctx.null_vectors(l)), np.stack(hier.vecs[l])) < 1e-9, l
        assert rel_err(to_host(ctx.coarse_op(l + 1)), hier.ops[l + 1].Y) < 1e-9, l


@pytest.mark.parametrize("n_pass", [1, 3])
def test_fp32_setup_close_to_oracle(n_pass):
    # mixed-precision contexts relax and adapt the near-null vectors in FP32 (Gram-Schmidt and
    # the Galerkin build stay FP64): the vectors and coarse operators agree with the FP64 oracle
    # setup to FP32 rounding amplified by the relaxation, and both solve in the same number of
    # outer iterations
    mg = _mg()
    dims = (32, 32)
    lat = Lattice(dims)
    U, _, _ = inputs.schwinger_links(32, 6.0, sweeps=200, workload_id=5)
    p = setup.MGParams(levels=3, blocks=((4, 4), (2, 2)), Nv=(8, 8), n_pass=n_pass, seed=777, coarsest_lu_max=4096)
    hier = setup.adaptive_setup(U, 0.02, lat, p)
    gp = mg.mg_default_params(levels=3, blocks=[(4, 4), (2, 2)], Nv=[8, 8], n_pass=n_pass, seed=777,
                              coarsest_lu_max=4096, precision=1)
    ctx = mg.Context.setup(to_dev(U), 0.02, dims, gp)
    for l in range(2):
        assert rel_err(to_host(ctx.null_vectors(l)), np.stack(hier.vecs[l])) < 1e-4, l
        assert rel_err(to_host(ctx.coarse_op(l + 1)), hier.ops[l + 1].Y) < 1e-4, l
    import torch
    chi = inputs.gaussian_source(*dims, seed=9)
    psi = torch.empty((1024, 2), dtype=torch.complex128, device="cuda")
    st = ctx.solve(to_dev(chi), psi, 1e-10)
    _, info = solvers.mg_solve(hier, chi, 1e-10)
    assert st["converged"] and abs(st["iters"] - info["iters"]) <= 1


@pytest.mark.parametrize("dims,lu_max", [((32, 32), 100000), ((32, 32), 0), ((64, 64), 0)])
def test_coarsest_solve_matches_oracle(dims, lu_max):
    # the coarsest exact solve alone: dense LU, or the persistent GCR kernel to 1e-12
    import torch
    U, _, _ = inputs.schwinger_links(dims[0], 6.0, sweeps=100, workload_id=5)
    hier, ctx, _ = make_pair(dims, 0.02, [(4, 4), (2, 2)], [8, 8], U, coarsest_lu_max=lu_max, coarsest_tol=1e-12)
    n, k = ctx.level_size(2)
    b = inputs.gaussian_complex(n * k, 8, 80).reshape(n, k)
    x = torch.empty((n, k), dtype=torch.complex128, device="cuda")
    iters, ms = ctx.coarsest_solve(to_dev(b), x)
    assert (iters == 0) == (lu_max > 0) and ms > 0
    want = np.linalg.solve(solvers.stencil_matrix(hier.ops[2]), b.reshape(-1)).reshape(n, k)
    assert rel_err(to_host(x), want) < 1e-9


def test_mixed_precision_vcycle_close_to_oracle():
    # FP32 smoother / transfers / coarse operators (FP64 coarsest) against the FP64 oracle cycle:
    # the difference is FP32 rounding amplified by the cycle, far below the cycle's own action
    import torch
    dims = (32, 32)
    U, _, _ = inputs.schwinger_links(32, 6.0, sweeps=100, workload_id=5)
    hier, ctx, _ = make_pair(dims, 0.02, [(4, 4), (2, 2)], [8, 8], U, precision=1, coarsest_lu_max=4096)
    b = inputs.gaussian_source(*dims, seed=6)
    x = torch.empty((1024, 2), dtype=torch.complex128, device="cuda")
    ctx.vcycle(to_dev(b), x)
    want = solvers.vcycle(hier, 0, b)
    err = rel_err(to_host(x), want)
    assert err < 1e-5, err


def test_update_mass_matches_oracle():
    import torch
    dims = (32, 32)
    U, _, _ = inputs.schwinger_links(32, 6.0, sweeps=100, workload_id=5)
    hier, ctx, _ = make_pair(dims, 0.0, [(4, 4), (2, 2)], [8, 8], U, coarsest_lu_max=4096)
    # a cycle at the old mass first: its captured graph must not survive the mass change
    b0 = inputs.gaussian_source(*dims, seed=8)
    x0 = torch.empty((1024, 2), dtype=torch.complex128, device="cuda")
    ctx.vcycle(to_dev(b0), x0)
    ctx.update_mass(0.31)
    setup.update_mass(hier, 0.31)
    for l in (1, 2):
        assert rel_err(to_host(ctx.coarse_op(l)), hier.ops[l].Y) < 1e-13
    b = inputs.gaussian_source(*dims, seed=7)
    x = torch.empty((1024, 2), dtype=torch.complex128, device="cuda")
    ctx.vcycle(to_dev(b), x)
    assert rel_err(to_host(x), solvers.vcycle(hier, 0, b)) < 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_is_bitwise_reproducible(precision):
    # fixed-order reductions everywhere: two runs give identical bits
    import torch
    import paper_0707_4018_gb300 as mg
    L = 64
    U = to_dev(inputs.links_from_angles(inputs.metropolis_u1_2d(L, L, 6.0, 100, seed=3)[0]))
    chi = to_dev(inputs.gaussian_source(L, L, seed=4))
    outs = []
    for _ in range(2):
        ctx = mg.Context.setup(U, 0.0, (L, L), mg.mg_default_params(levels=3, blocks=[(4, 4), (2, 2)], Nv=[8, 8],
                                                                     precision=precision, coarsest_lu_max=0,
                                                                     coarsest_tol=1e-3))
        psi = torch.empty_like(chi)
        ctx.solve(chi, psi, 1e-10)
        outs.append(to_host(psi))
        ctx.close()
    assert np.array_equal(outs[0].view(np.uint64), outs[1].view(np.uint64))


@pytest.mark.parametrize("kernel", ["cluster", "smem_fp32_stencil", "large32"])
def test_fp32_stencil_coarsest_solve_meets_its_tolerance(kernel, monkeypatch):
    # mixed precision with a loose coarsest tolerance: the one-cluster FP32 GCR, (cluster kernel
    # switched off) A M stored and applied in FP32 inside the whole-chip FP64 GCR, or (both
    # switched off, the path of large coarsest levels) the whole-chip FP32 GCR with FP64 sums;
    # the solution meets the tolerance against the oracle's FP64 coarse operator
    import torch
    if kernel != "cluster":
        monkeypatch.setenv("MG_NO_CLUSTER_COARSEST", "1")
    if kernel == "large32":
        monkeypatch.setenv("MG_NO_SMEM_COARSEST", "1")
    dims = (64, 64)
    U, _, _ = inputs.schwinger_links(64, 6.0, sweeps=100, workload_id=5)
    hier, ctx, _ = make_pair(dims, 0.02, [(4, 4), (2, 2)], [8, 8], U, precision=1, coarsest_lu_max=0,
                             coarsest_tol=1e-4)
    n, k = ctx.level_size(2)
    A = solvers.stencil_matrix(hier.ops[2])
    for seed in (8, 9):
        b = inputs.gaussian_complex(n * k, seed, 80).reshape(n, k)
        x = torch.empty((n, k), dtype=torch.complex128, device="cuda")
        iters, _ = ctx.coarsest_solve(to_dev(b), x)
        res = np.linalg.norm(b.reshape(-1) - A @ to_host(x).reshape(-1)) / np.linalg.norm(b)
        assert 0 < iters < 200 and res <= 1.5e-4, (iters, res)


@pytest.mark.parametrize("kernel", ["cluster", "smem"])
def test_mixed_solve_with_loose_coarsest_reaches_true_residual(kernel, monkeypatch):
    # the bench's configuration (3 levels, coarsest tolerance 0.2): the setup's batched V-cycles
    # (one cluster per vector) and the solve's cycles; the FP64 outer loop reaches 1e-10
    import torch
    import paper_0707_4018_gb300 as mg
    if kernel != "cluster":
        monkeypatch.setenv("MG_NO_CLUSTER_COARSEST", "1")
    L = 128
    U, _, _ = inputs.schwinger_links(L, 6.0, sweeps=200, workload_id=5)
    p = mg.mg_default_params(levels=3, blocks=[(4, 4), (2, 2)], Nv=[8, 8], precision=1, coarsest_tol=0.2,
                             coarsest_lu_max=0)
    ctx = mg.Context.setup(to_dev(U), 0.02, (L, L), p)
    chi = inputs.gaussian_source(L, L, seed=12)
    psi = torch.empty((L * L, 2), dtype=torch.complex128, device="cuda")
    st = ctx.solve(to_dev(chi), psi, 1e-10)
    res = np.linalg.norm(chi - wilson.apply_D(U, to_host(psi), 0.02, Lattice((L, L)))) / np.linalg.norm(chi)
    assert st["converged"] and res <= 1e-10 and st["coarsest_iters"] > 0
    ctx.close()
