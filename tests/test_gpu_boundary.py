"""The boundary calls that serve the paper's reuse of one setup (its near-null space is
found once and then serves further masses and right-hand sides): saved setups, setups of
several configurations at once, mg_solve with nrhs > 1, and the timing and cost fields
of mg_stats. Solves are checked bit for bit against the paths they must reproduce and
by the true residual the oracle recomputes."""
import os

import numpy as np
import pytest

import inputs
from oracle import wilson
from oracle.lattice import Lattice
from tests._util import to_dev, to_host

pytestmark = pytest.mark.gpu


def _p2(precision, levels=3, **kw):
    import paper_0707_4018_gb300 as mg
    if levels == 3:
        return mg.mg_default_params(levels=3, blocks=[(4, 4), (2, 2)], Nv=[8, 8], precision=precision, n_pass=3,
                                    coarsest_tol=0.2, **kw)
    return mg.mg_default_params(levels=2, blocks=[(4, 4)], Nv=[8], precision=precision, n_pass=3, **kw)


@pytest.mark.parametrize("precision,levels", [(0, 2), (1, 3), (0, 3)])
def test_save_load_reproduces_solves_bitwise(tmp_path, precision, levels):
    import torch
    import paper_0707_4018_gb300 as mg
    L = 64
    dims = (L, L)
    U, _, _ = inputs.schwinger_links(L, 6.0, sweeps=200, workload_id=13)
    Ud = to_dev(U)
    m = 0.03
    p = _p2(precision, levels)
    a = mg.Context.setup(Ud, m, dims, p)
    chi = to_dev(inputs.gaussian_source(L, L, seed=5))
    psi_a = torch.empty_like(chi)
    st_a = a.solve(chi, psi_a, 1e-10)
    path = str(tmp_path / "setup.mgs")
    a.save(path)
    vec_a = [a.null_vectors(l).clone() for l in range(levels - 1)]
    Y_a = [a.coarse_op(l).clone() for l in range(1, levels)]
    a.close()
    b = mg.Context.load(path, Ud, dims)
    assert b.params.levels == levels and b.mass == m
    for l in range(levels - 1):
        assert torch.equal(b.null_vectors(l), vec_a[l])
    for l in range(1, levels):
        assert torch.equal(b.coarse_op(l), Y_a[l - 1])
    psi_b = torch.empty_like(chi)
    st_b = b.solve(chi, psi_b, 1e-10)
    assert st_b["converged"] and st_b["iters"] == st_a["iters"]
    assert torch.equal(psi_a, psi_b)
    # the rebuild runs no relaxation: it is cheaper than the setup it replaces
    assert 0.0 < st_b["setup_s"] and 0.0 < st_a["setup_s"]
    res = np.linalg.norm(to_host(chi) - wilson.apply_D(U, to_host(psi_b), m, Lattice(dims)))
    assert res / np.linalg.norm(to_host(chi)) <= 1e-10
    b.close()


def test_load_rejects_other_links_and_corrupt_files(tmp_path):
    import paper_0707_4018_gb300 as mg
    L = 32
    dims = (L, L)
    U, _, _ = inputs.schwinger_links(L, 6.0, sweeps=50, workload_id=14)
    a = mg.Context.setup(to_dev(U), 0.05, dims, _p2(0, levels=2))
    path = str(tmp_path / "s.mgs")
    a.save(path)
    a.close()
    U2, _, _ = inputs.schwinger_links(L, 6.0, sweeps=51, workload_id=14)
    with pytest.raises(mg.MGError) as e:
        mg.Context.load(path, to_dev(U2), dims)
    assert e.value.code == 1 and "digest" in str(e.value)
    raw = bytearray(open(path, "rb").read())
    raw[-5] ^= 0x40  # one flipped bit in the stored vectors
    bad = str(tmp_path / "bad.mgs")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(mg.MGError) as e:
        mg.Context.load(bad, to_dev(U), dims)
    assert e.value.code == 1 and "corrupt" in str(e.value)
    short = str(tmp_path / "short.mgs")
    open(short, "wb").write(bytes(raw[: len(raw) // 2]))
    with pytest.raises(mg.MGError):
        mg.Context.load(short, to_dev(U), dims)


def test_save_load_4d_bitwise(tmp_path):
    import torch
    import paper_0707_4018_gb300 as mg
    dims = (8, 8, 8, 8)
    U = inputs.su3_links(dims, seed=31)
    Ud = to_dev(U)
    p = mg.mg_default_params(levels=2, blocks=[(4, 4, 4, 4)], Nv=[6], precision=1, chiral_split=1, n_pass=1,
                             nu_setup=30, coarsest_tol=0.05, coarsest_restart=32)
    a = mg.Context.setup(Ud, 0.05, dims, p)
    chi = to_dev(np.ascontiguousarray(inputs.gaussian_spinor(8 ** 4, 12, 7, 0)))
    psi_a = torch.empty_like(chi)
    st_a = a.solve(chi, psi_a, 1e-10)
    path = str(tmp_path / "s4.mgs")
    a.save(path)
    a.close()
    b = mg.Context.load(path, Ud, dims)
    psi_b = torch.empty_like(chi)
    st_b = b.solve(chi, psi_b, 1e-10)
    assert st_a["converged"] and st_b["iters"] == st_a["iters"]
    assert torch.equal(psi_a, psi_b)
    b.close()


def test_setup_batch_equals_single_setups():
    import torch
    import paper_0707_4018_gb300 as mg
    sizes = [(32, 32), (64, 32), (64, 64)]
    Us = [inputs.schwinger_links(d[0], 6.0, sweeps=100, workload_id=15)[0] if d[0] == d[1] else
          inputs.links_from_angles(inputs.metropolis_u1_2d(d[0], d[1], 6.0, 100, seed=77)[0]) for d in sizes]
    ms = [0.04, 0.05, 0.06]
    ps = [_p2(1, levels=2), _p2(0, levels=2), _p2(1, levels=3)]
    Ud = [to_dev(U) for U in Us]
    batch = mg.Context.setup_batch(Ud, ms, sizes, ps)
    for i, d in enumerate(sizes):
        single = mg.Context.setup(Ud[i], ms[i], d, ps[i])
        for l in range(ps[i].levels - 1):
            assert torch.equal(batch[i].null_vectors(l), single.null_vectors(l))
        chi = to_dev(inputs.gaussian_source(d[0], d[1], seed=20 + i))
        x0, x1 = torch.empty_like(chi), torch.empty_like(chi)
        s0 = batch[i].solve(chi, x0, 1e-10)
        single.solve(chi, x1, 1e-10)
        assert s0["converged"] and torch.equal(x0, x1)
        res = np.linalg.norm(to_host(chi) - wilson.apply_D(Us[i], to_host(x0), ms[i], Lattice(d)))
        assert res / np.linalg.norm(to_host(chi)) <= 1e-10
        single.close()
        batch[i].close()


def test_setup_batch_reports_the_failing_configuration():
    import paper_0707_4018_gb300 as mg
    U, _, _ = inputs.schwinger_links(32, 6.0, sweeps=20, workload_id=16)
    good = _p2(0, levels=2)
    bad = mg.mg_default_params(levels=2, blocks=[(5, 4)], Nv=[8])
    with pytest.raises(mg.MGError) as e:
        mg.Context.setup_batch([to_dev(U), to_dev(U)], [0.1, 0.1], [(32, 32), (32, 32)], [good, bad])
    assert e.value.code == 1 and "configuration 1" in str(e.value)


def test_solve_nrhs_equals_solve_batch_and_stats():
    import torch
    import paper_0707_4018_gb300 as mg
    L = 64
    U, _, _ = inputs.schwinger_links(L, 6.0, sweeps=200, workload_id=13)
    p = _p2(1, levels=3, max_rhs=4)
    ctx = mg.Context.setup(to_dev(U), 0.03, (L, L), p)
    chi = torch.stack([to_dev(inputs.gaussian_source(L, L, seed=40 + k)) for k in range(3)])
    x_n, x_b = torch.empty_like(chi), torch.empty_like(chi)
    st_n = ctx.solve_nrhs(chi, x_n, 1e-10)
    st_b = ctx.solve_batch(chi, x_b, 1e-10)
    assert torch.equal(x_n, x_b)
    for a, b in zip(st_n, st_b):
        assert a["converged"] and a["iters"] == b["iters"]
        assert a["fine_D_apps"] == a["level_apps"][0] > 0
        assert abs(a["solve_s"] - a["ms"] * 1e-3) < 1e-12 and a["setup_s"] > 0
    x1 = torch.empty_like(chi[0])
    st1 = ctx.solve(chi[0], x1, 1e-10)
    # one outer iteration applies D once (w = D z) plus, per V-cycle, 2 nu + 1 fine applications
    nu = p.nu_pre + p.nu_post
    assert st1["fine_D_apps"] >= st1["iters"] * (1 + nu)
    ctx.close()
