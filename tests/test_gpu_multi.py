"""mg_solve_multi: the solves of several contexts (different lattices, configurations, masses and
precisions) in one graph launch, each outer flexible GCR running as a conditional WHILE loop on the
device. Every solution meets the tolerance by the oracle's FP64 true residual, with outer iteration
counts close to the host-driven loop's."""
import numpy as np
import pytest

import inputs
from oracle import wilson
from oracle.lattice import Lattice
from tests._util import to_dev, to_host

pytestmark = pytest.mark.gpu


def _case(L0, L1, beta, seed):
    th, _ = inputs.metropolis_u1_2d(L0, L1, beta, 200, seed=seed)
    return inputs.links_from_angles(th)


def test_multi_solve_several_configurations():
    import torch
    import paper_0707_4018_gb300 as mg
    specs = [((64, 64), 6.0, 0.03, 1, 3), ((32, 64), 3.0, 0.05, 0, 2), ((128, 128), 10.0, 0.02, 1, 3),
             ((64, 64), 6.0, 0.1, 1, 2)]
    ctxs, Us, chis, psis, single = [], [], [], [], []
    for i, (dims, beta, m, prec, levels) in enumerate(specs):
        U = _case(dims[0], dims[1], beta, 100 + i)
        blocks = [(4, 4), (2, 2)][: levels - 1]
        p = mg.mg_default_params(levels=levels, blocks=blocks, Nv=[8] * (levels - 1), precision=prec, n_pass=3,
                                 coarsest_tol=0.2, coarsest_lu_max=0 if levels == 3 else 2048)
        ctx = mg.Context.setup(to_dev(U), m, dims, p)
        chi = to_dev(inputs.gaussian_source(dims[0], dims[1], seed=7 + i))
        ref = torch.empty_like(chi)
        single.append(ctx.solve(chi, ref, 1e-10))
        ctxs.append(ctx)
        Us.append(U)
        chis.append(chi)
        psis.append(torch.empty_like(chi))
    st = mg.solve_multi(ctxs, chis, psis, 1e-10)
    for i, (dims, beta, m, prec, levels) in enumerate(specs):
        res = np.linalg.norm(to_host(chis[i]) - wilson.apply_D(Us[i], to_host(psis[i]), m, Lattice(dims)))
        assert st[i]["converged"] and res / np.linalg.norm(to_host(chis[i])) <= 1e-10, (i, st[i])
        assert st[i]["fine_D_apps"] > 0 and st[i]["graphs"]
        assert abs(st[i]["iters"] - single[i]["iters"]) <= max(3, single[i]["iters"] // 5), (st[i]["iters"],
                                                                                            single[i]["iters"])
    # a second call on the same contexts gives the same iterates (deterministic loop)
    psis2 = [torch.empty_like(c) for c in chis]
    st2 = mg.solve_multi(ctxs, chis, psis2, 1e-10)
    for i in range(len(specs)):
        assert st2[i]["iters"] == st[i]["iters"] and torch.equal(psis2[i], psis[i])
    for c in ctxs:
        c.close()


def test_multi_solve_rejects_repeated_context():
    import torch
    import paper_0707_4018_gb300 as mg
    U = _case(32, 32, 6.0, 5)
    ctx = mg.Context.setup(to_dev(U), 0.05, (32, 32), mg.mg_default_params(n_pass=2))
    chi = to_dev(inputs.gaussian_source(32, 32, seed=1))
    with pytest.raises(mg.MGError) as e:
        mg.solve_multi([ctx, ctx], [chi, chi], [torch.empty_like(chi), torch.empty_like(chi)], 1e-10)
    assert e.value.code == 1
    ctx.close()


def test_multi_solve_batches_of_right_hand_sides():
    # contexts with several right-hand sides each, solved in lockstep inside their WHILE loops;
    # with 8 or more vectors in FP32 cycles the coarse residual applies run on tensor cores
    import torch
    import paper_0707_4018_gb300 as mg
    specs = [((64, 64), 6.0, 0.03, 1, 8), ((32, 64), 3.0, 0.05, 1, 3), ((64, 32), 10.0, 0.04, 0, 2)]
    ctxs, Us, chis, psis, nrhs = [], [], [], [], []
    for i, (dims, beta, m, prec, nr) in enumerate(specs):
        U = _case(dims[0], dims[1], beta, 200 + i)
        p = mg.mg_default_params(levels=3, blocks=[(4, 4), (2, 2)], Nv=[8, 8], precision=prec, n_pass=3,
                                 coarsest_tol=0.2, coarsest_lu_max=0, max_rhs=8)
        ctx = mg.Context.setup(to_dev(U), m, dims, p)
        chi = torch.stack([to_dev(inputs.gaussian_source(dims[0], dims[1], seed=30 + 10 * i + v)) for v in range(nr)])
        ctxs.append(ctx)
        Us.append(U)
        chis.append(chi)
        psis.append(torch.empty_like(chi))
        nrhs.append(nr)
    st = mg.solve_multi(ctxs, chis, psis, 1e-10, nrhs=nrhs)
    assert len(st) == sum(nrhs)
    e = 0
    for i, (dims, beta, m, prec, nr) in enumerate(specs):
        ref = torch.empty_like(chis[i])
        sb = ctxs[i].solve_batch(chis[i], ref, 1e-10)
        for v in range(nr):
            x = to_host(psis[i][v])
            b = to_host(chis[i][v])
            res = np.linalg.norm(b - wilson.apply_D(Us[i], x, m, Lattice(dims))) / np.linalg.norm(b)
            assert st[e]["converged"] and res <= 1e-10, (i, v, st[e], res)
            assert st[e]["iters"] <= sb[v]["iters"] + max(4, sb[v]["iters"] // 4), (st[e]["iters"], sb[v]["iters"])
            e += 1
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("kernel", ["smem", "large32", "large64"])
def test_concurrent_cooperative_coarsest_solves(kernel, monkeypatch):
    # Contexts whose coarsest solve is a cooperative kernel (grid barriers over many CTAs): their
    # setups run at once (mg_setup_batch, one stream each), their solves run from several host
    # threads and from one multi-context graph. Cooperative launches pass through one lane per
    # device, so none of them waits on CTAs that another one keeps off the GPU: every call
    # succeeds, and the results equal those of the same contexts run one at a time.
    import threading
    import torch
    import paper_0707_4018_gb300 as mg
    monkeypatch.setenv("MG_NO_CLUSTER_COARSEST", "1")
    if kernel != "smem":
        monkeypatch.setenv("MG_NO_SMEM_COARSEST", "1")
    tol_c = 1e-8 if kernel == "large64" else 0.2
    n = 6
    dims = (64, 64)
    Us = [_case(64, 64, 6.0, 300 + i) for i in range(n)]
    ms = [0.03 + 0.01 * i for i in range(n)]
    p = mg.mg_default_params(levels=3, blocks=[(4, 4), (2, 2)], Nv=[8, 8], precision=1, n_pass=2,
                             coarsest_tol=tol_c, coarsest_lu_max=0)
    together = mg.Context.setup_batch([to_dev(U) for U in Us], ms, [dims] * n, [p] * n)
    alone = [mg.Context.setup(to_dev(U), m, dims, p) for U, m in zip(Us, ms)]
    chis = [to_dev(inputs.gaussian_source(64, 64, seed=40 + i)) for i in range(n)]
    ref = [torch.empty_like(c) for c in chis]
    st_ref = [alone[i].solve(chis[i], ref[i], 1e-10) for i in range(n)]
    # host threads, one solve each, all at once
    out = [torch.empty_like(c) for c in chis]
    st_thr = [None] * n
    err = []

    def run(i):
        try:
            st_thr[i] = together[i].solve(chis[i], out[i], 1e-10)
        except Exception as e:  # noqa: BLE001 - reported below
            err.append(e)
    th = [threading.Thread(target=run, args=(i,)) for i in range(n)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not err, err
    torch.cuda.synchronize()
    for i in range(n):
        assert st_thr[i]["converged"] and st_thr[i]["iters"] == st_ref[i]["iters"], (i, st_thr[i], st_ref[i])
        assert torch.equal(out[i], ref[i])
    # one graph launch for all of them
    outm = [torch.empty_like(c) for c in chis]
    st_m = mg.solve_multi(together, chis, outm, 1e-10)
    for i in range(n):
        res = np.linalg.norm(to_host(chis[i]) - wilson.apply_D(Us[i], to_host(outm[i]), ms[i], Lattice(dims)))
        assert st_m[i]["converged"] and res / np.linalg.norm(to_host(chis[i])) <= 1e-10, (i, st_m[i])
    for c in together + alone:
        c.close()
