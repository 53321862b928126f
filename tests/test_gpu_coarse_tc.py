"""Tensor-core coarse apply (mg_coarse_apply_mrhs): BF16 operands, FP32 sums.

Two comparisons per case:
- against the oracle's stencil apply in FP64 of the same operands rounded to BF16 (round to
  nearest even, emulated in numpy from the FP32 values): the only difference left is the
  FP32 summation of 80 products per output, bounded per site by 1e-5 of sum |Y| |x|;
- against the exact FP64 apply: the BF16 rounding error, stated (about 2^-8 of sum |Y| |x|).
"""
import numpy as np
import pytest

import inputs
from oracle.coarse import StencilOperator
from oracle.lattice import Lattice
from tests._util import to_dev, to_host

pytestmark = pytest.mark.gpu


def bf16(a):
    """float32 values rounded to bfloat16 (round to nearest, ties to even), as float32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def bf16c(z):
    z = np.asarray(z, dtype=np.complex64)
    return bf16(z.real).astype(np.float64) + 1j * bf16(z.imag).astype(np.float64)


@pytest.mark.parametrize("level", [1, 2])
@pytest.mark.parametrize("nrhs", [1, 8, 13, 16])
def test_tensor_core_apply_matches_bf16_reference(level, nrhs):
    import torch
    import paper_0707_4018_gb300 as mg
    dims = (64, 64)
    U, _, _ = inputs.schwinger_links(64, 6.0, sweeps=100, workload_id=5)
    p = mg.mg_default_params(levels=3, blocks=[(4, 4), (2, 2)], Nv=[8, 8], precision=1, n_pass=2)
    ctx = mg.Context.setup(to_dev(U), 0.05, dims, p)
    n_sites, n_int = ctx.level_size(level)
    side = (dims[0] // (4 if level == 1 else 8), dims[1] // (4 if level == 1 else 8))
    lat = Lattice(side)
    assert lat.volume == n_sites and n_int == 8
    Y = to_host(ctx.coarse_op(level)).reshape(n_sites, 5, 8, 8)
    x = np.stack([inputs.gaussian_complex(n_sites * 8, 70 + level, 900 + k).reshape(n_sites, 8)
                  for k in range(nrhs)]).astype(np.complex64)
    out = torch.empty((nrhs, n_sites, 8), dtype=torch.complex64, device="cuda")
    ctx.coarse_apply_mrhs(level, to_dev(x), out)
    got = to_host(out).astype(np.complex128)
    Yb = bf16c(Y.astype(np.complex64))
    op_b = StencilOperator(Yb, lat)
    op_abs = StencilOperator(np.abs(Yb), lat)
    op_exact = StencilOperator(Y, lat)
    worst_emul, worst_exact = 0.0, 0.0
    for k in range(nrhs):
        xb = bf16c(x[k])
        ref = op_b.apply(xb)
        bound = op_abs.apply(np.abs(xb)).real
        worst_emul = max(worst_emul, float(np.max(np.abs(got[k] - ref) / bound)))
        exact = op_exact.apply(x[k].astype(np.complex128))
        worst_exact = max(worst_exact, float(np.max(np.abs(got[k] - exact) / bound)))
    assert worst_emul <= 1e-5, worst_emul
    # the BF16 rounding of both operands: at most about 2 * 2^-8 of sum |Y| |x| per site
    assert worst_exact <= 1e-2, worst_exact


def test_tensor_core_apply_needs_fp32_context():
    import torch
    import paper_0707_4018_gb300 as mg
    dims = (32, 32)
    U = inputs.hot_links(*dims, seed=2)
    ctx = mg.Context.setup(to_dev(U), 0.1, dims, mg.mg_default_params(levels=3, blocks=[(4, 4), (2, 2)],
                                                                       Nv=[8, 8], precision=0))
    x = torch.zeros((2, 64, 8), dtype=torch.complex64, device="cuda")
    with pytest.raises(mg.MGError) as e:
        ctx.coarse_apply_mrhs(1, x, torch.empty_like(x))
    assert e.value.code == 6


def test_autotuner_picks_a_tile_shape_and_keeps_results():
    import torch
    import paper_0707_4018_gb300 as mg
    dims = (32, 32)
    U = inputs.hot_links(*dims, seed=3)
    ctx = mg.Context.setup(to_dev(U), 0.2, dims, mg.mg_default_params(levels=3, blocks=[(4, 4), (2, 2)],
                                                                       Nv=[8, 8], precision=1, n_pass=1))
    n_sites, _ = ctx.level_size(1)
    x = torch.from_numpy(np.stack([inputs.gaussian_complex(n_sites * 8, 77, k) for k in range(11)])
                         .astype(np.complex64).reshape(11, n_sites, 8)).cuda()
    y1, y2 = torch.empty_like(x), torch.empty_like(x)
    ctx.coarse_apply_mrhs(1, x, y1)  # first call: the six shapes are timed
    ctx.coarse_apply_mrhs(1, x, y2)  # cached shape
    rep = mg.autotune_report()
    key = "coarse_apply_tc/8x8/nvec11"
    assert key in rep and 0 <= rep[key] < 6, rep
    assert torch.equal(y1, y2)
    # the split-operand forms are built for the 4d level only; out-of-range modes are rejected
    for mode, code in ((2, 6), (3, 6), (4, 1), (-1, 1)):
        with pytest.raises(mg.MGError) as e:
            ctx.coarse_apply_mrhs(1, x, y2, mode)
        assert e.value.code == code, (mode, e.value.code)


@pytest.mark.parametrize("nrhs", [1, 8, 12, 16])
def test_tensor_core_apply_4d_matches_bf16_reference(nrhs):
    import torch
    import paper_0707_4018_gb300 as mg
    dims = (8, 8, 8, 16)
    U = inputs.su3_links(dims, seed=31)
    p = mg.mg_default_params(levels=2, blocks=[(4, 4, 4, 4)], Nv=[24], precision=1, chiral_split=1, n_pass=1,
                             nu_setup=4)
    ctx = mg.Context.setup(to_dev(U), 0.1, dims, p)
    n_sites, n_int = ctx.level_size(1)
    lat = Lattice((2, 2, 2, 4))
    assert lat.volume == n_sites and n_int == 48
    Y = to_host(ctx.coarse_op(1))  # [j][dir][row][col]
    x = np.stack([inputs.gaussian_complex(n_sites * 48, 80, 900 + k).reshape(n_sites, 48)
                  for k in range(nrhs)]).astype(np.complex64)
    out_tc = torch.empty((nrhs, n_sites, 48), dtype=torch.complex64, device="cuda")
    out_cc = torch.empty_like(out_tc)
    ctx.coarse_apply_mrhs(1, to_dev(x), out_tc, True)
    ctx.coarse_apply_mrhs(1, to_dev(x), out_cc, False)
    got, cc = to_host(out_tc).astype(np.complex128), to_host(out_cc).astype(np.complex128)
    Yb = bf16c(Y.astype(np.complex64))
    op_b, op_abs, op_exact = StencilOperator(Yb, lat), StencilOperator(np.abs(Yb), lat), StencilOperator(Y, lat)
    worst_emul = worst_exact = worst_cc = 0.0
    for k in range(nrhs):
        xb = bf16c(x[k])
        bound = op_abs.apply(np.abs(xb)).real
        exact = op_exact.apply(x[k].astype(np.complex128))
        worst_emul = max(worst_emul, float(np.max(np.abs(got[k] - op_b.apply(xb)) / bound)))
        worst_exact = max(worst_exact, float(np.max(np.abs(got[k] - exact) / bound)))
        worst_cc = max(worst_cc, float(np.max(np.abs(cc[k] - exact) / bound)))
    assert worst_emul <= 1e-5, worst_emul       # only the FP32 summation of 432 products differs
    assert worst_exact <= 1e-2, worst_exact     # the BF16 rounding of both operands
    assert worst_cc <= 1e-5, worst_cc           # the FP32 CUDA-core path
    # split operands: vectors as BF16 hi + lo (the operator's rounding is left), then the operator
    # too (hi hi + hi lo + lo hi: the dropped lo lo term and the FP32 sums are left)
    for mode, bound_emul, bound_exact in ((2, 1e-5, 1e-2), (3, None, 2e-5)):
        out_s = torch.empty_like(out_tc)
        ctx.coarse_apply_mrhs(1, to_dev(x), out_s, mode)
        got_s = to_host(out_s).astype(np.complex128)
        w_emul = w_exact = 0.0
        for k in range(nrhs):
            bound = op_abs.apply(np.abs(x[k]).astype(np.float64)).real
            exact = op_exact.apply(x[k].astype(np.complex128))
            w_exact = max(w_exact, float(np.max(np.abs(got_s[k] - exact) / bound)))
            if bound_emul is not None:  # the exact product with the BF16 operator
                w_emul = max(w_emul, float(np.max(np.abs(got_s[k] - op_b.apply(x[k].astype(np.complex128))) / bound)))
        assert w_exact <= bound_exact, (mode, w_exact)
        if bound_emul is not None:
            assert w_emul <= bound_emul, (mode, w_emul)
    assert w_exact < worst_exact / 50  # the split operator gains more than 5 bits over BF16
    with pytest.raises(mg.MGError):
        ctx.coarse_apply_mrhs(1, to_dev(x), out_tc, 4)
    ctx.close()
