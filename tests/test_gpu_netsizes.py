"""The network sizes of Table 1 (GRU hidden size m x stacked cells n, m in
{32, 64}, n in {1, 2, 3}) on the tensor-core kernels against the oracle: one
recurrent step for many patches, the gradient of the Eq. 7 loss by
backpropagation through time, Adam learning, and a whole DNN-MG time step.
Also Table 1's own networks (bias-free GRUs, one dense layer, 51 inputs,
18 outputs) with their parameter counts.  Tolerances as for the default
64 x 2 network: outputs 5e-3 and hidden states 2e-3 relative L2 (bfloat16
operands, FP32 accumulation), gradient 5e-3 (1e-2 per parameter block)
against the oracle rounding its backward's product inputs as the kernels
do, loss 1e-3, DNN-MG states 1e-4."""
import ctypes

import numpy as np
import pytest

import synthetic
from oracle import dnnmg, fem, mesh, net, newton
from tests.gpu_util import lib, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SIZES = [(32, 1), (64, 1), (32, 2), (64, 2), (32, 3), (64, 3)]


def _ctx(dn, m, n, **kw):
    return dn.Context(level_solve=2, hidden=m, gru_layers=n, **kw)


@pytest.mark.parametrize("m,n", SIZES)
@pytest.mark.parametrize("P", [1000, 61440])
def test_patch_infer_matches_oracle(m, n, P):
    dn = lib()
    ctx = _ctx(dn, m, n)
    spec = net.NetSpec(hidden=m, layers=n)
    assert ctx.num_params() == spec.num_params()
    w = synthetic.random_weights(m + n, spec.num_params(), 0.25).astype(np.float32)
    ctx.set_weights(w)
    x = net.bf16_round(synthetic.random_patch_inputs(P + n, (P, spec.c_in)))
    h = synthetic.random_patch_inputs(P + m, (n, P, m), 0.5).astype(np.float32).astype(np.float64)
    hg = torch.from_numpy(h).float().cuda()
    out = ctx.patch_infer(torch.from_numpy(x).to(torch.bfloat16).cuda(), hg)
    y_ref, h_ref = net.step_forward(spec, spec.unflatten(w.astype(np.float64)), x, h, bf16=True)
    assert rel(out.double().cpu().numpy(), y_ref) < 5e-3
    assert rel(hg.double().cpu().numpy(), h_ref) < 2e-3


@pytest.mark.parametrize("m,n", SIZES)
def test_gradient_matches_oracle(m, n):
    dn = lib()
    B, T = 48, 3
    ctx = _ctx(dn, m, n, train_batch=B, train_seq=T)
    spec = net.NetSpec(hidden=m, layers=n)
    w = synthetic.random_weights(7 * m + n, spec.num_params(), 0.2).astype(np.float32)
    ctx.set_weights(w)
    X = net.bf16_round(synthetic.random_patch_inputs(m + 3 * n, (B, T, spec.c_in)))
    Y = synthetic.random_patch_inputs(m + 3 * n + 1, (B, T, spec.c_out), 0.3)
    Xg = torch.from_numpy(X).to(torch.bfloat16).cuda().contiguous()
    Yg = torch.from_numpy(Y).float().cuda().contiguous()
    g = torch.empty(ctx.num_params(), dtype=torch.float32, device="cuda")
    loss = ctypes.c_float()
    ctx._check(ctx.lib.dnnmg_train_grad(ctx.h, dn._ptr(Xg), dn._ptr(Yg), B, T, dn._ptr(g),
                                        ctypes.byref(loss)))
    g = g.double().cpu().numpy()
    L_ref, g_ref = net.sequence_backward(spec, spec.unflatten(w.astype(np.float64)), X,
                                         Y.astype(np.float32).astype(np.float64), bf16=True,
                                         bf16_grad=True)
    assert abs(loss.value - L_ref) < 1e-3 * L_ref, (loss.value, L_ref)
    assert rel(g, g_ref) < 5e-3, rel(g, g_ref)
    o = 0
    for name, shape in spec.shapes():
        k = int(np.prod(shape))
        assert rel(g[o:o + k], g_ref[o:o + k]) < 1e-2, (name, rel(g[o:o + k], g_ref[o:o + k]))
        o += k
    # Adam learns on this batch
    losses = [ctx.train_step(Xg, Yg, B, T, 1e-3) for _ in range(20)]
    assert losses[-1] < 0.8 * losses[0], losses


TABLE1 = [(32, 1, 8544), (64, 1, 23232), (32, 2, 14688), (64, 2, 47808), (32, 3, 20832),
          (64, 3, 72384)]


@pytest.mark.parametrize("m,n,count", TABLE1)
def test_table1_networks_match_oracle(m, n, count):
    """Table 1's networks on the kernels: bias-free GRUs and a single dense
    layer m -> 18, 51 inputs (3 * 51 + 18 = 171, the linear coefficient of
    the table's parameter counts).  dnnmg_num_params gives the table's count;
    one recurrent step over many patches and the gradient match the oracle's
    variant; Adam learns; DNN-MG steps are refused (their patch features are
    40, not 51)."""
    dn = lib()
    B, T, P = 48, 3, 3000
    ctx = _ctx(dn, m, n, mlp_width=0, net_bias=0, net_inputs=51, train_batch=B, train_seq=T)
    spec = net.NetSpec(c_in=51, hidden=m, layers=n, mlp=0, c_out=18, bias=False)
    assert ctx.num_params() == spec.num_params() == count
    assert ctx.net_dims() == (51, 18)
    w = synthetic.random_weights(3 * m + n, spec.num_params(), 0.25).astype(np.float32)
    ctx.set_weights(w)
    params = spec.unflatten(w.astype(np.float64))
    x = net.bf16_round(synthetic.random_patch_inputs(P + 7 * n, (P, 51)))
    h = synthetic.random_patch_inputs(P + m + 1, (n, P, m), 0.5).astype(np.float32).astype(np.float64)
    hg = torch.from_numpy(h).float().cuda()
    out = ctx.patch_infer(torch.from_numpy(x).to(torch.bfloat16).cuda().contiguous(), hg)
    y_ref, h_ref = net.step_forward(spec, params, x, h, bf16=True)
    assert rel(out.double().cpu().numpy(), y_ref) < 5e-3
    assert rel(hg.double().cpu().numpy(), h_ref) < 2e-3
    X = net.bf16_round(synthetic.random_patch_inputs(5 * m + n, (B, T, 51)))
    Y = synthetic.random_patch_inputs(5 * m + n + 1, (B, T, 18), 0.3)
    Xg = torch.from_numpy(X).to(torch.bfloat16).cuda().contiguous()
    Yg = torch.from_numpy(Y).float().cuda().contiguous()
    g = torch.empty(ctx.num_params(), dtype=torch.float32, device="cuda")
    loss = ctypes.c_float()
    ctx._check(ctx.lib.dnnmg_train_grad(ctx.h, dn._ptr(Xg), dn._ptr(Yg), B, T, dn._ptr(g),
                                        ctypes.byref(loss)))
    g = g.double().cpu().numpy()
    L_ref, g_ref = net.sequence_backward(spec, params, X, Y.astype(np.float32).astype(np.float64),
                                         bf16=True, bf16_grad=True)
    assert abs(loss.value - L_ref) < 1e-3 * L_ref, (loss.value, L_ref)
    assert rel(g, g_ref) < 5e-3, rel(g, g_ref)
    o = 0
    for name, shape in spec.shapes():
        k = int(np.prod(shape))
        assert rel(g[o:o + k], g_ref[o:o + k]) < 1e-2, (name, rel(g[o:o + k], g_ref[o:o + k]))
        o += k
    losses = [ctx.train_step(Xg, Yg, B, T, 1e-3) for _ in range(20)]
    assert losses[-1] < 0.9 * losses[0], losses   # no biases, one dense layer: slower
    with pytest.raises(dn.DnnmgError) as e:
        ctx.step(dn.NET)
    assert e.value.code == dn.ERR_ARG


@pytest.mark.parametrize("m,n", [(32, 1), (32, 3), (64, 1)])
def test_two_replaced_levels_sizes_match_oracle(m, n):
    """The 104-input, 50-output network of two replaced levels at other
    sizes: one recurrent step and the gradient."""
    dn = lib()
    B, T, P = 32, 2, 700
    ctx = _ctx(dn, m, n, replaced_levels=2, train_batch=B, train_seq=T)
    spec = net.NetSpec(c_in=104, c_out=50, hidden=m, layers=n)
    assert ctx.num_params() == spec.num_params() and ctx.net_dims() == (104, 50)
    w = synthetic.random_weights(5 * m + n, spec.num_params(), 0.2).astype(np.float32)
    ctx.set_weights(w)
    params = spec.unflatten(w.astype(np.float64))
    x = net.bf16_round(synthetic.random_patch_inputs(P + 2 * n, (P, 104)))
    h = synthetic.random_patch_inputs(P + m, (n, P, m), 0.5).astype(np.float32).astype(np.float64)
    hg = torch.from_numpy(h).float().cuda()
    out = ctx.patch_infer(torch.from_numpy(x).to(torch.bfloat16).cuda(), hg)
    y_ref, h_ref = net.step_forward(spec, params, x, h, bf16=True)
    assert rel(out.double().cpu().numpy(), y_ref) < 5e-3
    assert rel(hg.double().cpu().numpy(), h_ref) < 2e-3
    X = net.bf16_round(synthetic.random_patch_inputs(m + n, (B, T, 104)))
    Y = synthetic.random_patch_inputs(m + n + 1, (B, T, 50), 0.3)
    Xg = torch.from_numpy(X).to(torch.bfloat16).cuda().contiguous()  # held for the call
    Yg = torch.from_numpy(Y).float().cuda().contiguous()
    g = torch.empty(ctx.num_params(), dtype=torch.float32, device="cuda")
    loss = ctypes.c_float()
    ctx._check(ctx.lib.dnnmg_train_grad(ctx.h, dn._ptr(Xg), dn._ptr(Yg), B, T, dn._ptr(g),
                                        ctypes.byref(loss)))
    L_ref, g_ref = net.sequence_backward(spec, params, X, Y.astype(np.float32).astype(np.float64),
                                         bf16=True, bf16_grad=True)
    assert abs(loss.value - L_ref) < 1e-3 * L_ref
    assert rel(g.double().cpu().numpy(), g_ref) < 5e-3


@pytest.mark.parametrize("m,n", [(32, 3), (64, 1)])
def test_dnnmg_step_matches_oracle(m, n):
    dn = lib()
    ob = synthetic.obstacle_block(1000)
    L, nu, dt = 2, 0.01, 0.01
    ctx = dn.Context(level_solve=L, precision=dn.FP64, obstacle_i0=ob[0], obstacle_j0=ob[1],
                     nu=nu, dt=dt, newton_tol=1e-12, hidden=m, gru_layers=n)
    spec = net.NetSpec(hidden=m, layers=n)
    w = synthetic.random_weights(13 + m + n, spec.num_params(), 0.05).astype(np.float32)
    ctx.set_weights(w)
    levels = mesh.hierarchy(L, obstacle=ob)
    fine = mesh.Level(L + 1, obstacle=ob)
    opt = newton.SolverOptions(newton_tol=1e-12)
    prm = fem.Params(nu=nu, dt=dt)
    params = spec.unflatten(w.astype(np.float64))
    x = mesh.initial_state(levels[-1])
    state = dict(bL=None, vcorr=None, h=np.zeros((n, len(levels[-1].fluid_cells), m)))
    for k in range(2):
        st = ctx.step(dn.NET)
        x, state, info = dnnmg.time_step(levels, fine, x, state, spec, params, prm, opt)
        assert rel(ctx.get_state().cpu().numpy(), x) < 1e-4, (k, st)
        assert st["fallback"] == int(info["fallback"])


def test_sizes_outside_the_kernels_are_rejected():
    """64 x 3 with 104 inputs (two replaced levels) exceeds the shared
    memory of one CTA; other hidden sizes and depths have no kernel."""
    dn = lib()
    for kw in (dict(hidden=64, gru_layers=3, replaced_levels=2), dict(hidden=48, gru_layers=2),
               dict(hidden=64, gru_layers=4)):
        ctx = dn.Context(level_solve=2, **kw)
        with pytest.raises(dn.DnnmgError) as e:
            ctx.set_weights(np.zeros(ctx.num_params(), np.float32))
        assert e.value.code == dn.ERR_ARG
    ok = dn.Context(level_solve=2, hidden=64, gru_layers=2, replaced_levels=2)
    ok.set_weights(np.zeros(ok.num_params(), np.float32))
