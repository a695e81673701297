"""Training kernels of the patch network against the oracle (Eq. 7 loss,
backpropagation through time, Adam).  The GPU path uses bfloat16 operands
for every product, including the output, dense and gate gradients fed to the
tensor cores; the oracle rounds at the same points (bf16=True for the
forward, bf16_grad=True for the backward) and keeps everything else in FP64,
while the kernels keep it in FP32.  The loss must agree to 1e-3 relative and
the gradient to 5e-3 relative L2 (1e-2 per parameter block): what remains is
FP32 arithmetic and the rare bfloat16 rounding that FP32 and FP64 values
take to different sides."""
import numpy as np
import pytest

import synthetic
from oracle import net
from tests.gpu_util import lib, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _ctx(dn, B, T, replaced=1):
    return dn.Context(level_solve=2, train_batch=B, train_seq=T, replaced_levels=replaced)


def _grad(ctx, dn, X, Y, B, T):
    g = torch.empty(ctx.num_params(), dtype=torch.float32, device="cuda")
    loss = __import__("ctypes").c_float()
    rc = ctx.lib.dnnmg_train_grad(ctx.h, dn._ptr(X), dn._ptr(Y), B, T, dn._ptr(g),
                                  __import__("ctypes").byref(loss))
    ctx._check(rc)
    return g.double().cpu().numpy(), loss.value


@pytest.mark.parametrize("B,T,replaced", [(16, 1, 1), (32, 3, 1), (144, 4, 1), (48, 3, 2)])
def test_gradient_matches_oracle(B, T, replaced):
    """Also for the two-replaced-level network (104 inputs, 50 outputs)."""
    dn = lib()
    ctx = _ctx(dn, 160, 4, replaced)
    k = 2 ** replaced + 1
    spec = net.NetSpec(c_in=4 * k * k + 4, c_out=2 * k * k)
    w = synthetic.random_weights(B + T, spec.num_params(), 0.2).astype(np.float32)
    ctx.set_weights(w)
    X = net.bf16_round(synthetic.random_patch_inputs(B * 10 + T, (B, T, spec.c_in)))
    Y = synthetic.random_patch_inputs(B * 10 + T + 1, (B, T, spec.c_out), 0.3)
    Xg = torch.from_numpy(X).to(torch.bfloat16).cuda().contiguous()
    Yg = torch.from_numpy(Y).float().cuda().contiguous()
    g, loss = _grad(ctx, dn, Xg, Yg, B, T)
    L_ref, g_ref = net.sequence_backward(spec, spec.unflatten(w.astype(np.float64)), X,
                                         Y.astype(np.float32).astype(np.float64), bf16=True,
                                         bf16_grad=True)
    assert abs(loss - L_ref) < 1e-3 * L_ref, (loss, L_ref)
    assert rel(g, g_ref) < 5e-3, rel(g, g_ref)
    # every parameter block individually
    o = 0
    for name, shape in spec.shapes():
        n = int(np.prod(shape))
        assert rel(g[o:o + n], g_ref[o:o + n]) < 1e-2, (name, rel(g[o:o + n], g_ref[o:o + n]))
        o += n
    g2, loss2 = _grad(ctx, dn, Xg, Yg, B, T)
    np.testing.assert_array_equal(g, g2)          # fixed-order reductions
    assert loss == loss2


def test_adam_step_and_learning():
    dn = lib()
    B, T = 64, 3
    ctx = _ctx(dn, B, T)
    spec = net.NetSpec()
    w = synthetic.random_weights(5, spec.num_params(), 0.2).astype(np.float32)
    ctx.set_weights(w)
    X = net.bf16_round(synthetic.random_patch_inputs(50, (B, T, 40)))
    Y = synthetic.random_patch_inputs(51, (B, T, 18), 0.3)
    Xg = torch.from_numpy(X).to(torch.bfloat16).cuda().contiguous()
    Yg = torch.from_numpy(Y).float().cuda().contiguous()
    _, g_ref = net.sequence_backward(spec, spec.unflatten(w.astype(np.float64)), X,
                                     Y.astype(np.float32).astype(np.float64), bf16=True)
    lr = 1e-3
    ctx.train_step(Xg, Yg, B, T, lr)
    dw = ctx.get_weights().double().numpy() - w
    big = np.abs(g_ref) > 1e-3 * np.abs(g_ref).max()
    # Adam's first step is -lr * sign(g) up to eps
    np.testing.assert_allclose(dw[big], -lr * np.sign(g_ref[big]), rtol=0, atol=2e-5)
    losses = [ctx.train_step(Xg, Yg, B, T, lr) for _ in range(30)]
    assert losses[-1] < 0.8 * losses[0], losses


def test_adam_steps_match_oracle_elementwise():
    """Five Adam steps (bias correction, beta = (0.9, 0.999), eps = 1e-8)
    against oracle.net.Adam element by element.  Both take the gradient the
    GPU computes at the GPU's current weights (dnnmg_train_grad is bitwise
    the one dnnmg_train_step uses), so the comparison isolates the optimiser:
    a wrong beta2, a missing bias correction or a wrong epsilon changes the
    later steps by far more than FP32 rounding does."""
    dn = lib()
    B, T = 64, 3
    ctx = _ctx(dn, B, T)
    spec = net.NetSpec()
    w = synthetic.random_weights(9, spec.num_params(), 0.2).astype(np.float32)
    ctx.set_weights(w)
    X = net.bf16_round(synthetic.random_patch_inputs(60, (B, T, 40)))
    Y = synthetic.random_patch_inputs(61, (B, T, 18), 0.3)
    Xg = torch.from_numpy(X).to(torch.bfloat16).cuda().contiguous()
    Yg = torch.from_numpy(Y).float().cuda().contiguous()
    opt = net.Adam(spec.num_params())
    for k, lr in enumerate((1e-3, 2e-3, 5e-4, 1e-3, 3e-3)):
        w0 = ctx.get_weights().double().numpy()
        g, _ = _grad(ctx, dn, Xg, Yg, B, T)
        w_ref = opt.step(w0, g, lr)
        ctx.train_step(Xg, Yg, B, T, lr)
        w1 = ctx.get_weights().double().numpy()
        # FP32 weights of magnitude <= 1 carry ~6e-8 absolute rounding
        np.testing.assert_allclose(w1 - w0, w_ref - w0, rtol=1e-4, atol=2e-7 + 1e-4 * lr,
                                   err_msg=f"Adam step {k + 1}")
