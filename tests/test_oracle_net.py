"""Pins of the oracle's patch network (Sec. 2.2, Sec. 3.1, Table 1, Eq. 7):
parameter counts of Table 1, forward pass against PyTorch's GRU and Linear in
FP64, backward against central differences and PyTorch autograd, Adam
against torch.optim.Adam, and bfloat16 rounding against torch's."""
import numpy as np
import pytest
import torch

from oracle import net

TABLE1 = [(32, 1, 8544), (64, 1, 23232), (32, 2, 14688), (64, 2, 47808), (32, 3, 20832), (64, 3, 72384)]


@pytest.mark.parametrize("m,n,count", TABLE1)
def test_table1_parameter_counts(m, n, count):
    """Table 1's networks are bias-free GRUs plus one dense layer with
    3 * inputs + outputs = 171 (e.g. 51 inputs, 18 outputs)."""
    assert net.NetSpec(c_in=51, hidden=m, layers=n, mlp=0, c_out=18, bias=False).num_params() == count


def test_default_network_size():
    spec = net.NetSpec()
    assert spec.num_params() == 55954
    assert spec.flops_per_patch_step() == 110080


def _torch_model(spec, w):
    p = spec.unflatten(w)
    gru = torch.nn.GRU(spec.c_in, spec.hidden, spec.layers, batch_first=True, bias=spec.bias).double()
    with torch.no_grad():
        for l in range(spec.layers):
            getattr(gru, f"weight_ih_l{l}").copy_(torch.from_numpy(p[f"W_ih{l}"]))
            getattr(gru, f"weight_hh_l{l}").copy_(torch.from_numpy(p[f"W_hh{l}"]))
            if spec.bias:
                getattr(gru, f"bias_ih_l{l}").copy_(torch.from_numpy(p[f"b_ih{l}"]))
                getattr(gru, f"bias_hh_l{l}").copy_(torch.from_numpy(p[f"b_hh{l}"]))
    l1 = torch.nn.Linear(spec.hidden, spec.mlp).double()
    l2 = torch.nn.Linear(spec.mlp, spec.c_out).double()
    with torch.no_grad():
        l1.weight.copy_(torch.from_numpy(p["W1"]))
        l1.bias.copy_(torch.from_numpy(p["b1"]))
        l2.weight.copy_(torch.from_numpy(p["W2"]))
        l2.bias.copy_(torch.from_numpy(p["b2"]))
    return gru, l1, l2


def _torch_params(spec, gru, l1, l2):
    out = []
    for l in range(spec.layers):
        out += [getattr(gru, f"weight_ih_l{l}"), getattr(gru, f"weight_hh_l{l}"),
                getattr(gru, f"bias_ih_l{l}"), getattr(gru, f"bias_hh_l{l}")]
    return out + [l1.weight, l1.bias, l2.weight, l2.bias]


def test_forward_matches_torch_gru_fp64():
    spec = net.NetSpec(c_in=40, hidden=16, layers=2, mlp=24, c_out=18)
    rng = np.random.default_rng(0)
    w = rng.uniform(-0.4, 0.4, spec.num_params())
    X = rng.standard_normal((5, 7, spec.c_in))
    Y, h = net.sequence_forward(spec, spec.unflatten(w), X)
    gru, l1, l2 = _torch_model(spec, w)
    with torch.no_grad():
        o, hT = gru(torch.from_numpy(X))
        Yt = l2(torch.relu(l1(o))).numpy()
    np.testing.assert_allclose(Y, Yt, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(h, hT.numpy(), rtol=1e-12, atol=1e-13)


def test_backward_matches_autograd_and_finite_differences():
    spec = net.NetSpec(c_in=12, hidden=8, layers=2, mlp=10, c_out=6)
    rng = np.random.default_rng(1)
    w = rng.uniform(-0.5, 0.5, spec.num_params())
    X = rng.standard_normal((4, 5, spec.c_in))
    Y = rng.standard_normal((4, 5, spec.c_out))
    L, g = net.sequence_backward(spec, spec.unflatten(w), X, Y)
    gru, l1, l2 = _torch_model(spec, w)
    o, _ = gru(torch.from_numpy(X))
    Lt = torch.mean((l2(torch.relu(l1(o))) - torch.from_numpy(Y)) ** 2)
    Lt.backward()
    gt = torch.cat([t.grad.reshape(-1) for t in _torch_params(spec, gru, l1, l2)]).numpy()
    assert abs(L - Lt.item()) < 1e-13
    np.testing.assert_allclose(g, gt, rtol=1e-10, atol=1e-13)
    for i in rng.choice(spec.num_params(), 12, replace=False):
        e = np.zeros_like(w)
        e[i] = 1e-6
        Lp = net.loss(net.sequence_forward(spec, spec.unflatten(w + e), X)[0], Y)
        Lm = net.loss(net.sequence_forward(spec, spec.unflatten(w - e), X)[0], Y)
        assert abs((Lp - Lm) / 2e-6 - g[i]) < 1e-7 * max(1.0, abs(g[i]))


def test_backward_single_dense_layer_variant():
    spec = net.NetSpec(c_in=7, hidden=5, layers=3, mlp=0, c_out=4, bias=False)
    rng = np.random.default_rng(2)
    w = rng.uniform(-0.5, 0.5, spec.num_params())
    X, Y = rng.standard_normal((3, 4, 7)), rng.standard_normal((3, 4, 4))
    _, g = net.sequence_backward(spec, spec.unflatten(w), X, Y)
    for i in range(0, spec.num_params(), 17):
        e = np.zeros_like(w)
        e[i] = 1e-6
        Lp = net.loss(net.sequence_forward(spec, spec.unflatten(w + e), X)[0], Y)
        Lm = net.loss(net.sequence_forward(spec, spec.unflatten(w - e), X)[0], Y)
        assert abs((Lp - Lm) / 2e-6 - g[i]) < 1e-7 * max(1.0, abs(g[i]))


def test_adam_matches_torch():
    rng = np.random.default_rng(3)
    w0 = rng.standard_normal(50)
    grads = [rng.standard_normal(50) for _ in range(6)]
    opt = net.Adam(50)
    w = w0.copy()
    for k, g in enumerate(grads):
        w = opt.step(w, g, 1e-2 * (1 + k))
    wt = torch.tensor(w0, requires_grad=True)
    topt = torch.optim.Adam([wt], lr=1e-2)
    for k, g in enumerate(grads):
        for grp in topt.param_groups:
            grp["lr"] = 1e-2 * (1 + k)
        wt.grad = torch.from_numpy(g)
        topt.step()
    np.testing.assert_allclose(w, wt.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(4)
    a = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-8, 8, 10000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875]])
    t = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(net.bf16_round(a), t)


def _q_t(t):
    """bfloat16 rounding of a float64 tensor through float32 (the oracle's path)."""
    return t.float().to(torch.bfloat16).double()


def _ste(t):
    """bfloat16-rounded value whose gradient passes through unchanged."""
    return t + (_q_t(t) - t).detach()


def test_bf16_gradient_rounding_matches_autograd_with_hooks():
    """bf16_grad=True against PyTorch autograd on a GRU built cell by cell:
    the forward uses rounded weights and rounded product inputs (straight-
    through, as the oracle's forward), and backward hooks round the gradients
    of the output, of the dense pre-activation and of both gate
    pre-activation vectors of every layer.  Autograd supplies the chain rule,
    so a rounding point put at the wrong place, dropped, or a term that
    skips the rounded value, shows up here."""
    spec = net.NetSpec(c_in=12, hidden=8, layers=2, mlp=10, c_out=6)
    rng = np.random.default_rng(7)
    w = rng.uniform(-0.5, 0.5, spec.num_params())
    B, T = 5, 4
    X = net.bf16_round(rng.standard_normal((B, T, spec.c_in)))
    Y = rng.standard_normal((B, T, spec.c_out))
    L, g = net.sequence_backward(spec, spec.unflatten(w), X, Y, bf16=True, bf16_grad=True)
    _, g_plain = net.sequence_backward(spec, spec.unflatten(w), X, Y, bf16=True)
    p = spec.unflatten(w)
    H = spec.hidden
    tp = {}
    for k, v in p.items():
        t = torch.from_numpy(net.bf16_round(v) if k.startswith("W") else v.copy())
        tp[k] = t.requires_grad_(True)
    hook = lambda gr: _q_t(gr)
    h = [torch.zeros(B, H, dtype=torch.float64) for _ in range(spec.layers)]
    Xt = torch.from_numpy(X)
    outs = []
    for t in range(T):
        inp = Xt[:, t]
        for l in range(spec.layers):
            gi = inp @ tp[f"W_ih{l}"].T + tp[f"b_ih{l}"]
            gh = _ste(h[l]) @ tp[f"W_hh{l}"].T + tp[f"b_hh{l}"]
            gi.register_hook(hook)
            gh.register_hook(hook)
            r = torch.sigmoid(gi[:, :H] + gh[:, :H])
            z = torch.sigmoid(gi[:, H:2 * H] + gh[:, H:2 * H])
            n = torch.tanh(gi[:, 2 * H:] + r * gh[:, 2 * H:])
            h[l] = (1 - z) * n + z * h[l]
            inp = _ste(h[l])
        a1 = inp @ tp["W1"].T + tp["b1"]
        a1.register_hook(hook)
        y = _ste(torch.relu(a1)) @ tp["W2"].T + tp["b2"]
        y.register_hook(hook)
        outs.append(y)
    Lt = torch.mean((torch.stack(outs, 1) - torch.from_numpy(Y)) ** 2)
    Lt.backward()
    gt = torch.cat([tp[k].grad.reshape(-1) for k in spec.param_names()]).numpy()
    assert abs(L - Lt.item()) < 1e-13
    np.testing.assert_allclose(g, gt, rtol=1e-9, atol=1e-13)
    # the rounding is a real, bounded perturbation of the unrounded gradient
    d = np.linalg.norm(g - g_plain) / np.linalg.norm(g_plain)
    assert 1e-5 < d < 2e-2, d
