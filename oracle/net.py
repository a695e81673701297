"""Patch network of DNN-MG: stacked GRUs + dense layers (oracle, test only).

Sec. 2.2 and Sec. 3.1: the network N acts on each patch separately, is
recurrent with memory (stacked GRU cells, hidden size m, n cells stacked)
and ends in dense layers that output the velocity correction d of the
patch's fine nodes; it is trained with the loss of Eq. 7.

Readings:
  * GRU gates follow PyTorch (the paper used PyTorch, Sec. 3.1):
      r = sigma(W_ir x + b_ir + W_hr h + b_hr)
      z = sigma(W_iz x + b_iz + W_hz h + b_hz)
      n = tanh(W_in x + b_in + r * (W_hn h + b_hn))
      h' = (1 - z) * n + z * h
  * after the GRUs: Linear(H -> F) + ReLU, Linear(F -> C_out); with F = 0
    a single Linear(H -> C_out), the dense layer of Table 1's networks;
  * flat parameter order, per GRU layer l: W_ih (3H x C_l, gate rows r,z,n),
    W_hh (3H x H), b_ih (3H), b_hh (3H); then W1 (F x H), b1 (F),
    W2 (C_out x F), b2 (C_out).  The bias-free variant of Table 1 simply
    drops the biases;
  * loss (Eq. 7) as the mean over steps, patches and outputs of the squared
    difference (a mean instead of a sum only rescales the learning rate);
  * Adam with bias correction (the paper does not name its optimiser).

`bf16=True` rounds to bfloat16 exactly where the tensor-core path feeds a
matrix product: weights, the input x, the hidden state multiplied by W_hh,
the input of every layer above the first and the ReLU output.  Everything
else stays FP64.  In the backward pass, `bf16_grad=True` also rounds the
gradients that feed a product: the output gradient dY, the gradient of the
dense layer's pre-activation, and the gate gradients of every GRU layer
(both the products with the weights and the weight and bias gradients then
use the rounded values).
"""
import numpy as np


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), via float32."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(a))


class NetSpec:
    def __init__(self, c_in=40, hidden=64, layers=2, mlp=128, c_out=18, bias=True):
        self.c_in, self.hidden, self.layers = c_in, hidden, layers
        self.mlp, self.c_out, self.bias = mlp, c_out, bias

    def shapes(self):
        """(name, shape) in flat order."""
        H, out = self.hidden, []
        for l in range(self.layers):
            c = self.c_in if l == 0 else H
            out += [(f"W_ih{l}", (3 * H, c)), (f"W_hh{l}", (3 * H, H))]
            if self.bias:
                out += [(f"b_ih{l}", (3 * H,)), (f"b_hh{l}", (3 * H,))]
        if self.mlp:
            out += [("W1", (self.mlp, H))]
            if self.bias:
                out += [("b1", (self.mlp,))]
        out += [("W2", (self.c_out, self.mlp or H))]
        if self.bias:
            out += [("b2", (self.c_out,))]
        return out

    def num_params(self):
        return int(sum(np.prod(s) for _, s in self.shapes()))

    def unflatten(self, w):
        p, o = {}, 0
        for name, s in self.shapes():
            n = int(np.prod(s))
            p[name] = w[o:o + n].reshape(s)
            o += n
        if not self.bias:
            H = self.hidden
            for l in range(self.layers):
                p[f"b_ih{l}"] = np.zeros(3 * H)
                p[f"b_hh{l}"] = np.zeros(3 * H)
            p["b1"], p["b2"] = np.zeros(self.mlp), np.zeros(self.c_out)
        return p

    def param_names(self):
        return [name for name, _ in self.shapes()]

    def flatten(self, p):
        return np.concatenate([p[name].ravel() for name, _ in self.shapes()])

    def flops_per_patch_step(self):
        """Multiply-add FLOPs (2 per MAC) of one forward step of one patch."""
        H, macs = self.hidden, 0
        for l in range(self.layers):
            c = self.c_in if l == 0 else H
            macs += 3 * H * c + 3 * H * H
        macs += (self.mlp * H + self.c_out * self.mlp) if self.mlp else self.c_out * H
        return 2 * macs


def _sig(a):
    return 1.0 / (1.0 + np.exp(-a))


def _q(a, bf16):
    return bf16_round(a) if bf16 else a


def step_forward(spec, p, x, h, bf16=False, cache=None):
    """One time step for a batch of patches.

    x [P, C_in], h [layers, P, H] -> (y [P, C_out], h_new [layers, P, H]).
    """
    H = spec.hidden
    inp = _q(x, bf16)
    h_new = np.empty_like(h)
    layer_cache = []
    for l in range(spec.layers):
        Wih, Whh = _q(p[f"W_ih{l}"], bf16), _q(p[f"W_hh{l}"], bf16)
        hq = _q(h[l], bf16)
        gi = inp @ Wih.T + p[f"b_ih{l}"]
        gh = hq @ Whh.T + p[f"b_hh{l}"]
        r = _sig(gi[:, :H] + gh[:, :H])
        z = _sig(gi[:, H:2 * H] + gh[:, H:2 * H])
        n = np.tanh(gi[:, 2 * H:] + r * gh[:, 2 * H:])
        h_new[l] = (1.0 - z) * n + z * h[l]
        layer_cache.append((inp, hq, h[l], r, z, n, gh[:, 2 * H:]))
        inp = _q(h_new[l], bf16)
    if spec.mlp:
        a1 = inp @ _q(p["W1"], bf16).T + p["b1"]
        y1 = _q(np.maximum(a1, 0.0), bf16)
    else:
        a1, y1 = None, inp
    y = y1 @ _q(p["W2"], bf16).T + p["b2"]
    if cache is not None:
        cache.append((layer_cache, inp, a1, y1))
    return y, h_new


def sequence_forward(spec, p, X, bf16=False, h0=None, cache=None):
    """X [B, T, C_in] -> Y [B, T, C_out], hidden starting at zero (or h0)."""
    B, T, _ = X.shape
    h = np.zeros((spec.layers, B, spec.hidden)) if h0 is None else h0.copy()
    Y = np.empty((B, T, spec.c_out))
    for t in range(T):
        Y[:, t], h = step_forward(spec, p, X[:, t], h, bf16, cache)
    return Y, h


def loss(Ypred, Y):
    """Eq. 7 as a mean of squared differences."""
    return float(np.mean((Ypred - Y) ** 2))


def sequence_backward(spec, p, X, Y, bf16=False, bf16_grad=False):
    """Loss and gradient (flat, FP64) by backpropagation through time.

    Weight gradients are taken with respect to the (rounded) weights the
    forward pass used.  bf16_grad: round the gradients that enter a matrix
    product to bfloat16 (see the module docstring).
    """
    qg = (lambda a: bf16_round(a)) if bf16_grad else (lambda a: a)
    B, T, _ = X.shape
    H = spec.hidden
    cache = []
    Yp, _ = sequence_forward(spec, p, X, bf16, cache=cache)
    Lval = loss(Yp, Y)
    dY = 2.0 * (Yp - Y) / Yp.size
    g = {k: np.zeros_like(v) for k, v in p.items()}
    W = {k: _q(v, bf16) if k.startswith("W") else v for k, v in p.items()}
    dh_next = np.zeros((spec.layers, B, H))
    for t in range(T - 1, -1, -1):
        layer_cache, top, a1, y1 = cache[t]
        dy = qg(dY[:, t])
        g["W2"] += dy.T @ y1
        g["b2"] += dy.sum(0)
        if spec.mlp:
            da1 = qg((dy @ W["W2"]) * (a1 > 0))
            g["W1"] += da1.T @ top
            g["b1"] += da1.sum(0)
            dinp = da1 @ W["W1"]
        else:
            dinp = dy @ W["W2"]
        dh_prev = np.zeros_like(dh_next)
        for l in range(spec.layers - 1, -1, -1):
            inp, hq, hprev, r, z, n, ghn = layer_cache[l]
            dh = dinp + dh_next[l]
            dn = dh * (1.0 - z)
            dz = dh * (hprev - n)
            dan = dn * (1.0 - n * n)
            dr = dan * ghn
            dar = dr * r * (1.0 - r)
            daz = dz * z * (1.0 - z)
            dgi = qg(np.concatenate([dar, daz, dan], axis=1))
            dgh = qg(np.concatenate([dar, daz, dan * r], axis=1))
            g[f"W_ih{l}"] += dgi.T @ inp
            g[f"b_ih{l}"] += dgi.sum(0)
            g[f"W_hh{l}"] += dgh.T @ hq
            g[f"b_hh{l}"] += dgh.sum(0)
            dh_prev[l] = dh * z + dgh @ W[f"W_hh{l}"]
            dinp = dgi @ W[f"W_ih{l}"]
        dh_next = dh_prev
    return Lval, spec.flatten(g)


class Adam:
    """Adam with bias correction, beta = (0.9, 0.999), eps = 1e-8."""

    def __init__(self, n, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m, self.v, self.t = np.zeros(n), np.zeros(n), 0
        self.b1, self.b2, self.eps = beta1, beta2, eps

    def step(self, w, g, lr):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return w - lr * mh / (np.sqrt(vh) + self.eps)
