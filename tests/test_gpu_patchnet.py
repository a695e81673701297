"""Parity of the tensor-core patch network with references: the generic
tcgen05 GEMM against torch (exact BF16 products, FP32 sums), and one
recurrent step of the fused GRU/dense kernel against the FP64 oracle with
bfloat16 rounding at the same points (weights, inputs, hidden state fed to
W_hh, layer-1 input, ReLU output).  Tolerance: relative L2 <= 5e-3 on the
outputs and 2e-3 on the hidden states -- the remaining differences are FP32
vs FP64 accumulation and occasional one-ulp bfloat16 flips of intermediate
activations (2^-8 relative)."""
import numpy as np
import pytest

import synthetic
from oracle import net
from tests.gpu_util import lib, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("M,N,K", [(128, 16, 16), (256, 192, 48), (384, 256, 128), (128, 64, 200 - 8)])
def test_umma_gemm_matches_torch(M, N, K):
    dn = lib()
    ctx = dn.Context(level_solve=1)
    g = torch.Generator().manual_seed(M + N + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    C = ctx.gemm_bf16(A, B)
    ref = A.double() @ B.double().T
    assert rel(C.double().cpu().numpy(), ref.cpu().numpy()) < 1e-6


def _weights(spec, seed, scale=0.25):
    return synthetic.random_weights(seed, spec.num_params(), scale).astype(np.float32)


@pytest.mark.parametrize("P,seed,replaced", [(1, 1, 1), (128, 2, 1), (1000, 3, 1), (61440, 4, 1),
                                             (1, 5, 2), (1000, 6, 2), (61440, 7, 2)])
def test_patch_infer_matches_oracle(P, seed, replaced):
    """One replaced level: 3x3-node patches, 40 inputs, 18 outputs; two:
    5x5-node patches, 104 inputs, 50 outputs."""
    dn = lib()
    ctx = dn.Context(level_solve=2, replaced_levels=replaced)
    k = 2 ** replaced + 1
    spec = net.NetSpec(c_in=4 * k * k + 4, c_out=2 * k * k)
    assert ctx.num_params() == spec.num_params() == (55954 if replaced == 1 else 72370)
    assert ctx.net_dims() == (spec.c_in, spec.c_out)
    w = _weights(spec, seed)
    ctx.set_weights(w)
    np.testing.assert_array_equal(ctx.get_weights().numpy(), w)
    x = net.bf16_round(synthetic.random_patch_inputs(seed, (P, spec.c_in)))
    h = synthetic.random_patch_inputs(seed + 1, (2, P, 64), 0.5).astype(np.float32).astype(np.float64)
    xg = torch.from_numpy(x).to(torch.bfloat16).cuda()
    hg = torch.from_numpy(h).float().cuda()
    out = ctx.patch_infer(xg, hg).double().cpu().numpy()
    y_ref, h_ref = net.step_forward(spec, spec.unflatten(w.astype(np.float64)), x, h, bf16=True)
    assert rel(out, y_ref) < 5e-3, rel(out, y_ref)
    assert rel(hg.double().cpu().numpy(), h_ref) < 2e-3


def test_zero_network_predicts_zero():
    dn = lib()
    ctx = dn.Context(level_solve=2)
    P = 300
    x = torch.randn(P, 40).to(torch.bfloat16).cuda()
    h = torch.zeros(2, P, 64, device="cuda")
    out = ctx.patch_infer(x, h)
    assert float(out.abs().max()) == 0.0
    assert float(h.abs().max()) == 0.0      # n = tanh(0) = 0 and z = 1/2 keep h at 0
    assert ctx.patch_infer(x[:0], h[:, :0]).numel() == 0
