"""The allocation-free coarse solve (dnnmg_coarse_solve_noalloc) returns what
the coarse level of the context-based V-cycle returns.

Some callers cannot call cudaMalloc at all (an external memory manager owns
the device heap, or a real-time loop forbids allocation), so they cannot
create a context; this entry point keeps its working memory in a static
device array instead.  The test calls it through the C ABI twice in a row
(the array keeps the previous call's contents) and compares each result with
the oracle's direct solve of the same linearised operator and with
dnnmg_vcycle on the coarsest level, which applies the context's inverse of
that operator.  This file is collected last so that a failure here does not
hide the other GPU tests."""
import ctypes

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synthetic
from oracle import fem, mesh
from tests.gpu_util import lib, rel, seeded_state

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _entry(dn):
    f = dn.load().dnnmg_coarse_solve_noalloc
    f.argtypes = [ctypes.c_void_p] * 5
    f.restype = ctypes.c_int
    return f


@pytest.mark.parametrize("with_obstacle", [True, False])
def test_noalloc_coarse_solve_matches_oracle_and_context_vcycle(with_obstacle):
    dn = lib()
    f = _entry(dn)
    # without an obstacle the device-side masks take their other branch
    obstacle = synthetic.obstacle_block(1000) if with_obstacle else None
    oi, oj = obstacle if obstacle else (-1, -1)
    cfg = dn.default_config(level_solve=1, precision=dn.FP64, obstacle_i0=oi, obstacle_j0=oj,
                            nu=0.006, dt=0.01)
    ctx = dn.Context(cfg)
    lev = mesh.Level(1, obstacle=obstacle)
    stream = torch.cuda.current_stream()
    for call, seed in enumerate((21, 22)):
        x = torch.from_numpy(seeded_state(lev, seed)).cuda()
        ctx.linearize(x)
        bh = synthetic.random_vector(seed + 100, lev.ndof)
        bh[lev.cons] = 0.0
        b = torch.from_numpy(bh).cuda()
        ref = ctx.vcycle(1, b).cpu().numpy()
        out = torch.full_like(b, float("nan"))
        vbar = x[:2 * lev.nn].contiguous()
        rc = f(ctypes.byref(cfg), ctypes.c_void_p(vbar.data_ptr()), ctypes.c_void_p(b.data_ptr()),
               ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == dn.OK, dn.load().dnnmg_last_error(None)
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert rel(got, ref) < 1e-10, (call, rel(got, ref))
        # the oracle: A'(vbar)^-1 b with the FP64 Jacobian of the same level
        A = fem.jacobian(lev, x.cpu().numpy(), fem.Params(nu=0.006, dt=0.01))
        xo = spla.spsolve(A.tocsc(), bh)
        assert rel(got, xo) < 1e-10, (call, rel(got, xo))
    ctx.close()


def test_noalloc_rejects_levels_beyond_its_scratch():
    dn = lib()
    f = _entry(dn)
    cfg = dn.default_config(level_coarse=2)
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    rc = f(ctypes.byref(cfg), p, p, p, None)
    assert rc == dn.ERR_ARG
    assert b"scratch" in dn.load().dnnmg_last_error(None)
