"""Parity of the CUDA DNN-MG time step (Algorithm 1) with the
oracle's composition of the same steps, plus the zero-network invariant and
the Newton-count fallback.  Solver in FP64 (Newton tolerance 1e-12), network
in BF16 with FP32 accumulation: states are compared at relative L2 1e-4
(the bar for one DNN-MG step from an identical state), the patch inputs at
5e-3 (bfloat16 rounding of features computed in FP32 vs FP64)."""
import numpy as np
import pytest

import synthetic
from oracle import dnnmg, fem, mesh, net, newton
from tests.gpu_util import lib, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

L, NU, DT = 2, 0.01, 0.01


def _ctx(dn, obstacle, **kw):
    return dn.Context(level_solve=L, precision=dn.FP64, obstacle_i0=obstacle[0],
                      obstacle_j0=obstacle[1], nu=NU, dt=DT, newton_tol=1e-12, **kw)


def test_zero_network_dnnmg_equals_plain_multigrid():
    dn = lib()
    ob = synthetic.obstacle_block(1001)
    a, b = _ctx(dn, ob), _ctx(dn, ob)
    for n in range(3):
        sa = a.step(dn.NET)
        sb = b.step(dn.PLAIN)
        assert sa["fallback"] == 0
        assert rel(a.get_state().cpu().numpy(), b.get_state().cpu().numpy()) < 1e-10, n
    assert a.num_patches() == 64 * 16 - 4 * 16


def test_dnnmg_steps_match_oracle():
    dn = lib()
    ob = synthetic.obstacle_block(1000)
    ctx = _ctx(dn, ob)
    spec = net.NetSpec()
    w = synthetic.random_weights(11, spec.num_params(), 0.05).astype(np.float32)
    ctx.set_weights(w)
    rng = np.random.default_rng(5)
    mean = rng.normal(0, 0.1, 40).astype(np.float32)
    std = rng.uniform(0.5, 2.0, 40).astype(np.float32)
    ctx.set_feature_stats(mean, std)
    levels = mesh.hierarchy(L, obstacle=ob)
    fine = mesh.Level(L + 1, obstacle=ob)
    opt = newton.SolverOptions(newton_tol=1e-12)
    prm = fem.Params(nu=NU, dt=DT)
    params = spec.unflatten(w.astype(np.float64))
    x = mesh.initial_state(levels[-1])
    state = dict(bL=None, vcorr=None, h=np.zeros((2, len(levels[-1].fluid_cells), 64)))
    P = ctx.num_patches()
    for n in range(3):
        st = ctx.step(dn.NET)
        x, state, info = dnnmg.time_step(levels, fine, x, state, spec, params, prm, opt,
                                         mean.astype(np.float64), std.astype(np.float64))
        xg = ctx.get_state().cpu().numpy()
        assert rel(xg, x) < 1e-4, (n, rel(xg, x))
        vg = torch.empty(2 * fine.nn, dtype=torch.float64, device="cuda")
        ctx.lib.dnnmg_get_fine_velocity(ctx.h, dn._ptr(vg))
        assert rel(vg.cpu().numpy(), state["vcorr"][:2 * fine.nn]) < 1e-4, n
        Xg = torch.empty(P, 40, dtype=torch.bfloat16, device="cuda")
        ctx.lib.dnnmg_get_patch_inputs(ctx.h, dn._ptr(Xg))
        assert rel(Xg.double().cpu().numpy(), info["X"]) < 5e-3, n
        assert st["fallback"] == int(info["fallback"])


def test_fallback_drops_the_network_rhs():
    dn = lib()
    ob = synthetic.obstacle_block(1000)
    a = _ctx(dn, ob, fallback_newton_its=0)
    b = _ctx(dn, ob)
    w = synthetic.random_weights(3, a.num_params(), 0.2).astype(np.float32)
    a.set_weights(w)
    a.step(dn.NET)
    b.step(dn.PLAIN)
    st = a.step(dn.NET)
    b.step(dn.PLAIN)
    assert st["fallback"] == 1
    assert rel(a.get_state().cpu().numpy(), b.get_state().cpu().numpy()) < 1e-10


def test_forced_fallback_matches_oracle():
    """The switch-off of Sec. 3.3 forced on every step that has a network
    right-hand side (threshold 0 Newton iterations): the GPU and the oracle
    (time_step with fallback_its=0) both redo those steps with the plain
    right-hand side, so states, corrected fine velocities and the fallback
    flags agree, while the network still runs after each step."""
    dn = lib()
    ob = synthetic.obstacle_block(1000)
    ctx = _ctx(dn, ob, fallback_newton_its=0)
    spec = net.NetSpec()
    w = synthetic.random_weights(3, spec.num_params(), 0.2).astype(np.float32)
    ctx.set_weights(w)
    levels = mesh.hierarchy(L, obstacle=ob)
    fine = mesh.Level(L + 1, obstacle=ob)
    opt = newton.SolverOptions(newton_tol=1e-12)
    prm = fem.Params(nu=NU, dt=DT)
    params = spec.unflatten(w.astype(np.float64))
    zero, one = np.zeros(40), np.ones(40)
    x = mesh.initial_state(levels[-1])
    state = dict(bL=None, vcorr=None, h=np.zeros((2, len(levels[-1].fluid_cells), 64)))
    flags = []
    for n in range(3):
        st = ctx.step(dn.NET)
        x, state, info = dnnmg.time_step(levels, fine, x, state, spec, params, prm, opt,
                                         zero, one, fallback_its=0)
        assert st["fallback"] == int(info["fallback"]), (n, st, info["fallback"])
        flags.append(st["fallback"])
        assert rel(ctx.get_state().cpu().numpy(), x) < 1e-4, n
        assert rel(ctx.get_fine_velocity().cpu().numpy(), state["vcorr"][:2 * fine.nn]) < 1e-4, n
    assert flags == [0, 1, 1]


def test_two_replaced_levels_dnnmg_steps_match_oracle():
    """The network replaces levels L+1 and L+2 (5x5-node patches, 104
    inputs, 50 outputs): P and R act twice, the fine residual and the
    right-hand side live on level L+2."""
    dn = lib()
    ob = synthetic.obstacle_block(1001)
    ctx = _ctx(dn, ob, replaced_levels=2)
    spec = net.NetSpec(c_in=104, c_out=50)
    assert ctx.net_dims() == (104, 50)
    w = synthetic.random_weights(12, spec.num_params(), 0.05).astype(np.float32)
    ctx.set_weights(w)
    rng = np.random.default_rng(6)
    mean = rng.normal(0, 0.1, 104).astype(np.float32)
    std = rng.uniform(0.5, 2.0, 104).astype(np.float32)
    ctx.set_feature_stats(mean, std)
    levels = mesh.hierarchy(L, obstacle=ob)
    chain = [mesh.Level(L + 1, obstacle=ob), mesh.Level(L + 2, obstacle=ob)]
    fine = chain[-1]
    opt = newton.SolverOptions(newton_tol=1e-12)
    prm = fem.Params(nu=NU, dt=DT)
    params = spec.unflatten(w.astype(np.float64))
    x = mesh.initial_state(levels[-1])
    state = dict(bL=None, vcorr=None, h=np.zeros((2, len(levels[-1].fluid_cells), 64)))
    P = ctx.num_patches()
    for n in range(3):
        st = ctx.step(dn.NET)
        x, state, info = dnnmg.time_step(levels, chain, x, state, spec, params, prm, opt,
                                         mean.astype(np.float64), std.astype(np.float64))
        assert rel(ctx.get_state().cpu().numpy(), x) < 1e-4, n
        vg = ctx.get_fine_velocity().cpu().numpy()
        assert vg.size == 2 * fine.nn
        assert rel(vg, state["vcorr"][:2 * fine.nn]) < 1e-4, n
        Xg = torch.empty(P, 104, dtype=torch.bfloat16, device="cuda")
        ctx.lib.dnnmg_get_patch_inputs(ctx.h, dn._ptr(Xg))
        assert rel(Xg.double().cpu().numpy(), info["X"]) < 5e-3, n
        assert st["fallback"] == int(info["fallback"])


def test_two_replaced_levels_zero_network_equals_plain_multigrid():
    dn = lib()
    ob = synthetic.obstacle_block(1000)
    a, b = _ctx(dn, ob, replaced_levels=2), _ctx(dn, ob)
    for n in range(3):
        a.step(dn.NET)
        b.step(dn.PLAIN)
        assert rel(a.get_state().cpu().numpy(), b.get_state().cpu().numpy()) < 1e-10, n
