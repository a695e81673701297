"""The device corpus (dnnmg_make_corpus, Sec. 3.1: training data from plain
fine-level trajectories, localised to time steps and patches) against the
same trajectories driven call by call through the C ABI: contexts created
with each trajectory's viscosity and the spin-up time step, dnnmg_prolongate,
plain fine steps and one dnnmg_make_sample per step (whose own parity with
the oracle is tested elsewhere).  FP64 solvers; the Newton tolerance is 1e-12
on both sides, so the two routes agree to round-off of the converged
states."""
import ctypes

import numpy as np
import pytest

import synthetic
from tests.gpu_util import lib, rel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

L, DT = 2, 0.01


@pytest.mark.parametrize("replaced", [1, 2])
def test_make_corpus_equals_make_sample_over_the_same_trajectories(replaced):
    dn = lib()
    ob = synthetic.obstacle_block(1001)
    nus = [synthetic.viscosity(2000 + k, 0.004, 0.01) for k in range(2)]
    spin, spin_dt, relax, T = 4, 0.02, 1, 3
    common = dict(precision=dn.FP64, obstacle_i0=ob[0], obstacle_j0=ob[1], newton_tol=1e-12)
    ctx = dn.Context(level_solve=L, replaced_levels=replaced, nu=0.007, dt=DT, **common)
    fresh = dn.Context(level_solve=L, replaced_levels=replaced, nu=0.007, dt=DT, **common)
    X, Y = ctx.make_corpus(nus, spin, spin_dt, relax, T)
    P = ctx.num_patches()
    ci, co = ctx.net_dims()
    assert X.shape == (2, T, P, ci) and Y.shape == (2, T, P, co)
    for k, nu in enumerate(nus):
        coarse = dn.Context(level_solve=L, nu=nu, dt=spin_dt, **common)
        for _ in range(spin):
            coarse.step(dn.PLAIN)
        x = coarse.get_state()
        helper = dn.Context(level_solve=L, replaced_levels=replaced, nu=nu, dt=DT, **common)
        for r in range(replaced):
            x = helper.prolongate(L + r, x)
        fine = dn.Context(level_solve=L + replaced, nu=nu, dt=DT, **common)
        fine.set_state(x)
        for _ in range(relax):
            fine.step(dn.PLAIN)
        for n in range(T):
            prev = fine.get_state().clone()
            fine.step(dn.PLAIN)
            Xs, Ys = helper.make_sample(prev, fine.get_state())
            ex = rel(X[k, n].double().cpu().numpy(), Xs.double().cpu().numpy())
            ey = rel(Y[k, n].double().cpu().numpy(), Ys.double().cpu().numpy())
            assert ex < 1e-9 and ey < 1e-7, (k, n, ex, ey)
        for c in (coarse, helper, fine):
            c.close()
    # the context is back at the impulsive start with its configured physics
    np.testing.assert_array_equal(ctx.get_state().cpu().numpy(), fresh.get_state().cpu().numpy())
    ctx.step(dn.PLAIN)
    fresh.step(dn.PLAIN)
    assert rel(ctx.get_state().cpu().numpy(), fresh.get_state().cpu().numpy()) < 1e-12


def test_make_corpus_rejects_bad_arguments():
    dn = lib()
    ctx = dn.Context(level_solve=L, replaced_levels=1, precision=dn.FP64, nu=0.007, dt=DT)
    for args in (([0.005], 1, 0.0, 0, 1), ([-0.005], 1, 0.02, 0, 1), ([0.005], 1, 0.02, 0, 0),
                 ([0.005], -1, 0.02, 0, 1)):
        with pytest.raises(dn.DnnmgError) as e:
            ctx.make_corpus(*args)
        assert e.value.code == dn.ERR_ARG
    # a context without the network's patch level has no corpus to make
    plain = dn.Context(level_solve=L, replaced_levels=0, precision=dn.FP64, nu=0.007, dt=DT)
    buf = torch.empty(16, device="cuda")
    nu = (ctypes.c_double * 1)(0.005)
    rc = plain.lib.dnnmg_make_corpus(plain.h, 1, nu, 1, 0.02, 0, 1, dn._ptr(buf), dn._ptr(buf))
    assert rc == dn.ERR_STATE
