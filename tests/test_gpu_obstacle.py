"""Parity of the CUDA path with the oracle for the obstacle square snapped to
level-1 cells (the alternative geometry of Sec. 2.1's channel): at odd
level-1 offsets the 2h stabilisation patches of the coarse level are partly
solid, which only the coarse direct solve sees.  V-cycles (both persistent
kinds and the per-stage launches), plain time steps and DNN-MG steps
against the oracle; tolerances as for the level-0 block (1e-10 FP64, 1e-4
mixed, patch inputs 5e-3)."""
import numpy as np
import pytest

import synthetic
from oracle import dnnmg, fem, mesh, mg, net, newton
from tests.gpu_util import lib, rel, seeded_state

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _ctx(dn, L, precision, ob, nu=0.01, dt=0.01, **kw):
    return dn.Context(level_solve=L, precision=precision, obstacle_i0=ob[0], obstacle_j0=ob[1],
                      obstacle_level=ob[2], nu=nu, dt=dt, **kw)


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-4)])
@pytest.mark.parametrize("ob,split,mode", [((5, 3, 1), 0, -1), ((5, 3, 1), 3, 0),
                                           ((3, 2, 1), 3, 1), ((6, 2, 1), -1, -1),
                                           ((7, 3, 1), -1, -1)])
def test_snapped_obstacle_vcycle_matches_oracle(precision, tol, ob, split, mode):
    dn = lib()
    prm = fem.Params(nu=0.01, dt=0.01)
    L = 3
    ctx = _ctx(dn, L, precision, ob, prm.nu, prm.dt, persistent_vcycle=split,
               persistent_mode=mode)
    levels = mesh.hierarchy(L, obstacle=ob)
    lev = levels[-1]
    x = seeded_state(lev, 31)
    ctx.linearize(torch.from_numpy(x).cuda())
    b = synthetic.random_vector(81, lev.ndof)
    b[lev.cons] = 0.0
    xg = ctx.vcycle(L, torch.from_numpy(b).to(ctx.vdtype).cuda()).double().cpu().numpy()
    H = mg.Hierarchy(levels, x, prm)
    xr = mg.vcycle(H, len(levels) - 1, b)
    assert rel(xg, xr) < tol, rel(xg, xr)
    # the coarse solve alone (level 1, part-solid patches) is the exact solve
    lev1 = levels[0]
    b1 = synthetic.random_vector(82, lev1.ndof)
    b1[lev1.cons] = 0.0
    x1 = ctx.vcycle(1, torch.from_numpy(b1).to(ctx.vdtype).cuda()).double().cpu().numpy()
    assert rel(x1, mg.vcycle(H, 0, b1)) < (1e-12 if precision == 0 else 1e-6)


@pytest.mark.parametrize("precision", [0, 1])
def test_snapped_obstacle_steps_match_oracle(precision):
    dn = lib()
    ob = (5, 3, 1)
    prm = fem.Params(nu=0.01, dt=0.01)
    ntol = 1e-12 if precision == 0 else 1e-10
    ctx = _ctx(dn, 3, precision, ob, prm.nu, prm.dt, newton_tol=ntol)
    levels = mesh.hierarchy(3, obstacle=ob)
    opt = newton.SolverOptions(newton_tol=1e-12)
    x = mesh.initial_state(levels[-1])
    for n in range(3):
        st = ctx.step(dn.PLAIN)
        x, _, _, _ = newton.time_step(levels, x, prm, opt)
        xg = ctx.get_state().cpu().numpy()
        assert st["res_final"] <= ntol
        assert rel(xg, x) < (1e-10 if precision == 0 else 1e-4), (n, rel(xg, x), st)


def test_snapped_obstacle_dnnmg_steps_match_oracle():
    dn = lib()
    ob, L = (7, 1, 1), 2
    ctx = _ctx(dn, L, dn.FP64, ob, newton_tol=1e-12)
    spec = net.NetSpec()
    w = synthetic.random_weights(12, spec.num_params(), 0.05).astype(np.float32)
    ctx.set_weights(w)
    rng = np.random.default_rng(6)
    mean = rng.normal(0, 0.1, 40).astype(np.float32)
    std = rng.uniform(0.5, 2.0, 40).astype(np.float32)
    ctx.set_feature_stats(mean, std)
    levels = mesh.hierarchy(L, obstacle=ob)
    fine = mesh.Level(L + 1, obstacle=ob)
    opt = newton.SolverOptions(newton_tol=1e-12)
    prm = fem.Params(nu=0.01, dt=0.01)
    params = spec.unflatten(w.astype(np.float64))
    x = mesh.initial_state(levels[-1])
    state = dict(bL=None, vcorr=None, h=np.zeros((2, len(levels[-1].fluid_cells), 64)))
    P = ctx.num_patches()
    assert P == len(levels[-1].fluid_cells)
    for n in range(2):
        st = ctx.step(dn.NET)
        x, state, info = dnnmg.time_step(levels, fine, x, state, spec, params, prm, opt,
                                         mean.astype(np.float64), std.astype(np.float64))
        assert rel(ctx.get_state().cpu().numpy(), x) < 1e-4, n
        Xg = torch.empty(P, 40, dtype=torch.bfloat16, device="cuda")
        ctx.lib.dnnmg_get_patch_inputs(ctx.h, dn._ptr(Xg))
        assert rel(Xg.double().cpu().numpy(), info["X"]) < 5e-3, n
        assert st["fallback"] == int(info["fallback"])


def test_operator_on_part_solid_level_is_refused():
    """The operator kernels take whole patches: level 1 with the square at
    odd level-1 offsets is refused, level 2 (whole patches) matches the
    oracle, and at even offsets level 1 is whole and allowed."""
    dn = lib()
    prm = fem.Params(nu=0.01, dt=0.01)
    for ob, level1_ok in (((5, 3, 1), False), ((4, 2, 1), True)):
        ctx = _ctx(dn, 3, dn.FP64, ob, prm.nu, prm.dt)
        levels = mesh.hierarchy(3, obstacle=ob)
        x = seeded_state(levels[-1], 3)
        ctx.linearize(torch.from_numpy(x).cuda())
        H = mg.Hierarchy(levels, x, prm)
        for k, lev in enumerate(levels):
            w = torch.from_numpy(synthetic.random_vector(5 + k, lev.ndof)).cuda()
            if lev.ell == 1 and not level1_ok:
                with pytest.raises(dn.DnnmgError) as e:
                    ctx.apply(1, w)
                assert e.value.code == dn.ERR_ARG
                continue
            y = ctx.apply(lev.ell, w).cpu().numpy()
            assert rel(y, H.ops[k].A @ w.cpu().numpy()) < 1e-13, (ob, lev.ell)
