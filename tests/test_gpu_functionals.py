"""Parity of the CUDA functionals (Sec. 3.4) with the oracle through the C
ABI: J_div, drag and lift in residual form, and the relative l2 errors.
Both sides are FP64 with different summation orders: J_div to 1e-12
relative; drag and lift to 1e-12 of the sum of the absolute momentum rows
over the obstacle's boundary nodes (the terms they cancel from); errors to
1e-12 relative."""
import numpy as np
import pytest

from oracle import fem, functionals as fn, mesh
from tests.gpu_util import lib, seeded_state

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _ctx(dn, L, obstacle, prm, **kw):
    return dn.Context(level_solve=L, precision=dn.FP64, obstacle_i0=obstacle[0],
                      obstacle_j0=obstacle[1], nu=prm.nu, dt=prm.dt, **kw)


def _check(lev, got, x, prm, x_old):
    jd = fn.divergence(lev, x)
    d, l = fn.forces(lev, x, prm, x_old)
    ru, rv = fn.momentum_residual(lev, x, prm, x_old)
    gam = fn.obstacle_boundary(lev)
    scale = np.abs(ru[gam]).sum() + np.abs(rv[gam]).sum()
    assert abs(got[0] - jd) <= 1e-12 * jd, (got[0], jd)
    assert abs(got[1] - d) <= 1e-12 * scale, (got[1], d, scale)
    assert abs(got[2] - l) <= 1e-12 * scale, (got[2], l, scale)


@pytest.mark.parametrize("L,obstacle", [(2, (2, 1)), (3, (3, 1)), (5, (2, 1))])
@pytest.mark.parametrize("with_old", [True, False])
def test_functionals_match_oracle(L, obstacle, with_old):
    dn = lib()
    prm = fem.Params(nu=0.01, dt=0.02)
    ctx = _ctx(dn, L, obstacle, prm)
    lev = mesh.Level(L, obstacle=obstacle)
    x = seeded_state(lev, 30 + L)
    xo = seeded_state(lev, 40 + L) if with_old else None
    got = ctx.functionals(L, torch.from_numpy(x).cuda(),
                          torch.from_numpy(xo).cuda() if with_old else None)
    _check(lev, got, x, prm, xo)
    again = ctx.functionals(L, torch.from_numpy(x).cuda(),
                            torch.from_numpy(xo).cuda() if with_old else None)
    assert again == got                           # fixed-order sums


def test_functionals_on_every_level_of_a_two_level_dnnmg_context():
    """Levels below, at and above the solved one (the network's levels 5 and
    6 here; level 6 has more cells than one pass of the grid covers)."""
    dn = lib()
    prm = fem.Params(nu=0.004, dt=0.005)
    ctx = _ctx(dn, 4, (2, 1), prm, replaced_levels=2)
    for ell in (0, 1, 4, 5, 6):
        lev = mesh.Level(ell, obstacle=(2, 1))
        x = seeded_state(lev, 50 + ell)
        xo = seeded_state(lev, 60 + ell)
        got = ctx.functionals(ell, torch.from_numpy(x).cuda(), torch.from_numpy(xo).cuda())
        _check(lev, got, x, prm, xo)


def test_functionals_of_solver_steps():
    """Backward-Euler steps of the GPU solver from the impulsive start in the
    symmetric channel: oracle parity on its states, positive drag, and no
    lift beyond the solver tolerance."""
    dn = lib()
    prm = fem.Params(nu=0.05, dt=0.05)
    L = 3
    ctx = _ctx(dn, L, (2, 1), prm)
    lev = mesh.Level(L, obstacle=(2, 1))
    for _ in range(3):
        x_old = ctx.get_state().clone()
        ctx.step(dn.PLAIN)
    x = ctx.get_state()
    got = ctx.functionals(L, x, x_old)
    _check(lev, got, x.cpu().numpy(), prm, x_old.cpu().numpy())
    assert got[1] > 0.1
    assert abs(got[2]) < 1e-7 * got[1]


def test_relative_errors_match_oracle():
    dn = lib()
    prm = fem.Params(nu=0.01, dt=0.01)
    L = 4
    ctx = _ctx(dn, L, (3, 1), prm)
    lev = mesh.Level(L, obstacle=(3, 1))
    x = seeded_state(lev, 7)
    xr = seeded_state(lev, 8)
    got = ctx.relative_errors(L, torch.from_numpy(x).cuda(), torch.from_numpy(xr).cuda())
    ref = fn.relative_errors(lev, x, xr)
    np.testing.assert_allclose(got, ref, rtol=1e-12)
    xg = torch.from_numpy(x).cuda()
    assert ctx.relative_errors(L, xg, xg) == (0.0, 0.0)


def test_functionals_argument_errors():
    import ctypes
    dn = lib()
    prm = fem.Params(nu=0.01, dt=0.01)
    ctx = _ctx(dn, 2, (2, 1), prm)
    x = torch.zeros(ctx.ndof(2), dtype=torch.float64, device="cuda")
    out = (ctypes.c_double * 3)()
    for bad in (-1, 9):
        assert ctx.lib.dnnmg_functionals(ctx.h, bad, dn._ptr(x), None, out) == dn.ERR_ARG
        assert ctx.lib.dnnmg_relative_errors(ctx.h, bad, dn._ptr(x), dn._ptr(x), out) == dn.ERR_ARG
    assert ctx.lib.dnnmg_functionals(ctx.h, 2, None, None, out) == dn.ERR_ARG
    with pytest.raises(ValueError):
        ctx.functionals(2, x[:-1])
    lev = mesh.Level(2, obstacle=(2, 1))
    with pytest.raises(dn.DnnmgError) as e:
        ctx.relative_errors(2, torch.from_numpy(seeded_state(lev, 1)).cuda(), x)
    assert e.value.code == dn.ERR_NUMERICAL
